"""Dense Kronecker-assembled operators of Section 3 (test-only).

Builds the matrices exactly as printed: B_p of Example 1 for each boundary
type, and A_i of Eq. (Ai) with the species factor D in the LAST Kronecker slot
(species index fastest) and B_p at position d-i+1.  The oracle and the CUDA
library store the state species-major with x fastest, so ``to_paper`` /
``from_paper`` permute between the two orderings.  Dense solves use LAPACK
through numpy.linalg.solve; nothing here calls the oracle.
"""
from __future__ import annotations

import numpy as np

import oracle


def oracle_problem(w) -> oracle.Problem:
    """oracle.Problem for a workloads.Workload."""
    return oracle.Problem(n=w.n, bc=w.bc, D=w.D, reaction=w.reaction_id, params=w.params, k=w.k,
                          length=w.length, Dc=w.Dc)


def B_p(p: int, bc: int, h: float) -> np.ndarray:
    """Example 1: -(1/h^2) times the printed second-difference matrix."""
    T = np.zeros((p, p))
    for i in range(p):
        T[i, i] = -2.0
        if i > 0:
            T[i, i - 1] = 1.0
        if i < p - 1:
            T[i, i + 1] = 1.0
    if bc == oracle.NEUMANN:
        T[0, 1] = 2.0
        T[p - 1, p - 2] = 2.0
    if bc == oracle.PERIODIC:
        T[0, p - 1] = 1.0
        T[p - 1, 0] = 1.0
    return -T / (h * h)


def A_i(P: oracle.Problem, i: int) -> np.ndarray:
    """Eq. (Ai): I x ... x B_p (position d-i+1) x ... x I x D, i = 1..d (axis i-1).
    D is diag(P.D), or the full 2 x 2 matrix P.Dc of the coupled systems of
    Section 8 (the same Kronecker slot)."""
    d = P.dim
    Dm = np.diag(P.D) if getattr(P, "Dc", None) is None else np.asarray(P.Dc, dtype=np.float64).reshape(2, 2)
    factors = []
    for pos in range(1, d + 1):          # spatial Kronecker positions 1..d
        axis = d - pos                    # position d-i+1 holds axis i-1
        n = P.n[axis]
        factors.append(B_p(n, P.bc[axis], P.h(axis)) if axis == i - 1 else np.eye(n))
    M = factors[0]
    for F in factors[1:]:
        M = np.kron(M, F)
    return np.kron(M, Dm)


def to_paper(P: oracle.Problem, U: np.ndarray) -> np.ndarray:
    """state[s, (z,) y, x] -> paper vector with the species index fastest."""
    U = np.asarray(U).reshape(P.shape)
    return np.moveaxis(U, 0, -1).ravel()


def from_paper(P: oracle.Problem, v: np.ndarray) -> np.ndarray:
    shape = tuple(reversed(P.n)) + (P.nspecies,)
    return np.moveaxis(v.reshape(shape), -1, 0).copy()


def solve(P: oracle.Problem, i: int, gamma: float, v: np.ndarray, transpose=False) -> np.ndarray:
    """(I + (k/gamma) A_i)^{-1} v by dense LU (numpy.linalg.solve)."""
    A = A_i(P, i)
    M = np.eye(A.shape[0]) + (P.k / gamma) * A
    return np.linalg.solve(M.T if transpose else M, v)
