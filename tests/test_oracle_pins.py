"""Pins for the FP64 CPU oracle: it is checked here against what the paper and
the mathematics fix, never against a retyped copy of itself.

  * dense LU of the Kronecker-assembled operators of Eq. (Ai)  -> line solves,
    boundary matrices, axis order, species layout, Sherman-Morrison;
  * the framed scheme of Section 6 evaluated with dense solves  -> the step;
  * eigenmodes with analytic eigenvalues (F = 0 and F = -lambda u) -> R_RDP,
    R_01 and the predictor/corrector coefficients (Section 6);
  * D = 0  ->  Heun's method (textbook RK2);
  * conservation invariants (Neumann trapezoid sums, periodic sums);
  * second-order convergence (manufactured solution; Tables enztable/brutable);
  * reaction Jacobians / parameter derivatives by finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2001_11220_gb300 import workloads as W
from tests import dense_reference as dr

RNG = np.random.default_rng(12345)


def R_rdp(z):
    """Eq. (padenonlinear): (1 - 5z/12) / ((1 + z/3)(1 + z/4))."""
    return (1 - 5 * z / 12) / ((1 + z / 3) * (1 + z / 4))


# ------------------------------------------------------------ line solves --

@pytest.mark.parametrize("bc", [oracle.DIRICHLET, oracle.NEUMANN, oracle.PERIODIC])
@pytest.mark.parametrize("p", [3, 4, 7, 16])
@pytest.mark.parametrize("transpose", [False, True])
def test_line_solve_vs_dense(bc, p, transpose):
    r = 0.73
    h = 1.0
    M = np.eye(p) + r * dr.B_p(p, bc, h)
    b = RNG.standard_normal(p)
    x = oracle.line_solve(bc, r, b, transpose=transpose)
    ref = np.linalg.solve(M.T if transpose else M, b)
    assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("dims,bcs", [
    ((5, 4), (0, 0)), ((5, 4), (1, 1)), ((5, 4), (2, 2)), ((4, 6), (2, 1)),
    ((3, 4, 5), (0, 1, 2)), ((4, 3, 3), (1, 1, 1)), ((3, 3, 4), (2, 2, 2)),
])
@pytest.mark.parametrize("nspecies", [1, 2])
@pytest.mark.parametrize("transpose", [False, True])
def test_axis_solve_vs_kronecker_dense(dims, bcs, nspecies, transpose):
    D = (0.7, 0.2)[:nspecies]
    P = oracle.Problem(n=dims, bc=bcs, D=D, k=0.05, length=(1.0, 1.3, 0.8)[: len(dims)])
    U = RNG.standard_normal(P.shape)
    for axis in range(P.dim):
        for gamma in (1.0, 3.0, 4.0):
            got = oracle.axis_solve(P, axis, gamma, U, transpose=transpose)
            ref = dr.from_paper(P, dr.solve(P, axis + 1, gamma, dr.to_paper(P, U), transpose))
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), (axis, gamma)


def test_axis_apply_vs_kronecker_dense():
    P = oracle.Problem(n=(4, 5, 3), bc=(1, 2, 0), D=(0.3, 1.1), k=0.1)
    U = RNG.standard_normal(P.shape)
    for axis in range(3):
        ref = dr.from_paper(P, dr.A_i(P, axis + 1) @ dr.to_paper(P, U))
        assert np.allclose(oracle.axis_apply(P, axis, U), ref, rtol=1e-13, atol=1e-11)


def test_commutation_lemma():
    """Lemmas 1-2 (Section 4): A_i A_j = A_j A_i for the assembled operators."""
    P = oracle.Problem(n=(3, 4, 3), bc=(1, 2, 0), D=(0.3, 1.1), k=0.1)
    A = [dr.A_i(P, i) for i in (1, 2, 3)]
    for i in range(3):
        for j in range(3):
            assert np.allclose(A[i] @ A[j], A[j] @ A[i], atol=1e-9)


# --------------------------------------------------- the step vs the frame --

def _frame_dense(P, U, t, F):
    """The framed ETD-RDP-IF scheme of Section 6, every inverse a dense solve."""
    d, k = P.dim, P.k
    u = dr.to_paper(P, U)
    fu = dr.to_paper(P, F(U, t))

    def R(i, v):
        return 9 * dr.solve(P, i, 3.0, v) - 8 * dr.solve(P, i, 4.0, v)

    ustar = u + k * fu
    for i in range(1, d + 1):
        ustar = dr.solve(P, i, 1.0, ustar)
    fstar = dr.to_paper(P, F(dr.from_paper(P, ustar), t + k))
    g1 = 9 * u + 2 * k * fu
    g2 = 8 * u + 1.5 * k * fu
    for i in range(1, d):
        g1, g2 = R(i, g1), R(i, g2)
    out = dr.solve(P, d, 3.0, g1 + k * fstar) - dr.solve(P, d, 4.0, g2 + 0.5 * k * fstar)
    return dr.from_paper(P, out)


def _brusselator(a, b):
    def F(U, t):
        u, v = U
        return np.stack([a + u * u * v - (b + 1) * u, b * u - u * u * v])
    return F


@pytest.mark.parametrize("dims,bcs", [((6, 5), (1, 1)), ((5, 6), (2, 0)), ((4, 3, 5), (1, 2, 0)),
                                      ((3, 4, 4), (2, 2, 2))])
def test_step_vs_dense_frame(dims, bcs):
    a, b = 1.0, 3.4
    P = oracle.Problem(n=dims, bc=bcs, D=(0.02, 0.05), reaction=oracle.BRUSSELATOR, params=(a, b), k=0.07)
    U = np.stack([a + 0.1 * RNG.standard_normal(P.shape[1:]), b / a + 0.1 * RNG.standard_normal(P.shape[1:])])
    got = oracle.step(P, U, 0.3)
    ref = _frame_dense(P, U, 0.3, _brusselator(a, b))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_axis_order_matters():
    """Reading of the frame: axis d (slowest index) is the one carrying T_d/S_d with f(U*);
    transposing a 2D state therefore does not commute with a step."""
    a, b = 1.0, 3.4
    P = oracle.Problem(n=(6, 6), bc=(1, 1), D=(0.05, 0.05), reaction=oracle.BRUSSELATOR, params=(a, b), k=0.2)
    U = np.stack([a + 0.3 * RNG.standard_normal((6, 6)), b / a + 0.3 * RNG.standard_normal((6, 6))])
    s1 = oracle.step(P, U, 0.0)
    s2 = oracle.step(P, U.transpose(0, 2, 1).copy(), 0.0).transpose(0, 2, 1)
    assert np.max(np.abs(s1 - s2)) > 1e-6


# --------------------------------------------------- eigenmode closed forms --

def _mode(P, js):
    """separable eigenvector of every A_i and its eigenvalues mu_a of B_p."""
    vec = np.ones(())
    mus = []
    for a in range(P.dim):
        p, h, bc = P.n[a], P.h(a), P.bc[a]
        i = np.arange(p)
        j = js[a]
        if bc == oracle.DIRICHLET:     # sin(j pi x_i), x_i = (i+1) h
            v = np.sin(j * math.pi * (i + 1) * h)
            mu = 4 / h ** 2 * math.sin(j * math.pi * h / 2) ** 2
        elif bc == oracle.NEUMANN:     # cos(j pi x_i), x_i = i h
            v = np.cos(j * math.pi * i * h)
            mu = 4 / h ** 2 * math.sin(j * math.pi * h / 2) ** 2
        else:                          # cos(2 pi j x_i), x_i = i h
            v = np.cos(2 * math.pi * j * i * h)
            mu = 4 / h ** 2 * math.sin(math.pi * j * h) ** 2
        vec = np.multiply.outer(v, vec) if vec.ndim else v
        mus.append(mu)
    return vec, mus


@pytest.mark.parametrize("dims,bcs,js", [((9, 7), (0, 0), (2, 3)), ((9, 7), (1, 1), (1, 4)),
                                         ((8, 10), (2, 2), (1, 3)), ((6, 7, 8), (0, 1, 2), (2, 1, 3)),
                                         ((8, 8, 8), (2, 2, 2), (0, 1, 2))])
@pytest.mark.parametrize("k", [0.01, 0.4, 50.0])
def test_eigenmode_F0(dims, bcs, js, k):
    """F = 0: U_{n+1} = R_d...R_1 U_n (9T - 8S = R_RDP), so a mode decays by prod R_RDP(k D mu_a)."""
    D = (0.3, 0.05)
    P = oracle.Problem(n=dims, bc=bcs, D=D, reaction=oracle.ZERO, k=k)
    vec, mus = _mode(P, js)
    U = np.stack([vec, 2 * vec])
    nsteps = 3
    got = oracle.run(P, U, 0.0, nsteps)
    for s in range(2):
        fac = np.prod([R_rdp(k * D[s] * mu) for mu in mus]) ** nsteps
        ref = fac * U[s]
        assert np.max(np.abs(got[s] - ref)) <= 1e-12 * np.max(np.abs(U[s])), (s, fac)


def test_L_stability():
    """R_RDP(z) -> 0 as z -> infinity: a stiff mode is annihilated in one step (Section 6)."""
    P = oracle.Problem(n=(16, 16), bc=(0, 0), D=(1.0,), reaction=oracle.ZERO, k=1e6)
    vec, mus = _mode(P, (5, 7))
    got = oracle.step(P, vec[None], 0.0)
    assert np.max(np.abs(got)) < 1e-5 * np.max(np.abs(vec))
    assert abs(R_rdp(1e9)) < 1e-8 and abs(R_rdp(12 / 5)) < 1e-15


@pytest.mark.parametrize("dims,bcs", [((9, 7), (1, 0)), ((6, 7, 8), (0, 1, 2))])
def test_linear_reaction_closed_form(dims, bcs):
    """F = -lambda u on an eigenmode, z_a = k D mu_a, T(z) = 1/(1+z/3), S(z) = 1/(1+z/4),
    P(z) = 1/(1+z):  u* = (1 - k lambda) prod P(z_a) u,  c = prod_{a<d} R(z_a) u,
    u' = T(z_d)[(9 - 2k lambda) c - k lambda u*] - S(z_d)[(8 - 1.5 k lambda) c - 0.5 k lambda u*]."""
    lam, k, D = 1.7, 0.15, 0.08
    P = oracle.Problem(n=dims, bc=bcs, D=(D,), reaction=oracle.LINEAR, params=(-lam, 0.0), k=k)
    vec, mus = _mode(P, (1, 2, 1)[: len(dims)])
    z = [k * D * mu for mu in mus]
    ustar = (1 - k * lam) * np.prod([1 / (1 + zz) for zz in z])
    c = np.prod([R_rdp(zz) for zz in z[:-1]])
    T, S = 1 / (1 + z[-1] / 3), 1 / (1 + z[-1] / 4)
    fac = T * ((9 - 2 * k * lam) * c - k * lam * ustar) - S * ((8 - 1.5 * k * lam) * c - 0.5 * k * lam * ustar)
    got = oracle.step(P, vec[None], 0.0)
    assert np.max(np.abs(got[0] - fac * vec)) <= 1e-13 * np.max(np.abs(vec))


def test_zero_diffusion_is_heun():
    """D = 0: T = S = P = I and the scheme is u + k/2 (f(u) + f(u + k f(u))) pointwise."""
    a, b, k = 1.0, 3.4, 0.05
    P = oracle.Problem(n=(7, 5), bc=(1, 2), D=(0.0, 0.0), reaction=oracle.BRUSSELATOR, params=(a, b), k=k)
    U = np.stack([a + 0.2 * RNG.standard_normal((5, 7)), b / a + 0.2 * RNG.standard_normal((5, 7))])
    F = _brusselator(a, b)
    heun = U + 0.5 * k * (F(U, 0) + F(U + k * F(U, 0), k))
    assert np.max(np.abs(oracle.step(P, U, 0.0) - heun)) < 1e-14 * 10


# --------------------------------------------------------------- invariants --

def test_conservation_neumann_and_periodic():
    """F = 0: the trapezoid weights (1/2, 1, ..., 1, 1/2) are a left null vector of the
    Neumann B_p and the all-ones vector one of the periodic B_p, so the weighted sums are
    invariant under every (I + c A_i)^{-1} and hence under the step (9 - 8 = 1)."""
    P = oracle.Problem(n=(6, 7, 5), bc=(1, 2, 1), D=(0.4, 0.9), reaction=oracle.ZERO, k=0.3)
    U = RNG.standard_normal(P.shape)
    wts = []
    for a in range(3):
        w = np.ones(P.n[a])
        if P.bc[a] == oracle.NEUMANN:
            w[0] = w[-1] = 0.5
        wts.append(w)
    Wt = np.einsum("z,y,x->zyx", wts[2], wts[1], wts[0])
    V = oracle.run(P, U, 0.0, 5)
    for s in range(2):
        assert abs((Wt * V[s]).sum() - (Wt * U[s]).sum()) < 1e-12 * np.abs(U[s]).sum()


def test_constant_source_constant_state():
    """F = c, constant initial state, Neumann/periodic: U_n = U_0 + n k c exactly."""
    c, k = 0.37, 0.2
    P = oracle.Problem(n=(5, 6), bc=(1, 2), D=(0.5,), reaction=oracle.LINEAR, params=(0.0, c), k=k)
    U = np.full(P.shape, 1.25)
    V = oracle.run(P, U, 0.0, 7)
    assert np.max(np.abs(V - (1.25 + 7 * k * c))) < 1e-13


# ---------------------------------------------------------------- reaction --

@pytest.mark.parametrize("kind,params,S", [(oracle.LINEAR, (-0.7, 0.3), 2), (oracle.BRUSSELATOR, (1.0, 3.4), 2),
                                           (oracle.SCHNAKENBERG, (0.1, 0.9, 5.0), 2),
                                           (oracle.GRAY_SCOTT, (0.04, 0.06), 2), (oracle.ENZYME, (1.0, 0.8), 1),
                                           (oracle.CGL, (1.3,), 2)])
def test_reaction_derivatives_fd(kind, params, S):
    P = oracle.Problem(n=(5, 4), bc=(0, 0), D=(0.1,) * S, reaction=kind, params=params, k=0.1)
    U = 0.5 + 0.5 * RNG.random(P.shape)
    ybar = RNG.standard_normal(P.shape)
    out, pbar = oracle.reaction_vjp(P, U, 0.2, ybar)
    eps = 1e-6
    V = RNG.standard_normal(P.shape)
    fd = (np.sum(ybar * oracle.reaction(P, U + eps * V, 0.2)) - np.sum(ybar * oracle.reaction(P, U - eps * V, 0.2))) / (2 * eps)
    assert abs(fd - np.sum(out * V)) < 1e-7 * max(1, abs(fd))
    for j in range(len(params)):
        pp, pm = list(params), list(params)
        pp[j] += eps
        pm[j] -= eps
        Pp = oracle.Problem(n=P.n, bc=P.bc, D=P.D, reaction=kind, params=pp, k=0.1)
        Pm = oracle.Problem(n=P.n, bc=P.bc, D=P.D, reaction=kind, params=pm, k=0.1)
        fdp = (np.sum(ybar * oracle.reaction(Pp, U, 0.2)) - np.sum(ybar * oracle.reaction(Pm, U, 0.2))) / (2 * eps)
        assert abs(fdp - pbar[j]) < 1e-7 * max(1, abs(fdp)), j


def test_reaction_steady_states():
    """Homogeneous equilibria of the systems: F vanishes there."""
    cases = [(oracle.BRUSSELATOR, (1.0, 3.4), (1.0, 3.4)), (oracle.BRUSSELATOR, (2.0, 1.0), (2.0, 0.5)),
             (oracle.SCHNAKENBERG, (0.1, 0.9, 1000.0), (1.0, 0.9)), (oracle.GRAY_SCOTT, (0.04, 0.06), (1.0, 0.0))]
    for kind, params, st in cases:
        P = oracle.Problem(n=(3, 3), bc=(1, 1), D=(0.1, 0.1), reaction=kind, params=params, k=0.1)
        U = np.stack([np.full((3, 3), st[0]), np.full((3, 3), st[1])])
        assert np.max(np.abs(oracle.reaction(P, U, 0.0))) < 1e-12


def test_gray_scott_interior_equilibrium():
    """Gray-Scott with F = 0.04, kappa = 0.06 has the non-trivial homogeneous
    equilibrium (u, v) = (0.5, 0.2): u v = F + kappa and F (1 - u) = (F + kappa) v
    give 0.1 v^2 - 0.04 v + 0.004 = 0, a double root at v = 0.2.  Every term of
    the reaction is non-zero there (u v^2 = 0.02 = F (1 - u) = (F + kappa) v), so
    a swapped u^2 v or a wrong sign of any term moves F away from zero.  Nearby
    points must not be equilibria."""
    P = oracle.Problem(n=(3, 3), bc=(2, 2), D=(0.1, 0.1), reaction=oracle.GRAY_SCOTT, params=(0.04, 0.06), k=0.1)
    U = np.stack([np.full((3, 3), 0.5), np.full((3, 3), 0.2)])
    assert np.max(np.abs(oracle.reaction(P, U, 0.0))) < 1e-15
    for du, dv in ((0.01, 0.0), (0.0, 0.01), (-0.01, 0.01)):
        V = np.stack([np.full((3, 3), 0.5 + du), np.full((3, 3), 0.2 + dv)])
        assert np.min(np.abs(oracle.reaction(P, V, 0.0)).max(axis=0)) > 1e-4, (du, dv)


@pytest.mark.parametrize("kind,params,uv,f", [
    # hand-evaluated at (u, v) = (0.3, 0.7): -u v^2 + F (1 - u) = -0.147 + 0.028; u v^2 - (F + kappa) v = 0.147 - 0.07
    (oracle.GRAY_SCOTT, (0.04, 0.06), (0.3, 0.7), (-0.119, 0.077)),
    # a + u^2 v - (b + 1) u = 1 + 0.5 - 2.2; b u - u^2 v = 1.7 - 0.5 at (0.5, 2)
    (oracle.BRUSSELATOR, (1.0, 3.4), (0.5, 2.0), (-0.7, 1.2)),
    # gamma (a - u + u^2 v) = 2 (0.1 - 0.5 + 0.5); gamma (b - u^2 v) = 2 (0.9 - 0.5) at (0.5, 2)
    (oracle.SCHNAKENBERG, (0.1, 0.9, 2.0), (0.5, 2.0), (0.2, 0.8)),
])
def test_reaction_hand_values(kind, params, uv, f):
    """Two-species reactions at a point where u^2 v and u v^2 differ (Section 8's
    model equations evaluated by hand)."""
    P = oracle.Problem(n=(3, 3), bc=(1, 1), D=(0.1, 0.1), reaction=kind, params=params, k=0.1)
    U = np.stack([np.full((3, 3), uv[0]), np.full((3, 3), uv[1])])
    out = oracle.reaction(P, U, 0.0)
    assert np.max(np.abs(out[0] - f[0])) < 1e-14 and np.max(np.abs(out[1] - f[1])) < 1e-14


def test_manufactured_source_consistency():
    """u = e^{-t} prod sin(pi x_a) solves u_t = d Lap u - u/(1+u) + src with the continuous
    Laplacian: check the residual pointwise with analytic derivatives."""
    d = 0.8
    w = W.mms_3d(6).with_(D=(d,), params=(1.0, d))
    P = dr.oracle_problem(w)
    t = 0.37
    u = W.exact_mms(w, t)
    F = oracle.reaction(P, u, t)
    u_t = -u
    lap = -3 * math.pi ** 2 * u
    assert np.max(np.abs(u_t - (d * lap + F))) < 1e-13


# ----------------------------------------------------------- convergence --

def test_second_order_manufactured_3d():
    """Manufactured solution, Dirichlet cube, k = h: error vs the exact solution falls as h^2
    (space and time both second order)."""
    errs = []
    for p in (7, 15, 31):
        w = W.mms_3d(p)
        U = oracle.run(dr.oracle_problem(w), W.initial_state(w), 0.0, w.steps)
        errs.append(np.max(np.abs(U - W.exact_mms(w, w.steps * w.k))))
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    # pre-asymptotic at p = 7 (k = h = 1/8); the order approaches 2 from below (1.96 at p = 63)
    assert 1.7 < eoc[0] < 2.2 and 1.85 < eoc[1] < 2.2, (errs, eoc)


def _table(name):
    rows = []
    with open(__file__.rsplit("/", 1)[0] + f"/golden/{name}") as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, eps, eoc = line.split()
                rows.append((float(k), float(eps), None if eoc == "-" else float(eoc)))
    return rows


@pytest.mark.slow
def test_paper_brusselator_table():
    """Table brutable (Section 8.2): errors within a factor 1.5 of the printed ones and EOC
    within 0.3 of the printed EOC; reference = same scheme at k_min/16."""
    rows = _table("brusselator_table.txt")
    wref = W.brusselator_paper(81, rows[-1][0] / 16)
    Uref = oracle.run(dr.oracle_problem(wref), W.initial_state(wref), 0.0, wref.steps)
    errs = []
    for k, eps, _ in rows:
        w = W.brusselator_paper(81, k)
        errs.append(np.max(np.abs(oracle.run(dr.oracle_problem(w), W.initial_state(w), 0.0, w.steps) - Uref)))
    for (k, eps, _), e in zip(rows, errs):
        assert eps / 1.5 < e < eps * 1.5, (k, e, eps)
    for i in range(1, len(rows)):
        assert abs(math.log2(errs[i - 1] / errs[i]) - rows[i][2]) < 0.3


@pytest.mark.slow
def test_paper_enzyme_table_order():
    """Table enztable (Section 8.1): EOC within 0.25 of the printed values."""
    rows = _table("enzyme_table.txt")
    wref = W.enzyme_paper(79, rows[-1][0] / 16)
    Uref = oracle.run(dr.oracle_problem(wref), W.initial_state(wref), 0.0, wref.steps)
    errs = []
    for k, _, _ in rows:
        w = W.enzyme_paper(79, k)
        errs.append(np.max(np.abs(oracle.run(dr.oracle_problem(w), W.initial_state(w), 0.0, w.steps) - Uref)))
    for i in range(1, len(rows)):
        assert abs(math.log2(errs[i - 1] / errs[i]) - rows[i][2]) < 0.25


@pytest.mark.slow
def test_brusselator_3d_terminal_behaviour():
    """Section 8.2, 3D: Neumann, h = 1/10, k = 1/1000, D = 0.02.  With A = 1, B = 2
    (1 - A + B^2 >= 0) the point values approach (B, A/B) = (2, 1/2) by T = 5."""
    w = W.Workload("bru3d", (11, 11, 11), W.NEUMANN, (0.02, 0.02), "brusselator", (2.0, 1.0), 1e-3, 5000,
                   ic="brusselator_3d")
    U = oracle.run(dr.oracle_problem(w), W.initial_state(w), 0.0, w.steps)
    i = 3  # x = 0.3
    assert abs(U[0, i, i, i] - 2.0) < 1e-2 and abs(U[1, i, i, i] - 0.5) < 1e-2


# ----------------------------------------------------------------- adjoint --

@pytest.mark.parametrize("dims,bcs,kind,params", [
    ((5, 6), (1, 2), oracle.BRUSSELATOR, (1.0, 3.4)),
    ((4, 5, 3), (2, 0, 1), oracle.GRAY_SCOTT, (0.04, 0.06)),
    ((6, 5), (0, 0), oracle.SCHNAKENBERG, (0.1, 0.9, 3.0)),
])
def test_step_adjoint_vs_finite_differences(dims, bcs, kind, params):
    D = (0.03, 0.07)
    P = oracle.Problem(n=dims, bc=bcs, D=D, reaction=kind, params=params, k=0.1)
    U = 0.5 + 0.3 * RNG.random(P.shape)
    wbar = RNG.standard_normal(P.shape)
    Ubar, dD, dp = oracle.step_adjoint(P, U, 0.1, wbar)
    eps = 1e-6

    def J(Pq, V):
        return np.sum(wbar * oracle.step(Pq, V, 0.1))

    v = RNG.standard_normal(P.shape)
    fd = (J(P, U + eps * v) - J(P, U - eps * v)) / (2 * eps)
    assert abs(fd - np.sum(Ubar * v)) < 1e-7 * max(1, abs(fd))
    for s in range(2):
        Dp, Dm = list(D), list(D)
        Dp[s] += eps
        Dm[s] -= eps
        Pp = oracle.Problem(n=dims, bc=bcs, D=Dp, reaction=kind, params=params, k=0.1)
        Pm = oracle.Problem(n=dims, bc=bcs, D=Dm, reaction=kind, params=params, k=0.1)
        fdD = (J(Pp, U) - J(Pm, U)) / (2 * eps)
        assert abs(fdD - dD[s]) < 1e-6 * max(1, abs(fdD)), (s, fdD, dD[s])
    for j in range(len(params)):
        pp, pm = list(params), list(params)
        pp[j] += eps
        pm[j] -= eps
        Pp = oracle.Problem(n=dims, bc=bcs, D=D, reaction=kind, params=pp, k=0.1)
        Pm = oracle.Problem(n=dims, bc=bcs, D=D, reaction=kind, params=pm, k=0.1)
        fdp = (J(Pp, U) - J(Pm, U)) / (2 * eps)
        assert abs(fdp - dp[j]) < 1e-6 * max(1, abs(fdp)), (j, fdp, dp[j])


def test_grad_multistep_vs_finite_differences():
    w = W.gray_scott_3d(6, steps=4).with_(k=0.5, D=(0.01, 0.005))
    P = dr.oracle_problem(w)
    U0 = W.initial_state(w)
    target = W.initial_state(w, seed=7)
    loss, dU0, dD, dp = oracle.grad(P, U0, 0.0, target, w.steps)

    def L(Pq, V):
        r = oracle.run(Pq, V, 0.0, w.steps) - target
        return 0.5 * np.sum(r * r)

    assert abs(L(P, U0) - loss) < 1e-12 * loss
    eps = 1e-6
    v = RNG.standard_normal(P.shape)
    fd = (L(P, U0 + eps * v) - L(P, U0 - eps * v)) / (2 * eps)
    assert abs(fd - np.sum(dU0 * v)) < 1e-6 * max(1, abs(fd))
    for s in range(2):
        Dp, Dm = list(w.D), list(w.D)
        Dp[s] += eps
        Dm[s] -= eps
        fdD = (L(dr.oracle_problem(w.with_(D=tuple(Dp))), U0) - L(dr.oracle_problem(w.with_(D=tuple(Dm))), U0)) / (2 * eps)
        assert abs(fdD - dD[s]) < 1e-5 * max(1, abs(fdD))


def test_threads_do_not_change_results():
    """The OpenMP loops share out independent lines and points; every value
    must be bit-identical to the one-thread result."""
    import oracle
    P = oracle.Problem(n=(9, 7, 11), bc=(0, 2, 1), D=(0.7, 0.2), reaction=oracle.BRUSSELATOR,
                       params=(1.0, 3.0), k=0.01)
    U0 = 1.0 + 0.1 * np.random.default_rng(3).standard_normal(P.shape)
    prev = oracle.get_threads()
    try:
        oracle.set_threads(1)
        a = oracle.run(P, U0, 0.0, 3)
        oracle.set_threads(4)
        b = oracle.run(P, U0, 0.0, 3)
    finally:
        oracle.set_threads(prev)
    assert np.array_equal(a, b)


# ------------------------------------------------- complex Ginzburg-Landau --
# Section 8: u_t = u + (1 + i alpha) Lap u - (1 + i beta) u |u|^2 with alpha = 0,
# carried as two real species (Re u, Im u) with the same real D.

def test_cgl_reaction_hand_values():
    """F = u - (1 + i beta) u |u|^2 at u = 0.6 + 0.8 i (|u| = 1) with beta = 1.3 is
    -i beta u = 1.04 - 0.78 i; at u = 0.5 (|u|^2 = 0.25): 0.5 - 0.125 (1 + 1.3 i)
    = 0.375 - 0.1625 i."""
    P = oracle.Problem(n=(4, 4), bc=(2, 2), D=(1.0, 1.0), reaction=oracle.CGL, params=(1.3,), k=0.05)
    for (a, b), (fa, fb) in (((0.6, 0.8), (1.04, -0.78)), ((0.5, 0.0), (0.375, -0.1625))):
        U = np.stack([np.full((4, 4), a), np.full((4, 4), b)])
        F = oracle.reaction(P, U, 0.0)
        assert abs(F[0, 0, 0] - fa) < 1e-15 and abs(F[1, 0, 0] - fb) < 1e-15, (F[:, 0, 0], fa, fb)


def test_cgl_uniform_unit_modulus_state_rotates_at_second_order():
    """A uniform state of modulus 1 has zero Laplacian and F = -i beta u, so the exact
    solution is u(t) = e^{-i beta t} u0.  The scheme integrates this ODE at second
    order: halving k divides the error at T = 1 by about 4."""
    beta, T = 1.3, 1.0
    u0 = np.exp(0.4j)
    errs = []
    for k in (0.05, 0.025, 0.0125):
        P = oracle.Problem(n=(8, 8), bc=(2, 2), D=(1.0, 1.0), reaction=oracle.CGL, params=(beta,), k=k)
        U = np.stack([np.full((8, 8), u0.real), np.full((8, 8), u0.imag)])
        V = oracle.run(P, U, 0.0, int(round(T / k)))
        exact = u0 * np.exp(-1j * beta * T)
        errs.append(max(np.max(np.abs(V[0] - exact.real)), np.max(np.abs(V[1] - exact.imag))))
        assert np.max(np.abs(V - V[:, :1, :1])) < 1e-14   # stays uniform
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.2 for o in orders), (errs, orders)


def test_cgl_phase_equivariance():
    """The equation is invariant under u -> e^{i phi} u, and so is the scheme: real
    line matrices act on Re u and Im u alike and F(e^{i phi} u) = e^{i phi} F(u).  A
    rotated initial state gives the rotated solution (to rounding); a wrong sign or a
    swapped coupling term of F breaks this."""
    P = oracle.Problem(n=(12, 10), bc=(2, 2), D=(1.0, 1.0), reaction=oracle.CGL, params=(1.3,), k=0.05,
                       length=(6.0, 5.0))
    rng = np.random.default_rng(7)
    U = 0.5 * rng.standard_normal((2, 10, 12))
    phi = 0.9
    c, s = np.cos(phi), np.sin(phi)
    R = np.stack([c * U[0] - s * U[1], s * U[0] + c * U[1]])
    V = oracle.run(P, U, 0.0, 6)
    VR = oracle.run(P, R, 0.0, 6)
    rot = np.stack([c * V[0] - s * V[1], s * V[0] + c * V[1]])
    assert np.max(np.abs(VR - rot)) < 1e-13 * max(1.0, np.max(np.abs(V)))
    assert np.max(np.abs(V - U)) > 1e-2   # the run did something
