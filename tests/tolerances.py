"""FP32 error bound of one ETD-RDP-IF step against the FP64 oracle, derived
per workload from the line matrices.

One solve x = M^{-1} b of M = tridiag(-r, 1 + 2r, -r) runs two first-order
recurrences (forward and backward elimination, Section 7) whose multiplier
converges to lam(r) = 2r / (1 + 2r + sqrt(1 + 4r)) < 1, the decay factor of
M^{-1} away from its diagonal.  A rounding error of u = 2^-24 (relative) made
at one position reaches position i + j attenuated by lam^j, so the error a
recurrence leaves at a position is a weighted sum of independent roundings;
its root-sum-square is u / sqrt(1 - lam^2) =: u g(r).  Per axis the step
applies R = 9T - 8S (T: gamma = 3, S: gamma = 4; the |9| + |8| = 17
cancellation of the partial fractions of R_RDP, Section 6) and P (gamma = 1),
each solve with two recurrences:
    e_a = 2 (9 g(r_a / 3) + 8 g(r_a / 4) + g(r_a)),  r_a = k max_s D_s / h_a^2
and the step error is bounded by C u sum_a e_a with C = 3 for the rounding of
the state, the reaction and the pointwise combinations of the frame.  For
non-stiff lines (g ~ 1) this is about 216 u (2D) to 324 u (3D); the stiff
4096^2 periodic lines (r = 16777, g ~ 6-8) give about 1300 u.
"""
import math

import numpy as np

U_FP32 = 2.0 ** -24


def decay(r: float) -> float:
    """Decay factor of the inverse of tridiag(-r, 1 + 2r, -r) (the smaller root
    of lam^2 - (2 + 1/r) lam + 1 = 0), 0 for r = 0."""
    if r <= 0.0:
        return 0.0
    return 2.0 * r / ((1.0 + 2.0 * r) + math.sqrt(1.0 + 4.0 * r))


def gain(r: float) -> float:
    lam = decay(r)
    return 1.0 / math.sqrt(1.0 - lam * lam)


def decay_c(r: complex) -> float:
    """|lam| of the smaller root of lam^2 - (2 + 1/r) lam + 1 = 0 for the
    complex line matrices tridiag(-r, 1 + 2r, -r) of the coupled systems
    (r = k (p + i q) / h^2): the roots multiply to 1, so the smaller one has
    modulus below 1 whenever 2 + 1/r is not in [-2, 2] (Re r >= 0, r != 0)."""
    if r == 0:
        return 0.0
    b = 2.0 + 1.0 / r
    disc = np.sqrt(complex(b * b - 4.0))
    return float(min(abs((b - disc) / 2.0), abs((b + disc) / 2.0)))


def fp32_step_bound(w, C: float = 3.0) -> float:
    """Relative error bound (max over species of max|diff| / max|U|) of one
    FP32 step of workload w against the FP64 oracle.  Coupled workloads
    (w.Dc = [[p, -q], [q, p]]) take the decay factor of their complex line
    matrices, with the same count of recurrences and cancellations, and a
    factor 2 for the four real products of each complex multiply."""
    Dc = getattr(w, "Dc", None)
    total = 0.0
    for a in range(w.dim):
        if Dc is None:
            r = w.k * max(w.D) / w.h(a) ** 2
            total += 2.0 * (9.0 * gain(r / 3.0) + 8.0 * gain(r / 4.0) + gain(r))
        else:
            r = w.k * complex(Dc[0], Dc[2]) / w.h(a) ** 2
            g = [1.0 / math.sqrt(1.0 - decay_c(r / gm) ** 2) for gm in (3.0, 4.0, 1.0)]
            total += 4.0 * (9.0 * g[0] + 8.0 * g[1] + g[2])
    return C * U_FP32 * total


def fp32_ensemble_bound(works, nsteps: int = 1) -> float:
    """Bound for a set of instances run nsteps steps: the largest per-step
    bound, times the number of steps (errors of successive steps add)."""
    return nsteps * max(fp32_step_bound(w) for w in works)


def fp64_solve_error(w) -> float:
    """The FP32 step bound's arithmetic with the FP64 unit roundoff 2^-53: the
    relative error the FP64 line solves of one step leave in the state."""
    return fp32_step_bound(w) * 2.0 ** -29


def fp64_param_grad_bound(w, U, nsteps: int = 1, C: float = 10.0) -> float:
    """Relative bound for dL/dD and dL/dparams in FP64.  The GPU forms
    <lambda, B x> of every solve (I + r h^2 B) x = b as <lambda, b - x> / r,
    r = (k / gamma) D_s / h^2, so the solve error of x (fp64_solve_error) is
    amplified by |x| / |b - x| = |x| / (r |h^2 B x|): 1 plus the ratio of the
    state's magnitude to its second differences along each axis divided by r
    (gamma = 4, the worst species and axis), measured on the state U the
    gradient starts from.  Errors of successive reversed steps add (nsteps);
    C = 10 covers the FP64 sums over the grid and the smoothing of the state
    over the run (the ratio grows as diffusion smooths it)."""
    amp = 1.0
    for s in range(w.nspecies):
        x = np.asarray(U[s], dtype=np.float64)
        for a in range(w.dim):
            ax = x.ndim - 1 - a
            if w.bc[a] == 2:  # periodic
                d2 = 2.0 * x - np.roll(x, 1, ax) - np.roll(x, -1, ax)
            else:
                d2 = np.diff(x, 2, axis=ax)
            r = (w.k / 4.0) * w.D[s] / w.h(a) ** 2
            amp = max(amp, 1.0 + float(np.abs(x).max()) / (r * max(float(np.abs(d2).max()), 1e-300)))
    return C * nsteps * fp64_solve_error(w) * amp
