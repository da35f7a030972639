"""Seeded synthetic workloads: problem descriptions and initial states.

This module holds no arithmetic of the ETD-RDP-IF method: it only names
problems (grid, boundaries, diffusion coefficients, reaction and its
parameters, time step, step count) and draws initial states from a seeded
generator.  Both the CUDA path and the CPU oracle are fed from here, so parity
never depends on a random-number generator.

Problems mirror the paper's experiments (Section 8) and the reaction-diffusion
systems they use; sizes are the benchmark shapes.  Naming: n[a] grid nodes on
axis a (axis 0 = x, fastest), paper's convention per boundary type (Section 3,
Example 1): Dirichlet p interior nodes with h = L/(p+1), Neumann p nodes with
h = L/(p-1), periodic p nodes with h = L/p.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

DIRICHLET, NEUMANN, PERIODIC = 0, 1, 2
REACTIONS = {"zero": 0, "linear": 1, "brusselator": 2, "schnakenberg": 3, "gray_scott": 4, "enzyme": 5,
             "cgl": 6, "nls": 7}
BC_NAMES = {DIRICHLET: "dirichlet", NEUMANN: "neumann", PERIODIC: "periodic"}


@dataclass
class Workload:
    name: str
    n: tuple                 # nodes per axis, x first
    bc: tuple                # boundary type per axis
    D: tuple                 # diffusion coefficient per species
    reaction: str
    params: tuple
    k: float
    steps: int
    length: tuple = None
    t0: float = 0.0
    ic: str = "normal"       # initial-state recipe, see initial_state()
    ic_args: tuple = ()
    seed: int = 2001
    extra: dict = field(default_factory=dict)
    Dc: tuple = None         # coupled two-species diffusion matrix (row-major 2 x 2), or None

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if isinstance(self.bc, int):
            self.bc = (self.bc,) * len(self.n)
        if self.length is None:
            self.length = (1.0,) * len(self.n)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def nspecies(self) -> int:
        return len(self.D)

    @property
    def npoints(self) -> int:
        return int(np.prod(self.n))

    @property
    def shape(self) -> tuple:
        return (self.nspecies,) + tuple(reversed(self.n))

    @property
    def reaction_id(self) -> int:
        return REACTIONS[self.reaction]

    def h(self, axis: int) -> float:
        p, L = self.n[axis], self.length[axis]
        return {DIRICHLET: L / (p + 1), NEUMANN: L / (p - 1), PERIODIC: L / p}[self.bc[axis]]

    def coords(self, axis: int) -> np.ndarray:
        h = self.h(axis)
        i = np.arange(self.n[axis], dtype=np.float64)
        return (i + 1) * h if self.bc[axis] == DIRICHLET else i * h

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _grids(w: Workload):
    """coordinate arrays broadcast to the state layout (z, y, x)."""
    axes = [w.coords(a) for a in range(w.dim)]
    return np.meshgrid(*reversed(axes), indexing="ij")[::-1]  # x, y, (z)


def initial_state(w: Workload, seed: int | None = None) -> np.ndarray:
    """Initial state U[s][z][y][x] in float64 for the workload's recipe."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    shape = w.shape
    if w.ic == "normal":          # base_s + scale * N(0, 1)
        base, scale = w.ic_args
        U = np.empty(shape)
        for s in range(w.nspecies):
            U[s] = base[s] + scale * rng.standard_normal(shape[1:])
        return U
    if w.ic == "uniform":         # base_s + U(-amp, amp)
        base, amp = w.ic_args
        U = np.empty(shape)
        for s in range(w.nspecies):
            U[s] = base[s] + rng.uniform(-amp, amp, size=shape[1:])
        return U
    if w.ic == "sine":            # prod_a sin(pi x_a / L_a) (manufactured solution at t = 0)
        g = _grids(w)
        q = np.ones(shape[1:])
        for a in range(w.dim):
            q = q * np.sin(math.pi * g[a] / w.length[a])
        return q[None].repeat(w.nspecies, axis=0).copy()
    if w.ic == "constant":
        (vals,) = w.ic_args
        U = np.empty(shape)
        for s in range(w.nspecies):
            U[s] = vals[s]
        return U
    if w.ic == "brusselator_paper":   # Section 8.2: u1 = 1/2 + y, u2 = 1 + 5x
        g = _grids(w)
        return np.stack([0.5 + g[1], 1.0 + 5.0 * g[0]])
    if w.ic == "brusselator_3d":      # Section 8.2 3D: u1 = 1 + sin 2pi x sin 2pi y sin 2pi z, u2 = 3
        g = _grids(w)
        u1 = 1.0 + np.sin(2 * math.pi * g[0]) * np.sin(2 * math.pi * g[1]) * np.sin(2 * math.pi * g[2])
        return np.stack([u1, np.full_like(u1, 3.0)])
    if w.ic == "gray_scott":          # u = 1, v = 0, a seeded perturbed block, plus noise
        (noise,) = w.ic_args
        U = np.empty(shape)
        U[0] = 1.0
        U[1] = 0.0
        sl = tuple(slice(int(0.4 * m), max(int(0.4 * m) + 1, int(0.6 * m))) for m in shape[1:])
        U[0][sl] = 0.5
        U[1][sl] = 0.25
        U += noise * rng.standard_normal(shape)
        return U
    if w.ic == "cgl_pulses":          # Section 8 (CGL): Gaussian pulses (real part), imaginary part 0
        g = _grids(w)
        if w.dim == 2:
            centres, signs = ((50, 50), (100, 100), (100, 50)), (1.0, -1.0, 1.0)
        else:
            centres, signs = ((50, 50, 50), (100, 100, 100)), (1.0, -1.0)
        re = np.zeros(shape[1:])
        for c, sg in zip(centres, signs):
            re += sg * np.exp(-sum((g[a] - c[a]) ** 2 for a in range(w.dim)) / 1000.0)
        return np.stack([re, np.zeros_like(re)])
    if w.ic == "nls_exact":           # Section 8 (Schrodinger 2D): Psi(0) = cos(pi x) cos(pi y), real
        return exact_nls(w, 0.0)
    raise ValueError(f"unknown initial-state recipe {w.ic!r}")


def exact_nls(w: Workload, t: float) -> np.ndarray:
    """Section 8's exact Schrodinger solution e^{-it} prod_a cos(pi x_a), as (Re, Im)."""
    g = _grids(w)
    c = np.ones(g[0].shape)
    for a in range(w.dim):
        c = c * np.cos(math.pi * g[a] / w.length[a])
    return np.stack([math.cos(t) * c, -math.sin(t) * c])


def exact_mms(w: Workload, t: float) -> np.ndarray:
    """Exact solution e^{-t} prod_a sin(pi x_a / L_a) of the manufactured problem."""
    return math.exp(-t) * initial_state(w.with_(ic="sine"))


# ---------------------------------------------------------------- problems --

def brusselator_2d(p: int = 64, steps: int = 100, k: float = 0.01) -> Workload:
    """2D Brusselator, 2 species, Neumann, eps = 2e-3, a = 1, b = 3.4, FP64 case."""
    a, b = 1.0, 3.4
    return Workload("brusselator2d", (p, p), NEUMANN, (2e-3, 2e-3), "brusselator", (a, b), k, steps,
                    ic="normal", ic_args=((a, b / a), 0.1))


def mms_3d(p: int = 256) -> Workload:
    """3D scalar Dirichlet problem u_t = d Lap u - u/(1+u) + f(x,t), d = 1, with f manufactured
    so that u = e^{-t} sin(pi x) sin(pi y) sin(pi z); k = h = 1/(p+1), T = 1."""
    h = 1.0 / (p + 1)
    return Workload(f"mms3d_{p}", (p, p, p), DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), h, p + 1, ic="sine")


def schnakenberg_2d(p: int = 4096, steps: int = 1000) -> Workload:
    """2D Schnakenberg on the periodic unit square, a = 0.1, b = 0.9, gamma = 1000, D = (1, 10),
    k = 1e-4; steady state (a+b, b/(a+b)^2) = (1, 0.9) plus U(-1e-3, 1e-3) noise."""
    return Workload(f"schnakenberg2d_{p}", (p, p), PERIODIC, (1.0, 10.0), "schnakenberg", (0.1, 0.9, 1000.0),
                    1e-4, steps, ic="uniform", ic_args=((1.0, 0.9), 1e-3))


def gray_scott_3d(p: int = 256, steps: int = 200, seed: int = 2001) -> Workload:
    """3D Gray-Scott on the periodic unit cube, Du = 2e-5, Dv = 1e-5, F = 0.04, kappa = 0.06, k = 1."""
    return Workload(f"grayscott3d_{p}", (p, p, p), PERIODIC, (2e-5, 1e-5), "gray_scott", (0.04, 0.06),
                    1.0, steps, ic="gray_scott", ic_args=(1e-2,), seed=seed)


def ensemble(ninst: int = 512, steps: int = 500, seed: int = 2001,
             sizes=(64, 96, 128, 192, 256, 384, 512)) -> list:
    """Batched ensemble of independent 2D Brusselator instances with seeded sizes,
    a ~ U[0.5, 2], b ~ U[1.5, 4], eps ~ U[1e-4, 1e-2] (both species), boundary
    Neumann or periodic (same on both axes), k = 0.01."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(ninst):
        p = int(rng.choice(sizes))
        a = float(rng.uniform(0.5, 2.0))
        b = float(rng.uniform(1.5, 4.0))
        eps = float(rng.uniform(1e-4, 1e-2))
        bc = NEUMANN if rng.integers(0, 2) == 0 else PERIODIC
        out.append(Workload(f"ens{i}", (p, p), bc, (eps, eps), "brusselator", (a, b), 0.01, steps,
                            ic="normal", ic_args=((a, b / a), 0.1), seed=seed * 100003 + i))
    return out


def enzyme_paper(p: int = 79, k: float = 0.05) -> Workload:
    """Section 8.1: u_t = D Lap u - u/(1+u), D = 0.2, unit square, Dirichlet 0, u(x,0) = 1, T = 1."""
    return Workload("enzyme_paper", (p, p), DIRICHLET, (0.2,), "enzyme", (0.0, 0.0), k,
                    int(round(1.0 / k)), ic="constant", ic_args=((1.0,),))


def _cgl_coupling(alpha: float):
    """D = 1 + i alpha as the 2 x 2 matrix on (Re u, Im u); None for alpha = 0 (real diffusion)."""
    return None if alpha == 0.0 else (1.0, -alpha, alpha, 1.0)


def cgl_2d(p: int = 400, steps: int = 2000, ic: str = "cgl_pulses", beta: float = 1.3, seed: int = 2001,
           alpha: float = 0.0) -> Workload:
    """Section 8: complex Ginzburg-Landau u_t = u + (1 + i alpha) Lap u - (1 + i beta) u |u|^2,
    beta = 1.3, periodic [0, 200]^2, p = 400 (h = 1/2), k = 1/20, T = 100 (2000 steps); Gaussian
    pulses, or ic="normal": N(0, 1) field.  alpha = 0 (the paper's runs) is real diffusion (D = 1 on
    Re u and Im u); alpha != 0 couples them (complex line solves)."""
    ic_args = ((0.0, 0.0), 1.0) if ic == "normal" else ()
    name = f"cgl2d_{p}" if alpha == 0.0 else f"cgl2d_{p}_alpha{alpha:g}"
    return Workload(name, (p, p), PERIODIC, (1.0, 1.0), "cgl", (beta,), 0.05, steps,
                    length=(200.0, 200.0), ic=ic, ic_args=ic_args, seed=seed, Dc=_cgl_coupling(alpha))


def cgl_3d(p: int = 200, steps: int = 2000, beta: float = 1.3, alpha: float = 0.0) -> Workload:
    """Section 8: the same equation on periodic [0, 200]^3, p = 200 (h = 1), k = 1/20, T = 100,
    Gaussian pulses."""
    name = f"cgl3d_{p}" if alpha == 0.0 else f"cgl3d_{p}_alpha{alpha:g}"
    return Workload(name, (p, p, p), PERIODIC, (1.0, 1.0), "cgl", (beta,), 0.05, steps,
                    length=(200.0, 200.0, 200.0), ic="cgl_pulses", Dc=_cgl_coupling(alpha))


def nls_2d(p: int = 79, k: float = 0.0125, T: float = 1.0) -> Workload:
    """Section 8's 2D cubic Schrodinger example: i Psi_t + Lap Psi = q Psi on the unit square,
    Neumann, q = B + C |Psi|^2, B = (1 - 2 pi^2)(1 - cos^2(pi x) cos^2(pi y)), C = 1 - 2 pi^2,
    exact solution e^{-it} cos(pi x) cos(pi y); h = 1/78 (p = 79 nodes), k = 0.0125, T = 1.
    As u_t = Dm Lap u + F: Dm = [[0, -1], [1, 0]] (the complex i), F = q (w, -v)."""
    c = 1.0 - 2.0 * math.pi ** 2
    return Workload(f"nls2d_{p}", (p, p), NEUMANN, (1.0, 1.0), "nls", (0.0, c, c), k, int(round(T / k)),
                    ic="nls_exact", Dc=(0.0, -1.0, 1.0, 0.0))


def brusselator_paper(p: int = 81, k: float = 0.1) -> Workload:
    """Section 8.2 (Table brutable): D = 2e-3, A = 3.4, B = 1 (config form a = B, b = A), Neumann,
    u1 = 1/2 + y, u2 = 1 + 5x, T = 2."""
    return Workload("brusselator_paper", (p, p), NEUMANN, (2e-3, 2e-3), "brusselator", (1.0, 3.4), k,
                    int(round(2.0 / k)), ic="brusselator_paper")
