"""FP64 CPU oracle for the ETD-RDP-IF scheme (arXiv 2001.11220).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2001_11220_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``etd_oracle.c`` (plain C, one line at a time, no
blocking or fusion); this module only builds it with gcc and marshals numpy
arrays through ctypes.  See ``etd_oracle.h`` for what each function follows in
the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "etd_oracle.c")]
_HDR = os.path.join(_HERE, "etd_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

DIRICHLET, NEUMANN, PERIODIC = 0, 1, 2
ZERO, LINEAR, BRUSSELATOR, SCHNAKENBERG, GRAY_SCOTT, ENZYME, CGL, NLS = range(8)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, no -march).

    Built with OpenMP where gcc has it (independent lines and points are
    shared among host threads; each is computed exactly as in the serial
    loop), else serially.
    """
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp] + _SRC
    if subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
        subprocess.run(base + ["-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("length", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3),
        ("nspecies", ctypes.c_int),
        ("D", ctypes.c_double * 4),
        ("reaction", ctypes.c_int),
        ("params", ctypes.c_double * 8),
        ("k", ctypes.c_double),
        ("coupled", ctypes.c_int),
        ("Dc", ctypes.c_double * 4),
    ]


@dataclass
class Problem:
    """A reaction-diffusion problem on a d-dimensional box (Section 2).

    n[a] counts grid nodes on axis a in the paper's convention (Section 3,
    Example 1); axis 0 is x, the fastest index of the state U[s][z][y][x].
    Dc (optional, 2 species): the full 2 x 2 diffusion matrix, row-major, of
    the coupled systems of Section 8; D then only sets the species count.
    """

    n: tuple
    bc: tuple
    D: tuple
    reaction: int = ZERO
    params: tuple = ()
    k: float = 0.01
    length: tuple = None
    Dc: tuple = None
    dim: int = field(init=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.dim = len(self.n)
        if isinstance(self.bc, int):
            self.bc = (self.bc,) * self.dim
        self.bc = tuple(int(b) for b in self.bc)
        self.D = tuple(float(d) for d in self.D)
        if self.length is None:
            self.length = (1.0,) * self.dim
        self.length = tuple(float(v) for v in self.length)

    @property
    def nspecies(self) -> int:
        return len(self.D)

    @property
    def shape(self) -> tuple:
        """numpy shape of the state: (s, [z,] y, x)."""
        return (self.nspecies,) + tuple(reversed(self.n))

    def as_c(self) -> _Problem:
        c = _Problem()
        c.dim = self.dim
        for a in range(3):
            c.n[a] = self.n[a] if a < self.dim else 1
            c.length[a] = self.length[a] if a < self.dim else 1.0
            c.bc[a] = self.bc[a] if a < self.dim else 0
        c.nspecies = self.nspecies
        for s in range(4):
            c.D[s] = self.D[s] if s < self.nspecies else 0.0
        c.reaction = int(self.reaction)
        for j in range(8):
            c.params[j] = float(self.params[j]) if j < len(self.params) else 0.0
        c.k = float(self.k)
        c.coupled = 1 if self.Dc is not None else 0
        for j in range(4):
            c.Dc[j] = float(self.Dc[j]) if self.Dc is not None else 0.0
        return c

    def h(self, axis: int) -> float:
        p, L = self.n[axis], self.length[axis]
        return {DIRICHLET: L / (p + 1), NEUMANN: L / (p - 1), PERIODIC: L / p}[self.bc[axis]]

    def coords(self, axis: int) -> np.ndarray:
        h = self.h(axis)
        i = np.arange(self.n[axis], dtype=np.float64)
        return (i + 1) * h if self.bc[axis] == DIRICHLET else i * h


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        sig = {
            "oracle_line_solve": [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp],
            "oracle_axis_solve": [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp],
            "oracle_axis_apply": [P, ctypes.c_int, _dp, _dp],
            "oracle_reaction": [P, _dp, ctypes.c_double, _dp],
            "oracle_reaction_vjp": [P, _dp, ctypes.c_double, _dp, _dp, _dp],
            "oracle_step": [P, _dp, ctypes.c_double],
            "oracle_run": [P, _dp, ctypes.c_double, ctypes.c_long],
            "oracle_step_adjoint": [P, _dp, ctypes.c_double, _dp, _dp, _dp, _dp],
            "oracle_grad": [P, _dp, ctypes.c_double, _dp, ctypes.c_long, _dp, _dp, _dp, _dp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Host threads for the oracle's line and point loops; returns the count
    now in use (1 for a serial build)."""
    lib = _load()
    lib.oracle_set_threads(int(n))
    return lib.oracle_get_threads()


def get_threads() -> int:
    return _load().oracle_get_threads()


def _arr(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _check(rc: int, name: str):
    if rc != 0:
        raise ValueError(f"{name} rejected its arguments (rc={rc})")


def line_solve(bc: int, r: float, b, transpose: bool = False) -> np.ndarray:
    """Solve (I + r h^2 B_p) x = b for one line (Section 7 Thomas / Sherman-Morrison)."""
    b = _arr(b).copy()
    x = np.empty_like(b)
    _check(_load().oracle_line_solve(len(b), bc, r, int(transpose), _ptr(b), _ptr(x)), "line_solve")
    return x


def axis_solve(P: Problem, axis: int, gamma: float, U, transpose: bool = False) -> np.ndarray:
    """(I + (k/gamma) A_axis)^{-1} U over every line of the axis (Eq. Ai)."""
    c = P.as_c()
    src = _arr(U, P.shape).copy()
    out = np.empty_like(src)
    _check(_load().oracle_axis_solve(ctypes.byref(c), axis, gamma, int(transpose), _ptr(src), _ptr(out)), "axis_solve")
    return out


def axis_apply(P: Problem, axis: int, U) -> np.ndarray:
    c = P.as_c()
    src = _arr(U, P.shape).copy()
    out = np.empty_like(src)
    _check(_load().oracle_axis_apply(ctypes.byref(c), axis, _ptr(src), _ptr(out)), "axis_apply")
    return out


def reaction(P: Problem, U, t: float) -> np.ndarray:
    c = P.as_c()
    src = _arr(U, P.shape).copy()
    out = np.empty_like(src)
    _check(_load().oracle_reaction(ctypes.byref(c), _ptr(src), t, _ptr(out)), "reaction")
    return out


def reaction_vjp(P: Problem, U, t: float, ybar):
    c = P.as_c()
    src = _arr(U, P.shape).copy()
    yb = _arr(ybar, P.shape).copy()
    out = np.empty_like(src)
    pbar = np.zeros(8)
    _check(_load().oracle_reaction_vjp(ctypes.byref(c), _ptr(src), t, _ptr(yb), _ptr(out), _ptr(pbar)), "reaction_vjp")
    return out, pbar


def step(P: Problem, U, t: float) -> np.ndarray:
    """One ETD-RDP-IF step (framed scheme of Section 6); returns U_{n+1}."""
    c = P.as_c()
    u = _arr(U, P.shape).copy()
    _check(_load().oracle_step(ctypes.byref(c), _ptr(u), t), "step")
    return u


def run(P: Problem, U, t0: float, nsteps: int) -> np.ndarray:
    c = P.as_c()
    u = _arr(U, P.shape).copy()
    _check(_load().oracle_run(ctypes.byref(c), _ptr(u), t0, int(nsteps)), "run")
    return u


def step_adjoint(P: Problem, Un, t: float, Ubar_next):
    """Reverse mode of one step: (Ubar_n, dD[:s], dparams[8]); coupled problems
    return dD as the 4 entries d/dDc[s][t], row-major."""
    c = P.as_c()
    u = _arr(Un, P.shape).copy()
    ub = _arr(Ubar_next, P.shape).copy()
    out = np.empty_like(u)
    dD = np.zeros(4)
    dp = np.zeros(8)
    _check(_load().oracle_step_adjoint(ctypes.byref(c), _ptr(u), t, _ptr(ub), _ptr(out), _ptr(dD), _ptr(dp)), "step_adjoint")
    return out, (dD if P.Dc is not None else dD[: P.nspecies]), dp


def grad(P: Problem, U0, t0: float, target, nsteps: int):
    """loss = 1/2 |U_N - target|^2 and its gradients (dU0, dD[:s], dparams[8])."""
    c = P.as_c()
    u = _arr(U0, P.shape).copy()
    tg = _arr(target, P.shape).copy()
    dU0 = np.empty_like(u)
    loss = np.zeros(1)
    dD = np.zeros(4)
    dp = np.zeros(8)
    _check(_load().oracle_grad(ctypes.byref(c), _ptr(u), t0, _ptr(tg), int(nsteps), _ptr(loss), _ptr(dU0), _ptr(dD), _ptr(dp)), "grad")
    return float(loss[0]), dU0, (dD if P.Dc is not None else dD[: P.nspecies]), dp
