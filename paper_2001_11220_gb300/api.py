"""Torch-facing wrapper of the C ABI: device memory and streams come from
PyTorch, every step of the scheme runs in libetdrdpif's kernels.

    ctx = EtdRdpIf.from_workload(workload, precision="fp32")
    U = torch.tensor(initial_state, device="cuda", dtype=ctx.dtype)
    ctx.run(U, t0=0.0, nsteps=100)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B
from .workloads import REACTIONS, Workload


def _stream_handle(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_grid(n, bc, length=None) -> B.etd_grid:
    g = B.etd_grid()
    g.dim = len(n)
    bc = (bc,) * len(n) if isinstance(bc, int) else tuple(bc)
    length = length or (1.0,) * len(n)
    for a in range(3):
        g.n[a] = int(n[a]) if a < len(n) else 1
        g.bc[a] = int(bc[a]) if a < len(n) else 0
        g.length[a] = float(length[a]) if a < len(n) else 1.0
    return g


def make_reaction(kind, nspecies, params=()) -> B.etd_reaction:
    r = B.etd_reaction()
    r.kind = REACTIONS[kind] if isinstance(kind, str) else int(kind)
    r.nspecies = int(nspecies)
    for j in range(8):
        r.params[j] = float(params[j]) if j < len(params) else 0.0
    return r


class EtdRdpIf:
    """One ETD-RDP-IF problem on the current CUDA device."""

    def __init__(self, n, bc, D, reaction="zero", params=(), k=0.01, precision="fp64", length=None, stream=None,
                 Dc=None):
        """Dc (optional): the 2 x 2 diffusion matrix (row-major) of a coupled
        two-species problem, etd_create_coupled; D then only fixes the species
        count (two)."""
        self.lib = B.load()
        self.n = tuple(int(v) for v in n)
        self.D = tuple(float(d) for d in D)
        self.Dc = None if Dc is None else tuple(float(v) for v in Dc)
        self.k = float(k)
        self.precision = B.ETD_FP64 if precision in ("fp64", B.ETD_FP64) else B.ETD_FP32
        self.dtype = torch.float64 if self.precision == B.ETD_FP64 else torch.float32
        self.shape = (len(self.D),) + tuple(reversed(self.n))
        grid = make_grid(self.n, bc, length)
        rx = make_reaction(reaction, len(self.D), params)
        ctx = ctypes.c_void_p()
        if self.Dc is not None:
            Dm = (ctypes.c_double * 4)(*self.Dc)
            st = self.lib.etd_create_coupled(ctypes.byref(grid), Dm, ctypes.byref(rx), self.k, self.precision,
                                             _stream_handle(stream), ctypes.byref(ctx))
        else:
            Darr = (ctypes.c_double * len(self.D))(*self.D)
            st = self.lib.etd_create(ctypes.byref(grid), Darr, ctypes.byref(rx), self.k, self.precision,
                                     _stream_handle(stream), ctypes.byref(ctx))
        B.check(st, None)
        self.ctx = ctx

    @classmethod
    def from_workload(cls, w: Workload, precision="fp64", stream=None) -> "EtdRdpIf":
        return cls(w.n, w.bc, w.D, w.reaction, w.params, w.k, precision, w.length, stream, w.Dc)

    def _check_state(self, U: torch.Tensor):
        if not (U.is_cuda and U.dtype == self.dtype and U.is_contiguous() and tuple(U.shape) == self.shape):
            raise ValueError(f"state must be a contiguous CUDA {self.dtype} tensor of shape {self.shape}")

    def set_stream(self, stream=None):
        B.check(self.lib.etd_set_stream(self.ctx, _stream_handle(stream)), self.ctx)

    def step(self, U: torch.Tensor, t: float):
        self._check_state(U)
        B.check(self.lib.etd_step(self.ctx, ctypes.c_void_p(U.data_ptr()), float(t)), self.ctx)
        return U

    def run(self, U: torch.Tensor, t0: float, nsteps: int):
        self._check_state(U)
        B.check(self.lib.etd_run(self.ctx, ctypes.c_void_p(U.data_ptr()), float(t0), int(nsteps)), self.ctx)
        return U

    def run_host(self, U: torch.Tensor, t0: float, nsteps: int):
        """U: contiguous CPU tensor (pinned for speed); copies in/out inside the call."""
        if U.is_cuda or U.dtype != self.dtype or not U.is_contiguous() or tuple(U.shape) != self.shape:
            raise ValueError("run_host needs a contiguous CPU tensor of the state's dtype and shape")
        B.check(self.lib.etd_run_host(self.ctx, ctypes.c_void_p(U.data_ptr()), float(t0), int(nsteps)), self.ctx)
        return U

    def step_adjoint(self, Un: torch.Tensor, t: float, Ubar_next: torch.Tensor, Ubar_n: torch.Tensor = None):
        self._check_state(Un)
        self._check_state(Ubar_next)
        if Ubar_n is None:
            Ubar_n = torch.empty_like(Un)
        dD = (ctypes.c_double * len(self.D))()
        dp = (ctypes.c_double * 8)()
        B.check(self.lib.etd_step_adjoint(self.ctx, ctypes.c_void_p(Un.data_ptr()), float(t),
                                          ctypes.c_void_p(Ubar_next.data_ptr()), ctypes.c_void_p(Ubar_n.data_ptr()),
                                          dD, dp), self.ctx)
        return Ubar_n, np.array(dD[:]), np.array(dp[:])

    def grad(self, U0: torch.Tensor, t0: float, target: torch.Tensor, nsteps: int, ckpt_every: int = 20):
        self._check_state(U0)
        self._check_state(target)
        dU0 = torch.empty_like(U0)
        loss = ctypes.c_double()
        dD = (ctypes.c_double * len(self.D))()
        dp = (ctypes.c_double * 8)()
        B.check(self.lib.etd_grad(self.ctx, ctypes.c_void_p(U0.data_ptr()), float(t0),
                                  ctypes.c_void_p(target.data_ptr()), int(nsteps), int(ckpt_every),
                                  ctypes.byref(loss), ctypes.c_void_p(dU0.data_ptr()), dD, dp), self.ctx)
        return loss.value, dU0, np.array(dD[:]), np.array(dp[:])

    def run_vjp(self, U0: torch.Tensor, t0: float, nsteps: int, Ubar_N: torch.Tensor, ckpt_every: int = 20):
        """(dU0, dD, dparams) for the cotangent Ubar_N of the state after nsteps steps."""
        self._check_state(U0)
        self._check_state(Ubar_N)
        dU0 = torch.empty_like(U0)
        dD = (ctypes.c_double * len(self.D))()
        dp = (ctypes.c_double * 8)()
        B.check(self.lib.etd_run_vjp(self.ctx, ctypes.c_void_p(U0.data_ptr()), float(t0), int(nsteps),
                                     int(ckpt_every), ctypes.c_void_p(Ubar_N.data_ptr()),
                                     ctypes.c_void_p(dU0.data_ptr()), dD, dp), self.ctx)
        return dU0, np.array(dD[:]), np.array(dp[:])

    def autotune(self, U_work: torch.Tensor):
        self._check_state(U_work)
        B.check(self.lib.etd_autotune(self.ctx, ctypes.c_void_p(U_work.data_ptr())), self.ctx)

    def profile(self, enable: bool):
        B.check(self.lib.etd_profile(self.ctx, int(bool(enable))), self.ctx)

    def profile_read(self):
        """(ms[3], launches[3]) per sweep kind since the last read (synchronises)."""
        ms = (ctypes.c_double * 3)()
        ln = (ctypes.c_int64 * 3)()
        B.check(self.lib.etd_profile_read(self.ctx, ms, ln), self.ctx)
        return list(ms), list(ln)

    def check_finite(self, U: torch.Tensor) -> int:
        """-1 if every element of U is finite, else the smallest flat index of a
        NaN / infinity (etd_check_finite returns ETD_ERR_NONFINITE there)."""
        self._check_state(U)
        first = ctypes.c_int64(-1)
        st = self.lib.etd_check_finite(self.ctx, ctypes.c_void_p(U.data_ptr()), ctypes.byref(first))
        if st not in (B.ETD_OK, B.ETD_ERR_NONFINITE):
            B.check(st, self.ctx)
        return int(first.value)

    def info(self) -> dict:
        inf = B.etd_info()
        B.check(self.lib.etd_get_info(self.ctx, ctypes.byref(inf)), self.ctx)
        return {f: (list(getattr(inf, f)) if f in ("chunk", "lines_per_block", "staged", "pack", "grid_blocks") else getattr(inf, f))
                for f, _ in inf._fields_}

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.etd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EtdEnsemble:
    """Many independent problems (same dimension, species count, precision and
    time step; any grid size, boundaries, coefficients and reaction parameters)
    advanced together: one persistent kernel launch per time step covers every
    sweep of every instance (work queue, per-instance completion counters,
    bounded waits; a wait that runs out raises EtdError ETD_ERR_TIMEOUT)."""

    def __init__(self, workloads, precision="fp32", stream=None):
        self.lib = B.load()
        ws = list(workloads)
        if not ws:
            raise ValueError("empty ensemble")
        self.k = float(ws[0].k)
        if any(abs(w.k - self.k) > 0 for w in ws):
            raise ValueError("every instance needs the same time step k")
        self.S = ws[0].nspecies
        self.precision = B.ETD_FP64 if precision in ("fp64", B.ETD_FP64) else B.ETD_FP32
        self.dtype = torch.float64 if self.precision == B.ETD_FP64 else torch.float32
        self.shapes = [w.shape for w in ws]
        n = len(ws)
        grids = (B.etd_grid * n)(*[make_grid(w.n, w.bc, w.length) for w in ws])
        rx = (B.etd_reaction * n)(*[make_reaction(w.reaction, w.nspecies, w.params) for w in ws])
        D = (ctypes.c_double * (n * self.S))(*[d for w in ws for d in w.D])
        ctx = ctypes.c_void_p()
        B.check(self.lib.etd_batch_create(n, grids, D, rx, self.k, self.precision, _stream_handle(stream),
                                          ctypes.byref(ctx)), None)
        self.ctx = ctx
        self.n = n

    def _check_states(self, states):
        if len(states) != self.n:
            raise ValueError(f"expected {self.n} states")
        for U, shp in zip(states, self.shapes):
            if not (U.is_cuda and U.dtype == self.dtype and U.is_contiguous() and tuple(U.shape) == shp):
                raise ValueError("every state must be a contiguous CUDA tensor of its instance's shape and dtype")

    def run(self, states, t0: float, nsteps: int):
        self._check_states(states)
        ptrs = (ctypes.c_void_p * self.n)(*[U.data_ptr() for U in states])
        B.check(self.lib.etd_batch_run(self.ctx, ptrs, float(t0), int(nsteps)), self.ctx)
        return states

    def set_wait_limit(self, seconds: float):
        """Limit of each dependency wait inside the step kernel (default 1 s)."""
        B.check(self.lib.etd_batch_set_wait_limit(self.ctx, float(seconds)), self.ctx)

    def debug_hold(self, instance: int, axis: int = 0):
        """Test hook: the next run's wait on sweep `axis` of `instance` never
        releases, so that run raises ETD_ERR_TIMEOUT."""
        B.check(self.lib.etd_batch_debug_hold(self.ctx, int(instance), int(axis)), self.ctx)

    def autotune(self, work_states):
        """Pick the line-block shapes by timing candidates; work_states are scratch
        device states of the instances' shapes (overwritten)."""
        self._check_states(work_states)
        ptrs = (ctypes.c_void_p * self.n)(*[U.data_ptr() for U in work_states])
        B.check(self.lib.etd_batch_autotune(self.ctx, ptrs), self.ctx)

    def info(self) -> dict:
        inf = B.etd_info()
        B.check(self.lib.etd_get_info(self.ctx, ctypes.byref(inf)), self.ctx)
        return {f: (list(getattr(inf, f)) if f in ("chunk", "lines_per_block", "staged", "pack", "grid_blocks") else getattr(inf, f))
                for f, _ in inf._fields_}

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.etd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
