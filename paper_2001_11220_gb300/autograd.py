"""Differentiable ETD-RDP-IF runs for PyTorch.

``simulate(U0, D, params, ...)`` advances a state nsteps steps with the CUDA
library and returns U_N; gradients of any scalar function of U_N flow back to
U0 (device tensor), D and params (1-D float64 CPU tensors) through the
library's hand-written discrete adjoint (etd_run_vjp: checkpointed forward
pass, segment recomputation, transposed line solves).  No PyTorch operation
takes part in the step itself.
"""
from __future__ import annotations

import torch

from .api import EtdRdpIf

_SOLVERS = {}


def _solver(n, bc, reaction, k, D, params, precision, length):
    key = (tuple(n), bc if isinstance(bc, int) else tuple(bc), reaction, float(k), tuple(D), tuple(params),
           precision, None if length is None else tuple(length))
    s = _SOLVERS.get(key)
    if s is None:
        if len(_SOLVERS) > 16:
            _SOLVERS.clear()
        s = EtdRdpIf(n, bc, D, reaction, params, k, precision, length)
        _SOLVERS[key] = s
    return s


class EtdRun(torch.autograd.Function):
    """U_N = run(U0; D, params); backward = etd_run_vjp."""

    @staticmethod
    def forward(ctx, U0, D, params, solver, t0, nsteps, ckpt_every):
        U = U0.detach().clone()
        solver.run(U, t0, nsteps)
        ctx.save_for_backward(U0)
        ctx.solver, ctx.t0, ctx.nsteps, ctx.ckpt = solver, t0, nsteps, ckpt_every
        ctx.npar = params.numel()
        return U

    @staticmethod
    def backward(ctx, gU):
        (U0,) = ctx.saved_tensors
        dU0, dD, dp = ctx.solver.run_vjp(U0.detach().contiguous(), ctx.t0, ctx.nsteps,
                                         gU.detach().to(U0.dtype).contiguous(), ctx.ckpt)
        return (dU0, torch.tensor(dD, dtype=torch.float64), torch.tensor(dp[: ctx.npar], dtype=torch.float64),
                None, None, None, None)


def simulate(U0: torch.Tensor, D: torch.Tensor, params: torch.Tensor, *, n, bc, reaction: str, k: float,
             nsteps: int, t0: float = 0.0, ckpt_every: int = 20, length=None) -> torch.Tensor:
    """Differentiable run of nsteps ETD-RDP-IF steps.

    U0: contiguous CUDA tensor (s, [z,] y, x), float64 or float32 (sets the
    precision).  D: (s,) float64 CPU tensor.  params: reaction parameters,
    float64 CPU tensor.  Returns U_N (same dtype/device as U0).
    """
    precision = "fp64" if U0.dtype == torch.float64 else "fp32"
    solver = _solver(n, bc, reaction, k, D.detach().tolist(), params.detach().tolist(), precision, length)
    return EtdRun.apply(U0, D, params, solver, float(t0), int(nsteps), int(ckpt_every))
