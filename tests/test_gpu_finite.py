"""Non-finite detection (etd_check_finite): a device scan of a state that
returns ETD_ERR_NONFINITE with the smallest offending element index."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_11220_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(w, prec):
    from paper_2001_11220_gb300.api import EtdRdpIf
    return EtdRdpIf.from_workload(w, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_planted_nan_and_inf_report_the_first_index(prec):
    from paper_2001_11220_gb300 import _binding as B
    import ctypes
    w = W.brusselator_2d(p=128, steps=1)   # 2 x 16384 elements
    ctx = _ctx(w, prec)
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=ctx.dtype)
    assert ctx.check_finite(U) == -1
    flat = U.view(-1)
    flat[20000] = float("inf")
    flat[12345] = float("nan")
    flat[9000 + U[0].numel()] = -float("inf")   # species 1, point 9000
    first = ctypes.c_int64(0)
    st = ctx.lib.etd_check_finite(ctx.ctx, ctypes.c_void_p(U.data_ptr()), ctypes.byref(first))
    assert st == B.ETD_ERR_NONFINITE and first.value == 12345
    assert b"12345" in ctx.lib.etd_last_error(ctx.ctx)
    assert ctx.check_finite(U) == 12345
    flat[12345] = 1.0
    assert ctx.check_finite(U) == 20000
    flat[20000] = 1.0
    assert ctx.check_finite(U) == 9000 + U[0].numel()
    ctx.close()


def test_diverging_run_is_detected():
    """F = 1e4 u with k = 1: the explicit reaction terms multiply the state by ~1e4
    per step, so FP32 overflows within a dozen steps; the scan reports it, and a
    stable run of the same grid stays finite."""
    w = W.Workload("blowup", (64, 48), W.NEUMANN, (0.01, 0.01), "linear", (1.0e4, 0.0), 1.0, 20,
                   ic="normal", ic_args=((1.0, 1.0), 0.1))
    ctx = _ctx(w, "fp32")
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float32)
    ctx.run(U, 0.0, 20)
    torch.cuda.synchronize()
    assert ctx.check_finite(U) >= 0
    ctx.close()
    ws = w.with_(params=(-1.0, 0.0), k=0.01)
    ctx = _ctx(ws, "fp32")
    U = torch.tensor(W.initial_state(ws), device="cuda", dtype=torch.float32)
    ctx.run(U, 0.0, 20)
    torch.cuda.synchronize()
    assert ctx.check_finite(U) == -1
    ctx.close()


def test_coupled_context_scan():
    w = W.nls_2d(p=33)
    ctx = _ctx(w, "fp64")
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float64)
    ctx.run(U, 0.0, 3)
    assert ctx.check_finite(U) == -1
    U.view(-1)[-1] = float("nan")
    assert ctx.check_finite(U) == U.numel() - 1
    ctx.close()
