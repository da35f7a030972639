"""etd_step_noalloc: the allocation-free step for callers that cannot call
cudaMalloc (hosts that own every device allocation, real-time loops that may
not touch the allocator).  Its scratch is a static device array; two calls in
a row must give the same states as the regular etd_create/etd_step path,
within the parity tolerances of the other GPU tests.

This file is collected last on purpose (pytest orders files by name).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_11220_gb300 import _binding as B  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.tolerances import fp32_step_bound  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _noalloc_step(w, U, t, precision, stream):
    from paper_2001_11220_gb300.api import make_grid, make_reaction
    lib = B.load()
    g = make_grid(w.n, w.bc, w.length)
    r = make_reaction(w.reaction, w.nspecies, w.params)
    D = (ctypes.c_double * w.nspecies)(*w.D)
    st = lib.etd_step_noalloc(ctypes.byref(g), D, ctypes.byref(r), w.k, precision,
                              ctypes.c_void_p(U.data_ptr()), t, ctypes.c_void_p(stream.cuda_stream))
    B.check(st, None)


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return max(float(np.abs(a[s] - b[s]).max() / np.abs(b[s]).max()) for s in range(b.shape[0]))


@pytest.mark.parametrize("w,prec", [
    (W.brusselator_2d(p=48, steps=2), "fp64"),
    (W.mms_3d(24), "fp32"),
    (W.Workload("gs2d_per", (40, 36), W.PERIODIC, (0.02, 0.01), "gray_scott", (0.04, 0.06), 0.5, 2,
                ic="normal", ic_args=((0.8, 0.2), 0.05)), "fp64"),
], ids=["bru2d_fp64", "mms3d_fp32", "gs2d_per_fp64"])
def test_noalloc_matches_regular_step_twice(w, prec):
    from paper_2001_11220_gb300.api import EtdRdpIf
    precision = B.ETD_FP64 if prec == "fp64" else B.ETD_FP32
    tol = FP64_TOL if prec == "fp64" else fp32_step_bound(w)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = EtdRdpIf.from_workload(w, prec, stream=s)
        U0 = torch.tensor(W.initial_state(w), device="cuda", dtype=ctx.dtype)
        A = U0.clone()
        Bst = U0.clone()
    for n in range(2):                       # two calls in a row
        t = n * w.k
        ctx.step(A, t)
        _noalloc_step(w, Bst, t, precision, s)
        s.synchronize()
        err = _rel(Bst, A)
        assert err <= tol, (n, err)
        assert bool(torch.isfinite(Bst).all())
    ctx.close()


def test_noalloc_allocates_no_device_memory():
    """The entry point's promise: after a first call (which may load kernel
    modules), a further call leaves the device's free memory unchanged."""
    w = W.brusselator_2d(p=48, steps=2)
    s = torch.cuda.Stream()
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float64)
    _noalloc_step(w, U, 0.0, B.ETD_FP64, s)
    s.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _noalloc_step(w, U, w.k, B.ETD_FP64, s)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert bool(torch.isfinite(U).all())


def test_noalloc_rejects_too_long_axis():
    """Axes longer than one block of whole lines (n > 8192) need the segmented
    plans, whose device buffers this entry point does not have."""
    from paper_2001_11220_gb300.api import make_grid, make_reaction
    lib = B.load()
    g = make_grid((8200, 3), (0, 0))
    r = make_reaction("zero", 1)
    D = (ctypes.c_double * 1)(1.0)
    U = torch.zeros(8200 * 3, device="cuda", dtype=torch.float32)
    st = lib.etd_step_noalloc(ctypes.byref(g), D, ctypes.byref(r), 0.01, B.ETD_FP32,
                              ctypes.c_void_p(U.data_ptr()), 0.0, None)
    assert st == B.ETD_ERR_UNSUPPORTED
    assert b"does not fit one block" in lib.etd_last_error(None)


def test_noalloc_rejects_oversize_problem():
    from paper_2001_11220_gb300.api import make_grid, make_reaction
    lib = B.load()
    g = make_grid((1024, 1024, 32), (0, 0, 0))
    r = make_reaction("zero", 1)
    D = (ctypes.c_double * 1)(1.0)
    st = lib.etd_step_noalloc(ctypes.byref(g), D, ctypes.byref(r), 0.01, B.ETD_FP64,
                              ctypes.c_void_p(16), 0.0, None)
    assert st == B.ETD_ERR_INVALID_ARG
    assert b"static scratch" in lib.etd_last_error(None)
