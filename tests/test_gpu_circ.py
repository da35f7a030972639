"""Circulant sweeps of periodic axes (ETD_TILES kernel code 5) against the FP64
oracle.  The kernels solve every line matrix I + c B_p of a periodic axis
through its exact factorisation alpha (I - lambda E)(I - lambda E^-1) (two
cyclic first-order recurrences, chunk carries by lane scans) instead of the
Thomas tables of Section 7; the oracle keeps Thomas plus Sherman-Morrison, so
agreement pins the factorisation, the scans and the cyclic closures.

Cases cover one and several lines per warp (m = p / L chunks: 2 .. 32), lines
spanning several warps (m = 64 .. 512, a shared-memory step between the
warps), one and two species, 2D and 3D, and stiff lines (r = k D / h^2 up to
1.7e4, the 4096^2 benchmark's).  FP64: <= 1e-12 relative after 1 and 3 steps
(stiff lines: the condition bound eps (1 + 4 r) of the Sherman-Morrison test,
when larger); FP32: fp32_step_bound per step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.dense_reference import oracle_problem  # noqa: E402
from tests.tolerances import fp32_step_bound  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def case(name, n, bc, D, reaction, params=(), k=0.05, ic="normal", ic_args=None, length=None):
    S = len(D)
    if ic_args is None and ic == "normal":
        ic_args = ((0.8, 1.2)[:S], 0.1)
    return W.Workload(name, n, bc, D, reaction, params, k, 1, length=length, ic=ic, ic_args=ic_args or ())


def rel_err(a, ref):
    return max(float(np.max(np.abs(a[s] - ref[s])) / max(np.max(np.abs(ref[s])), 1e-300)) for s in range(ref.shape[0]))


CASES = [
    case("circ_x_tiny", (32, 9), (W.PERIODIC, W.NEUMANN), (0.3, 0.1), "gray_scott", (0.04, 0.06)),
    case("circ_x_256", (256, 20), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0)),
    case("circ_x_1024_gs", (1024, 8), (W.PERIODIC, W.DIRICHLET), (0.5, 2.0), "gray_scott", (0.04, 0.06), k=0.01),
    case("circ_x_512_lin", (512, 12), (W.PERIODIC, W.NEUMANN), (0.3,), "linear", (-0.7, 0.2), k=0.1),
    case("circ_x_4096_stiff", (4096, 6), W.PERIODIC, (1.0, 10.0), "schnakenberg", (0.1, 0.9, 1000.0), k=1e-4,
         ic="uniform", ic_args=((1.0, 0.9), 1e-3)),
    case("circ_3d_x", (128, 7, 6), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott", (0.04, 0.06),
         k=0.5),
    case("circ_x_bru", (64, 33), (W.PERIODIC, W.PERIODIC), (0.05, 0.02), "brusselator", (1.0, 3.4)),
]


def _tiles(w, L):
    return ",".join([f"{L}:0:5:1"] + ["0:0:0:1"] * (w.dim - 1))


def _fp64_bound(w):
    r = w.k * max(w.D) / w.h(0) ** 2
    return max(FP64_TOL, 2.0 ** -52 * (1 + 4 * r))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_circulant_first_sweep_vs_oracle(w, prec, monkeypatch):
    from paper_2001_11220_gb300.api import EtdRdpIf
    L = 8 if prec == "fp64" else 16
    monkeypatch.setenv("ETD_TILES", _tiles(w, L))
    ctx = EtdRdpIf.from_workload(w, prec)
    inf = ctx.info()
    assert inf["staged"][0] == 5 and inf["chunk"][0] == L, inf
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    P = oracle_problem(w)
    ref1 = oracle.run(P, U0, 0.3, 1)
    ref3 = oracle.run(P, U0, 0.3, 3)
    e1, e3 = rel_err(one, ref1), rel_err(three, ref3)
    print(f"{w.name} {prec} circulant: 1 step {e1:.3e}, 3 steps {e3:.3e}")
    if prec == "fp64":
        assert e1 <= _fp64_bound(w) and e3 <= _fp64_bound(w), (e1, e3, _fp64_bound(w))
    else:
        assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


def test_circulant_plan_rejects_unsupported_lines(monkeypatch):
    """Non-periodic axes and line lengths that are not L times a power of two
    fall back to the table kernels (the forced circulant plan is refused)."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    for w in (case("neu_x", (256, 8), W.NEUMANN, (0.1,), "linear", (-0.5, 0.0)),
              case("per_96", (96, 8), W.PERIODIC, (0.1,), "linear", (-0.5, 0.0))):
        monkeypatch.setenv("ETD_TILES", _tiles(w, 16))
        ctx = EtdRdpIf.from_workload(w, "fp32")
        assert ctx.info()["staged"][0] != 5
        ctx.close()


# Strided axes: 32 lines x wb chunks per block, a line split over p / (wb L)
# blocks of one thread-block cluster (1 .. 16)
STRIDED_CASES = [
    # (workload, per-axis kernel spec: "c" circulant on that axis, "-" default)
    (case("circ_y_256", (64, 256), (W.NEUMANN, W.PERIODIC), (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0)), "-c"),
    (case("circ_y_1024", (32, 1024), (W.DIRICHLET, W.PERIODIC), (0.5, 2.0), "gray_scott", (0.04, 0.06), k=0.01),
     "-c"),
    (case("circ_xy_512", (512, 512), W.PERIODIC, (0.05, 0.02), "brusselator", (1.0, 3.4)), "cc"),
    (case("circ_y_lin", (96, 512), (W.NEUMANN, W.PERIODIC), (0.3,), "linear", (-0.7, 0.2), k=0.1), "-c"),
    (case("circ_3d_mid", (32, 256, 5), (W.PERIODIC, W.PERIODIC, W.DIRICHLET), (0.02, 0.01), "gray_scott",
          (0.04, 0.06), k=0.5), "cc-"),
    (case("circ_3d_last", (32, 6, 512), (W.NEUMANN, W.DIRICHLET, W.PERIODIC), (0.02, 0.01), "gray_scott",
          (0.04, 0.06), k=0.5), "--c"),
    (case("circ_3d_all", (64, 128, 128), W.PERIODIC, (0.05, 0.02), "brusselator", (1.0, 3.4)), "ccc"),
    (case("circ_cgl_xy", (256, 512), W.PERIODIC, (1.0, 1.0), "cgl", (1.3,), ic_args=((0.0, 0.0), 1.0),
          length=(128.0, 256.0)), "cc"),
]


SHAPES = [("fp32", 16, 16), ("fp32", 16, 32), ("fp32", 8, 32), ("fp32", 32, 16), ("fp64", 8, 32),
          ("fp64", 16, 16)]


@pytest.mark.parametrize("prec,wb,nc", SHAPES, ids=[f"{p}-{a}x{b}" for p, a, b in SHAPES])
@pytest.mark.parametrize("w,spec", STRIDED_CASES, ids=[c[0].name for c in STRIDED_CASES])
def test_circulant_strided_sweeps_vs_oracle(w, spec, prec, wb, nc, monkeypatch):
    """(wb chunks, nc lines) per block; lines longer than wb L run as clusters."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    L = 8 if prec == "fp64" else 16
    for a, ch in enumerate(spec):
        st = int(np.prod(w.n[:a]))
        if ch == "c" and a > 0 and (w.n[a] % (wb * L) or w.n[a] // (wb * L) > 16 or st % nc):
            pytest.skip(f"axis {a} of n = {w.n[a]} does not split into {wb} x {L} blocks of {nc} lines")
    tiles = ",".join((f"{L}:{wb}:5:{nc}" if ch == "c" else "0:0:0:1") for a, ch in enumerate(spec))
    monkeypatch.setenv("ETD_TILES", tiles)
    ctx = EtdRdpIf.from_workload(w, prec)
    inf = ctx.info()
    for a, ch in enumerate(spec):
        if ch == "c":
            assert inf["staged"][a] == 5, (a, inf)
            if a > 0:
                assert inf["lines_per_block"][a] == nc, (a, inf)
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    P = oracle_problem(w)
    e1 = rel_err(one, oracle.run(P, U0, 0.3, 1))
    e3 = rel_err(three, oracle.run(P, U0, 0.3, 3))
    print(f"{w.name} {prec} circulant strided ({tiles}): 1 step {e1:.3e}, 3 steps {e3:.3e}")
    bound = max(_fp64_bound_axis(w, a) for a in range(w.dim))
    if prec == "fp64":
        assert e1 <= bound and e3 <= bound, (e1, e3, bound)
    else:
        assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


def _fp64_bound_axis(w, a):
    r = w.k * max(w.D) / w.h(a) ** 2
    return max(FP64_TOL, 2.0 ** -52 * (1 + 4 * r)) if w.bc[a] == W.PERIODIC else FP64_TOL


def test_circulant_strided_4096_stiff_fp32(monkeypatch):
    """The 4096^2 periodic benchmark grid's last sweep as 16-block clusters
    (16 lines x 16 chunks of 16 per block), one FP32 step against the oracle."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    w = W.schnakenberg_2d(4096)
    monkeypatch.setenv("ETD_TILES", "16:0:5:1,16:16:5:16")
    ctx = EtdRdpIf.from_workload(w, "fp32")
    inf = ctx.info()
    assert inf["staged"] == [5, 5, 0] and inf["pack"][1] == 16, inf
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=torch.float32)
    ctx.run(U, 0.0, 1)
    torch.cuda.synchronize()
    ctx.close()
    err = rel_err(U.double().cpu().numpy(), oracle.run(oracle_problem(w), U0, 0.0, 1))
    print(f"schnakenberg2d_4096 circulant x and y, one FP32 step: err {err:.3e}")
    assert err <= fp32_step_bound(w), (err, fp32_step_bound(w))
