"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances: FP64 <= 1e-12 relative (max over species of
max|U_gpu - U_oracle| / max|U_oracle|), after one step and at the end of a
run.  FP32: the error against the FP64 oracle is measured (printed with -s)
and bounded per step by fp32_step_bound(w) (tests/tolerances.py), derived per
workload from the decay factor of each axis's line matrices, the 17-fold
cancellation of R = 9T - 8S and the unit roundoff 2^-24; n steps: n times it.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.dense_reference import oracle_problem  # noqa: E402
from tests.tolerances import fp32_step_bound  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _api():
    from paper_2001_11220_gb300.api import EtdRdpIf
    return EtdRdpIf


def rel_err(a, ref):
    return max(float(np.max(np.abs(a[s] - ref[s])) / max(np.max(np.abs(ref[s])), 1e-300)) for s in range(ref.shape[0]))


def gpu_run(w, U0, nsteps, precision="fp64", t0=0.0):
    ctx = _api().from_workload(w, precision)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, t0, nsteps)
    torch.cuda.synchronize()
    out = U.double().cpu().numpy()
    ctx.close()
    return out


def oracle_run(w, U0, nsteps, t0=0.0):
    return oracle.run(oracle_problem(w), U0, t0, nsteps)


def case(name, n, bc, D, reaction, params=(), k=0.05, ic="normal", ic_args=None, length=None):
    S = len(D)
    if ic_args is None and ic == "normal":
        ic_args = ((0.8, 1.2)[:S], 0.1)
    return W.Workload(name, n, bc, D, reaction, params, k, 1, length=length, ic=ic, ic_args=ic_args or ())


ONE_STEP_CASES = [
    case("bru2d_neu_64", (64, 64), W.NEUMANN, (2e-3, 2e-3), "brusselator", (1.0, 3.4), k=0.01),
    case("bru2d_neu_ragged", (37, 23), W.NEUMANN, (0.02, 0.05), "brusselator", (1.0, 3.4)),
    case("enz2d_dir_src", (45, 31), W.DIRICHLET, (0.2,), "enzyme", (1.0, 0.2), ic="sine"),
    case("enz2d_dir_plain", (19, 40), W.DIRICHLET, (0.2,), "enzyme", (0.0, 0.0)),
    case("sch2d_per", (41, 29), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0)),
    case("gs2d_mixed", (33, 47), (W.PERIODIC, W.NEUMANN), (0.02, 0.01), "gray_scott", (0.04, 0.06), k=0.5),
    case("lin2d_dir_stiff", (130, 67), W.DIRICHLET, (3.0,), "linear", (-0.7, 0.2), k=0.5),
    case("min2d_dir", (3, 3), W.DIRICHLET, (0.3, 0.1), "linear", (0.5, 0.0)),
    case("min2d_neu", (3, 3), W.NEUMANN, (0.3, 0.1), "brusselator", (1.0, 3.4)),
    case("min2d_per", (3, 3), W.PERIODIC, (0.3, 0.1), "gray_scott", (0.04, 0.06)),
    case("long_x", (517, 5), (W.NEUMANN, W.PERIODIC), (0.5, 0.1), "brusselator", (1.0, 3.4)),
    case("long_y", (5, 517), (W.PERIODIC, W.DIRICHLET), (0.5, 0.1), "brusselator", (1.0, 3.4)),
    case("heun_D0", (21, 13), W.NEUMANN, (0.0, 0.0), "brusselator", (1.0, 3.4)),
    case("long_per_y", (6, 1100), (W.NEUMANN, W.PERIODIC), (0.5, 2.0), "schnakenberg", (0.1, 0.9, 10.0),
         k=0.01, ic="uniform", ic_args=((1.0, 0.9), 1e-2)),
    case("long_per_x", (1301, 7), (W.PERIODIC, W.DIRICHLET), (0.5, 2.0), "gray_scott", (0.04, 0.06), k=0.01),
    case("gs3d_mixed", (19, 17, 23), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott",
         (0.04, 0.06), k=0.5),
    case("mms3d_16", (16, 16, 16), W.DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), k=1 / 17, ic="sine"),
    case("bru3d_per", (33, 20, 9), W.PERIODIC, (0.05, 0.02), "brusselator", (1.0, 3.4)),
    case("min3d", (3, 3, 3), (W.DIRICHLET, W.NEUMANN, W.PERIODIC), (0.3, 0.1), "brusselator", (1.0, 3.4)),
    case("sch3d_stiff", (24, 24, 24), W.PERIODIC, (1.0, 10.0), "schnakenberg", (0.1, 0.9, 1000.0), k=1e-3,
         ic="uniform", ic_args=((1.0, 0.9), 1e-3)),
    # complex Ginzburg-Landau (Section 8, alpha = 0): Re u, Im u as two species, N(0, 1) field
    case("cgl2d_per", (40, 36), W.PERIODIC, (1.0, 1.0), "cgl", (1.3,), k=0.05, ic_args=((0.0, 0.0), 1.0),
         length=(20.0, 18.0)),
    case("cgl3d_per", (16, 12, 10), W.PERIODIC, (1.0, 1.0), "cgl", (1.3,), k=0.05, ic_args=((0.0, 0.0), 0.5),
         length=(16.0, 12.0, 10.0)),
]


@pytest.mark.parametrize("w", ONE_STEP_CASES, ids=lambda w: w.name)
def test_one_step_fp64_matches_oracle(w):
    U0 = W.initial_state(w)
    got = gpu_run(w, U0, 1, "fp64", t0=0.3)
    ref = oracle_run(w, U0, 1, t0=0.3)
    err = rel_err(got, ref)
    assert err <= FP64_TOL, err


FP32_CASES = ("cgl2d_per", "bru2d_neu_64", "bru2d_neu_ragged", "enz2d_dir_src", "enz2d_dir_plain", "sch2d_per", "gs2d_mixed",
              "gs3d_mixed", "mms3d_16", "bru3d_per", "long_per_y")


def test_stiff_periodic_fp64_within_condition_bound():
    """Periodic 1301-node lines at r = k D / h^2 ~ 1.7e6: the line matrices' condition
    number is up to 1 + 4r, so the forward error of any backward-stable solve may reach
    eps * (1 + 4r); the GPU result is held to that bound against the oracle."""
    w = case("long_per_x_stiff", (1301, 7), (W.PERIODIC, W.DIRICHLET), (0.5, 2.0), "gray_scott", (0.04, 0.06),
             k=0.5)
    r_max = w.k * max(w.D) * ((w.n[0]) / w.length[0]) ** 2
    bound = 2.0 ** -52 * (1 + 4 * r_max)
    U0 = W.initial_state(w)
    err = rel_err(gpu_run(w, U0, 1, "fp64", t0=0.3), oracle_run(w, U0, 1, t0=0.3))
    print(f"stiff periodic FP64 error {err:.3e} (bound {bound:.3e})")
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("w", [c for c in ONE_STEP_CASES if c.name in FP32_CASES], ids=lambda w: w.name)
def test_one_step_fp32_error_bounded(w):
    U0 = W.initial_state(w)
    got = gpu_run(w, U0, 1, "fp32", t0=0.3)
    ref = oracle_run(w, U0, 1, t0=0.3)
    err = rel_err(got, ref)
    print(f"FP32 one-step error {w.name}: {err:.3e}")
    assert err <= fp32_step_bound(w), (err, fp32_step_bound(w))


def test_brusselator_64_full_run_fp64_and_fp32():
    """2D Brusselator 64x64 Neumann, k = 0.01, 100 steps (T = 1)."""
    w = W.brusselator_2d()
    U0 = W.initial_state(w)
    ref = oracle_run(w, U0, w.steps)
    e64 = rel_err(gpu_run(w, U0, w.steps, "fp64"), ref)
    e32 = rel_err(gpu_run(w, U0, w.steps, "fp32"), ref)
    print(f"brusselator2d_64 100 steps: FP64 err {e64:.3e}  FP32 err {e32:.3e}")
    assert e64 <= FP64_TOL
    assert e32 <= 1e-4


@pytest.mark.parametrize("p", [32])
def test_mms3d_full_run(p):
    w = W.mms_3d(p)
    U0 = W.initial_state(w)
    ref = oracle_run(w, U0, w.steps)
    e64 = rel_err(gpu_run(w, U0, w.steps, "fp64"), ref)
    e32 = rel_err(gpu_run(w, U0, w.steps, "fp32"), ref)
    exact = W.exact_mms(w, w.steps * w.k)
    print(f"mms3d_{p}: FP64 err vs oracle {e64:.3e}, FP32 {e32:.3e}, oracle vs exact {rel_err(ref, exact):.3e}")
    assert e64 <= FP64_TOL
    assert e32 <= 1e-5


def test_mms3d_convergence_full_runs_fp64_and_fp32():
    """Second order in k = h on the manufactured 3D Dirichlet problem (Section 8.1's
    check, here on the GPU): full runs to T = 1 at p = 32, 64, 128, 256 in FP64 and
    FP32, error against the exact solution e^{-t} sin sin sin.  FP64 matches the
    oracle at p <= 64; the observed order of the FP64 errors approaches 2 (the
    oracle's own pin: 1.92, 1.96 from p = 15 to 63), and FP32 reaches the same
    accuracy as FP64 at every size (its rounding stays below the scheme's error)."""
    errs = {"fp64": [], "fp32": []}
    for p in (32, 64, 128, 256):
        w = W.mms_3d(p)
        U0 = W.initial_state(w)
        exact = W.exact_mms(w, w.steps * w.k)
        for prec in ("fp64", "fp32"):
            got = gpu_run(w, U0, w.steps, prec)
            errs[prec].append(float(np.max(np.abs(got - exact)) / np.max(np.abs(exact))))
            if prec == "fp64" and p <= 64:
                assert rel_err(got, oracle_run(w, U0, w.steps)) <= FP64_TOL
    eoc = {k: [math.log(v[i] / v[i + 1]) / math.log((2 * 32 * 2 ** i + 1) / (32 * 2 ** i + 1)) for i in range(3)]
           for k, v in errs.items()}
    print(f"mms3d T = 1 errors vs exact: FP64 {errs['fp64']}, FP32 {errs['fp32']}; EOC FP64 {eoc['fp64']}, "
          f"FP32 {eoc['fp32']}")
    assert all(1.85 < e < 2.15 for e in eoc["fp64"]), eoc
    for a, b in zip(errs["fp32"], errs["fp64"]):
        assert abs(a - b) <= 0.3 * b, (a, b)


def test_mms3d_256_one_step_full_size():
    """3D Dirichlet manufactured problem at the benchmark size 256^3, one step, FP64 and FP32."""
    w = W.mms_3d(256)
    U0 = W.initial_state(w)
    ref = oracle_run(w, U0, 1)
    e64 = rel_err(gpu_run(w, U0, 1, "fp64"), ref)
    e32 = rel_err(gpu_run(w, U0, 1, "fp32"), ref)
    print(f"mms3d_256 one step: FP64 err {e64:.3e}, FP32 err {e32:.3e}")
    assert e64 <= FP64_TOL
    assert e32 <= fp32_step_bound(w), (e32, fp32_step_bound(w))


def test_schnakenberg_4096_one_step_fp32():
    """2D periodic Schnakenberg 4096^2 (cyclic lines, Sherman-Morrison), FP32 state, one step."""
    w = W.schnakenberg_2d(4096)
    U0 = W.initial_state(w)
    ref = oracle_run(w, U0, 1)
    e32 = rel_err(gpu_run(w, U0, 1, "fp32"), ref)
    print(f"schnakenberg2d_4096 one step FP32 err {e32:.3e}")
    assert e32 <= fp32_step_bound(w), (e32, fp32_step_bound(w))


@pytest.mark.parametrize("name", ["mms3d_256", "schnakenberg2d_4096"])
def test_full_size_in_the_benchmark_configuration(name):
    """The benchmark workloads at full size in the launch configuration the
    benchmark times: tile shapes autotuned on a scratch state exactly as
    bench.py does (on 4096^2 this picks the cluster-segmented sweeps), then
    one FP32 step from the same state against the FP64 oracle."""
    w = W.mms_3d(256) if name == "mms3d_256" else W.schnakenberg_2d(4096)
    U0 = W.initial_state(w)
    ctx = _api().from_workload(w, "fp32")
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.autotune(U.clone())
    inf = ctx.info()
    ctx.run(U, 0.0, 1)
    torch.cuda.synchronize()
    out = U.double().cpu().numpy()
    ctx.close()
    err = rel_err(out, oracle_run(w, U0, 1))
    tiles = ",".join(f"{inf['chunk'][a]}:{inf['lines_per_block'][a]}:{inf['staged'][a]}:{inf['pack'][a]}"
                     for a in range(w.dim))
    print(f"{name} autotuned ({tiles}) one FP32 step: err {err:.3e}")
    assert err <= fp32_step_bound(w), (err, fp32_step_bound(w), tiles)


def test_run_host_matches_device_run():
    w = W.brusselator_2d(p=40, steps=7)
    U0 = W.initial_state(w)
    EtdRdpIf = _api()
    ctx = EtdRdpIf.from_workload(w, "fp64")
    U = torch.tensor(U0, device="cuda")
    ctx.run(U, 0.0, w.steps)
    H = torch.tensor(U0).pin_memory()
    ctx.run_host(H, 0.0, w.steps)
    torch.cuda.synchronize()
    assert torch.equal(U.cpu(), H)
    ctx.close()


@pytest.mark.parametrize("prec,steps,pinned", [("fp32", 1, True), ("fp32", 2, True), ("fp64", 3, False),
                                               ("fp32", 1, False)])
def test_run_host_direct_and_copied(prec, steps, pinned):
    """etd_run_host on pinned and pageable host buffers, one and several
    steps, FP32 and FP64: bit-identical to the same run on a device state."""
    w = W.gray_scott_3d(24, steps=steps)
    U0 = W.initial_state(w)
    EtdRdpIf = _api()
    ctx = EtdRdpIf.from_workload(w, prec)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.25, steps)
    H = torch.tensor(U0, dtype=ctx.dtype)
    if pinned:
        H = H.pin_memory()
    ctx.run_host(H, 0.25, steps)
    torch.cuda.synchronize()
    assert torch.equal(U.cpu(), H)
    ctx.close()


def test_graph_replay_matches_direct_launches():
    w = W.brusselator_2d(p=48, steps=9)
    U0 = W.initial_state(w)
    EtdRdpIf = _api()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = EtdRdpIf.from_workload(w, "fp32")
        A = torch.tensor(U0, device="cuda", dtype=torch.float32)
        B = A.clone()
        ctx.run(A, 0.0, w.steps)          # captured into a CUDA graph
        ctx.run(B, 0.0, w.steps)          # different buffer: captured again
        C = torch.tensor(U0, device="cuda", dtype=torch.float32)
        os.environ["ETD_NO_GRAPHS"] = "1"
        try:
            ctx.run(C, 0.0, w.steps)      # direct launches
        finally:
            del os.environ["ETD_NO_GRAPHS"]
    s.synchronize()
    assert torch.equal(A, B) and torch.equal(A, C)
    ctx.close()


def test_step_sequence_equals_run():
    w = W.brusselator_2d(p=30, steps=4)
    U0 = W.initial_state(w)
    EtdRdpIf = _api()
    ctx = EtdRdpIf.from_workload(w, "fp64")
    A = torch.tensor(U0, device="cuda")
    B = A.clone()
    ctx.run(A, 0.0, 4)
    for n in range(4):
        ctx.step(B, n * w.k)
    torch.cuda.synchronize()
    assert torch.equal(A, B)
    ctx.close()


def test_bad_state_rejected():
    w = W.brusselator_2d(p=16, steps=1)
    ctx = _api().from_workload(w, "fp64")
    with pytest.raises(ValueError):
        ctx.step(torch.zeros((2, 16, 16), device="cuda", dtype=torch.float32), 0.0)
    ctx.close()


def test_autotuned_tiles_keep_parity():
    """Every tile shape the autotuner may pick computes the same step: after
    tuning, one FP64 step still matches the oracle."""
    w = case("gs3d_tune", (40, 36, 33), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott",
             (0.04, 0.06), k=0.5)
    U0 = W.initial_state(w)
    EtdRdpIf = _api()
    ctx = EtdRdpIf.from_workload(w, "fp64")
    work = torch.tensor(U0, device="cuda")
    ctx.autotune(work)
    U = torch.tensor(U0, device="cuda")
    ctx.step(U, 0.3)
    torch.cuda.synchronize()
    err = rel_err(U.cpu().numpy(), oracle_run(w, U0, 1, t0=0.3))
    ctx.close()
    assert err <= FP64_TOL, err


# Line-pair mode (FP32 strided sweeps, two neighbouring lines per thread in
# packed two-lane arithmetic), forced through ETD_TILES on every strided axis
PAIR_CASES = [
    case("pair_bru2d_neu", (64, 64), W.NEUMANN, (2e-3, 2e-3), "brusselator", (1.0, 3.4), k=0.01),
    case("pair_sch2d_per", (40, 29), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0)),
    case("pair_gs2d_ragged", (34, 47), (W.PERIODIC, W.NEUMANN), (0.02, 0.01), "gray_scott", (0.04, 0.06), k=0.5),
    case("pair_gs3d", (20, 17, 23), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott",
         (0.04, 0.06), k=0.5),
    case("pair_mms3d", (16, 16, 16), W.DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), k=1 / 17, ic="sine"),
    case("pair_lin3d", (30, 22, 9), W.NEUMANN, (0.3,), "linear", (-0.7, 0.2), k=0.1),
    case("pair_long_per", (6, 1100), (W.NEUMANN, W.PERIODIC), (0.5, 2.0), "schnakenberg", (0.1, 0.9, 10.0),
         k=0.01, ic="uniform", ic_args=((1.0, 0.9), 1e-2)),
]


def pair_tiles(dim):
    return ",".join(["8:0:0:1"] + ["8:0:0:2"] * (dim - 1))


@pytest.mark.parametrize("w", PAIR_CASES, ids=lambda w: w.name)
def test_line_pairs_fp32_vs_oracle(w, monkeypatch):
    monkeypatch.setenv("ETD_TILES", pair_tiles(len(w.n)))
    ctx = _api().from_workload(w, "fp32")
    assert ctx.info()["pack"][1:len(w.n)] == [2] * (len(w.n) - 1)
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=torch.float32)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    e1 = rel_err(one, oracle_run(w, U0, 1, t0=0.3))
    e3 = rel_err(three, oracle_run(w, U0, 3, t0=0.3))
    print(f"{w.name}: FP32 line pairs vs FP64 oracle: 1 step {e1:.3e}, 3 steps {e3:.3e}")
    assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


def test_line_pairs_grad_matches_single_lines(monkeypatch):
    """The gradient's forward recomputation runs the pair kernels when they are
    planned: its FP32 result matches the one-line-per-thread gradient."""
    w = W.gray_scott_3d(16, steps=4).with_(k=0.5, D=(0.01, 0.005))
    U0 = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float32)
    tg = torch.tensor(W.initial_state(w, seed=5), device="cuda", dtype=torch.float32)
    out = []
    for tiles in (None, pair_tiles(3)):
        if tiles:
            monkeypatch.setenv("ETD_TILES", tiles)
        ctx = _api().from_workload(w, "fp32")
        out.append(ctx.grad(U0, 0.0, tg, 4, 2))
        ctx.close()
    (l0, g0, d0, p0), (l1, g1, d1, p1) = out
    assert abs(l1 - l0) <= 1e-5 * abs(l0)
    assert float((g1 - g0).abs().max() / g0.abs().max()) <= 1e-4
    assert np.max(np.abs(d1 - d0)) <= 1e-3 * np.max(np.abs(d0))


# FP32 tile kernels (shared-memory tiles of whole lines, compile-time tile
# geometry), forced through ETD_TILES: one line per thread on every axis, and
# line pairs on the strided axes
TILE_CASES = [
    case("tile_bru2d_neu", (64, 64), W.NEUMANN, (2e-3, 2e-3), "brusselator", (1.0, 3.4), k=0.01),
    case("tile_sch2d_per", (40, 28), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0)),
    case("tile_gs2d_ragged", (36, 47), (W.PERIODIC, W.NEUMANN), (0.02, 0.01), "gray_scott", (0.04, 0.06), k=0.5),
    case("tile_gs3d", (20, 16, 23), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott",
         (0.04, 0.06), k=0.5),
    case("tile_mms3d", (16, 16, 16), W.DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), k=1 / 17, ic="sine"),
    case("tile_lin3d", (28, 20, 37), W.NEUMANN, (0.3,), "linear", (-0.7, 0.2), k=0.1),
]


@pytest.mark.parametrize("pairs", [False, True], ids=["lines", "pairs"])
@pytest.mark.parametrize("w", TILE_CASES, ids=lambda w: w.name)
def test_tile_kernels_fp32_vs_oracle(w, pairs, monkeypatch):
    d = len(w.n)
    monkeypatch.setenv("ETD_TILES", ",".join(["8:16:2:1"] + ["8:16:2:%d" % (2 if pairs else 1)] * (d - 1)))
    ctx = _api().from_workload(w, "fp32")
    inf = ctx.info()
    assert inf["staged"][:d] == [2] * d, inf
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=torch.float32)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    e1 = rel_err(one, oracle_run(w, U0, 1, t0=0.3))
    e3 = rel_err(three, oracle_run(w, U0, 3, t0=0.3))
    print(f"{w.name} ({'pairs' if pairs else 'lines'}): FP32 tile kernels vs FP64 oracle: 1 step {e1:.3e}, "
          f"3 steps {e3:.3e}")
    assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


def test_tile_kernels_reject_misaligned_state(monkeypatch):
    """A state that is not 16-byte aligned is refused before any launch."""
    import ctypes
    from paper_2001_11220_gb300 import _binding as B
    w = TILE_CASES[0]
    monkeypatch.setenv("ETD_TILES", "8:16:2:1,8:16:2:1")
    ctx = _api().from_workload(w, "fp32")
    buf = torch.zeros(W.initial_state(w).size + 4, device="cuda", dtype=torch.float32)
    for call in (lambda p: ctx.lib.etd_step(ctx.ctx, ctypes.c_void_p(p), 0.0),
                 lambda p: ctx.lib.etd_run(ctx.ctx, ctypes.c_void_p(p), 0.0, 2)):
        with pytest.raises(B.EtdError, match="16-byte aligned"):
            B.check(call(buf.data_ptr() + 4), ctx.ctx)
    ctx.close()


# Segmented sweeps (long lines split over several blocks: segment summaries,
# a carry pass over the segments of every line, then the carried solves),
# forced through ETD_TILES ("L:lines:3:chunks per segment") on the long axes
SEG_CASES = [
    (case("seg_per_y", (6, 1100), (W.NEUMANN, W.PERIODIC), (0.5, 2.0), "schnakenberg", (0.1, 0.9, 10.0), k=0.01,
          ic="uniform", ic_args=((1.0, 0.9), 1e-2)), ["{L}:0:0:1", "{L}:8:3:16"]),
    (case("seg_per_x", (1301, 7), (W.PERIODIC, W.DIRICHLET), (0.5, 2.0), "gray_scott", (0.04, 0.06), k=0.01),
     ["{L}:8:3:16", "{L}:0:0:1"]),
    (case("seg_neu_dir_ragged", (517, 301), (W.NEUMANN, W.DIRICHLET), (0.5, 0.1), "brusselator", (1.0, 3.4)),
     ["{L}:8:3:8", "{L}:16:3:8"]),
    (case("seg_3d_middle", (8, 300, 6), (W.NEUMANN, W.PERIODIC, W.DIRICHLET), (0.02, 0.01), "gray_scott",
          (0.04, 0.06), k=0.5), ["{L}:0:0:1", "{L}:8:3:16", "{L}:0:0:1"]),
    (case("seg_3d_last_src", (12, 10, 270), W.DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), k=1 / 17, ic="sine"),
     ["{L}:0:0:1", "{L}:0:0:1", "{L}:4:3:16"]),
]


def seg_tiles(spec, L):
    return ",".join(x.format(L=L, M=128 // L) for x in spec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("w,spec", SEG_CASES, ids=[c[0].name for c in SEG_CASES])
def test_segmented_sweeps_vs_oracle(w, spec, prec, monkeypatch):
    monkeypatch.setenv("ETD_TILES", seg_tiles(spec, 4 if prec == "fp64" else 8))
    ctx = _api().from_workload(w, prec)
    inf = ctx.info()
    seg_axes = [a for a, x in enumerate(spec) if ":3:" in x]
    assert all(inf["staged"][a] == 3 for a in seg_axes), inf
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    e1 = rel_err(one, oracle_run(w, U0, 1, t0=0.3))
    e3 = rel_err(three, oracle_run(w, U0, 3, t0=0.3))
    print(f"{w.name} {prec} segmented: 1 step {e1:.3e}, 3 steps {e3:.3e}")
    if prec == "fp64":
        assert e1 <= FP64_TOL and e3 <= FP64_TOL, (e1, e3)
    else:
        assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


# Cluster-segmented sweeps ("L:lines:4:chunks per segment"): the segments of a
# line group run as one thread-block cluster (2 to 16 blocks, 9 and more on
# the non-portable cluster size) and exchange their summaries through
# distributed shared memory in a single launch per sweep
CLUSTER_CASES = [
    (case("clu_per_y", (6, 1100), (W.NEUMANN, W.PERIODIC), (0.5, 2.0), "schnakenberg", (0.1, 0.9, 10.0), k=0.01,
          ic="uniform", ic_args=((1.0, 0.9), 1e-2)), ["{L}:0:0:1", "{L}:8:4:32"]),
    (case("clu_per_x", (1301, 7), (W.PERIODIC, W.DIRICHLET), (0.5, 2.0), "gray_scott", (0.04, 0.06), k=0.01),
     ["{L}:8:4:32", "{L}:0:0:1"]),
    (case("clu_neu_dir_ragged", (517, 301), (W.NEUMANN, W.DIRICHLET), (0.5, 0.1), "brusselator", (1.0, 3.4)),
     ["{L}:8:4:16", "{L}:16:4:8"]),
    (case("clu_16_blocks", (2048, 5), (W.PERIODIC, W.NEUMANN), (0.5, 2.0), "schnakenberg", (0.1, 0.9, 10.0),
          k=0.01, ic="uniform", ic_args=((1.0, 0.9), 1e-2)), ["{L}:8:4:{M}", "{L}:0:0:1"]),
    (case("clu_3d_middle", (8, 300, 6), (W.NEUMANN, W.PERIODIC, W.DIRICHLET), (0.02, 0.01), "gray_scott",
          (0.04, 0.06), k=0.5), ["{L}:0:0:1", "{L}:8:4:16", "{L}:0:0:1"]),
    (case("clu_3d_last_src", (12, 10, 270), W.DIRICHLET, (1.0,), "enzyme", (1.0, 1.0), k=1 / 17, ic="sine"),
     ["{L}:0:0:1", "{L}:0:0:1", "{L}:4:4:16"]),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("w,spec", CLUSTER_CASES, ids=[c[0].name for c in CLUSTER_CASES])
def test_cluster_segmented_sweeps_vs_oracle(w, spec, prec, monkeypatch):
    L = 4 if prec == "fp64" else 8
    monkeypatch.setenv("ETD_TILES", seg_tiles(spec, L))
    ctx = _api().from_workload(w, prec)
    inf = ctx.info()
    seg_axes = [a for a, x in enumerate(spec) if ":4:" in x]
    assert all(inf["staged"][a] == 4 for a in seg_axes), inf
    assert inf["launches_per_step"] == w.dim, inf  # one launch per sweep
    U0 = W.initial_state(w)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.3, 1)
    torch.cuda.synchronize()
    one = U.double().cpu().numpy()
    ctx.run(U, 0.3 + w.k, 2)
    torch.cuda.synchronize()
    three = U.double().cpu().numpy()
    ctx.close()
    e1 = rel_err(one, oracle_run(w, U0, 1, t0=0.3))
    e3 = rel_err(three, oracle_run(w, U0, 3, t0=0.3))
    print(f"{w.name} {prec} cluster-segmented ({seg_tiles(spec, L)}): 1 step {e1:.3e}, 3 steps {e3:.3e}")
    if prec == "fp64":
        assert e1 <= FP64_TOL and e3 <= FP64_TOL, (e1, e3)
    else:
        assert e1 <= fp32_step_bound(w) and e3 <= 3 * fp32_step_bound(w), (e1, e3, fp32_step_bound(w))


def test_cgl_2d_paper_pulses_fp64_and_fp32():
    """Section 8's 2D CGL run (periodic [0, 200]^2, alpha = 0, beta = 1.3, k = 1/20,
    Gaussian pulses) at p = 64 for 40 steps: FP64 matches the oracle, FP32 stays
    within the derived per-step bound times the linear growth e^T of the equation."""
    w = W.cgl_2d(64, steps=40)
    U0 = W.initial_state(w)
    ref = oracle_run(w, U0, w.steps)
    g64 = gpu_run(w, U0, w.steps, "fp64")
    assert rel_err(g64, ref) <= FP64_TOL
    g32 = gpu_run(w, U0, w.steps, "fp32")
    e32 = rel_err(g32, ref)
    print(f"cgl2d_64 40 steps: FP64 {rel_err(g64, ref):.2e}, FP32 {e32:.2e} vs oracle")
    assert e32 <= w.steps * fp32_step_bound(w) * math.exp(w.steps * w.k)


@pytest.mark.parametrize("w", [c for c in ONE_STEP_CASES if c.name in ("bru2d_neu_64", "bru2d_neu_ragged", "gs2d_mixed",
                                                                       "gs3d_mixed", "bru3d_per", "cgl2d_per")],
                         ids=lambda w: w.name)
def test_staged_kernels_forced_fp64_matches_oracle(w, monkeypatch):
    """The staged (persistent, cp.async double-buffered) table kernels, which small
    problems no longer take by default, forced on every axis (ETD_TILES kernel code 1)."""
    monkeypatch.setenv("ETD_TILES", ",".join(["4:0:1:1"] * len(w.n)))
    U0 = W.initial_state(w)
    ctx = _api().from_workload(w, "fp64")
    staged = ctx.info()["staged"][:len(w.n)]
    ctx.close()
    assert any(k == 1 for k in staged), staged
    got = gpu_run(w, U0, 1, "fp64")
    assert rel_err(got, oracle_run(w, U0, 1)) <= FP64_TOL


@pytest.mark.parametrize("shape,bc", [((16384, 3), W.NEUMANN), ((16384, 3), W.PERIODIC),
                                      ((3, 16384), W.DIRICHLET), ((3, 16384), W.PERIODIC)],
                         ids=["x_neumann", "x_periodic", "y_dirichlet", "y_periodic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_longest_lines_the_api_accepts(shape, bc, prec):
    """Lines of 16384 nodes (the largest n etd_create takes) along x and along y, on
    the plans the library picks for them: one step against the oracle (FP64 1e-12,
    FP32 the per-step bound)."""
    w = case(f"maxline_{shape[0]}x{shape[1]}", shape, bc, (1e-6, 2e-6), "brusselator", (1.0, 3.4), k=0.01)
    U0 = W.initial_state(w)
    got = gpu_run(w, U0, 1, prec)
    ref = oracle_run(w, U0, 1)
    e = rel_err(got, ref)
    tol = FP64_TOL if prec == "fp64" else fp32_step_bound(w)
    print(f"{w.name} {W.BC_NAMES[bc]} {prec}: {e:.2e} (tol {tol:.2e})")
    assert e <= tol
