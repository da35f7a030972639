"""GPU reverse mode against the FP64 oracle's discrete adjoint (itself pinned
to finite differences in test_oracle_pins.py).

Tolerances (FP64): state adjoint and dL/dU0 <= 1e-12 relative (the forward
bar); over a 40-step run 1e-11.  dL/dD and dL/dparams: fp64_param_grad_bound
(tests/tolerances.py), the FP64 solve error amplified by the cancellation of
b - x in <lambda, B x> = <lambda, b - x> / r (measured on the starting state),
times the number of reversed steps.  The block sums are reduced in a fixed order, so repeated runs are
bit-identical.  FP32: the error of the FP32 gradient against
the FP64 oracle gradient is measured and stated.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.dense_reference import oracle_problem  # noqa: E402
from tests.tolerances import fp64_param_grad_bound as pbound  # noqa: E402

pytestmark = pytest.mark.gpu


def _ctx(w, prec):
    from paper_2001_11220_gb300.api import EtdRdpIf
    return EtdRdpIf.from_workload(w, prec)


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def case(name, n, bc, D, reaction, params, k, ic_args):
    return W.Workload(name, n, bc, D, reaction, params, k, 1, ic="normal", ic_args=ic_args)


STEP_CASES = [
    case("bru2d_neu", (37, 23), W.NEUMANN, (0.02, 0.05), "brusselator", (1.0, 3.4), 0.05, ((1.0, 3.4), 0.1)),
    case("sch2d_per", (24, 20), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0), 0.02, ((1.0, 0.9), 0.05)),
    case("gs2d_mixed", (19, 26), (W.PERIODIC, W.DIRICHLET), (0.02, 0.01), "gray_scott", (0.04, 0.06), 0.5,
         ((0.8, 0.2), 0.05)),
    case("gs3d_mixed", (13, 11, 9), (W.PERIODIC, W.NEUMANN, W.DIRICHLET), (0.02, 0.01), "gray_scott",
         (0.04, 0.06), 0.5, ((0.8, 0.2), 0.05)),
    case("lin3d_neu", (10, 12, 7), W.NEUMANN, (0.3,), "linear", (-0.7, 0.2), 0.1, ((1.0,), 0.2)),
    W.mms_3d(12).with_(name="mms3d_12"),
    case("cgl2d_per", (24, 20), W.PERIODIC, (1.0, 1.0), "cgl", (1.3,), 0.05, ((0.0, 0.0), 0.5)).with_(
        length=(12.0, 10.0)),
    # periodic axes with whole chunks take the circulant adjoint (every axis here)
    case("gs3d_per_circ", (16, 8, 24), W.PERIODIC, (0.02, 0.01), "gray_scott", (0.04, 0.06), 0.5,
         ((0.8, 0.2), 0.05)),
    case("sch2d_per_circ", (32, 40), W.PERIODIC, (0.01, 0.1), "schnakenberg", (0.1, 0.9, 10.0), 0.02,
         ((1.0, 0.9), 0.05)),
    # 700-node periodic lines take the warp-cooperative chunk scan; h = 0.1 keeps the
    # dL/dD sum as well conditioned as the cases above (at h = 1/700, r = k D / h^2 ~ 4e5
    # and a one-ulp change of U_n moves the oracle's dL/dD by 3e-12 relative)
    case("long_per", (9, 700), (W.NEUMANN, W.PERIODIC), (0.3, 1.5), "gray_scott", (0.04, 0.06), 0.5,
         ((0.8, 0.2), 0.05)).with_(length=(0.8, 70.0)),
]


@pytest.mark.parametrize("w", STEP_CASES, ids=lambda w: w.name)
def test_step_adjoint_fp64_matches_oracle(w):
    rng = np.random.default_rng(7)
    U0 = W.initial_state(w)
    ub = rng.standard_normal(U0.shape)
    ctx = _ctx(w, "fp64")
    Un = torch.tensor(U0, device="cuda")
    Ubn = torch.tensor(ub, device="cuda")
    got, dD, dp = ctx.step_adjoint(Un, 0.2, Ubn)
    torch.cuda.synchronize()
    ref, rdD, rdp = oracle.step_adjoint(oracle_problem(w), U0, 0.2, ub)
    ctx.close()
    print(f"{w.name} step adjoint: state {rel(got.cpu().numpy(), ref):.2e}, dD {rel(dD, rdD):.2e}")
    assert rel(got.cpu().numpy(), ref) <= 1e-12
    assert rel(dD, rdD) <= pbound(w, U0), (dD, rdD, pbound(w, U0))
    npar = len(w.params)
    if npar and np.max(np.abs(rdp[:npar])) > 0:
        assert rel(dp[:npar], rdp[:npar]) <= pbound(w, U0), (dp, rdp, pbound(w, U0))


@pytest.mark.parametrize("w,nsteps,ckpt", [
    (case("bru2d_grad", (20, 16), W.NEUMANN, (0.02, 0.03), "brusselator", (1.0, 3.4), 0.05, ((1.0, 3.4), 0.1)), 7, 3),
    (W.gray_scott_3d(12, steps=5).with_(k=0.5, D=(0.01, 0.005)), 5, 2),
    (W.mms_3d(10).with_(name="mms3d_10"), 4, 4),
], ids=["bru2d", "gs3d", "mms3d"])
def test_grad_fp64_matches_oracle(w, nsteps, ckpt):
    U0 = W.initial_state(w)
    target = W.initial_state(w, seed=99) * 0.9
    ctx = _ctx(w, "fp64")
    loss, dU0, dD, dp = ctx.grad(torch.tensor(U0, device="cuda"), 0.0, torch.tensor(target, device="cuda"),
                                 nsteps, ckpt)
    rloss, rdU0, rdD, rdp = oracle.grad(oracle_problem(w), U0, 0.0, target, nsteps)
    ctx.close()
    print(f"grad {w.name}: dU0 {rel(dU0.cpu().numpy(), rdU0):.2e}, dD {rel(dD, rdD):.2e}")
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    assert rel(dU0.cpu().numpy(), rdU0) <= 1e-12
    assert rel(dD, rdD) <= pbound(w, U0, nsteps), (dD, rdD, pbound(w, U0, nsteps))
    npar = len(w.params)
    if np.max(np.abs(rdp[:npar])) > 0:
        assert rel(dp[:npar], rdp[:npar]) <= pbound(w, U0, nsteps), (dp, rdp, pbound(w, U0, nsteps))


def test_grad_checkpoint_interval_does_not_change_result():
    """Recomputation from checkpoints repeats the forward arithmetic exactly and
    the block sums are reduced in a fixed order: every spacing, and a repeated
    call, give bit-identical loss and gradients."""
    w = case("bru2d_ck", (16, 12), W.NEUMANN, (0.02, 0.03), "brusselator", (1.0, 3.4), 0.05, ((1.0, 3.4), 0.1))
    U0 = torch.tensor(W.initial_state(w), device="cuda")
    tg = torch.tensor(W.initial_state(w, seed=3), device="cuda")
    ctx = _ctx(w, "fp64")
    a = ctx.grad(U0, 0.0, tg, 9, 1)
    b = ctx.grad(U0, 0.0, tg, 9, 4)
    c = ctx.grad(U0, 0.0, tg, 9, 9)
    d = ctx.grad(U0, 0.0, tg, 9, 1)
    ctx.close()
    for x in (b, c, d):
        assert x[0] == a[0]
        assert torch.equal(x[1], a[1])
        assert np.array_equal(x[2], a[2]) and np.array_equal(x[3], a[3])


def test_grad_dD_matches_gpu_finite_differences():
    """Independent of the oracle: central differences of the GPU forward loss in D."""
    w = W.gray_scott_3d(12, steps=4).with_(k=0.5, D=(0.01, 0.005))
    U0 = W.initial_state(w)
    target = W.initial_state(w, seed=5)
    ctx = _ctx(w, "fp64")
    _, _, dD, _ = ctx.grad(torch.tensor(U0, device="cuda"), 0.0, torch.tensor(target, device="cuda"), w.steps, 2)
    ctx.close()
    eps = 1e-6

    def L(D):
        c = _ctx(w.with_(D=D), "fp64")
        U = torch.tensor(U0, device="cuda")
        c.run(U, 0.0, w.steps)
        torch.cuda.synchronize()
        r = U.cpu().numpy() - target
        c.close()
        return 0.5 * float(np.sum(r * r))

    for s in range(2):
        Dp, Dm = list(w.D), list(w.D)
        Dp[s] += eps
        Dm[s] -= eps
        fd = (L(tuple(Dp)) - L(tuple(Dm))) / (2 * eps)
        assert abs(fd - dD[s]) <= 1e-6 * max(1.0, abs(fd)), (s, fd, dD[s])


def test_grayscott_32_gradient_fp32_and_fp64_vs_oracle():
    """3D Gray-Scott periodic copy at 32^3 (k = 1, checkpoint every 20 steps): the FP64 GPU
    gradient matches the FP64 oracle gradient; the FP32 error is stated."""
    nsteps = 40
    w = W.gray_scott_3d(32, steps=nsteps)
    U0 = W.initial_state(w)
    target = W.initial_state(w, seed=2002)
    rloss, rdU0, rdD, rdp = oracle.grad(oracle_problem(w), U0, 0.0, target, nsteps)
    out = {}
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        ctx = _ctx(w, prec)
        out[prec] = ctx.grad(torch.tensor(U0, device="cuda", dtype=dt), 0.0,
                             torch.tensor(target, device="cuda", dtype=dt), nsteps, 20)
        ctx.close()
    l64, g64, d64, p64 = out["fp64"]
    l32, g32, d32, p32 = out["fp32"]
    e_g32 = rel(g32.double().cpu().numpy(), rdU0)
    e_d32 = rel(d32, rdD)
    e_p32 = rel(p32[:2], rdp[:2])
    print(f"grayscott3d_32 {nsteps} steps: FP32 gradient error vs FP64 oracle: dU0 {e_g32:.3e}, "
          f"dD {e_d32:.3e}, dparams {e_p32:.3e}; FP64: dU0 {rel(g64.cpu().numpy(), rdU0):.3e}")
    assert abs(l64 - rloss) <= 1e-12 * abs(rloss)
    assert rel(g64.cpu().numpy(), rdU0) <= 1e-11
    assert rel(d64, rdD) <= pbound(w, U0, nsteps) and rel(p64[:2], rdp[:2]) <= pbound(w, U0, nsteps)
    assert e_g32 <= 1e-3 and e_d32 <= 1e-2 and e_p32 <= 1e-2


def test_adjoint_rejects_zero_diffusion():
    from paper_2001_11220_gb300._binding import EtdError
    w = case("d0", (8, 8), W.NEUMANN, (0.0, 0.1), "brusselator", (1.0, 3.4), 0.05, ((1.0, 3.4), 0.1))
    ctx = _ctx(w, "fp64")
    U = torch.tensor(W.initial_state(w), device="cuda")
    with pytest.raises(EtdError):
        ctx.step_adjoint(U, 0.0, U.clone())
    ctx.close()


def test_autograd_simulate_matches_oracle_adjoint():
    """torch.autograd through simulate() for a loss that is not the built-in misfit
    (sum of w * U_N^2): compared with the oracle's step adjoints chained by hand."""
    from paper_2001_11220_gb300.autograd import simulate
    w = case("bru2d_ag", (18, 14), W.NEUMANN, (0.02, 0.03), "brusselator", (1.0, 3.4), 0.05, ((1.0, 3.4), 0.1))
    nsteps = 6
    U0 = W.initial_state(w)
    rng = np.random.default_rng(11)
    wt = rng.random(U0.shape)
    U0t = torch.tensor(U0, device="cuda", requires_grad=True)
    Dt = torch.tensor(w.D, dtype=torch.float64, requires_grad=True)
    pt = torch.tensor(w.params, dtype=torch.float64, requires_grad=True)
    UN = simulate(U0t, Dt, pt, n=w.n, bc=w.bc, reaction=w.reaction, k=w.k, nsteps=nsteps, ckpt_every=4)
    loss = (torch.tensor(wt, device="cuda") * UN * UN).sum()
    loss.backward()
    # oracle: forward states, then chained step adjoints with cotangent 2 w U_N
    P = oracle_problem(w)
    states = [U0]
    for i in range(nsteps):
        states.append(oracle.step(P, states[-1], i * w.k))
    ub = 2 * wt * states[-1]
    dD = np.zeros(2)
    dp = np.zeros(8)
    for i in reversed(range(nsteps)):
        ub, d1, p1 = oracle.step_adjoint(P, states[i], i * w.k, ub)
        dD += d1
        dp += p1
    assert rel(U0t.grad.cpu().numpy(), ub) <= 1e-12
    assert rel(Dt.grad.numpy(), dD) <= pbound(w, U0, nsteps)
    assert rel(pt.grad.numpy(), dp[:2]) <= pbound(w, U0, nsteps)


@pytest.mark.parametrize("kernel", [3, 4], ids=["segmented", "cluster"])
def test_grad_with_segmented_forward_sweeps(kernel, monkeypatch):
    """The gradient's forward recomputation runs segmented sweeps (a long
    periodic middle axis split over blocks; 4: the blocks of a line group as
    one thread-block cluster): the FP64 gradient still matches the oracle's."""
    w = case("seg_grad", (8, 300, 6), (W.NEUMANN, W.PERIODIC, W.DIRICHLET), (0.02, 0.01), "gray_scott",
             (0.04, 0.06), 0.5, ((0.8, 0.2), 0.05))
    monkeypatch.setenv("ETD_TILES", f"4:0:0:1,4:8:{kernel}:16,4:0:0:1")
    U0 = W.initial_state(w)
    target = W.initial_state(w, seed=99) * 0.9
    ctx = _ctx(w, "fp64")
    assert ctx.info()["staged"][1] == kernel
    loss, dU0, dD, dp = ctx.grad(torch.tensor(U0, device="cuda"), 0.0, torch.tensor(target, device="cuda"), 3, 2)
    rloss, rdU0, rdD, rdp = oracle.grad(oracle_problem(w), U0, 0.0, target, 3)
    ctx.close()
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    assert rel(dU0.cpu().numpy(), rdU0) <= 1e-12
    assert rel(dD, rdD) <= pbound(w, U0, 3), (dD, rdD)


def test_grad_fp32_repeatable():
    """FP32 gradient of the 3D Gray-Scott problem: two identical calls give
    bit-identical loss, dL/dU0, dL/dD and dL/dparams (fixed-order block sums)."""
    w = W.gray_scott_3d(16, steps=4).with_(k=0.5, D=(0.01, 0.005))
    U0 = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float32)
    tg = torch.tensor(W.initial_state(w, seed=5), device="cuda", dtype=torch.float32)
    ctx = _ctx(w, "fp32")
    a = ctx.grad(U0, 0.0, tg, 4, 2)
    b = ctx.grad(U0, 0.0, tg, 4, 2)
    ctx.close()
    assert a[0] == b[0] and torch.equal(a[1], b[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_circulant_adjoint_matches_table_adjoint(prec, monkeypatch):
    """On periodic axes with whole chunks the adjoint sweeps run on the circulant
    factorisation; the line-table kernels (ETD_ADJ_CIRC=0) solve the same systems.
    Both gradients of a 3D Gray-Scott run agree to rounding (FP64) or within the
    FP32 precision."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    w = W.gray_scott_3d(16, steps=3).with_(k=0.5, D=(0.01, 0.005))
    U0 = W.initial_state(w)
    tgt = W.initial_state(w, seed=99)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("ETD_ADJ_CIRC", flag)
        ctx = EtdRdpIf.from_workload(w, prec)
        U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
        T = torch.tensor(tgt, device="cuda", dtype=ctx.dtype)
        loss, dU0, dD, dp = ctx.grad(U, 0.0, T, 3, 2)
        out[flag] = (loss, dU0.double().cpu().numpy(), dD, dp)
        ctx.close()
    a, b = out["1"], out["0"]
    tol = 1e-11 if prec == "fp64" else 2e-4
    assert abs(a[0] - b[0]) <= tol * abs(b[0])
    assert np.max(np.abs(a[1] - b[1])) <= tol * np.max(np.abs(b[1]))
    assert np.max(np.abs(a[2] - b[2])) <= tol * 10 * np.max(np.abs(b[2]))
