"""Batched ensemble (one persistent launch per step over many uneven
instances, or one launch per sweep kind) against the FP64 oracle, instance by
instance; the bounded dependency waits of the persistent step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.dense_reference import oracle_problem  # noqa: E402
from tests.tolerances import fp32_step_bound  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel(a, b):
    return max(float(np.max(np.abs(a[s] - b[s])) / np.max(np.abs(b[s]))) for s in range(b.shape[0]))


def small_ensemble(n=14, seed=5):
    ws = W.ensemble(ninst=n, steps=3, seed=seed, sizes=(3, 7, 20, 33, 48, 64, 70))
    # ragged rectangles too
    ws[0] = ws[0].with_(n=(37, 21))
    ws[1] = ws[1].with_(n=(5, 66), bc=(W.PERIODIC, W.NEUMANN))
    return ws


@pytest.mark.parametrize("tuned", [False, True], ids=["planned", "autotuned"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ensemble_matches_oracle_per_instance(prec, tuned):
    from paper_2001_11220_gb300.api import EtdEnsemble
    ws = small_ensemble()
    dt = torch.float64 if prec == "fp64" else torch.float32
    U0 = [W.initial_state(w) for w in ws]
    states = [torch.tensor(u, device="cuda", dtype=dt) for u in U0]
    ens = EtdEnsemble(ws, prec)
    if tuned:  # shapes picked by timing candidates on scratch copies
        ens.autotune([U.clone() for U in states])
    ens.run(states, 0.1, 3)
    torch.cuda.synchronize()
    worst = 0.0
    for w, u0, U in zip(ws, U0, states):
        ref = oracle.run(oracle_problem(w), u0, 0.1, 3)
        e = rel(U.double().cpu().numpy(), ref)
        worst = max(worst, e)
        assert e <= (FP64_TOL if prec == "fp64" else 3 * fp32_step_bound(w)), (w.name, w.n, w.bc, e)
    print(f"ensemble {prec} ({'autotuned' if tuned else 'planned'}): worst per-instance error vs oracle "
          f"after 3 steps {worst:.3e}")
    ens.close()


def test_ensemble_graph_replay_and_pointer_change():
    from paper_2001_11220_gb300.api import EtdEnsemble
    ws = small_ensemble(6, seed=9)
    U0 = [W.initial_state(w) for w in ws]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ens = EtdEnsemble(ws, "fp64", stream=s)
        A = [torch.tensor(u, device="cuda") for u in U0]
        B = [torch.tensor(u, device="cuda") for u in U0]
        ens.run(A, 0.0, 4)      # captured graph
        ens.run(B, 0.0, 2)      # new pointers: arguments rebuilt
        ens.run(B, 2 * ws[0].k, 2)
    s.synchronize()
    for a, b in zip(A, B):
        assert torch.equal(a, b)
    ens.close()


def test_ensemble_full_size_sampled_instances():
    """The 512-instance Brusselator ensemble (sizes 64..512, Neumann/periodic, FP32): 2 steps
    on the GPU; 4 sampled instances compared with the FP64 oracle."""
    from paper_2001_11220_gb300.api import EtdEnsemble
    ws = W.ensemble(ninst=512, steps=2)
    states = [torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float32) for w in ws]
    ens = EtdEnsemble(ws, "fp32")
    ens.run(states, 0.0, 2)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    for i in sorted(rng.choice(len(ws), 4, replace=False)):
        w = ws[i]
        ref = oracle.run(oracle_problem(w), W.initial_state(w), 0.0, 2)
        e = rel(states[i].double().cpu().numpy(), ref)
        print(f"ensemble instance {i} n={w.n} bc={w.bc}: FP32 error vs FP64 oracle {e:.3e}")
        assert e <= 2 * fp32_step_bound(w), (e, fp32_step_bound(w))
    ens.close()


def small_ensemble_3d(seed=3):
    """Five small 3D Brusselator instances of uneven, ragged shapes and mixed boundaries."""
    rng = np.random.default_rng(seed)
    shapes = [(9, 12, 17), (16, 16, 16), (20, 8, 11), (5, 7, 6), (24, 10, 13)]
    out = []
    for i, n in enumerate(shapes):
        a, b = float(rng.uniform(0.5, 2.0)), float(rng.uniform(1.5, 4.0))
        eps = float(rng.uniform(1e-3, 1e-2))
        bc = W.PERIODIC if i % 2 else W.NEUMANN
        out.append(W.Workload(f"e3d{i}", n, bc, (eps, 0.5 * eps), "brusselator", (a, b), 0.01, 3,
                              ic="normal", ic_args=((a, b / a), 0.1), seed=seed * 7919 + i))
    return out


def _run_ensemble(ws, prec, nsteps, env=None, t0=0.0):
    import os
    from paper_2001_11220_gb300.api import EtdEnsemble
    dt = torch.float64 if prec == "fp64" else torch.float32
    old = {k: os.environ.get(k) for k in (env or {})}
    os.environ.update(env or {})
    try:
        ens = EtdEnsemble(ws, prec)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    states = [torch.tensor(W.initial_state(w), device="cuda", dtype=dt) for w in ws]
    ens.run(states, t0, nsteps)
    torch.cuda.synchronize()
    info = ens.info()
    ens.close()
    return states, info


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim", [2, 3])
def test_persistent_step_is_one_launch_and_equals_per_sweep_launches(dim, prec):
    """The persistent step (one launch per step, work queue, completion counters)
    with the line tables on every instance gives the same states, bit for bit, as
    one launch per sweep kind; either work-list order (axis by axis, or instance
    groups interleaved) gives the same states; and the default persistent step,
    which solves periodic whole-chunk lines on the circulant factorisation,
    matches the oracle instance by instance."""
    ws = small_ensemble(10, seed=12) if dim == 2 else small_ensemble_3d()
    one, info1 = _run_ensemble(ws, prec, 3)
    tables, _ = _run_ensemble(ws, prec, 3, {"ETD_ENSEMBLE_CIRC": "0"})
    per_sweep, info2 = _run_ensemble(ws, prec, 3, {"ETD_ENSEMBLE_PERSISTENT": "0"})
    grouped, _ = _run_ensemble(ws, prec, 3, {"ETD_ENSEMBLE_WINDOW_MB": "0.001"})
    assert info1["launches_per_step"] == 1 and info2["launches_per_step"] == dim
    for w, a, b, c, d in zip(ws, one, per_sweep, grouped, tables):
        assert torch.equal(d, b), w.n
        assert torch.equal(a, c), w.n
    for w, U in zip(ws, one):
        ref = oracle.run(oracle_problem(w), W.initial_state(w), 0.0, 3)
        e = rel(U.double().cpu().numpy(), ref)
        assert e <= (FP64_TOL if prec == "fp64" else 3 * fp32_step_bound(w)), (w.n, e)


@pytest.mark.parametrize("dim", [2, 3])
def test_persistent_step_wait_runs_out_and_context_recovers(dim):
    """A dependency counter seeded so that it never reaches its target: the
    bounded wait runs out after the short limit, the call returns
    ETD_ERR_TIMEOUT naming the instance and axis, the counters are reset, and
    the next run on fresh states matches the oracle."""
    import time
    from paper_2001_11220_gb300 import _binding as B
    from paper_2001_11220_gb300.api import EtdEnsemble
    ws = small_ensemble(8, seed=4) if dim == 2 else small_ensemble_3d()
    ens = EtdEnsemble(ws, "fp64")
    ens.set_wait_limit(0.05)
    hold_axis = dim - 2
    ens.debug_hold(3, hold_axis)
    states = [torch.tensor(W.initial_state(w), device="cuda") for w in ws]
    t = time.perf_counter()
    with pytest.raises(B.EtdError) as ei:
        ens.run(states, 0.0, 3)
    waited = time.perf_counter() - t
    assert ei.value.status == B.ETD_ERR_TIMEOUT
    assert f"instance 3 axis {hold_axis + 1}" in str(ei.value), str(ei.value)
    assert waited < 5.0, waited
    with pytest.raises(B.EtdError) as bad:
        ens.set_wait_limit(0.0)
    assert bad.value.status == B.ETD_ERR_INVALID_ARG
    fresh = [torch.tensor(W.initial_state(w), device="cuda") for w in ws]
    ens.run(fresh, 0.0, 3)
    torch.cuda.synchronize()
    for w, U in zip(ws, fresh):
        ref = oracle.run(oracle_problem(w), W.initial_state(w), 0.0, 3)
        assert rel(U.cpu().numpy(), ref) <= FP64_TOL, w.n
    ens.close()
