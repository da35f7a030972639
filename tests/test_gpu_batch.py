"""Batched ensemble (one launch per sweep kind over many uneven instances)
against the FP64 oracle, instance by instance."""
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
