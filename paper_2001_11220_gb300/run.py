"""Run a named synthetic workload for a number of steps on cuda:0 (used for
profiling captures).

    python -m paper_2001_11220_gb300.run --workload mms3d --p 256 --precision fp32 --steps 4
    python -m paper_2001_11220_gb300.run --workload grayscott3d --p 256 --steps 2 --grad
      (--grad: the misfit gradient over the steps, one checkpoint segment)
    python -m paper_2001_11220_gb300.run --workload cgl3d --p 200 --alpha 0.5 --steps 2
      (complex Ginzburg-Landau; --alpha != 0 couples Re u and Im u: complex line kernels)
    python -m paper_2001_11220_gb300.run --workload nls2d --p 79 --precision fp64 --steps 80
    python -m paper_2001_11220_gb300.run --workload ensemble --p 512 --steps 3
      (the batched ensemble of --p instances, one persistent launch per step)
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def workload(name: str, p: int, alpha: float = 0.0):
    from paper_2001_11220_gb300 import workloads as W
    if name == "cgl2d":
        return W.cgl_2d(p, alpha=alpha)
    if name == "cgl3d":
        return W.cgl_3d(p, alpha=alpha)
    if name == "nls2d":
        return W.nls_2d(p)
    if name == "mms3d":
        return W.mms_3d(p)
    if name == "brusselator2d":
        return W.brusselator_2d(p)
    if name == "schnakenberg2d":
        return W.schnakenberg_2d(p)
    if name == "grayscott3d":
        return W.gray_scott_3d(p)
    raise SystemExit(f"unknown workload {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mms3d")
    ap.add_argument("--p", type=int, default=256)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--grad", action="store_true")
    ap.add_argument("--alpha", type=float, default=0.0)
    args = ap.parse_args()
    import torch

    from paper_2001_11220_gb300 import workloads as W
    from paper_2001_11220_gb300.api import EtdEnsemble, EtdRdpIf
    if args.workload == "ensemble":
        ws = W.ensemble(args.p, steps=args.steps)
        ens = EtdEnsemble(ws, args.precision)
        states = [torch.tensor(W.initial_state(x), device="cuda", dtype=ens.dtype) for x in ws]
        torch.cuda.synchronize()
        t = time.perf_counter()
        ens.run(states, 0.0, args.steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        ok = all(bool(torch.isfinite(U).all()) for U in states)
        print(f"ensemble of {args.p} instances {args.precision}: {args.steps} steps in {dt * 1e3:.2f} ms, "
              f"info {ens.info()}, finite={ok}")
        ens.close()
        return
    w = workload(args.workload, args.p, args.alpha)
    ctx = EtdRdpIf.from_workload(w, args.precision)          # default stream: direct launches
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=ctx.dtype)
    torch.cuda.synchronize()
    t = time.perf_counter()
    if args.grad:
        target = torch.tensor(W.initial_state(w.with_(seed=w.seed + 1)), device="cuda", dtype=ctx.dtype)
        ctx.grad(U, 0.0, target, args.steps, args.steps)
    else:
        for n in range(args.steps):
            ctx.step(U, n * w.k)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    print(f"{w.name} {args.precision}: {args.steps} steps in {dt * 1e3:.2f} ms, info {ctx.info()}, "
          f"finite={bool(torch.isfinite(U).all())}")
    ctx.close()


if __name__ == "__main__":
    main()
