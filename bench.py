"""Benchmark of one ETD-RDP-IF step on GB300.

Workload: 3D scalar Dirichlet problem u_t = Lap u - u/(1+u) + f(x,t) on the
unit cube, f manufactured so u = e^{-t} sin(pi x) sin(pi y) sin(pi z) is
exact, 256^3 interior nodes, k = h = 1/257, FP32 state and arithmetic (the
FP64 reference mode is timed beside it).  A "step" is one full ETD-RDP-IF
step: the three fused axis sweeps (F(U_n), predictor, R_1/P_1 on x; R_2/P_2 on
y; P_3, F(U*), corrector T_3/S_3 on z).  Metric: cell-species-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp32|fp64]

Under torchrun (N > 1) every rank advances its own independent replica of
the workload (the single-grid step has no exchange step: "replicas only"),
value = all ranks' cell-species-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ETD-RDP-IF cell-species-steps/s"
UNIT = "cell-species-steps/s"
P_BENCH = 256


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources that compile into the forward sweep kernels (their DRAM traffic
# depends on nothing else but the tile shapes, recorded beside each entry)
SWEEP_SOURCES = ("etd_internal.h", "etd_tables.h", "etd_sweep.cuh", "etd_sweep_smem.cuh", "etd_sweep_launch.cuh",
                 "etd_sweep_f32.cu", "etd_sweep_f64.cu", "etd_sweep_cluster.cu")


def _csrc_hash() -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2001_11220_gb300", "csrc")
    for fn in SWEEP_SOURCES:
        with open(os.path.join(cs, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str, tile: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel sources or that sweep's tile shape changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except Exception:
        return None
    ent = tab.get(workload, {}).get(kernel)
    if not ent or ent.get("csrc_hash") != _csrc_hash() or ent.get("tile") != tile:
        return None
    return float(ent["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"etd_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def oracle_baseline(w, sample_steps: int = 1, threads: int = 1):
    """Time the FP64 CPU oracle (as it stands) on a bounded sample of the
    workload: sample_steps steps of the full grid on `threads` host threads
    (OpenMP over the independent lines and points).  Returns (units/s,
    seconds, threads actually used)."""
    import oracle
    from paper_2001_11220_gb300 import workloads as W
    oracle.build()
    used = oracle.set_threads(threads)
    P = oracle.Problem(n=w.n, bc=w.bc, D=w.D, reaction=w.reaction_id, params=w.params, k=w.k, length=w.length)
    U0 = W.initial_state(w)
    t = time.perf_counter()
    oracle.run(P, U0, 0.0, sample_steps)
    dt = time.perf_counter() - t
    units = w.npoints * w.nspecies * sample_steps
    return units / dt, dt, used


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baselines(w):
    """The oracle on all host cores (3 steps of the full grid) and on one
    core (1 step), about 15 s of CPU time in all on a 16-core host."""
    v, dt, used = oracle_baseline(w, 3, host_cores())
    v1, dt1, _ = oracle_baseline(w, 1, 1)
    return {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"3 oracle steps of the full {P_BENCH}^3 grid (FP64, OpenMP over lines and points, "
                      f"{used} threads, {dt:.1f} s)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"1 oracle step of the full {P_BENCH}^3 grid (FP64, 1 thread, {dt1:.1f} s)"}}


def workload_desc(w, precision):
    return {"workload": f"mms3d_{P_BENCH}: 3D Dirichlet u_t = Lap u - u/(1+u) + f, {P_BENCH}^3 interior nodes, "
                        f"k = h = 1/{P_BENCH + 1}, manufactured u = e^-t sin sin sin",
            "points": w.npoints, "species": w.nspecies, "precision": precision,
            "l2": "inputs larger than L2: each sweep streams 4-6 fields of %d MB" % (w.npoints * (4 if precision == "fp32" else 8) // 2**20)}


def _timed(fn, stream, reps=1):
    """device time of fn() on stream (CUDA events), ms per call"""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_workloads(EtdRdpIf, W, stream, world, rank, barrier):
    """Throughput of the other benchmark problems (cell-species-steps/s):
    forward + adjoint (checkpointed gradient) on the main workload and on the
    256^3 periodic Gray-Scott problem, the 4096^2 periodic Schnakenberg step,
    and the 512-instance Brusselator ensemble."""
    import torch
    from paper_2001_11220_gb300.api import EtdEnsemble
    out = {}

    def mk(w, prec):
        with torch.cuda.stream(stream):
            c = EtdRdpIf.from_workload(w, prec, stream=stream)
            U = torch.tensor(W.initial_state(w), device="cuda", dtype=c.dtype)
            c.autotune(U.clone())    # tile shapes per axis, timed on a scratch copy of the state
        return c, U

    # forward + adjoint: etd_grad over 20 steps, checkpoint every 10 (main workload)
    w = W.mms_3d(P_BENCH)
    c, U = mk(w, "fp32")
    T = U.clone()
    nst = 20
    ms = _timed(lambda: c.grad(U, 0.0, T, nst, 10), stream)
    out["mms3d_256_fp32_fwd_adjoint"] = {"value": w.npoints * w.nspecies * nst / (ms / 1e3), "unit": UNIT,
                                         "ms_per_step": ms / nst, "steps": nst, "ckpt_every": 10}
    c.close()
    del U, T
    # 3D Gray-Scott periodic 256^3, 2 species, k = 1: forward and checkpointed gradient (ckpt 20)
    w = W.gray_scott_3d(256, steps=20)
    c, U = mk(w, "fp32")
    tg = torch.tensor(W.initial_state(w, seed=2002), device="cuda", dtype=torch.float32)
    V = U.clone()
    msf = _timed(lambda: c.run(V, 0.0, 20), stream)
    msg = _timed(lambda: c.grad(U, 0.0, tg, 20, 20), stream)
    units = w.npoints * w.nspecies * 20
    out["grayscott3d_256_fp32"] = {"fwd": units / (msf / 1e3), "fwd_adjoint": units / (msg / 1e3), "unit": UNIT,
                                   "fwd_ms_per_step": msf / 20, "fwd_adjoint_ms_per_step": msg / 20}
    c.close()
    del U, V, tg
    # 2D Schnakenberg periodic 4096^2 (cyclic lines, FP64 Sherman-Morrison scalar), FP32 state
    w = W.schnakenberg_2d(4096, steps=20)
    c, U = mk(w, "fp32")
    ms = _timed(lambda: c.run(U, 0.0, 20), stream)
    inf = c.info()
    tiles = [f"{inf['chunk'][a]}:{inf['lines_per_block'][a]}:{inf['staged'][a]}:{inf['pack'][a]}" for a in range(2)]
    # per-sweep device times (CUDA events around each sweep, a separate run) against the HBM peak
    c.profile(True)
    c.profile_read()
    c.run(U, 0.0, 20)
    torch.cuda.synchronize()
    sweep_ms, sweep_n = c.profile_read()
    c.profile(False)
    peak, _ = _peaks()
    fld = w.nspecies * w.npoints * 4
    per_sweep = {}
    for name, kind, a in (("sweep_first_x", 0, 0), ("sweep_last_y", 2, 1)):
        t = sweep_ms[kind] / max(1, sweep_n[kind]) / 1e3
        per_sweep[name] = {"ms": t * 1e3, "achieved_gbs": 4 * fld / t / 1e9, "frac": 4 * fld / t / 1e9 / peak,
                           "traffic": _traffic(name, "schnakenberg2d_4096_fp32", tiles[a])}
    out["schnakenberg2d_4096_fp32"] = {"value": w.npoints * w.nspecies * 20 / (ms / 1e3), "unit": UNIT,
                                       "ms_per_step": ms / 20, "tiles": ",".join(tiles),
                                       "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak,
                                                    "step_frac": inf["algorithmic_bytes"] / (ms / 20 / 1e3) / 1e9 / peak,
                                                    "algorithmic_bytes_per_step": inf["algorithmic_bytes"],
                                                    "per_sweep": per_sweep}}
    c.close()
    del U
    # batched ensemble: 512 Brusselator instances 64^2 .. 512^2, FP32, one launch per sweep
    from paper_2001_11220_gb300.parallel import aggregate, shard
    ws_all = W.ensemble(512, steps=20)
    ws = [ws_all[i] for i in shard(len(ws_all), world, rank)]   # instances are independent: shard by rank
    with torch.cuda.stream(stream):
        ens = EtdEnsemble(ws, "fp32", stream=stream)
        states = [torch.tensor(W.initial_state(x), device="cuda", dtype=torch.float32) for x in ws]
        ens.autotune([U.clone() for U in states])   # line-block shapes timed on scratch copies
    barrier()
    ms = _timed(lambda: ens.run(states, 0.0, 20), stream)
    units = sum(x.npoints * x.nspecies for x in ws) * 20
    ms_max, units_all, thr = aggregate(ms, units)
    out["ensemble512_brusselator_fp32"] = {"value": thr, "unit": UNIT, "ms_per_step": ms_max / 20,
                                           "instances": len(ws_all), "cell_species": int(units_all) // 20,
                                           "scaling": "strong (instances sharded across ranks)"}
    ens.close()
    return out


def run_reference(args):
    """--impl reference: the CPU oracle, timed on the host cores on a bounded
    sample of the same workload (each 'step' = one oracle step of 256^3)."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2001_11220_gb300 import workloads as W
    w = W.mms_3d(P_BENCH)
    # every timed "step" is one oracle step of the full grid on all host cores
    # (~10 s of CPU time); the run stops after K steps or a 60 s budget
    times = []
    cores = host_cores()
    while len(times) < max(1, args.steps) and sum(times) < 60.0:
        v, dt, used = oracle_baseline(w, 1, cores)
        times.append(dt)
    dt = sum(times)
    value = w.npoints * w.nspecies * len(times) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * dt / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{len(times)} oracle step(s) of the full {P_BENCH}^3 grid, FP64, "
                                       f"OpenMP over lines and points, {used} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2001_11220_gb300 import build as libbuild
    from paper_2001_11220_gb300 import workloads as W
    from paper_2001_11220_gb300.api import EtdRdpIf

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    libbuild.build()
    W_ = max(3, args.warmup)
    K = max(1, args.steps)

    w = W.mms_3d(P_BENCH)
    U0 = W.initial_state(w)
    stream = torch.cuda.Stream()
    units_per_step = w.npoints * w.nspecies

    def make(prec):
        with torch.cuda.stream(stream):
            ctx = EtdRdpIf.from_workload(w, prec, stream=stream)
            U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
        return ctx, U

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(ctx, U, K, profile, tag="etd_timed_steps"):
        # warm-up (untimed), then K steps between a barrier + synchronize on both sides
        ctx.run(U, 0.0, W_)
        torch.cuda.synchronize()
        if profile:
            ctx.profile(True)
            ctx.profile_read()
        barrier()
        torch.cuda.synchronize()
        if not profile:
            ctx.run(U, W_ * w.k, K)       # builds and caches the CUDA graph of this K-step run
            torch.cuda.synchronize()
            barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(tag)   # profilers can keep just these launches
        e0.record(stream)
        ctx.run(U, W_ * w.k, K)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        per = None
        if profile:
            per = ctx.profile_read()
            ctx.profile(False)
        return ms, per

    # ---- main measurement: FP32 (or --precision) with per-sweep events
    ctx, U = make(args.precision)
    if not args.no_autotune:
        with torch.cuda.stream(stream):
            Wk = U.clone()
        ctx.autotune(Wk)                      # tile shapes timed per axis on a scratch state
        del Wk
    info = ctx.info()
    # tile shapes per axis in the ETD_TILES format (L:lines:staged:pack), to reproduce in a profiler run
    tiles = ",".join(f"{info['chunk'][a]}:{info['lines_per_block'][a]}:{info['staged'][a]}:{info['pack'][a]}"
                     for a in range(w.dim))
    with ClockSampler(local) as clk:
        ms, per = timed(ctx, U, K, profile=True)
    clocks = clk.summary()
    from paper_2001_11220_gb300.parallel import aggregate, shard
    ms_max, _, value = aggregate(ms, units_per_step * K)   # max time over ranks, summed work

    # per-sweep roofline: dominant kernel = largest total device time
    kinds = ["sweep_first_x", "sweep_middle_y", "sweep_last_z"]
    sweep_ms, sweep_launches = per
    dom = max(range(3), key=lambda i: sweep_ms[i])
    rb = 4 if args.precision == "fp32" else 8
    fields = {0: 4, 1: 6, 2: 4}[dom]                       # fields read + written per point
    alg_bytes = fields * w.nspecies * w.npoints * rb       # per launch
    avg_s = sweep_ms[dom] / sweep_launches[dom] / 1e3
    achieved = alg_bytes / avg_s / 1e9
    peak, peak_src = _peaks()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic(kinds[dom], f"mms3d_{P_BENCH}_{args.precision}", tiles.split(",")[dom]),
            "kernel": kinds[dom], "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": alg_bytes,
            "per_sweep_ms": {kinds[i]: sweep_ms[i] / max(1, sweep_launches[i]) for i in range(3)},
            "step_frac": (info["algorithmic_bytes"] / (ms_max / K / 1e3) / 1e9) / peak}
    launches = int(sum(sweep_launches))

    # ---- FP64 reference mode (same workload), for the speedup at stated accuracy
    extra = {}
    if args.precision == "fp32":
        ctx64, U64 = make("fp64")
        if not args.no_autotune:
            with torch.cuda.stream(stream):
                Wk = U64.clone()
            ctx64.autotune(Wk)
            del Wk
        K64 = max(3, K // 5)
        ms64, _ = timed(ctx64, U64, K64, profile=False, tag="etd_timed_steps_fp64")
        v64 = units_per_step * K64 / (ms64 / 1e3)
        # accuracy of FP32 against the FP64 path (which matches the FP64 oracle) after 5 steps
        with torch.cuda.stream(stream):
            A = torch.tensor(U0, device="cuda", dtype=torch.float32)
            B64 = torch.tensor(U0, device="cuda", dtype=torch.float64)
        ctx.run(A, 0.0, 5)
        ctx64.run(B64, 0.0, 5)
        torch.cuda.synchronize()
        err = float((A.double() - B64).abs().max() / B64.abs().max())
        extra = {"fp64": {"value": v64, "ms_per_step": ms64 / K64},
                 "speedup_fp32_over_fp64": value / world / v64,
                 "fp32_rel_err_vs_fp64_after_5_steps": err}
        ctx64.close()
        del U64, B64

    # ---- end to end through the C ABI with a pinned host buffer, every step
    Hst = torch.tensor(U0, dtype=ctx.dtype).pin_memory()
    ctx.run_host(Hst, 0.0, 1)
    barrier()
    t0 = time.perf_counter()
    for n in range(args.e2e_steps):
        ctx.run_host(Hst, n * w.k, 1)
    t1 = time.perf_counter()
    e2e_t = torch.tensor([t1 - t0], device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_v = world * units_per_step * args.e2e_steps / float(e2e_t.item())
    state_bytes = info["state_bytes"]

    # ---- further workloads on this GPU (each a few device-timed steps)
    others = {} if args.no_extra else extra_workloads(EtdRdpIf, W, stream, world, rank, barrier)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W_,
                "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": dict(workload_desc(w, args.precision), parallelism="replicas" if world > 1 else "single",
                               chunk=info["chunk"][:3], lines_per_block=info["lines_per_block"][:3],
                               staged=info["staged"][:3], tiles=tiles, autotuned=not args.no_autotune),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes},
                "gpu_launches": launches, "clocks": clocks}
        line.update(extra)
        line["workloads"] = others
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
