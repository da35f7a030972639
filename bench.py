"""Benchmark of one ETD-RDP-IF step on GB300.

Headline workload: 2D Schnakenberg reaction-diffusion on the periodic unit
square, u_t = Lap u + 1000 (0.1 - u + u^2 v), v_t = 10 Lap v + 1000 (0.9 - u^2 v),
4096^2 nodes, 2 species, k = 1e-4, FP32 state and arithmetic (cyclic lines:
the circulant kernels, or the table kernels with Sherman-Morrison, whichever
the autotuner times faster).  A "step" is one full ETD-RDP-IF step: the two
fused axis sweeps (F(U_n), predictor, R_1/P_1 on x; P_2, F(U*), corrector
T_2/S_2 on y).  Metric: cell-species-steps/s, timed over K steps replayed from
one captured CUDA graph (the path etd_run gives users).

Beside it: the per-sweep event-timed run behind the roofline, the end-to-end
rate through etd_run_host (host buffer copied in and out every step), the 3D
manufactured 256^3 problem in FP32 and FP64 (speed-up at the accuracy each
reaches against the exact solution), the 3D Gray-Scott 256^3 forward and
checkpointed gradient, the 64^2 Brusselator in FP64 (microseconds per step),
the 512-instance ensemble, and the CPU oracle on the host cores.

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
P_HEAD = 4096      # headline grid: 4096^2 periodic Schnakenberg
P_3D = 256         # 3D manufactured and Gray-Scott grids


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
                 "etd_sweep_f32.cu", "etd_sweep_f64.cu", "etd_sweep_cluster.cu", "etd_circ.h", "etd_circ.cuh",
                 "etd_circ.cu", "etd_circ_rk_first.cu", "etd_circ_rk_strided.cu")


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
    wl = tab.get(workload, {})
    ent = wl.get(kernel)
    if not ent or ent.get("tile") != tile:   # captures of other tile shapes of the same kernel
        ent = wl.get(kernel + "_by_tile", {}).get(tile)
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
    P = oracle.Problem(n=w.n, bc=w.bc, D=w.D, reaction=w.reaction_id, params=w.params, k=w.k, length=w.length,
                          Dc=w.Dc)
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


def cpu_baselines(w, name):
    """The oracle on all host cores (3 steps of the full grid) and on one
    core (1 step): a bounded sample of the workload, about 15 s of CPU time."""
    v, dt, used = oracle_baseline(w, 3, host_cores())
    v1, dt1, _ = oracle_baseline(w, 1, 1)
    return {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"3 oracle steps of the full {name} grid (FP64, OpenMP over lines and points, "
                      f"{used} threads, {dt:.1f} s)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"1 oracle step of the full {name} grid (FP64, 1 thread, {dt1:.1f} s)"}}


def head_workload(W):
    return W.schnakenberg_2d(P_HEAD)


def workload_desc(w, precision):
    fb = w.npoints * (4 if precision == "fp32" else 8)
    return {"workload": f"schnakenberg2d_{P_HEAD}: 2D periodic Schnakenberg u_t = Lap u + 1000 (0.1 - u + u^2 v), "
                        f"v_t = 10 Lap v + 1000 (0.9 - u^2 v), {P_HEAD}^2 nodes, 2 species, k = 1e-4, "
                        f"IC (1, 0.9) + U(-1e-3, 1e-3)",
            "points": w.npoints, "species": w.nspecies, "precision": precision,
            "l2": f"inputs larger than L2: each sweep streams 4 fields of {2 * fb // 2**20} MB (2 species)"}


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


def tiles_of(info, dim):
    # tile shapes per axis in the ETD_TILES format (L:lines:kernel:pack), to reproduce in a profiler run
    return ",".join(f"{info['chunk'][a]}:{info['lines_per_block'][a]}:{info['staged'][a]}:{info['pack'][a]}"
                    for a in range(dim))


SWEEP_FIELDS = {0: 4, 1: 6, 2: 4}   # fields read + written per point: first, middle, last sweep


def sweep_roofline(ctx, U, w, nsteps, rb, peak, workload_key, tiles):
    """Per-sweep device times from a profiled run (CUDA events around every
    sweep launch on the context's stream) and their HBM rooflines."""
    import torch
    ctx.profile(True)
    ctx.profile_read()
    ctx.run(U, 0.0, nsteps)
    torch.cuda.synchronize()
    sweep_ms, sweep_n = ctx.profile_read()
    ctx.profile(False)
    names = {0: "sweep_first_x", 1: "sweep_middle_y", 2: "sweep_last_" + ("y" if w.dim == 2 else "z")}
    tl = tiles.split(",")
    out = {}
    for kind in range(3):
        if sweep_n[kind] == 0:
            continue
        t = sweep_ms[kind] / sweep_n[kind] / 1e3
        alg = SWEEP_FIELDS[kind] * w.nspecies * w.npoints * rb
        axis = {0: 0, 1: 1, 2: w.dim - 1}[kind]
        out[names[kind]] = {"ms": t * 1e3, "launches": sweep_n[kind], "algorithmic_bytes_per_launch": alg,
                            "achieved_gbs": alg / t / 1e9, "frac": alg / t / 1e9 / peak,
                            "traffic": _traffic(names[kind], workload_key, tl[axis])}
    return out, int(sum(sweep_n))


def extra_workloads(EtdRdpIf, W, stream, world, rank, barrier, peak, include_fp64=True):
    """The other benchmark problems (cell-species-steps/s, each a few
    device-timed steps replayed from a graph)."""
    import torch
    from paper_2001_11220_gb300.api import EtdEnsemble
    out = {}

    def mk(w, prec, tune=True):
        with torch.cuda.stream(stream):
            c = EtdRdpIf.from_workload(w, prec, stream=stream)
            U = torch.tensor(W.initial_state(w), device="cuda", dtype=c.dtype)
            if tune:
                c.autotune(U.clone())    # tile shapes per axis, timed on a scratch copy of the state
        return c, U

    # 3D manufactured 256^3 (Dirichlet, 1 species): FP32 and FP64 throughput, and
    # the accuracy each reaches at T = 1 (k = h, 257 steps) against the exact solution
    w = W.mms_3d(P_3D)
    res = {}
    for prec in ("fp32", "fp64") if include_fp64 else ("fp32",):
        c, U = mk(w, prec)
        rb = 4 if prec == "fp32" else 8
        nst = 20 if prec == "fp32" else 5
        ms = _timed(lambda: c.run(U, 0.0, nst), stream)
        tiles = tiles_of(c.info(), 3)
        per, _ = sweep_roofline(c, U, w, 3, rb, peak, f"mms3d_{P_3D}_{prec}", tiles)
        with torch.cuda.stream(stream):
            V = torch.tensor(W.initial_state(w), device="cuda", dtype=c.dtype)
        c.run(V, 0.0, w.steps)               # the whole run to T = 1
        torch.cuda.synchronize()
        exact = W.exact_mms(w, w.steps * w.k)
        err = float(abs(V.double().cpu().numpy() - exact).max() / abs(exact).max())
        res[prec] = {"value": w.npoints * nst / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / nst, "tiles": tiles,
                     "per_sweep": per, "err_vs_exact_at_T1": err,
                     "step_frac": c.info()["algorithmic_bytes"] / (ms / nst / 1e3) / 1e9 / peak}
        c.close()
        del U, V
    if include_fp64:
        res["speedup_fp32_over_fp64"] = res["fp32"]["value"] / res["fp64"]["value"]
        res["accuracy_note"] = ("error of the full run (T = 1, 257 steps, k = h = 1/257) against the exact "
                                "solution: the scheme's own error (second order in h) bounds both precisions")
    out[f"mms3d_{P_3D}"] = res
    # forward + adjoint (etd_grad over 20 steps, checkpoint every 10) on the manufactured problem
    c, U = mk(w, "fp32")
    T = U.clone()
    nst = 20
    ms = _timed(lambda: c.grad(U, 0.0, T, nst, 10), stream)
    out[f"mms3d_{P_3D}_fp32_fwd_adjoint"] = {"value": w.npoints * w.nspecies * nst / (ms / 1e3), "unit": UNIT,
                                             "ms_per_step": ms / nst, "steps": nst, "ckpt_every": 10}
    c.close()
    del U, T
    # 3D Gray-Scott periodic 256^3, 2 species, k = 1: forward and checkpointed gradient (ckpt 20)
    w = W.gray_scott_3d(P_3D, steps=20)
    c, U = mk(w, "fp32")
    tg = torch.tensor(W.initial_state(w, seed=2002), device="cuda", dtype=torch.float32)
    V = U.clone()
    msf = _timed(lambda: c.run(V, 0.0, 20), stream)
    tiles = tiles_of(c.info(), 3)
    per, _ = sweep_roofline(c, V, w, 3, 4, peak, f"grayscott3d_{P_3D}_fp32", tiles)
    msg = _timed(lambda: c.grad(U, 0.0, tg, 20, 20), stream)
    units = w.npoints * w.nspecies * 20
    alg = c.info()["algorithmic_bytes"]
    # reverse step (per step of the gradient, FP32, 2 species, N points; one checkpoint segment,
    # whose states and first/middle sweep outputs the forward pass keeps): ADJ_LAST (reads
    # Ubar', c_U, c_f, w; writes 3: 7 fields), ADJ_MIDDLE (3 adjoint + 3 forward fields read,
    # 3 written: 9), ADJ_FIRST (3 adjoint + U_n read, Ubar_n written: 5)
    rev_fields = 7 + 9 + 5
    fb = w.nspecies * w.npoints * 4
    # one adjoint step alone (etd_step_adjoint: the forward x and y sweeps of U_n, 4 + 6 fields,
    # then the three adjoint sweeps), CUDA events around the call
    ubar = torch.ones_like(U)
    msa = _timed(lambda: c.step_adjoint(U, 0.0, ubar), stream, reps=5)
    adj_fields = 4 + 6 + rev_fields
    # the full gradient run of the adjoint configuration: 200 steps, checkpoint every 20 (every
    # segment but the last is recomputed: 14 more fields per step for 9 of the 10 segments)
    ms200 = _timed(lambda: c.grad(U, 0.0, tg, 200, 20), stream)
    out[f"grayscott3d_{P_3D}_fp32"] = {
        "fwd": units / (msf / 1e3), "fwd_adjoint": units / (msg / 1e3), "unit": UNIT,
        "fwd_ms_per_step": msf / 20, "fwd_adjoint_ms_per_step": msg / 20, "tiles": tiles,
        "fwd_adjoint_over_fwd": msg / msf,
        "grad_200_steps_ckpt20_ms_per_step": ms200 / 200,
        "grad_200_steps_ckpt20_over_fwd": (ms200 / 200) / (msf / 20),
        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "per_sweep": per,
                     "fwd_step_frac": alg / (msf / 20 / 1e3) / 1e9 / peak,
                     "fwd_adjoint_algorithmic_bytes_per_step": alg + rev_fields * fb,
                     "fwd_adjoint_step_frac": (alg + rev_fields * fb) / (msg / 20 / 1e3) / 1e9 / peak,
                     "adjoint_step": {"ms": msa, "algorithmic_bytes": adj_fields * fb,
                                      "achieved_gbs": adj_fields * fb / (msa / 1e3) / 1e9,
                                      "frac": adj_fields * fb / (msa / 1e3) / 1e9 / peak,
                                      "note": "etd_step_adjoint: forward x, y sweeps of U_n (10 fields) + "
                                              "ADJ_LAST 7, ADJ_MIDDLE 9, ADJ_FIRST 5 fields"}}}
    c.close()
    del U, V, tg
    # 2D Brusselator 64^2 Neumann, FP64, 100 steps (T = 1): L2-resident, microseconds per step
    w = W.brusselator_2d()
    c, U = mk(w, "fp64", tune=False)
    ms = _timed(lambda: c.run(U, 0.0, w.steps), stream, reps=3)
    out["brusselator2d_64_fp64"] = {"value": w.npoints * w.nspecies * w.steps / (ms / 1e3), "unit": UNIT,
                                    "us_per_step": ms * 1e3 / w.steps, "steps": w.steps,
                                    "note": "whole 100-step run replayed from one graph; the state (64 KB) "
                                            "stays in L2, so the step is launch- and latency-bound"}
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
    cells = int(units_all) // 20
    out["ensemble512_brusselator_fp32"] = {"value": thr, "unit": UNIT, "ms_per_step": ms_max / 20,
                                           "instances": len(ws_all), "cell_species": cells,
                                           "step_frac": 8 * cells * 4 / (ms_max / 20 / 1e3) / 1e9 / peak,
                                           "scaling": "strong (instances sharded across ranks)"}
    ens.close()
    # Section 8's complex Ginzburg-Landau runs (alpha = 0, beta = 1.3, k = 1/20, T = 100, periodic,
    # Gaussian pulses): 2D [0,200]^2 at p = 400 and 3D [0,200]^3 at p = 200, FP32; the whole
    # 2000-step run time extrapolated from the timed steps, beside the paper's Fortran times
    # (Intel i7-4790, Table tableginz / tableginz2) as context
    for wcgl, nst, paper_s in ((W.cgl_2d(400), 200, {"fortran_1_thread_s": 86.66, "fortran_3_threads_s": 53.98,
                                                      "matlab_s": 95.65}),
                               (W.cgl_3d(200), 40, {"fortran_1_thread_s": 8260.91, "fortran_3_threads_s": 5287.64,
                                                    "matlab_s": 9673.13})):
        c, U = mk(wcgl, "fp32")
        ms = _timed(lambda: c.run(U, 0.0, nst), stream)
        out[f"{wcgl.name}_fp32"] = {"value": wcgl.npoints * wcgl.nspecies * nst / (ms / 1e3), "unit": UNIT,
                                    "ms_per_step": ms / nst,
                                    "full_run_s": ms / nst * wcgl.steps / 1e3, "steps_full_run": wcgl.steps,
                                    "tiles": tiles_of(c.info(), wcgl.dim),
                                    "step_frac": c.info()["algorithmic_bytes"] / (ms / nst / 1e3) / 1e9 / peak,
                                    "paper_cpu_context": paper_s}
        c.close()
        del U
    # coupled two-species diffusion (complex line kernels, etd_create_coupled): the same CGL runs
    # with alpha = 0.5 (D = 1 + 0.5 i), and Section 8's 2D Schrodinger run (p = 79, k = 0.0125,
    # T = 1, Neumann, FP64); per-sweep rooflines from profiled launches
    for wc, prec, nst in ((W.cgl_2d(400, alpha=0.5), "fp32", 200), (W.cgl_3d(200, alpha=0.5), "fp32", 40),
                          (W.nls_2d(), "fp64", 80)):
        c, U = mk(wc, prec, tune=False)
        rb = 4 if prec == "fp32" else 8
        ms = _timed(lambda: c.run(U, 0.0, nst), stream)
        tiles = tiles_of(c.info(), wc.dim)
        per, _ = sweep_roofline(c, U, wc, 2, rb, peak, f"{wc.name}_{prec}", tiles)
        out[f"{wc.name}_{prec}"] = {"value": wc.npoints * wc.nspecies * nst / (ms / 1e3), "unit": UNIT,
                                    "ms_per_step": ms / nst, "us_per_step": ms / nst * 1e3,
                                    "full_run_s": ms / nst * wc.steps / 1e3, "steps_full_run": wc.steps,
                                    "tiles": tiles, "kernel": "complex line kernel (staged = 6)",
                                    "step_frac": c.info()["algorithmic_bytes"] / (ms / nst / 1e3) / 1e9 / peak,
                                    "per_sweep": per}
        c.close()
        del U
    # Section 8's 1D Schrodinger soliton (d = 1, one fused sweep per step): the whole run, 10800
    # steps of 361 Neumann nodes in FP64, replayed from one graph
    import math
    import numpy as np
    x = -80.0 + 0.5 * np.arange(361)
    psi = math.sqrt(0.02) * np.exp(0.05j * x) / np.cosh(0.1 * x)
    with torch.cuda.stream(stream):
        c = EtdRdpIf((361,), (W.NEUMANN,), (1.0, 1.0), "nls", (0.0, -1.0, 0.0), 0.01, "fp64", (180.0,),
                     stream=stream, Dc=(0.0, -1.0, 1.0, 0.0))
        U = torch.tensor(np.stack([psi.real, psi.imag]), device="cuda", dtype=torch.float64)
    ms = _timed(lambda: c.run(U, 0.0, 10800), stream, reps=2)
    out["nls1d_361_fp64"] = {"value": 361 * 2 * 10800 / (ms / 1e3), "unit": UNIT, "us_per_step": ms * 1e3 / 10800,
                             "full_run_s": ms / 1e3, "steps_full_run": 10800,
                             "note": "one 361-node line: a single warp, latency-bound"}
    c.close()
    return out


def run_reference(args):
    """--impl reference: the CPU oracle, timed on the host cores on a bounded
    sample of the same workload (each 'step' = one oracle step of 4096^2)."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2001_11220_gb300 import workloads as W
    w = head_workload(W)
    # every timed "step" is one oracle step of the full grid on all host cores
    # (a few seconds); the run stops after K steps or a 60 s budget
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
                             "sample": f"{len(times)} oracle step(s) of the full {P_HEAD}^2 grid, FP64, "
                                       f"OpenMP over lines and points, {used} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
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

    w = head_workload(W)
    U0 = W.initial_state(w)
    stream = torch.cuda.Stream()
    units_per_step = w.npoints * w.nspecies
    rb = 4 if args.precision == "fp32" else 8
    peak, peak_src = _peaks()

    def barrier():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        ctx = EtdRdpIf.from_workload(w, args.precision, stream=stream)
        U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    if not args.no_autotune:
        with torch.cuda.stream(stream):
            Wk = U.clone()
        ctx.autotune(Wk)                      # tile shapes timed per axis on a scratch state
        del Wk
    info = ctx.info()
    tiles = tiles_of(info, w.dim)

    # ---- headline: K steps replayed from one captured CUDA graph (etd_run)
    ctx.run(U, 0.0, W_)                      # warm-up (untimed)
    ctx.run(U, W_ * w.k, K)                  # builds and caches the graph of this K-step run
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("etd_timed_steps")   # profilers can keep just these launches
        e0.record(stream)
        ctx.run(U, W_ * w.k, K)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    barrier()
    clocks = clk.summary()
    ms = e0.elapsed_time(e1)
    from paper_2001_11220_gb300.parallel import aggregate
    ms_max, _, value = aggregate(ms, units_per_step * K)   # max time over ranks, summed work
    launches = K * info["launches_per_step"]
    finite = bool(torch.isfinite(U).all())

    # ---- per-sweep roofline from a separate profiled run (direct launches, events per sweep)
    per, _ = sweep_roofline(ctx, U, w, min(K, 200), rb, peak, f"schnakenberg2d_{P_HEAD}_{args.precision}", tiles)
    dom = max(per, key=lambda k: per[k]["ms"])            # dominant kernel: longest sweep
    roof = {"bound": "hbm", "achieved": per[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": per[dom]["frac"], "traffic": per[dom]["traffic"], "kernel": dom,
            "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_bytes_per_launch": per[dom]["algorithmic_bytes_per_launch"],
            "per_sweep": per,
            "step_frac": (info["algorithmic_bytes"] / (ms_max / K / 1e3) / 1e9) / peak,
            "algorithmic_bytes_per_step": info["algorithmic_bytes"]}

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
    ctx.close()
    del U, Hst

    # ---- further workloads on this GPU (each a few device-timed steps)
    others = {} if args.no_extra else extra_workloads(EtdRdpIf, W, stream, world, rank, barrier, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(w, f"{P_HEAD}^2")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W_,
                "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": dict(workload_desc(w, args.precision), parallelism="replicas" if world > 1 else "single",
                               timed_path="etd_run: K steps replayed from one captured CUDA graph",
                               chunk=info["chunk"][:2], lines_per_block=info["lines_per_block"][:2],
                               staged=info["staged"][:2], grid_blocks=info["grid_blocks"][:2], tiles=tiles,
                               autotuned=not args.no_autotune, state_finite=finite),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes},
                "gpu_launches": launches, "clocks": clocks}
        line["workloads"] = others
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
