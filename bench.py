"""Benchmark of the FFT--HSS preconditioned GMRES hot path on one B300.

Workload (default): the 3D periodic 128^3 grid (2,097,152 nodes, 8.4M unknowns),
smooth synthetic field m = normalise((cos 2pi z sin 2pi x, sin 2pi z sin 2pi y,
cos 2pi x) + 1e-3 seeded noise), alpha = 0.1, h = (0, 0, 0.5), lambda = 0.5,
dt = 4x the explicit exchange limit, Crank--Nicolson-type midpoint steps with
Picard iteration, each linear solve by flexible GMRES(30) with the FFT--HSS
application and its inner matvec in FP32 and the Arnoldi process, least
squares, true residual and nodal update in FP64, rtol 1e-10.

One step = one midpoint time step (right-hand side, every Picard solve with all
its FFT--HSS applications and Arnoldi steps, the nodal update and the drift).
value = FFT--HSS applications per second over the timed steps (all ranks).
Also reported: the same system solved by all-FP64 FFT--HSS GMRES vs the FP32
flexible solve (ms per solve, same rtol), the isolated FP32 apply at 128^3 and
256^3 (applies/s and algorithmic GB/s), the dominant kernel class against its
roofline (timed live with CUDA events on the context's stream during the timed
steps), the oracle on the host cores, and an end-to-end figure through host
buffers.  Inputs (fields, the Krylov basis) are far larger than the 126 MB L2.

--impl reference runs the CPU oracle (the plain FP64 reference written from the
paper) on the same workload: each step is one oracle FFT--HSS application of the
128^3 field (radix-2 FFT mode), a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT-HSS applies/s + HBM GB/s; GMRES solve ms at 128^3, FP32-prec FGMRES vs FP64"
UNIT = "applies/s"
WORKLOAD = "llg-midpoint-3d-128: 128^3 periodic, smooth field, alpha 0.1, dt 4x explicit limit, FP32-flex FGMRES(30)"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6400.0, "fallback": True}


# DRAM traffic per launch of the dominant class (dram__bytes_read.sum + dram__bytes_write.sum),
# from one ncu capture of 90 arnoldi_pass launches of this workload at 128^3 (launches that
# returned at once left out); to be re-taken whenever the Arnoldi kernels change.
ARNOLDI_TRAFFIC_BYTES = 371.3e6
ARNOLDI_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum averaged over 90 non-empty "
                        "arnoldi_pass launches of this workload (exact-count kernels, fused reduction)")
# the same for the FP32-pair passes (gs_pass_staged), 90 launches of this workload
PAIR_TRAFFIC_BYTES = 392.5e6
PAIR_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum averaged over 90 gs_pass_staged "
                     "launches of this workload (profiles/gs_pass_staged_128cube_dram.md)")


def aggregate_over_ranks(dist, ms, counts, device):
    """Whole-job figures of N independent replicas: the timed region lasts as long as the
    slowest rank (MAX over ranks of the per-rank CUDA-event time), the work done is the SUM
    over ranks of each counter.  dist is torch.distributed (or None for one rank); device
    holds the reduction tensors ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None:
        return float(ms), {k: float(v) for k, v in counts.items()}
    import torch
    keys = sorted(counts)
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(counts[k]) for k in keys], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), {k: float(v) for k, v in zip(keys, c.tolist())}


def workload_params(n=128):
    import numpy as np
    alpha = 0.1
    sig_max = 3 * (math.pi * n) ** 2           # max |xi|^2 on the unit cube (Nyquist |k| = n/2)
    k_ex = 2 * alpha / ((1 + alpha ** 2) * sig_max)
    return dict(alpha=alpha, k=4 * k_ex, k_ex=k_ex, h=(0.0, 0.0, 0.5), lam=0.5, n=(n, n, n))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """Model name and logical core count of the host, for the CPU-baseline lines."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "host_cores": os.cpu_count()}


def _oracle_inputs_file(n):
    """The 128^3 workload's field and a saddle vector, written once to a temporary .npz so
    that worker processes load them instead of regenerating them."""
    import numpy as np
    from paper_2607_15290_b300 import inputs as I
    f = tempfile.NamedTemporaryFile(suffix=".npz", delete=False)
    f.close()
    np.savez(f.name, m=I.smooth3d(n), p=I.random_saddle_vector(n, seed=5))
    return f.name


def _oracle_apply_worker(path, n, prm_kw, warmup, count):
    """One single-threaded oracle process: `warmup` untimed then `count` timed FP64 FFT--HSS
    applications (radix-2 FFT mode).  Returns (wall-clock start, end) of the timed ones."""
    import numpy as np
    import oracle as O
    d = np.load(path)
    m, p = d["m"], d["p"]
    g = O.Grid(n)
    prm = O.Params(**prm_kw)
    O.set_transform(O.FFT)
    for _ in range(warmup):
        O.ffthss_apply(g, prm, m, p)
    t0 = time.time()
    for _ in range(count):
        O.ffthss_apply(g, prm, m, p)
    return t0, time.time()


def _oracle_processes():
    """Independent oracle processes to run at once: one per logical core, capped by the
    available host memory (about 0.7 GB per 128^3 process)."""
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable")) / 2 ** 20
        cores = max(1, min(cores, int(avail / 1.0)))
    except (OSError, StopIteration, ValueError):
        pass
    return cores


def oracle_apply_throughput(procs, warmup, count):
    """Oracle FFT--HSS applications/s with `procs` independent single-threaded processes
    (spawned), each doing `warmup` + `count` applications of the 128^3 field; the oracle's
    arithmetic is unchanged, the processes only run side by side.  Rate = procs * count /
    (last end - first start of the timed applications)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    w = workload_params()
    prm_kw = dict(alpha=w["alpha"], k=w["k"], theta=0.5, lam=w["lam"], h=w["h"])
    path = _oracle_inputs_file(w["n"])
    try:
        with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as pool:
            futs = [pool.submit(_oracle_apply_worker, path, w["n"], prm_kw, warmup, count) for _ in range(procs)]
            spans = [f.result() for f in futs]
    finally:
        os.unlink(path)
    t0 = min(a for a, _ in spans)
    t1 = max(b for _, b in spans)
    return procs * count / (t1 - t0), t1 - t0


def oracle_baseline(iters_per_solve=None, solves_per_step=None, seconds=10.0):
    """The oracle as it stands on the host cores, on bounded samples of the 128^3 workload:
      * single thread: FP64 FFT--HSS applications (radix-2 FFT mode) for ~`seconds`, and one
        saddle matvec;
      * all cores: one independent single-threaded oracle process per core (memory allowing),
        two applications each after one untimed;
      * one GMRES solve and one midpoint step, extrapolated from the single-thread apply and
        matvec times with the GPU run's iterations per solve and solves per step (each
        oracle GMRES iteration is one matvec and one application; the initial and final
        residuals add two more of each; the Gram--Schmidt work is left out, so these are
        lower bounds).  A full oracle solve at this size takes about a minute or more,
        which does not fit a bounded sample."""
    import oracle as O
    from paper_2607_15290_b300 import inputs as I
    w = workload_params()
    g = O.Grid(w["n"])
    prm = O.Params(alpha=w["alpha"], k=w["k"], theta=0.5, lam=w["lam"], h=w["h"])
    m = I.smooth3d(w["n"])
    p = I.random_saddle_vector(w["n"], seed=5)
    O.set_transform(O.FFT)
    O.ffthss_apply(g, prm, m, p)
    t0 = time.perf_counter()
    count = 0
    while True:
        O.ffthss_apply(g, prm, m, p)
        count += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    O.saddle_apply(g, prm, m, p)
    matvec_s = time.perf_counter() - t1
    O.set_transform(O.DFT)
    apply_s = dt / count
    procs = _oracle_processes()
    rate_all, span = oracle_apply_throughput(procs, 1, 2)
    out = {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle",
           "sample": f"{procs} independent single-threaded oracle processes, 2 FP64 FFT-HSS applications each "
                     f"of the 128^3 field (radix-2 FFT mode) after 1 untimed, {span:.1f} s",
           "single_thread": {"value": count / dt, "unit": UNIT, "cores": 1,
                             "sample": f"{count} applications in {dt:.1f} s",
                             "apply_s": apply_s, "saddle_matvec_s": matvec_s},
           **host_cpu()}
    if iters_per_solve is not None:
        solve_s = (iters_per_solve + 2) * (apply_s + matvec_s)
        out["single_thread"]["solve_s_extrapolated"] = solve_s
        out["single_thread"]["extrapolation"] = (
            f"(iterations per solve {iters_per_solve:.2f} + 2) x (apply + matvec), Gram-Schmidt left out: lower bound")
        if solves_per_step is not None:
            out["single_thread"]["step_s_extrapolated"] = solve_s * solves_per_step
            out["single_thread"]["solves_per_step"] = solves_per_step
    return out


def run_reference(args):
    """The oracle on the host cores as the reference arm: each step is one FP64 FFT--HSS
    application of the 128^3 field in every one of `procs` independent single-threaded
    oracle processes (one per core, memory allowing); value = applications/s of all of them."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = _oracle_processes()
    value, span = oracle_apply_throughput(procs, args.warmup, args.steps)
    sample = (f"{procs} independent single-threaded oracle processes, {args.steps} FP64 FFT-HSS applications "
              f"each of the 128^3 field (radix-2 FFT mode) after {args.warmup} untimed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": span / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "reference_step": f"one oracle FFT-HSS apply in each of {procs} processes"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                            **host_cpu()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def dtype_string(gs, ch):
    """the arithmetic the timed step computes in"""
    import paper_2607_15290_b300 as L
    parts = ["FP32 FFT-HSS + inner matvec"]
    if gs == L.GS_F32X2:
        parts.append("Gram-Schmidt in FP32-pair arithmetic on a basis whose first vector is FP64 and later ones FP32 pairs")
    else:
        parts.append("FP64 Gram-Schmidt")
    if ch == L.CHAIN_F32X2:
        parts.append("true residuals and right-hand side through FP32-pair Fourier chains (FP64 in and out)")
    else:
        parts.append("FP64 true residuals and right-hand side")
    parts.append("FP64 least squares and update")
    return "f32+f64 (" + "; ".join(parts) + ")"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--roofline-class", default="arnoldi", choices=["xfwd", "axis", "xinv", "arnoldi"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison and apply sweep legs")
    ap.add_argument("--apply-sweep", default="", help="only time the isolated FFT-HSS apply on these grids, "
                    "e.g. '256^3,128^3,1024^2' (one JSON line each, with a per-pass breakdown)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "matvec-fp64", "matvec-f32x2"],
                    help="what --apply-sweep times: the FFT-HSS apply (FP32 or FP64), or the saddle matvec with "
                         "an FP64 or an FP32-pair Fourier chain")
    ap.add_argument("--no-autotune", action="store_true",
                    help="--apply-sweep with the default launch shapes (for profiling the passes alone)")
    ap.add_argument("--ensemble", action="store_true", help="only the 96-problem batched ensemble (5 Euler steps)")
    ap.add_argument("--adjoint", action="store_true", help="only the 512^2 adjoint timing (16 midpoint steps)")
    ap.add_argument("--precond-compare", action="store_true",
                    help="only the comparison of preconditioners and the shift sweep on the one-step Euler "
                         "system with the manufactured right-hand side (2D)")
    ap.add_argument("--mesh-study", action="store_true",
                    help="only the random right-hand-side mesh study (fixed k vs bounded stiffness, 2D)")
    ap.add_argument("--midpoint-2d", action="store_true",
                    help="only the 1024^2 FP64 midpoint workload (20 steps, smooth and broadband fields): "
                         "iterations per solve, nodal drift, dissipation residual")
    ap.add_argument("--gs-arith", default="f32x2", choices=["fp64", "f32x2"],
                    help="arithmetic of the flexible solves' Gram-Schmidt passes: FP32 pairs on a "
                         "planar-pair basis (default) or FP64 multiply-adds")
    ap.add_argument("--chain-arith", default="f32x2", choices=["fp64", "f32x2"],
                    help="arithmetic of the FP64-accurate Fourier chains (true residuals, right-hand side): "
                         "FP32 pairs (default) or FP64")
    ap.add_argument("--axis-shapes", default="",
                    help="skip the autotuner and set the FP32 axis-pass shapes, e.g. "
                         "'y-forward=register(E8,TW16);z=tma(TW8);y-inverse=register(E8,TW16)'")
    ap.add_argument("--pass-plan", default="five", choices=["five", "cluster"],
                    help="3D FP32 round trips: five HBM passes, or x/y transforms in one cluster per plane")
    ap.add_argument("--n", type=int, default=128,
                    help="grid points per axis of the midpoint workload (128; smaller only for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_sweep:
        return apply_sweep(args)
    if args.ensemble:
        return ensemble_leg(args)
    if args.adjoint:
        return adjoint_leg(args)
    if args.precond_compare:
        return precond_compare_leg(args)
    if args.mesh_study:
        return mesh_study_leg(args)
    if args.midpoint_2d:
        return midpoint_2d_leg(args)

    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = workload_params(args.n)
    n = w["n"]
    N = n[0] * n[1] * n[2]
    ctx = L.Context(n)
    prm = L.Params(alpha=w["alpha"], k=w["k"], theta=0.5, lam=w["lam"], h_ext=w["h"])
    gs = L.GS_F32X2 if args.gs_arith == "f32x2" else L.GS_FP64
    ch = L.CHAIN_F32X2 if args.chain_arith == "f32x2" else L.CHAIN_FP64
    opts = L.Opts(restart=30, rtol=1e-10, precision=L.PREC_FP32_FLEX, picard_tol=1e-10, picard_max=50, gs_arith=gs,
                  chain_arith=ch)
    ctx.set_pass_plan(L.PLAN_CLUSTER if args.pass_plan == "cluster" else L.PLAN_FIVE)
    if args.axis_shapes:
        # shapes a live run picked, replayed (a profiler distorts the tuner's timings)
        for item in args.axis_shapes.split(";"):
            slot, shape = item.split("=")
            ctx.set_axis_shape(slot.strip(), shape.strip())
        tuning = "fixed FP32 shapes: " + args.axis_shapes
    else:
        tuning = ctx.autotune()       # launch shapes of the axis passes, picked on this device
    m0 = torch.tensor(I.smooth3d(n), device="cuda")
    x = ctx.empty(4)
    mA, mB = m0.clone(), ctx.empty(3)
    stream = ctx.stream

    def step(m_in, m_out, vprev):
        _, _, info = L.llg_step_midpoint(ctx, prm, opts, m_in, vprev, m_out, x)
        return info

    vprev = None
    for _ in range(args.warmup):
        step(mA, mB, vprev)
        vprev = x[:3].clone()
        mA, mB = mB, mA

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # the timed trajectory's starting state, kept in pinned host memory for the end-to-end leg
    start_m = mA.cpu().pin_memory()
    start_v = vprev.cpu().pin_memory()

    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launches()
    barrier()
    clocks.start()
    ctx.profile_begin(args.roofline_class)
    ev0.record(stream)
    applies = solves = iters = 0
    drift = 0.0
    for _ in range(args.steps):
        info = step(mA, mB, vprev)
        applies += info["applies"]
        solves += info["picard_iters"]
        iters += info["iters"]
        drift = max(drift, info["max_len_drift"])
        vprev = x[:3].clone()
        mA, mB = mB, mA
    ev1.record(stream)
    barrier()
    prof = ctx.profile_end()
    clk = clocks.stop()
    gpu_launches = ctx.launches() - l0
    ms = ev0.elapsed_time(ev1)
    ms, totals = aggregate_over_ranks(dist, ms, {"applies": applies, "solves": solves, "steps": args.steps},
                                      "cuda")
    value = totals["applies"] / (ms / 1e3)

    extras = {}
    pk = peaks()
    e2e = end_to_end(L, ctx, prm, opts, start_m, start_v, args.steps)
    if not args.no_extras and rank == 0:
        extras = extras_leg(L, I, ctx, prm, w, m0, args, gs)
    fp64_peak = ctx.probe_fma_rate(True)
    fp32_peak = ctx.probe_fma_rate(False)

    # roofline of the profiled (dominant) kernel class
    avg_ms = prof["ms"] / max(prof["launches"], 1)
    if args.roofline_class == "arnoldi" and gs == L.GS_F32X2:
        # FP32-pair passes: the FP64 unit is no longer the bound; the basis reads are
        achieved = prof["bytes"] / (prof["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": PAIR_TRAFFIC_BYTES if args.n == 128 else None,
                "traffic_note": PAIR_TRAFFIC_NOTE,
                "algorithmic_bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                "kernel": "gs_pass_staged (CGS2 multi-dot/update, FP32-pair arithmetic on a planar-pair basis, "
                          "operands staged in shared memory by bulk copies)",
                "launches": prof["launches"], "avg_launch_ms": avg_ms,
                "fp64_equivalent_tflops": prof["flops"] / (prof["ms"] / 1e3) / 1e12,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" + (" (fallback)" if pk.get("fallback") else "")}
    elif args.roofline_class == "arnoldi":
        achieved = prof["flops"] / (prof["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": ARNOLDI_TRAFFIC_BYTES if args.n == 128 else None,
                "traffic_note": ARNOLDI_TRAFFIC_NOTE, "algorithmic_bytes_per_launch": prof["bytes"] / max(prof["launches"], 1),
                "kernel": "arnoldi_pass (FP64 CGS2 multi-dot/update)", "launches": prof["launches"],
                "avg_launch_ms": avg_ms, "hbm_gbs_at_algorithmic_bytes": prof["bytes"] / (prof["ms"] / 1e3) / 1e9,
                "peak_source": "FP64 FMA rate measured live on this device (llg_probe_fma_rate); nominal 1.25"}
    else:
        achieved = prof["bytes"] / (prof["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": args.roofline_class,
                "launches": prof["launches"], "avg_launch_ms": avg_ms,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" + (" (fallback)" if pk.get("fallback") else "")}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_string(gs, ch),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(n), "nodes": N, "unknowns": 4 * N, "alpha": w["alpha"],
                   "dt": w["k"], "dt_over_explicit_limit": 4.0, "lambda": w["lam"], "h_ext": list(w["h"]),
                   "restart": 30, "rtol": 1e-10, "picard_tol": 1e-10, "gram_schmidt": args.gs_arith,
                   "fp64_accurate_chains": args.chain_arith,
                   "pass_plan": args.pass_plan,
                   "l2": "inputs larger than L2 (fields 50-67 MB each, Krylov basis ~2 GB)",
                   "parallelism": f"replicas x{world} (independent problems, no collective)"},
        "solves_per_s": totals["solves"] / (ms / 1e3), "steps_per_s": totals["steps"] / (ms / 1e3),
        "gmres_iters_per_solve": iters / max(solves, 1), "max_len_drift": drift,
        "roofline": roof, "gpu_launches": gpu_launches, "clocks": clk, "e2e": e2e,
        "fp64_fma_tflops_measured": fp64_peak, "fp32_fma_tflops_measured": fp32_peak,
        "autotune": tuning.strip().splitlines(),
    }
    out.update(extras)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = oracle_baseline(iters / max(solves, 1), totals["solves"] / totals["steps"])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def end_to_end(L, ctx, prm, opts, start_m, start_v, steps, chunks=8):
    """The timed trajectory again, from the same starting state, through host buffers: every
    step copies m^n and v^{n-1/2} from pinned host memory to the device, runs the midpoint
    step through the C ABI and copies m^{n+1} and v^{n+1/2} back to the same host buffers,
    which feed the next step.  Same steps, same warm start, same work per step as the timed
    region, so ms_per_step compares directly; the copies are inside the timed region.

    The round trip between two steps is pipelined over `chunks` pieces of each array on two
    streams: piece k goes device -> host while piece k-1 goes host -> device (the host link is
    full duplex), every piece's upload waiting for its own download."""
    import torch
    mh = start_m.clone().pin_memory()
    vh = start_v.clone().pin_memory()
    md, vd, mo, xx = ctx.empty(3), ctx.empty(3), ctx.empty(3), ctx.empty(4)
    stream = ctx.stream
    s_down, s_up = torch.cuda.Stream(), torch.cuda.Stream()

    def pieces(t):
        flat = t.reshape(-1)
        step = -(-flat.numel() // chunks)
        return [flat[i:i + step] for i in range(0, flat.numel(), step)]

    applies = 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    with torch.cuda.stream(stream):
        md.copy_(mh, non_blocking=True)
        vd.copy_(vh, non_blocking=True)
    for it in range(steps):
        _, _, info = L.llg_step_midpoint(ctx, prm, opts, md, vd, mo, xx)
        applies += info["applies"]
        done = torch.cuda.Event()
        done.record(stream)
        s_down.wait_event(done)
        s_up.wait_event(done)
        last = it == steps - 1
        ups = []
        with torch.cuda.stream(s_down):
            # v^{n+1/2} is the velocity part of x (its first three planes, contiguous)
            down = list(zip(pieces(mh), pieces(mo))) + list(zip(pieces(vh), pieces(xx[:3])))
            for h, d in down:
                h.copy_(d, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_down)
                ups.append(ev)
        if not last:
            with torch.cuda.stream(s_up):
                up = list(zip(pieces(md), pieces(mh))) + list(zip(pieces(vd), pieces(vh)))
                for (d, h), ev in zip(up, ups):
                    s_up.wait_event(ev)
                    d.copy_(h, non_blocking=True)
            stream.wait_stream(s_up)
        stream.wait_stream(s_down)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - w0) * 1e3
    t = e0.elapsed_time(e1)
    return {"value": applies / (t / 1e3), "unit": UNIT, "h2d_bytes_per_step": (mh.numel() + vh.numel()) * 8,
            "d2h_bytes_per_step": (mh.numel() + vh.numel()) * 8, "steps": steps, "ms_per_step": t / steps,
            "wall_ms_per_step": wall / steps, "applies_per_step": applies / steps,
            "note": "the timed trajectory from its starting state, with m^n and v^{n-1/2} copied in from pinned "
                    "host memory and m^{n+1}, v^{n+1/2} copied back every step (the round trip pipelined in "
                    f"{chunks} pieces per array on two streams, downloads and uploads overlapping)"}


def cufft_apply_compare(L, I, ctx, prm, nn, ours_ms):
    """Comparison point: the same FP32 FFT-HSS apply with cuFFT (torch.fft R2C/C2R over the
    three velocity components) for Algorithm 1's transforms and PyTorch elementwise kernels
    for the symbol division and the closed-form nodal inverse (unfused).  Checked against
    the library's apply on the same inputs, then timed with CUDA events."""
    import numpy as np
    import torch
    nx, ny, nz = nn
    N = nx * ny * nz
    two_pi = 2.0 * np.pi
    fz = torch.fft.fftfreq(nz, d=1.0 / nz, device="cuda", dtype=torch.float64) * two_pi
    fy = torch.fft.fftfreq(ny, d=1.0 / ny, device="cuda", dtype=torch.float64) * two_pi
    fx = torch.fft.rfftfreq(nx, d=1.0 / nx, device="cuda", dtype=torch.float64) * two_pi
    sigma = fz[:, None, None] ** 2 + fy[None, :, None] ** 2 + fx[None, None, :] ** 2
    chat = (1.0 + prm.alpha ** 2) * prm.c_ex
    inv = (1.0 / (prm.alpha + prm.theta * prm.k * chat * sigma + prm.lam)).to(torch.float32)
    lam = float(prm.lam)
    m = torch.tensor(I.smooth3d(nn), device="cuda").float()
    p = torch.randn((4, nz, ny, nx), device="cuda", dtype=torch.float32)

    def apply():
        w = torch.fft.irfftn(torch.fft.rfftn(p[:3], dim=(1, 2, 3)) * inv, s=(nz, ny, nx), dim=(1, 2, 3))
        q4 = p[3] / lam
        d = 1.0 / (lam * lam + (m * m).sum(0))
        z = torch.empty_like(p)
        z[:3] = (lam * w - torch.linalg.cross(m, w, dim=0) - m * q4) * d
        z[3] = (lam * q4 + (m * w).sum(0)) * d
        return z

    ref = L.llg_ffthss_apply_f32(ctx, prm, m, p)
    torch.cuda.synchronize()
    diff = float((apply() - ref).abs().max() / ref.abs().max())
    for _ in range(3):
        apply()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        apply()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"ms": ms, "applies_per_s": 1e3 / ms, "ours_ms": ours_ms, "ours_speedup": ms / ours_ms,
            "max_rel_diff_vs_ours": diff, "what": "torch.fft (cuFFT) R2C/C2R + unfused PyTorch elementwise nodal inverse"}


def extras_leg(L, I, ctx, prm, w, m0, args, gs):
    """FP32-flexible vs all-FP64 solve of one identical system and the isolated apply sweep.
    Runs after the timed region."""
    import torch
    ex = {}
    n = w["n"]
    stream = ctx.stream

    def events_ms(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # the first Picard system of a midpoint step from m0: A(m0; theta=1/2) x = b
    b = ctx.empty(4)
    x0 = ctx.empty(4)
    L.llg_step_midpoint(ctx, prm, L.Opts(picard_max=1, rtol=1e-3), m0, None, ctx.empty(3), x0,
                        raise_on_error=False)
    # right-hand side of that system: b = A x0 (a consistent system with a known solution)
    L.llg_saddle_apply(ctx, prm, m0, x0, out=b)
    res = {}
    for name, prec in (("fp32flex", L.PREC_FP32_FLEX), ("fp64", L.PREC_FP64)):
        o = L.Opts(restart=30, rtol=1e-10, precision=prec, gs_arith=gs)
        times, its, rr, err = [], 0, 0.0, 0.0
        for rep in range(4):
            x = torch.zeros_like(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            x, info = L.llg_gmres_solve(ctx, prm, o, m0, b, x)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
            its, rr = info["iters"], info["rel_res_true"]
            err = float((x - x0).abs().max() / x0.abs().max())
        times.sort()
        res[name] = {"ms": times[len(times) // 2], "iters": its, "rel_res_true": rr, "rel_err_vs_known_x": err}
    ex["solve_128"] = res
    ex["solve_ms_fp32flex"] = res["fp32flex"]["ms"]
    ex["solve_ms_fp64"] = res["fp64"]["ms"]
    ex["speedup_fp32flex_vs_fp64"] = res["fp64"]["ms"] / res["fp32flex"]["ms"]

    # isolated FP32 FFT-HSS apply: 128^3 (this context) and 256^3
    def apply_rate(c2, nn):
        N = nn[0] * nn[1] * nn[2]
        c2.autotune(fp64=False, fp32=True)
        mm = torch.tensor(I.smooth3d(nn), device="cuda").float()
        p = torch.randn((4,) + tuple(reversed(nn)), device="cuda", dtype=torch.float32)
        z = torch.empty_like(p)
        t = events_ms(lambda: L.llg_ffthss_apply_f32(c2, prm, mm, p, out=z), 20)
        algo = (11 + 24) * 4 * N        # inputs v, r, m + output z, and the 5-pass plan's 4 spectral passes
        floor = 11 * 4 * N
        return {"ms": t, "applies_per_s": 1e3 / t, "gbs_algorithmic_5pass": algo / t / 1e6,
                "gbs_io_floor": floor / t / 1e6}
    ex["apply_fp32_128"] = apply_rate(ctx, n)
    c256 = L.Context((256, 256, 256))
    ex["apply_fp32_256"] = apply_rate(c256, (256, 256, 256))
    ex["cufft_apply_fp32"] = {"128": cufft_apply_compare(L, I, ctx, prm, n, ex["apply_fp32_128"]["ms"]),
                              "256": cufft_apply_compare(L, I, c256, prm, (256, 256, 256), ex["apply_fp32_256"]["ms"])}
    c256.close()
    torch.cuda.empty_cache()

    return ex


def apply_sweep(args):
    """Isolated FFT-HSS apply (FP32 or FP64) per grid: time per apply (CUDA events over
    args.steps applies after args.warmup), algorithmic bytes of the pass plan, and the same
    split by pass class from the library's live per-launch timing."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    pk = peaks()
    for spec in args.apply_sweep.split(","):
        base, dim = spec.split("^")
        n = (int(base),) * int(dim)
        N = int(np.prod(n))
        ctx = L.Context(n)
        ctx.set_pass_plan(L.PLAN_CLUSTER if args.pass_plan == "cluster" else L.PLAN_FIVE)
        f32 = args.precision == "fp32"
        if args.axis_shapes:
            for item in args.axis_shapes.split(";"):
                slot, shape = item.split("=")
                ctx.set_axis_shape(slot.strip(), shape.strip())
            tuning = "fixed FP32 shapes: " + args.axis_shapes
        else:
            tuning = "" if args.no_autotune else ctx.autotune(fp64=not f32, fp32=f32)
        dt = torch.float32 if f32 else torch.float64
        m = torch.tensor(I.smooth3d(n) if len(n) == 3 else I.smooth2d(n), device="cuda").to(dt)
        p = torch.randn((4,) + tuple(reversed(n)), device="cuda", dtype=dt)
        z = torch.empty_like(p)
        prm = L.Params(alpha=0.1, k=workload_params(max(n))["k"], theta=0.5, lam=0.5)
        fn = {"fp32": lambda: L.llg_ffthss_apply_f32(ctx, prm, m, p, out=z),
              "fp64": lambda: L.llg_ffthss_apply(ctx, prm, m, p, out=z),
              "matvec-fp64": lambda: L.llg_saddle_apply(ctx, prm, m, p, out=z),
              "matvec-f32x2": lambda: L.llg_saddle_apply_f32x2(ctx, prm, m, p, out=z)}[args.precision]
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(args.steps):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        w = 4 if f32 else 8
        # the cluster plan's grids (128^2 and 256^2 planes) make three passes of the FP32 apply
        passes = 3 if len(n) == 2 or (args.pass_plan == "cluster" and f32 and n[0] == n[1] and n[0] in (128, 256)) else 5
        # nodal words: the apply reads v (3), then m and r (3 + 1) and writes z (4); the matvec
        # reads v (3), then m and x (3 + 4) and writes y (4); every spectral pass reads and
        # writes 3 words a node
        nodal = 14 if args.precision.startswith("matvec") else 11
        algo = (nodal + 6 * (passes - 1)) * w * N
        out = {"grid": list(n), "precision": args.precision, "ms_per_apply": ms, "applies_per_s": 1e3 / ms,
               "gbs_algorithmic": algo / ms / 1e6, "frac_of_hbm": algo / ms / 1e6 / pk["hbm_gbs"],
               "algorithmic_bytes": algo, "passes": passes, "autotune": tuning.strip().splitlines()}
        for cls in ("xfwd", "axis", "xinv"):
            ctx.profile_begin(cls)
            for _ in range(args.steps):
                fn()
            r = ctx.profile_end()
            out[cls] = {"ms_per_apply": r["ms"] / args.steps, "launches_per_apply": r["launches"] / args.steps,
                        "gbs": r["bytes"] / (r["ms"] / 1e3) / 1e9 if r["ms"] else None,
                        "gflops": r["flops"] / (r["ms"] / 1e3) / 1e9 if r["ms"] else None}
        print(json.dumps(out), flush=True)
        ctx.close()
        del m, p, z
        torch.cuda.empty_cache()


def precond_compare_leg(args):
    """One projected-Euler step (k = 1e-2, alpha = 0.2, GMRES(50), rtol 1e-8) from the
    manufactured solution at t = 0 with its forcing at t = k, on (0, 2 pi)^2: GMRES iterations
    and median solve time (3 runs after one warm-up, CUDA events) for the split FFT-HSS, the
    shifted symmetric part and no preconditioner, N = 32 ... 1024; then the shift sweep
    lambda = 2^-3 ... 2^4 for N = 64, 128, 256.  The paper's counts and CPU times are quoted
    as context (its hardware, its SciPy GMRES)."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    alpha, k = 0.2, 1e-2
    names = {L.PC_FFTHSS: "ffthss", L.PC_HERMITIAN: "symmetric_part", L.PC_NONE: "none"}
    paper = {"ffthss": {32: 11, 64: 11, 128: 11, 256: 11}, "symmetric_part": {n: 18 for n in (32, 64, 128, 256)},
             "none": {32: 22, 256: 175}}

    def step(ctx, m, f, lam, pc, reps):
        prm = L.Params(alpha=alpha, k=k, lam=lam, h_field=f)
        opts = L.Opts(restart=50, rtol=1e-8, max_iters=20000, preconditioner=pc)
        times, info = [], None
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(ctx.stream)
            _, _, info = L.llg_step_euler(ctx, prm, opts, m)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            if r > 0:
                times.append(e0.elapsed_time(e1))
        times.sort()
        return info["iters"], times[len(times) // 2]

    rows = []
    for N in (32, 64, 128, 256, 512, 1024):
        n = (N, N)
        ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
        m0, _ = I.manufactured2d(n, 0.0, alpha)
        _, f0 = I.manufactured2d(n, k, alpha)
        m, f = torch.tensor(m0, device="cuda"), torch.tensor(f0, device="cuda")
        row = {"N": N}
        for pc in (L.PC_FFTHSS, L.PC_HERMITIAN, L.PC_NONE):
            its, ms = step(ctx, m, f, 0.5, pc, 1 if (pc == L.PC_NONE and N >= 512) else 3)
            row[names[pc]] = {"iters": its, "ms": ms, "paper_iters": paper[names[pc]].get(N)}
        row["speedup_ffthss_vs_none"] = row["none"]["ms"] / row["ffthss"]["ms"]
        rows.append(row)
        ctx.close()
    sweep = {}
    lams = [0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0]
    for N in (64, 128, 256):
        n = (N, N)
        ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
        m0, _ = I.manufactured2d(n, 0.0, alpha)
        _, f0 = I.manufactured2d(n, k, alpha)
        m, f = torch.tensor(m0, device="cuda"), torch.tensor(f0, device="cuda")
        sweep[N] = [step(ctx, m, f, lam, L.PC_FFTHSS, 1)[0] for lam in lams]
        ctx.close()
    print(json.dumps({"leg": "precond_compare", "system": "one Euler step, k 1e-2, alpha 0.2, lambda 0.5, GMRES(50), "
                      "rtol 1e-8, manufactured right-hand side on (0,2pi)^2", "rows": rows,
                      "lambda_sweep": {"lambdas": lams, "iters": sweep,
                                       "paper": "minimum 10 at lambda 0.25 on N = 64, 128, 256; 32, 39, 42 at lambda 16"},
                      "paper_times_s": {"ffthss_256": 0.236, "speedup_vs_none_256": 15.45,
                                        "hardware": "AMD Ryzen 7 9800X3D, serial SciPy pocketfft"}}), flush=True)


def midpoint_2d_leg(args):
    """1024^2 periodic unit square, FP64 throughout, alpha = 0.02, midpoint scheme for 20 steps
    at 13.3x the linearised explicit exchange limit (Picard and GMRES(30) tolerances 1e-10),
    for the smooth field and the broadband field (|k|^-1.5 spectrum, seeded): GMRES
    iterations per linear solve, Picard iterations per step, worst nodal length drift, worst
    discrete dissipation residual, and step time (CUDA events, after one warm-up step)."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    n = (1024, 1024)
    alpha = 0.02
    k = 13.3 * 2 * alpha / ((1 + alpha ** 2) * 2 * (math.pi * n[0]) ** 2)
    ctx = L.Context(n)
    ctx.autotune(fp64=True, fp32=False)
    prm = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    opts = L.Opts(restart=30, rtol=1e-10, picard_tol=1e-10, picard_max=60, diagnostics=1)
    out = {"leg": "midpoint_2d", "grid": list(n), "alpha": alpha, "dt": k, "dt_over_explicit_limit": 13.3, "fields": {}}
    for field in ("smooth", "broadband"):
        m0 = I.smooth2d(n) if field == "smooth" else I.broadband(n, seed=20260725)
        m = torch.tensor(m0, device="cuda")
        L.llg_step_midpoint(ctx, prm, opts, m, None)      # warm-up
        vprev = None
        iters = solves = 0
        drift = diss = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        for _ in range(20):
            m, x, info = L.llg_step_midpoint(ctx, prm, opts, m, vprev)
            vprev = x[:3].contiguous()
            iters += info["iters"]
            solves += info["picard_iters"]
            drift = max(drift, info["max_len_drift"])
            diss = max(diss, abs(info["dissipation_residual"]) / max(abs(info["energy_before"]), 1e-300))
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        out["fields"][field] = {"gmres_iters_per_solve": iters / solves, "picard_iters_per_step": solves / 20,
                                "max_len_drift": drift, "max_rel_dissipation_residual": diss,
                                "ms_per_step": ms, "steps_per_s": 1e3 / ms}
    ctx.close()
    print(json.dumps(out), flush=True)


def mesh_study_leg(args):
    """Sec. 4.5's mesh study on the GPU: the velocity right-hand side replaced by three seeded
    normalised Gaussian vectors (seeds 20260724-26; not the paper's NumPy vectors), multiplier
    part zero, FFT-HSS GMRES(50) in FP64 at rtol 1e-8, the Sec. 4.3 field; fixed k = 1e-2 and
    bounded stiffness kN^2 = 10.24, N = 32 ... 1024.  Median/min/max iterations and median
    solve time; the paper's medians quoted as context."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    paper = {"fixed": {32: 55, 256: 608}, "bounded": {32: 55, 256: 56}}
    rows = []
    for regime in ("fixed", "bounded"):
        for N in (32, 64, 128, 256, 512, 1024):
            k = 1e-2 if regime == "fixed" else 10.24 / N ** 2
            n = (N, N)
            ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
            m0, _ = I.manufactured2d(n, 0.0, 0.2)
            m = torch.tensor(m0, device="cuda")
            prm = L.Params(alpha=0.2, k=k, theta=1.0, lam=0.5)
            opts = L.Opts(restart=50, rtol=1e-8, max_iters=20000)
            its, times, worst = [], [], 0.0
            for seed in (20260724, 20260725, 20260726):
                b = torch.tensor(I.gaussian_rhs(n, seed), device="cuda")
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(ctx.stream)
                _, info = L.llg_gmres_solve(ctx, prm, opts, m, b)
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                its.append(info["iters"])
                times.append(e0.elapsed_time(e1))
                worst = max(worst, info["rel_res_true"])
            ctx.close()
            rows.append({"regime": regime, "N": N, "k": k, "iters_median": sorted(its)[1], "iters_min": min(its),
                         "iters_max": max(its), "ms_median": sorted(times)[1], "worst_rel_res": worst,
                         "paper_median": paper[regime].get(N)})
    print(json.dumps({"leg": "mesh_study", "rows": rows}), flush=True)


def ensemble_leg(args):
    """96 independent 2D problems (32 each of 128^2, 256^2, 512^2), alpha ~ U[0.01, 0.5],
    dt = U[2, 16] x the explicit exchange limit, seeded smooth/broadband mixes, h = (0,0,0.5),
    5 projected-Euler steps each with FP32-flexible GMRES(30) at rtol 1e-10: one persistent
    launch (block count from the ensemble autotuner) vs the same problems one at a time
    through the context API."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    steps = 5
    specs = [(n, alpha, c * 2 * alpha / ((1 + alpha ** 2) * 2 * (np.pi * n) ** 2), f)
             for n, alpha, c, f in I.ensemble_mix()]
    # the ensemble kernel's Gram-Schmidt passes are FP64; the one-at-a-time path runs the same
    opts = L.Opts(restart=30, rtol=1e-10, max_iters=900, precision=L.PREC_FP32_FLEX, gs_arith=L.GS_FP64)
    stream = torch.cuda.Stream()
    probs = [{"n": (n, n), "params": L.Params(alpha=a, k=k, lam=0.5, h_ext=(0.0, 0.0, 0.5)),
              "m": torch.tensor(f, device="cuda"), "x": torch.zeros((4, n, n), dtype=torch.float64, device="cuda")}
             for n, a, k, f in specs]
    m0 = [p["m"].clone() for p in probs]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ens = L.Ensemble(probs, opts, stream=stream)
        blocks = ens.autotune()
        for p, m in zip(probs, m0):
            p["m"].copy_(m)
        ens.run(1)                                   # warm-up (captures the graph for 1 step)
        for p, m in zip(probs, m0):
            p["m"].copy_(m)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos, used_graph = ens.run(steps)
        e1.record(stream)
    stream.synchronize()
    ms_ens = e0.elapsed_time(e1)
    # the same problems one at a time (one context per grid size, one Euler step per call)
    ctxs = {n: L.Context((n, n)) for n in (128, 256, 512)}
    for c in ctxs.values():
        c.autotune(fp64=True, fp32=True)
    seq = [m.clone() for m in m0]
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    iters_seq = 0
    for idx, (n, a, k, f) in enumerate(specs):
        prm = probs[idx]["params"]
        m = seq[idx]
        for _ in range(steps):
            m, x, info = L.llg_step_euler(ctxs[n], prm, opts, m)
            iters_seq += info["iters"]
        seq[idx] = m
    t1.record()
    torch.cuda.synchronize()
    ms_seq = t0.elapsed_time(t1)
    diff = max(float((p["m"] - s_).abs().max()) for p, s_ in zip(probs, seq))
    solves = len(specs) * steps
    out = {"leg": "ensemble", "problems": len(specs), "steps": steps, "grids": "32 x 128^2, 32 x 256^2, 32 x 512^2",
           "gram_schmidt": "fp64",
           "ensemble_ms": ms_ens, "ensemble_solves_per_s": solves / (ms_ens / 1e3),
           "sequential_ms": ms_seq, "sequential_solves_per_s": solves / (ms_seq / 1e3),
           "speedup_vs_one_at_a_time": ms_seq / ms_ens, "persistent_blocks": blocks, "cuda_graph": used_graph,
           "max_abs_diff_vs_one_at_a_time": diff,
           "iters_per_solve_ensemble": sum(i["iters"] for i in infos) / solves,
           "iters_per_solve_sequential": iters_seq / solves,
           "worst_rel_res": max(i["rel_res_true"] for i in infos),
           "statuses": sorted(set(i["status"] for i in infos))}
    print(json.dumps(out), flush=True)
    ens.close()


def adjoint_leg(args):
    """Gradient of L = 1/2 |m(T) - m_target|^2 w.r.t. alpha, h and m0 through 16 midpoint steps on
    512^2 at dt = 8x the explicit limit, checkpoint every 4 steps: forward time vs gradient time."""
    import numpy as np
    import torch
    import paper_2607_15290_b300 as L
    from paper_2607_15290_b300 import inputs as I
    from paper_2607_15290_b300.autograd import midpoint_trajectory
    n = (512, 512)
    ctx = L.Context(n)
    ctx.autotune(fp64=True, fp32=False)
    alpha = 0.1
    k = 8 * 2 * alpha / ((1 + alpha ** 2) * 2 * (np.pi * 512) ** 2)
    m0 = torch.tensor(I.smooth2d(n, seed=41), device="cuda")
    tgt = torch.tensor(I.smooth2d(n, seed=42, noise=0.2), device="cuda")
    opts = L.Opts(rtol=1e-10, picard_tol=1e-10, restart=30)
    res = {}
    for rep in range(2):
        a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
        h = torch.tensor([0.0, 0.0, 0.5], dtype=torch.float64, requires_grad=True)
        m = m0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mT = midpoint_trajectory(ctx, m, a, h, k, 16, opts=opts, checkpoint=4)
        loss = 0.5 * ((mT - tgt) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        res = {"forward_s": t1 - t0, "gradient_s": t2 - t1, "gradient_over_forward": (t2 - t1) / (t1 - t0),
               "dL_dalpha": float(a.grad), "dL_dh": h.grad.tolist(), "loss": float(loss.detach())}
    out = {"leg": "adjoint", "grid": list(n), "steps": 16, "checkpoint": 4, "dt_over_explicit_limit": 8.0,
           "rtol": 1e-10, **res}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
