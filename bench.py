#!/usr/bin/env python
"""Benchmark of the narrow-band GRF posterior solve on one node.

Workload (default): the 200-frame object sequence -- a seeded spherical-
harmonic blob in a 512^3 grid at 2 mm, band +-24 voxels (7.2 M band
voxels), 200 depth frames 512x384 on a spiral orbit, 128 probes.

One step = the whole hot path on that synthetic depth sequence, inputs
already resident in device memory: build_band -> integrate_depth ->
solve_mean -> estimate_variance -> extract_surface -> score_views.  The
headline value is the time to posterior, solve_mean + estimate_variance
(FP32 vectors, FP64 inner products and refinement), read from CUDA events
on the library's stream: the probes to rel_tol 1e-6, the mean to 1e-8 (the
tolerance at which it meets the 1e-3-voxel parity bar; its 1e-6 time is
reported beside it).  Also reported: the full step time; the same metric end
to end through the C ABI with pinned host buffers (H2D of the frames and D2H
of mu and s inside the timed region); the roofline of the dominant kernel
(the probe solver's iteration, event-timed by bf_bench_kernel) and of the
single-RHS SpMV on the same band with L2 flushed; the posterior in its
unbatched, block and learned-warm-start forms; and the CPU oracle timed on a
bounded sample of the same workload.

Multi-GPU (torchrun, one process per GPU): one posterior per job with its
K probes split across the ranks (bf_estimate_variance_range with scale 1/K,
then one NCCL all-reduce of s); the mean, the mesh and the view scores are
computed on rank 0.  Strong scaling: value = max-over-ranks time per
posterior.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "posterior solve s (mean+diag var) at 1e-6 rel residual; SpMV GB/s vs HBM peak"

# DRAM bytes (read + write) per launch of the probe solver's iteration, from one ncu capture of that kernel on
# the band it was taken on (dram__bytes_read.sum + dram__bytes_write.sum, mean of an x-writing and an x-holding
# launch); keyed by (band voxels, block width); valid for the kernel as it was when captured.
BLK_IT_TRAFFIC = {(7221796, 32): 9154034688}  # the object band at R = 32: 10.08 GB (x written) and 8.23 GB (held)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blob512",
                    help="blob512 | union256 | sphere64 | sphere64_k256 | blob1024 | blob512_b5 (--kernel only; "
                         "blob1024: the blob512 object at 1 mm on a 1024^3 grid, band +-48 voxels, 200 frames "
                         "1024x768, 61 M voxels; blob512_b5: the blob512 object with a band of +-5 voxels)")
    ap.add_argument("--K", type=int, default=None, help="probes (default: the workload's, 128 for blob512)")
    ap.add_argument("--tol", type=float, default=1e-6, help="relative residual of the probe solves")
    ap.add_argument("--mean-tol", type=float, default=1e-8,
                    help="relative residual of the timed mean solve (1e-8: the 1e-3-voxel parity tolerance)")
    ap.add_argument("--rhs-block", type=int, default=0, help="probe block width (0 = the library's autotuner)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the unbatched / block / learned-warm-start comparison of the posterior")
    ap.add_argument("--cpu-probes", type=int, default=8, help="oracle probe solves in the CPU-baseline sample")
    ap.add_argument("--kernel", default=None,
                    choices=["block_iter", "spmv", "spmm", "spmv27", "net_forward", "net_train", "net_conv",
                             "net_conv_mma", "net_wgrad"],
                    help="time one kernel alone on the workload's band (for profiling): --warmup untimed and "
                         "--steps timed launches; prints one JSON line with its throughput")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for k, n in enumerate(names) if any(r[3 + k].lower() == "active" for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(args, **kw):
    import synth
    w = synth.make_workload(args.workload, threads=os.cpu_count() or 0, **kw)
    K = args.K or w.K
    return w, K


def workload_desc(w, K, args):
    """The workload string of the bench line's config (both arms)."""
    return (f"{w.name}: {w.n}^3 grid at {w.h * 1e3:g} mm, band +-{w.band_vox:g}, {w.T} views "
            f"{w.intr[4]}x{w.intr[5]}, K={K} probes at rel_tol {args.tol:g}, mean at rel_tol {args.mean_tol:g}")


# ----------------------------------------------------------------- oracle

def oracle_system(w):
    """Untimed set-up of the oracle's posterior system for workload w."""
    import oracle
    b = oracle.build_band_w(w)
    d, hd, _ = oracle.integrate_w(b, w)
    qd, rhs = oracle.assemble(b, d, hd, w.lam, w.lam_b)
    return b, qd, rhs


def oracle_mean_time(w, system, tol):
    import oracle
    b, qd, rhs = system
    t0 = time.perf_counter()
    oracle.pcg(b, w.lam, qd, rhs, tol=tol)
    return time.perf_counter() - t0


def oracle_probe_time(w, system, tol, k):
    """Wall time of the oracle's solve of probe k (one Hutchinson term)."""
    import oracle
    b, qd, rhs = system
    t0 = time.perf_counter()
    oracle.hutchinson(b, w.lam, qd, 1, w.seed, tol=tol, k0=k)
    return time.perf_counter() - t0


def cpu_cores():
    return len(os.sched_getaffinity(0))


def oracle_sample_desc(w, N, K, n_probes, args):
    return (f"{w.name}: oracle (FP64 CSR PCG, OpenMP over {cpu_cores()} threads) on N={N} band voxels: the mean "
            f"solve at rel_tol {args.mean_tol:g} and {n_probes} of the {K} probe solves at rel_tol {args.tol:g} "
            f"timed; the posterior time is the mean solve + {K} x the mean probe-solve time (extrapolated "
            f"linearly from the {n_probes} probes)")


def run_reference(args, world, rank):
    """The CPU oracle as the reference arm (rank 0 only).  Set-up (band,
    observations, assembly, and one timing of the mean solve) is untimed;
    each step then times one probe solve (probe k = step index), a bounded
    sample of the workload; value = t_mean + K x the mean probe time."""
    if rank != 0:
        return
    w, K = make_workload(args)
    system = oracle_system(w)
    t_mean = oracle_mean_time(w, system, args.mean_tol)
    probe = []
    for i in range(args.warmup + args.steps):
        t = oracle_probe_time(w, system, args.tol, i % K)
        if i >= args.warmup:
            probe.append(t)
    t_probe = statistics.mean(probe)
    v = t_mean + K * t_probe
    sample = oracle_sample_desc(w, system[0].N, K, len(probe), args) + \
        f"; each step is one probe solve ({t_probe:.3f} s); the mean solve took {t_mean:.3f} s"
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_probe * 1e3, "higher_is_better": False,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(w, K, args), "parallelism": "CPU oracle on rank 0"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2602_19697_gb300 import bfsdf, build
    from paper_2602_19697_gb300.sharding import probe_range

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w, K = make_workload(args)
    stream = torch.cuda.Stream(dev)
    ctx = bfsdf.Context(local, stream.cuda_stream)
    depth = torch.from_numpy(w.depth).to(dev)
    poses = torch.from_numpy(w.poses).to(dev)
    cand = torch.from_numpy(w.cand_poses).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    R = args.rhs_block
    k0, k1 = probe_range(rank, world, K)
    lead = rank == 0

    def variance(band, s):
        """s for the job's K probes: this rank's share, then the sum over ranks."""
        if world == 1:
            return band.estimate_variance(s, K=K, seed=0, rel_tol=args.tol, rhs_block=R).iters
        it = 0
        if k1 > k0:
            it = band.estimate_variance_range(s, k0, k1, seed=0, rel_tol=args.tol, rhs_block=R, scale=1.0 / K).iters
        else:
            s.zero_()
        import torch.distributed as dist
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        return it

    def step():
        with torch.cuda.stream(stream):
            return _step()

    def _step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        ev[0].record(stream)
        band = ctx.build_band_w(w, depth, poses)
        ev[1].record(stream)
        band.integrate_depth(depth, poses, w.intr)
        ev[2].record(stream)
        mu = torch.empty(band.N, device=dev)
        s = torch.empty(band.N, device=dev)
        im = band.solve_mean(mu, rel_tol=args.mean_tol) if lead else None
        ev[3].record(stream)
        vi = variance(band, s)
        ev[4].record(stream)
        tris, best = 0, -1
        if lead:
            V, F = band.extract_surface(mu, device=dev)
            tris = int(F.shape[0])
        ev[5].record(stream)
        if lead:
            U, best = band.score_views(mu, s, cand, w.cand_intr)
        ev[6].record(stream)
        stream.synchronize()
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(6)]
        info = dict(N=band.N, NB=band.NB, mean_iters=im.iters if im else None, var_iters=vi, tris=tris,
                    best_view=best)
        return band, t, info

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()

    for _ in range(args.warmup):
        b, _, _ = step()
        b.free()
        flush_l2()
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    l0 = bfsdf.launch_count()
    times, info = [], None
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        b, t, info = step()
        times.append(t)
        b.free()
        flush_l2()
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    launches = (bfsdf.launch_count() - l0) // max(args.steps, 1)
    clocks = clk.stop()

    post = [t[2] + t[3] for t in times]     # solve_mean + estimate_variance (ms)
    stepms = [sum(t) for t in times]
    post_s = max_over_ranks(world, statistics.mean(post) / 1e3)
    step_s = max_over_ranks(world, statistics.mean(stepms) / 1e3)
    value = post_s                            # one posterior per job (probes shared by the ranks)

    # ---- the mean at the probes' tolerance, and the rooflines on this band (untimed for the headline)
    hbm, peak_kind = peaks()
    band = ctx.build_band_w(w, depth, poses)
    band.integrate_depth(depth, poses, w.intr)
    N, NB = band.N, band.NB
    mu = torch.empty(N, device=dev)
    ms_mean6 = []
    for i in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush_l2()
        e0.record(stream)
        i6 = band.solve_mean(mu, rel_tol=args.tol)
        e1.record(stream)
        stream.synchronize()
        ms_mean6.append(e0.elapsed_time(e1))
    R_used, tune_ms = (R, None) if R else band.autotune_rhs_block(max(k1 - k0, 1))
    s = torch.empty(N, device=dev)
    band.estimate_variance(s, K=R_used, seed=0, rel_tol=args.tol, rhs_block=R_used)
    band.bench_kernel(bfsdf.BF_KERNEL_BLOCK_ITER, R=R_used, reps=5)
    ms_iter = band.bench_kernel(bfsdf.BF_KERNEL_BLOCK_ITER, R=R_used, reps=20)
    # algorithmic bytes of one probe-solver iteration (per voxel row of R
    # columns): r, w, s, p read and p, r', s', w' written (32 B per column),
    # the correction x read and written every second iteration (4 B per
    # column on average; the timed launches alternate the two kinds), Q_jj
    # and 1/Q_jj read (8 B); the neighbour gathers of the SpMM are not
    # counted (they come from shared memory and L2 by design)
    bytes_it = N * (R_used * 36 + 8)
    achieved = bytes_it / (ms_iter * 1e-3) / 1e9
    traffic = BLK_IT_TRAFFIC.get((N, R_used))
    roof = {"kernel": "k_blk_it<%d> (one probe-solver iteration: vector updates and w = Q u in one pass, "
                      "the dominant kernel)" % R_used, "bound": "hbm",
            "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "peak_kind": peak_kind, "traffic": traffic, "bytes_per_launch": bytes_it,
            "ms_per_launch": round(ms_iter, 5),
            "timing": "20 back-to-back launches (after 5 untimed) between CUDA events on the library stream (working set "
                      f"{bytes_it / 1e9:.2f} GB per launch, larger than L2)"}
    spmv = spmv_roofline(band, stream, hbm, peak_kind)
    band.free()

    # ---- end to end through the C ABI: pinned host frames in, host mu and s out
    e2e = None
    if not args.no_e2e:
        dh = torch.from_numpy(w.depth).pin_memory()
        ph = torch.from_numpy(w.poses).pin_memory()
        muh = torch.empty(N, dtype=torch.float32).pin_memory()  # result buffers, allocated once
        sh = torch.empty(N, dtype=torch.float32).pin_memory()
        sd = torch.empty(N, dtype=torch.float32, device=dev)
        e2e_t = []
        for i in range(2 + args.steps):
            stream.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):  # the step's inputs, copied once for the two calls that read them
                dd = dh.to(dev, non_blocking=True)
                pd = ph.to(dev, non_blocking=True)
                b = ctx.build_band_w(w, dd, pd)
                b.integrate_depth(dd, pd, w.intr)
                if b.N != N:
                    raise RuntimeError("band size differs between runs")
                if lead:
                    b.solve_mean(muh, rel_tol=args.mean_tol)
                if world == 1:
                    b.estimate_variance(sh, K=K, seed=0, rel_tol=args.tol, rhs_block=R)
                else:
                    variance(b, sd)
                    if lead:
                        sh.copy_(sd, non_blocking=True)
            stream.synchronize()
            dt = time.perf_counter() - t0
            if i >= 2:
                e2e_t.append(dt)
            b.free()
        e2e_s = max_over_ranks(world, statistics.mean(e2e_t))
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(w.depth.nbytes + w.poses.nbytes),
               "d2h_bytes_per_step": int(2 * N * 4),
               "note": "pinned host frames copied to the device once per step, then build_band + integrate_depth "
                       "+ solve_mean + estimate_variance through the C ABI, mu and s written to pinned host memory"}

    cmp_ = None
    if world == 1 and not args.no_compare:
        cmp_ = compare_forms(ctx, stream, w, K, args, flush_l2)

    cpu = None
    if lead and not args.no_cpu_baseline:
        system = oracle_system(w)
        t_mean = oracle_mean_time(w, system, args.mean_tol)
        tp = [oracle_probe_time(w, system, args.tol, k) for k in range(min(args.cpu_probes, K))]
        est = t_mean + K * statistics.mean(tp)
        cpu = {"value": est, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": oracle_sample_desc(w, N, K, len(tp), args)}

    if lead:
        mean_t = [statistics.mean(x) for x in zip(*times)]
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_desc(w, K, args),
                           "N_band": info["N"], "bricks": info["NB"], "rhs_block": R_used,
                           "rhs_block_choice": "autotuned" if not R else "fixed",
                           "autotune_ms_per_iter_r8_r16_r32": None if tune_ms is None else [round(float(v), 5) for v in tune_ms],
                           "l2": "inputs larger than L2 (the probe block's vectors are several GB) and a 512 MB "
                                 "buffer written between timed steps",
                           "parallelism": "single GPU" if world == 1 else f"probes sharded over {world} ranks, "
                                                                            "one NCCL all-reduce of s"},
                "breakdown_ms": {"build_band": mean_t[0], "integrate_depth": mean_t[1],
                                 "solve_mean": mean_t[2], "estimate_variance": mean_t[3],
                                 "extract_surface": mean_t[4], "score_views": mean_t[5],
                                 "solve_mean_at_probe_tol": round(statistics.median(ms_mean6), 4)},
                "iters": {"mean": info["mean_iters"], "mean_at_probe_tol": i6.iters,
                          "variance_total": info["var_iters"]},
                "roofline": roof, "spmv": spmv, "compare": cmp_, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "wall_s": round(wall, 3)}
        print(json.dumps(line), flush=True)


def spmv_roofline(band, stream, hbm, peak_kind):
    """Single-RHS SpMV on the band: single launches after writing and then
    reading 1 GB (L2 flushed, its dirty lines written back), median of 20."""
    import numpy as np
    import torch

    from paper_2602_19697_gb300 import bfsdf
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.float32, device=dev)
    clean = torch.zeros(256 * 1024 * 1024, dtype=torch.float32, device=dev)
    band.bench_kernel(bfsdf.BF_KERNEL_SPMV, reps=3)
    ms = []
    for i in range(20):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            clean.sum()
        stream.synchronize()
        ms.append(band.bench_kernel(bfsdf.BF_KERNEL_SPMV, reps=1))
    nbytes = band.N * 12 + band.NB * 152
    gbs = nbytes / (float(np.median(ms)) * 1e-3) / 1e9
    del flush, clean
    return {"kernel": "k_spmv_t (7-point SpMV, single RHS: a warp per brick, runs bulk-copied)", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(gbs / hbm, 4), "peak_kind": peak_kind, "ms_median": round(float(np.median(ms)), 5),
            "bytes": nbytes, "bytes_per_voxel": round(nbytes / band.N, 3),
            "l2": "1 GB written, then another 1 GB read, before each of 20 single launches; median"}


def compare_forms(ctx, stream, w, K, args, flush_l2):
    """Time to posterior on the same band in three forms, each run twice and
    the second run reported: the probes one at a time (unbatched single-RHS
    PCG), block PCG at the autotuned width, and block PCG with the mean
    warm-started by the learned network (trained here on seeded sphere
    instances) and the network's variance surrogate judged by 16 probes."""
    import torch

    import synth
    from paper_2602_19697_gb300 import bfsdf, learned

    dev = torch.device("cuda", torch.cuda.current_device())
    depth, poses = torch.from_numpy(w.depth).to(dev), torch.from_numpy(w.poses).to(dev)
    band = ctx.build_band_w(w, depth, poses)
    band.integrate_depth(depth, poses, w.intr)
    N = band.N

    def posterior(rhs_block, net=None):
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            mu, s = torch.empty(N, device=dev), torch.empty(N, device=dev)
            flush_l2()
            e0.record(stream)
            if net is None:
                im = band.solve_mean(mu, rel_tol=args.tol)
                iv = band.estimate_variance(s, K=K, seed=0, rel_tol=args.tol, rhs_block=rhs_block)
                acc = None
            else:
                lsh = torch.empty(N, device=dev)
                net.forward(band, mu, lsh)
                im = band.solve_mean(mu, rel_tol=args.tol, warm=True)
                iv, _, _, acc = band.surrogate_variance(lsh, s, K=K, K_judge=16, seed=0, rel_tol=args.tol,
                                                        rhs_block=rhs_block)
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1), im.iters, iv.iters, acc

    posterior(1)
    plain_ms, plain_mi, plain_vi, _ = posterior(1)
    posterior(0)
    block_ms, block_mi, block_vi, _ = posterior(0)
    data = [learned.make_example(ctx, synth.make_workload("sphere64", variant=i)) for i in range(50)]
    net = bfsdf.Net(ctx, seed=0)
    learned.train(net, data, epochs=20, lr=1e-3)
    posterior(0, net)
    warm_ms, warm_mi, warm_vi, acc = posterior(0, net)
    band.free()
    return {"note": "time to posterior (mean + variance, both at rel_tol %g), each form run twice, second run" % args.tol,
            "posterior_ms": {"unbatched_single_rhs_pcg": round(plain_ms, 3), "block_pcg_autotuned": round(block_ms, 3),
                             "block_pcg_learned_warm_start": round(warm_ms, 3)},
            "iters": {"unbatched": [plain_mi, plain_vi], "block": [block_mi, block_vi],
                      "learned": [warm_mi, warm_vi]},
            "surrogate_bricks_accepted": acc, "bricks": band.NB}


def kernel_workload(name):
    import synth
    if name == "blob1024":  # the object at twice the linear resolution, same physical band
        return synth.make_workload("blob512", n=1024, band_vox=48.0, image_scale=2.0, threads=os.cpu_count() or 0)
    if name == "blob512_b5":  # the object with a band of +-5 voxels
        return synth.make_workload("blob512", band_vox=5.0, threads=os.cpu_count() or 0)
    return synth.make_workload(name, threads=os.cpu_count() or 0)


def run_kernel(args):
    """One kernel of the path, launched alone through the library's timing
    entries (CUDA events on the library stream).  The SpMV is timed as single
    launches after writing and then reading 1 GB (L2 flushed), median of
    --steps; the other kernels as --steps back-to-back launches."""
    import numpy as np
    import torch

    from paper_2602_19697_gb300 import bfsdf, build
    build.build()
    ctx = bfsdf.Context(0)
    w = kernel_workload(args.workload)
    depth, poses = torch.from_numpy(w.depth).cuda(), torch.from_numpy(w.poses).cuda()
    band = ctx.build_band_w(w, depth, poses)
    band.integrate_depth(depth, poses, w.intr, trilinear=args.kernel == "spmv27")
    N, NB, R = band.N, band.NB, (args.rhs_block or 32)
    out = {"kernel": args.kernel, "workload": args.workload, "N_band": N, "bricks": NB}
    if args.kernel == "block_iter":
        which = bfsdf.BF_KERNEL_BLOCK_ITER
        band.bench_kernel(which, R=R, reps=max(args.warmup, 1))
        ms = band.bench_kernel(which, R=R, reps=max(args.steps, 1))
        nbytes = N * (R * 36 + 8)
        out.update(ms_per_launch=ms, bytes_per_launch=nbytes, achieved_gbs=nbytes / (ms * 1e-3) / 1e9)
    elif args.kernel in ("spmv", "spmm", "spmv27"):
        which = bfsdf.BF_KERNEL_SPMM if args.kernel == "spmm" else bfsdf.BF_KERNEL_SPMV
        band.bench_kernel(which, R=R, reps=max(args.warmup, 1))
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.float32, device="cuda")
        clean = torch.zeros(256 * 1024 * 1024, dtype=torch.float32, device="cuda")
        ms = []
        for i in range(max(args.steps, 1)):
            flush.fill_(float(i))
            clean.sum()
            torch.cuda.synchronize()
            ms.append(band.bench_kernel(which, R=R, reps=1))
        # x (or X) and Q_jj (or the 27 coefficients of the trilinear rows' precision) read, y (or Y) written,
        # brick metadata
        nbytes = {"spmv": N * 12 + NB * (128 + 24), "spmm": N * (8 * R + 4) + NB * (128 + 24),
                  "spmv27": N * (27 * 4 + 8) + NB * (128 + 16)}[args.kernel]
        med = float(np.median(ms))
        hbm, peak_kind = peaks()
        out.update(ms_per_launch=med, ms_min=min(ms), bytes_per_launch=nbytes,
                   achieved_gbs=nbytes / (med * 1e-3) / 1e9, peak_gbs=hbm, peak_kind=peak_kind,
                   frac=nbytes / (med * 1e-3) / 1e9 / hbm, bytes_per_voxel=nbytes / N,
                   columns=(R if args.kernel == "spmm" else 1),
                   l2="1 GB written, then another 1 GB read, before each single launch; median")
    else:
        net = bfsdf.Net(ctx, seed=0)
        which = {"net_forward": bfsdf.BF_NET_BENCH_FORWARD, "net_train": bfsdf.BF_NET_BENCH_TRAIN,
                 "net_conv": bfsdf.BF_NET_BENCH_CONV, "net_wgrad": bfsdf.BF_NET_BENCH_WGRAD,
                 "net_conv_mma": bfsdf.BF_NET_BENCH_CONV_MMA}[args.kernel]
        flops = {"net_forward": bfsdf.NET_FLOPS_FWD, "net_train": 3 * bfsdf.NET_FLOPS_FWD - 2 * 1000 * 27 * 2 * 32,
                 "net_conv": bfsdf.NET_FLOPS_CONV, "net_wgrad": bfsdf.NET_FLOPS_CONV,
                 "net_conv_mma": bfsdf.NET_FLOPS_CONV}[args.kernel] * NB
        net.bench(band, which, reps=max(args.warmup, 1))
        ms = net.bench(band, which, reps=max(args.steps, 1))
        out.update(ms_per_rep=ms, flops_per_rep=flops, achieved_tflops=flops / (ms * 1e-3) / 1e12)
    print(json.dumps(out))


def main():
    args = parse()
    if args.kernel:
        run_kernel(args)
        return
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
