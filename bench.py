#!/usr/bin/env python
"""Benchmark of the Feldman-Cousins hot path on one GB300 (or N replicas).

Workload (one step = one full FC job): the D=2 100x100 grid, N_full = 90 bins
collapsed pairwise to 45, every one of the 10^4 grid points a true point with
U = 1000 universes (10^7 fits), covariance refit until the best fit repeats
(<= 5 scans), tensor-core screen + certified double-float rescoring.  Each step
starts from a cold covariance cache (fc_set_frac_cov), so covariance builds,
inversions and q-vectors are inside the timed region.

Metric: chi2 evals/s = sum over universe-scans of G (the chi2 values a scan
decides its minimum over), whole job, inputs resident in HBM.  The line also
carries universes/s, the plain binary64 GPU fit on a sample (same metric), an
end-to-end figure through the C ABI with host buffers, the roofline of the
dominant kernel, the CPU oracle on a bounded sample, and the SM clocks seen.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
  python bench.py --serve      (cfg4 stream: p50/p99 job latency)
  python bench.py --sweep      (job time vs universes and vs grid points)
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

METRIC = "chi2 evals/s"
UNIT = "chi2 evals/s"

# DRAM bytes (read + write) per screened universe row of the tensor-core screen on the
# 100x100 grid with N 90->45 (K = 48): an ncu capture of one top-8 launch over 10^6
# universes (the current kernel, parallel top-k insertion) read 367.0 MB and wrote
# 56.3 MB.  The traffic is the rows' A images, the q-step rows of their covariance
# slots and the candidate lists, so a launch's traffic is taken as proportional to the
# rows it screens.
SCREEN_DRAM_BYTES_PER_ROW_CFG2 = 423.3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_sample(w, target_s: float, nthreads: int, seed: int = 0, max_points: int = 16):
    """Time the CPU oracle on a bounded sample of the workload (points spread over the grid)."""
    import numpy as np

    import oracle

    oracle.build()
    # calibrate on a tiny sample, then scale the universe count to about target_s
    pts_all = np.linspace(0, w.G - 1, max_points).round().astype(np.int64)
    t0 = time.perf_counter()
    _, _, ns = oracle.run_points(w.S, w.F, pts_all[:1], seed, 16, collapse=w.collapse, n_fit=w.n_fit,
                                 max_iter=w.max_iter, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_u = dt / 16 * nthreads
    n_univ = max(nthreads, int(target_s * nthreads / max(per_u, 1e-9)))
    P = int(min(max_points, max(1, n_univ // 64)))
    U = max(1, n_univ // P)
    pts = pts_all[np.linspace(0, max_points - 1, P).round().astype(int)]
    t0 = time.perf_counter()
    _, _, ns = oracle.run_points(w.S, w.F, pts, seed, U, collapse=w.collapse, n_fit=w.n_fit,
                                 max_iter=w.max_iter, nthreads=nthreads)
    dt = time.perf_counter() - t0
    evals = float(ns.astype(np.int64).sum()) * w.G
    return {"value": evals / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{P} true points x {U} universes of {w.name}, {evals:.3e} chi2 evals in {dt:.1f} s",
            "universes_per_s": P * U / dt}


def resid_fp32_ops(n: int) -> int:
    """binary32 operations of one double-float residual chi2 = |W (s - d)|^2 over n bins: 10 per element of
    r = s - d, 12 per double-float multiply-add (n(n+1)/2 of them in W r, n in the squares), 45 to combine the
    four partial sums of a row, 3 to round the total."""
    return 6 * n * n + 73 * n + 3


def _cfg3_step(fc, ctx, peak_bf16):
    """One cold-cache step of the D=3 workload (2048 points x 500 universes), CUDA-event timed after one
    untimed step: where the per-universe covariance refits decide the cost."""
    import torch

    import workloads

    w = workloads.cfg3()
    gid = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    tuning = fc.fc_autotune(ctx, gid)     # q-vector kernel, screen depth / buffering, rows per covariance slot
    opts = dict(precision=fc.FC_PREC_MIXED, top_k=8, max_iter=w.max_iter)
    n = len(w.points) * w.U
    dev = torch.device("cuda", torch.cuda.current_device())
    ps = torch.from_numpy(w.points).to(dev)
    outs = (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.int64, device=dev),
            torch.empty(n, dtype=torch.int8, device=dev))
    fc.fc_set_frac_cov(ctx, gid, w.F)
    fc.fc_run_points(ctx, gid, ps, 1, w.U, opts, *outs)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fc.fc_run_points(ctx, gid, ps, 2, w.U, opts, *outs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = fc.fc_get_stats(ctx)
    fc.fc_unload_grid(ctx, gid)
    ms = st["ms_total"]
    achieved = st["screen_flops"] / (st["ms_screen"] / 1e3) / 1e12 if st["ms_screen"] > 0 else 0.0
    return {"workload": f"cfg3: D=3 64^3 grid (262144 points), N=120, {len(w.points)} true points x {w.U} universes, "
                        "<= 5 scans, top-8, cold covariance cache", "autotuned": tuning,
            "ms_per_step": ms, "wall_ms": wall * 1e3, "value": st["chi2_evals"] / (ms / 1e3), "unit": UNIT,
            "universes_per_s": n / (ms / 1e3),
            "stage_ms": {k: st[k] for k in ("ms_fake", "ms_cov", "ms_prep", "ms_screen", "ms_rescore")},
            "scans": st["scans"], "distinct_cov": st["distinct_cov"],
            "screen_fill": st["screen_rows"] / max(1, 128 * st["screen_tiles"]),
            "screen_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_bf16, "unit": "TFLOP/s",
                                "frac": achieved / peak_bf16}}


def _cfg4_below_saturation(fc, device, rate, window, drain):
    """The serving stream (cfg4 pool, 80 GB budget) offered below its saturation rate: p50/p99 latency."""
    import numpy as np

    import workloads

    pool = workloads.cfg4_pool()
    ctx = fc.fc_create(device, 80 << 30, None)
    try:
        gids = []
        for w in pool:
            g = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
            fc.fc_set_frac_cov(ctx, g, w.F)
            gids.append(g)
        sizes = [w.G for w in pool]
        for g, G in zip(gids, sizes):
            fc.fc_run_points(ctx, g, np.array([G // 2], np.int64), 1, 128)
        r = _serve_stream(fc, ctx, gids, sizes, rate, window, 7, drain)
    finally:
        fc.fc_destroy(ctx)
    r["workload"] = ("cfg4 serving stream: 8 resident grids (D 2-4, G log-U[1e3,1e6], N U{40..200}), one true point "
                     "per job, U log-U[100,1e4], Poisson arrivals, 80 GB budget")
    return r


def _dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch.distributed as dist

    dist.init_process_group("gloo")
    return dist.get_rank(), int(os.environ.get("LOCAL_RANK", "0")), ws, dist


def _combine_ranks(dist, ms: float, evals: float, univ: float):
    """Whole-job figures of N replicas: the slowest rank's time, the sum of every rank's work."""
    import torch

    t = torch.tensor([ms, evals, univ], dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])


def replica_seed(rank: int) -> int:
    """Seed offset of a replica: ranks draw disjoint Philox keys, so their universes are independent."""
    return 1000003 * rank


def run_reference(args):
    """The reference arm: the CPU oracle, timed on the host cores (rank 0 only)."""
    rank, _, ws, dist = _dist_init()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import workloads

    w = workloads.cfg2()
    nthreads = len(os.sched_getaffinity(0))
    oracle.build()
    P, U = 2, max(nthreads, 4 * nthreads)
    pts = np.array([2550, 7575], np.int64)[:P]

    def step(seed):
        t0 = time.perf_counter()
        _, _, ns = oracle.run_points(w.S, w.F, pts, seed, U, collapse=w.collapse, n_fit=w.n_fit,
                                     max_iter=w.max_iter, nthreads=nthreads)
        return float(ns.astype(np.int64).sum()) * w.G, time.perf_counter() - t0

    for i in range(args.warmup):
        step(1000 + i)
    ev = tt = 0.0
    for i in range(args.steps):
        e, t = step(i)
        ev += e
        tt += t
    value = ev / tt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "cfg2 sample: 100x100 grid, N 90->45, 2 true points x "
                                   f"{U} universes per step (CPU oracle)", "max_iter": w.max_iter},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{P} points x {U} universes per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cfg5(workloads, args):
    """cfg5's workload: host spectra (stored grid), or its shape model when the grid is recomputed."""
    if args.recompute:
        return workloads.cfg5_model(U=args.universes or 16)
    return workloads.cfg5(U=args.universes or 16)


def _load_grid(fc, ctx, w):
    """A workload's grid: from its host spectra, or recomputed from its shape model (S is None)."""
    if w.S is None:
        m = w.meta["model"]
        return fc.fc_load_grid_osc(ctx, m["axes"], m["terms"], m["b"], m["f"], m["L"], m["E"], w.collapse, w.n_fit,
                                   recompute=True)
    return fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)


def run_native(args):
    import numpy as np
    import torch

    import paper_2002_07858_gb300 as fc
    import workloads

    rank, local_rank, ws, dist = _dist_init()
    torch.cuda.set_device(local_rank)
    fc.load()
    if args.config == "cfg3":
        w = workloads.cfg3(U=args.universes or 500)
        pts = w.points if args.points is None else w.points[np.linspace(0, len(w.points) - 1, args.points).astype(int)]
        desc = (f"cfg3: D=3 64^3 grid (262144 points), N=120 (K=128), {len(pts)} seeded true points x {w.U} "
                f"universes, <= {w.max_iter} scans, top-{args.top_k}")
        l2 = "working set per step > L2 (screen B image 134 MB, q-vectors 6.3 MB per covariance)"
    elif args.config == "cfg5":
        w = _cfg5(workloads, args)
        pts = w.points if args.points is None else w.points[np.linspace(0, len(w.points) - 1, args.points).astype(int)]
        desc = (f"cfg5: D=6 16^6 grid (16777216 points), N=64, {len(pts)} seeded true points x {w.U} universes "
                f"(one batch of {len(pts) * w.U}), <= {w.max_iter} scans, top-{args.top_k}"
                + (", spectra recomputed from the shape model (none stored)" if args.recompute else ""))
        l2 = "working set per step > L2 (screen B image 4.3 GB, q-vectors 0.4 GB per covariance)"
    else:
        w = workloads.cfg2(U=args.universes or 1000)
        P_all = w.G if args.points is None else args.points
        pts = (np.linspace(0, w.G - 1, P_all).round().astype(np.int64) if args.points
               else np.arange(w.G, dtype=np.int64))
        desc = (f"cfg2: D=2 100x100 grid, N 90->45 (pair collapse), all 1e4 true points x {w.U} universes, "
                f"<= {w.max_iter} scans, top-{args.top_k}")
        l2 = "working set per step > L2 (fake data 1.8 GB, screen A-tiles ~2 GB, q-vectors 0.8 GB)"
    P, U = len(pts), w.U
    n = P * U
    stream = torch.cuda.Stream()
    ctx = fc.fc_create(local_rank, 0, stream.cuda_stream)
    bytes0 = fc.fc_get_stats(ctx)["device_bytes"]
    gid = _load_grid(fc, ctx, w)
    grid_bytes = fc.fc_get_stats(ctx)["device_bytes"] - bytes0
    fc.fc_set_frac_cov(ctx, gid, w.F)
    # kernel choices and tile shape (rows per covariance slot) picked by the library's autotuner
    tuning = fc.fc_autotune(ctx, gid)
    dev = torch.device("cuda", local_rank)
    ps_dev = torch.from_numpy(pts).to(dev)
    dchi2 = torch.empty(n, dtype=torch.float64, device=dev)
    best = torch.empty(n, dtype=torch.int64, device=dev)
    nsc = torch.empty(n, dtype=torch.int8, device=dev)
    opts = dict(precision=fc.FC_PREC_MIXED, top_k=args.top_k, max_iter=w.max_iter)
    seed_base = replica_seed(rank)

    def step(i, ps=ps_dev, outs=(dchi2, best, nsc)):
        fc.fc_set_frac_cov(ctx, gid, w.F)          # cold covariance cache: every step builds its own
        fc.fc_run_points(ctx, gid, ps, seed_base + i, U, opts, *outs)
        return fc.fc_get_stats(ctx)

    for i in range(args.warmup):
        step(10_000 + i)
    torch.cuda.synchronize()
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            stats.append(step(i))
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    evals = float(sum(s["chi2_evals"] for s in stats))
    univ = float(sum(s["universes"] for s in stats))
    if dist:
        ms, evals, univ = _combine_ranks(dist, ms, evals, univ)
    value = evals / (ms / 1e3)

    # ---- stage breakdown and roofline of the dominant kernel (event-timed inside the library)
    keys = ["ms_fake", "ms_cov", "ms_prep", "ms_screen", "ms_rescore", "ms_fallback", "ms_scan64", "ms_finish"]
    stage = {k: sum(s[k] for s in stats) / len(stats) for k in keys}
    peaks, peak_src = _peaks()
    scr_ms = sum(s["ms_screen"] for s in stats)
    scr_flops = sum(s["screen_flops"] for s in stats)
    scr_launch = sum(s["screen_launches"] for s in stats)
    achieved = scr_flops / (scr_ms / 1e3) / 1e12 if scr_ms > 0 else 0.0
    scr_rows = sum(s["screen_rows"] for s in stats)
    traffic = None
    if args.config == "cfg2" and scr_launch > 0:
        # bytes per launch, scaled from the captured launch by the rows screened
        traffic = SCREEN_DRAM_BYTES_PER_ROW_CFG2 * scr_rows / scr_launch
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    roofline = {"kernel": "k_screen (tcgen05 BF16 hi/lo screen + fused top-k)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"bf16_tflops_sustained ({peak_src})", "traffic": traffic,
                "traffic_source": ("DRAM bytes per launch: an ncu capture of one top-8 launch (423.3 B per "
                                   "screened row) scaled by the rows each launch screens") if traffic else None,
                "flops_per_eval": 2 * w.n_fit, "launches": scr_launch,
                "avg_launch_ms": scr_ms / max(scr_launch, 1)}

    # ---- end to end through the C ABI with host (pinned) buffers
    e2e = None
    if rank == 0 or ws > 1:
        ps_h = torch.from_numpy(pts).pin_memory()
        d_h = torch.empty(n, dtype=torch.float64).pin_memory()
        b_h = torch.empty(n, dtype=torch.int64).pin_memory()
        s_h = torch.empty(n, dtype=torch.int8).pin_memory()
        step(20_000, ps_h, (d_h, b_h, s_h))
        t0 = time.perf_counter()
        e_ev = 0.0
        for i in range(args.steps):
            e_ev += step(i, ps_h, (d_h, b_h, s_h))["chi2_evals"]
        dt = time.perf_counter() - t0
        e2e = {"value": e_ev * ws / dt, "unit": UNIT, "h2d_bytes_per_step": int(P * 8 + w.n_full ** 2 * 8),
               "d2h_bytes_per_step": int(n * (8 + 8 + 1))}

    line = None
    if rank == 0:
        # measured fma rates of this GPU: denominators of the binary64 and double-float rooflines
        fp64_peak, fp32_peak = fc.fc_measure_peaks(ctx)
        # ---- rescoring: double-float residuals on the FP32 pipe (binary32 operations / s against the fma probe)
        n_res = sum(s["residuals"] for s in stats)
        res_ms = sum(s["ms_rescore"] for s in stats)
        res_ops = n_res * resid_fp32_ops(w.n_fit) / (res_ms / 1e3) / 1e12 if res_ms > 0 else 0.0
        roofline_rescoring = {"kernel": "k_resid_tiles / k_list_chunks (double-float residual chi2)",
                              "bound": "alu", "achieved": res_ops, "peak": fp32_peak / 2.0, "unit": "Top/s",
                              "frac": res_ops / (fp32_peak / 2.0) if fp32_peak else None,
                              "peak_source": "fc_measure_peaks binary32 fma probe (this run), 1 op per fma",
                              "residuals_per_step": n_res / len(stats),
                              "ops_per_residual": resid_fp32_ops(w.n_fit)}
        # ---- plain binary64 GPU fit on a sample (same metric)
        plain = None
        if not args.no_plain:
            n_pp = args.plain_points if args.plain_points is not None else (20 if args.config == "cfg2" else 1)
            pp = torch.from_numpy(np.linspace(0, w.G - 1, n_pp).round().astype(np.int64)).to(dev)
            m = n_pp * U
            outs = (torch.empty(m, dtype=torch.float64, device=dev), torch.empty(m, dtype=torch.int64, device=dev),
                    torch.empty(m, dtype=torch.int8, device=dev))
            fc.fc_set_frac_cov(ctx, gid, w.F)
            fc.fc_run_points(ctx, gid, pp, 77, U, dict(precision=fc.FC_PREC_FP64), *outs)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fc.fc_set_frac_cov(ctx, gid, w.F)
            a.record(stream)
            fc.fc_run_points(ctx, gid, pp, 78, U, dict(precision=fc.FC_PREC_FP64), *outs)
            b.record(stream)
            torch.cuda.synchronize()
            st = fc.fc_get_stats(ctx)
            pv = st["chi2_evals"] / (a.elapsed_time(b) / 1e3)
            # the scan kernel's own rate: 2 N_fit binary64 flops per chi2 eval (one fma per bin)
            scan_tf = 2.0 * w.n_fit * st["chi2_evals"] / (st["ms_scan64"] / 1e3) / 1e12 if st["ms_scan64"] else 0.0
            plain = {"value": pv, "unit": UNIT, "sample": f"{n_pp} true points x {U} universes, "
                                                          "cold covariance cache", "mixed_speedup": value / ws / pv,
                     "stage_ms": {k: st[k] for k in ("ms_fake", "ms_cov", "ms_scan64", "ms_finish")},
                     "scan_roofline": {"kernel": "k_scan64 (register-tiled binary64 y.s contraction)",
                                       "bound": "fp64", "achieved": scan_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                                       "frac": scan_tf / fp64_peak if fp64_peak else None,
                                       "peak_source": "fc_measure_peaks (binary64 fma probe, this run)"}}
        extras = {}
        if not args.no_extras and args.config == "cfg2":
            extras["cfg3"] = _cfg3_step(fc, ctx, peak)
            extras["cfg4_below_saturation"] = _cfg4_below_saturation(fc, local_rank, args.serve_rate_low,
                                                                       args.serve_seconds_low, args.serve_drain)
        cpu = None
        if not args.no_cpu_baseline and w.S is not None:  # the oracle scans host spectra
            cpu = _oracle_sample(w, args.cpu_seconds, len(os.sched_getaffinity(0)))
        clocks = clk.summary()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": ("bf16 hi/lo x3 screen with f32 accumulation; rescoring in double-float "
                                                      "(2 x f32, ~48 bits); f64 covariances"),
                "data": "synthetic",
                "config": {"workload": desc,
                           "global_batch": n * ws, "true_points": P, "universes_per_point": U,
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "covariance_cache": "cold every step", "autotuned": tuning,
                           "grid_device_bytes": grid_bytes, "l2": l2},
                "universes_per_s": univ / (ms / 1e3),
                "plain_fp64_gpu": plain,
                "stage_ms_per_step": stage,
                "scan_counts": {k: sum(s[k] for s in stats) for k in ("scans", "screened", "rescored", "fallback",
                                                                      "distinct_cov")},
                "roofline": roofline, "roofline_rescoring": roofline_rescoring,
                "measured_fma_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), **extras}
        print(json.dumps(line), flush=True)
    fc.fc_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _serve_stream(fc, ctx, gids, sizes, rate, duration, seed, drain_s):
    """Submit a cfg4 Poisson stream in real time, poll to completion; latency = submit -> done."""
    import numpy as np

    import workloads

    jobs = workloads.cfg4_jobs(sizes, rate, duration, seed)
    pending, lat, failed, evals, univ = {}, [], 0, 0, 0
    errors = {}
    t0 = time.perf_counter()
    i = 0
    while i < len(jobs) or pending:
        now = time.perf_counter() - t0
        while i < len(jobs) and jobs[i][0] <= now:
            _, k, p, sd, U = jobs[i]
            tk, outs = fc.fc_submit(ctx, gids[k], np.array([p], np.int64), sd, U, want_nscans=True)
            pending[tk] = (k, U, outs)
            i += 1
        for tk in list(pending):
            try:
                st, ms = fc.fc_poll(ctx, tk)
            except fc.FCError as e:
                failed += 1
                errors[str(e)] = errors.get(str(e), 0) + 1
                pending.pop(tk)
                continue
            if st == fc.FC_PENDING:
                continue
            k, U, outs = pending.pop(tk)
            lat.append(ms)
            evals += int(outs[2].astype(np.int64).sum()) * sizes[k]
            univ += U
        if now > duration + drain_s:
            for tk in list(pending):
                fc.fc_cancel(ctx, tk)
            t_cancel = time.perf_counter()
            while pending and time.perf_counter() - t_cancel < 120.0:
                for tk in list(pending):
                    try:
                        st, _ = fc.fc_poll(ctx, tk)
                    except fc.FCError:
                        st = None
                    if st != fc.FC_PENDING:
                        pending.pop(tk)
                time.sleep(0.01)
            break
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    a = np.array(lat) if lat else np.array([float("nan")])
    return {"offered_jobs_per_s": rate, "window_s": duration, "jobs": len(jobs), "completed": len(lat),
            "failed": failed, "dropped": len(jobs) - len(lat) - failed, "wall_s": wall,
            "p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max()),
            "throughput_jobs_per_s": len(lat) / wall, "chi2_evals_per_s": evals / wall,
            "universes_per_s": univ / wall, "errors": errors}


def run_serve(args):
    """Serving stream (cfg4): a pool of resident grids, Poisson job arrivals, continuous batching.

    Prints one JSON line with p50/p99 job latency at the offered rate (default
    50 jobs/s, an overload on one GPU: its throughput is the saturation
    throughput) and at half that measured throughput (utilisation < 1)."""
    import numpy as np
    import torch

    import paper_2002_07858_gb300 as fc
    import workloads

    rank, local_rank, ws, dist = _dist_init()
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    fc.load()
    pool = workloads.cfg4_pool()
    ctx = fc.fc_create(local_rank, 80 << 30, None)
    gids = []
    for w in pool:
        g = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
        fc.fc_set_frac_cov(ctx, g, w.F)
        gids.append(g)
    sizes = [w.G for w in pool]
    # warm-up: one small job per grid (scratch, lanes, a few covariances)
    for g, G in zip(gids, sizes):
        fc.fc_run_points(ctx, g, np.array([G // 2], np.int64), 1, 128)
    with ClockSampler(local_rank) as clk:
        over = _serve_stream(fc, ctx, gids, sizes, args.serve_rate, args.serve_seconds, 0, args.serve_drain)
        low_rate = max(0.05, 0.5 * over["throughput_jobs_per_s"])
        low = _serve_stream(fc, ctx, gids, sizes, low_rate, args.serve_seconds_low, 1, args.serve_drain)
    line = {"metric": "p50/p99 job latency", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "value": low["p99_ms"], "data": "synthetic",
            "config": {"workload": "cfg4 serving stream: 8 resident grids (D 2-4, G log-U[1e3,1e6], N U{40..200}), "
                                   "one true point per job, U log-U[100,1e4], Poisson arrivals",
                       "grids": [w.name for w in pool], "hbm_budget_bytes": 80 << 30,
                       "precision": "mixed (tensor-core screen + double-float rescoring)", "max_iter": 5},
            "overload": over, "below_saturation": low, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    fc.fc_destroy(ctx)


def run_sweep(args):
    """Scaling laws of the FC job (§4, Figs. 2, 3 and 7 re-measured on one GPU).

    Series 1: the 100x100 grid (N 90->45), every point a true point, U swept
    (the paper: run time linear in N_univ).  Series 2: U = 1000 at every point
    of an n x n grid of the same generator, n swept (the paper: run time
    quadratic in the number of grid points, since every point is scanned over
    the whole grid).  Each configuration: one untimed job, then one job timed
    with CUDA events on the library's stream (cold covariance cache both
    times).  Prints one JSON line with ms per job, chi2 evals/s ("velocity",
    Fig. 7), universes/s and the log-log slope of each series."""
    import numpy as np
    import torch

    import paper_2002_07858_gb300 as fc
    import workloads

    fc.load()
    stream = torch.cuda.Stream()
    ctx = fc.fc_create(0, 0, stream.cuda_stream)
    opts = dict(precision=fc.FC_PREC_MIXED, top_k=8, max_iter=5)

    def job(n_axis, U):
        S, F, _ = workloads.osc_2d(n_axis, n_axis, 90, seed=0)
        gid = fc.fc_load_grid(ctx, S, workloads.pair_collapse(90), 45)
        G = S.shape[0]
        dev = torch.device("cuda", 0)
        ps = torch.arange(G, dtype=torch.int64, device=dev)
        outs = (torch.empty(G * U, dtype=torch.float64, device=dev), torch.empty(G * U, dtype=torch.int64, device=dev),
                torch.empty(G * U, dtype=torch.int8, device=dev))
        fc.fc_set_frac_cov(ctx, gid, F)
        fc.fc_run_points(ctx, gid, ps, 5, U, opts, *outs)
        torch.cuda.synchronize()
        fc.fc_set_frac_cov(ctx, gid, F)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fc.fc_run_points(ctx, gid, ps, 6, U, opts, *outs)
        b.record(stream)
        torch.cuda.synchronize()
        st = fc.fc_get_stats(ctx)
        fc.fc_unload_grid(ctx, gid)
        ms = a.elapsed_time(b)
        return {"grid": f"{n_axis}x{n_axis}", "G": G, "U": U, "ms": ms, "chi2_evals_per_s": st["chi2_evals"] / ms * 1e3,
                "universes_per_s": G * U / ms * 1e3, "scans_per_universe": st["scans"] / (G * U)}

    def slope(xs, ys):
        return float(np.polyfit(np.log(xs), np.log(ys), 1)[0])

    with ClockSampler(0) as clk:
        by_u = [job(100, U) for U in (125, 250, 500, 1000, 2000)]
        by_g = [job(n, 1000) for n in (25, 50, 71, 100, 141, 200)]
    big_u = [r for r in by_u if r["U"] >= 500]
    big_g = [r for r in by_g if r["G"] >= 5000]
    line = {"metric": "FC job time scaling", "unit": "ms", "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "D=2 n x n grids of the 100x100 generator, N 90->45, every grid point a true "
                                   "point, <= 5 scans, top-8, mixed precision"},
            "vs_universes": by_u, "vs_grid_points": by_g,
            "slope_time_vs_U": slope([r["U"] for r in big_u], [r["ms"] for r in big_u]),
            "slope_time_vs_G": slope([r["G"] for r in big_g], [r["ms"] for r in big_g]),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    fc.fc_destroy(ctx)


def run_once(args):
    """One untimed FC job (for profilers): the configured points x universes, stats printed as JSON."""
    import numpy as np

    import paper_2002_07858_gb300 as fc
    import workloads

    fc.load()
    if args.config in ("cfg3", "cfg5"):
        w = workloads.cfg3(U=args.universes or 500) if args.config == "cfg3" else _cfg5(workloads, args)
        pts = w.points if args.points is None else w.points[np.linspace(0, len(w.points) - 1, args.points).astype(int)]
    else:
        w = workloads.cfg2(U=args.universes or 1000)
        pts = np.linspace(0, w.G - 1, args.points).round().astype(np.int64) if args.points else w.points
    ctx = fc.fc_create(0)
    gid = _load_grid(fc, ctx, w)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    fc.fc_run_points(ctx, gid, pts, 1, w.U, dict(precision=args.precision, top_k=args.top_k))
    print(json.dumps({"once": {"points": int(len(pts)), "universes": w.U, **fc.fc_get_stats(ctx)}}), flush=True)
    fc.fc_destroy(ctx)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="cfg2", choices=["cfg2", "cfg3", "cfg5"],
                    help="cfg2 (the metric's workload, default), cfg3 (D=3, N=120, 2048 points x 500) or "
                         "cfg5 (D=6, 16^6 points, N=64, 256 points x 16)")
    ap.add_argument("--universes", type=int, default=None, help="universes per true point (default: the config's)")
    ap.add_argument("--points", type=int, default=None, help="true points (default: all 10^4)")
    ap.add_argument("--top-k", type=int, default=None, help="candidates per universe (default 8; cfg5: 16)")
    ap.add_argument("--plain-points", type=int, default=None, help="plain binary64 sample (default 20; cfg3, cfg5: 1)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--once", action="store_true", help="run one untimed job and print its stats (for profilers)")
    ap.add_argument("--precision", type=int, default=1, help="with --once: 1 = mixed, 0 = plain fp64")
    ap.add_argument("--serve", action="store_true", help="cfg4 serving stream: p50/p99 job latency (own JSON line)")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="offered jobs/s of the overload stream")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window of the overload stream")
    ap.add_argument("--serve-seconds-low", type=float, default=15.0, help="arrival window below saturation")
    ap.add_argument("--serve-rate-low", type=float, default=1.5,
                    help="offered jobs/s of the default line's below-saturation cfg4 stream")
    ap.add_argument("--recompute", action="store_true",
                    help="cfg5: keep the grid as its shape model (no spectra stored; FC_GRID_RECOMPUTE)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the cfg3 step and the cfg4 below-saturation stream of the default line")
    ap.add_argument("--serve-drain", type=float, default=240.0, help="seconds after a window before cancelling")
    ap.add_argument("--sweep", action="store_true", help="job time vs universes and vs grid size (own JSON line)")
    args = ap.parse_args()
    if args.top_k is None:
        args.top_k = 16 if args.config == "cfg5" else 8
    if args.once:
        run_once(args)
    elif args.sweep:
        run_sweep(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
