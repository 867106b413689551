#!/usr/bin/env python3
"""Benchmark: batched VEGAS evaluation of all third-order Hugenholtz diagrams of
pure neutron matter over a density scan (3 diagrams x kF in {0.8, ..., 1.7} fm^-1,
2^22 samples per integral per iteration), on one B300.

A step is one VEGAS iteration over all 30 integrals: Philox sampling, VEGAS map,
integrand, per-chunk sums and histograms, the fixed-order reduction, the
combination of the iteration into each estimate and the grid refinement.
The headline arm runs it batched (one persistent launch per iteration, CUDA
graph) in mixed precision; the FP64 batched path and the plain per-diagram FP64
loop run the same workload beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "integrand evals/s; diagrams to 0.1% err/s vs plain FP64 loop; p50/p99 EOS latency"
UNIT = "integrand evals/s"
KF_SCAN = [round(0.8 + 0.1 * i, 2) for i in range(10)]
SAMPLES = 1 << 22
ORDER = 3
WORKLOAD = "third-order Hugenholtz diagrams (pp, hh, ph), pure neutron matter, kF 0.8..1.7 fm^-1 (10 points), 12D, 2^22 samples/iteration"

# FP64 operations per sample of an order-3 integral, mixed precision (FP32 sampling map), in the
# formulation of csrc/mbpt_device.cuh.  A sample that fails a Fermi step by more than the FP32 error
# bound is rejected by the FP32 pre-test with no FP64 work.  A live sample: chord momenta 3 products
# + |l|^2 3 = 6 per chord (24; the chord Jacobians, the VEGAS Jacobian and the weight's constant factor
# are one FP32 mantissa product), tree lines 6 sums + |k|^2 3 = 9 per line (18), energy denominators
# (7 sums, 1 product), weight (2 products), Newton reciprocal of the denominator product (4), sum w and
# sum w^2 (2) = 58.
# (About 1 % of samples lie near a Fermi surface and are placed with the FP64 map instead.)
FP64_OPS_LIVE = 58.0
# dram__bytes_read.sum + dram__bytes_write.sum of one k_iterate_256x2 launch on the 30 x 2^20 profiling case
# (profiles/k_iterate_third_order_scan.md): records, grids and chunk slots, as many chunks (128 per integral)
# as the benchmark launch; not proportional to samples
TRAFFIC_BYTES = 676608
# nominal FP64 rate of the recipe (1.25 TFLOP/s, FMA = 2 flops) in FP64 instructions per second
FP64_PEAK_NOMINAL = 1.25e12 / 2.0
# measured DFMA rate on this machine's B300 (paper_2603_24532_b300/csrc/pipe_peaks.cu, profiles/pipe_peaks_b300.md),
# FP64 thread operations per second at the SM clock of that run; scaled to the clock seen under load
FP64_PEAK_MEASURED = 4.73e11
FP64_PEAK_MEASURED_MHZ = 1938.5


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def slowest_rank_ms(dist, t_ms: float, device) -> float:
    """The step time of the job: the maximum over ranks (every rank holds its own replicas, so the
    job's throughput is all ranks' units over the slowest rank's time)."""
    if dist is None:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: float, t_ms: float) -> float:
    """Whole-job throughput (weak scaling: every rank processes the same units)."""
    return world * units_per_rank / (t_ms * 1e-3)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_integrals(M, ctx, precision, seed_base=1, stream_base=0, map_kind=0):
    descs = M.mbpt_generate(ORDER)
    gs, meta = [], []
    for ki, kf in enumerate(KF_SCAN):
        ph = M.physics(kF_n=kf, kF_p=0.0, K_max=kf + 6.0, map_kind=map_kind)
        for d in descs:
            sid = stream_base + 100 * ki + d.diagram_id
            cfg = M.vegas_cfg(samples=SAMPLES, seed=seed_base, stream_id=sid, precision=precision)
            gs.append(M.mbpt_create_diagram(ctx, d, ph, cfg))
            meta.append((kf, d.diagram_id))
    return gs, meta


def l2_flush(torch, buf):
    buf.add_(1)


def run_gpu(args):
    import torch

    from paper_2603_24532_b300 import mbpt as M

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    arena = torch.empty(32 << 30, dtype=torch.uint8, device=dev)   # chunk slots of the largest batch at the smallest tuned chunks
    ctx = M.mbpt_ctx_create(local, arena.numel(), arena_ptr=arena.data_ptr())
    stream = torch.cuda.ExternalStream(M.mbpt_ctx_stream(ctx), device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)    # 256 MiB > 126 MB L2

    def timed_steps(gs, k, per_diagram=False):
        ms_it, ms_step = [], []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.add_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            if per_diagram:
                it = 0.0
                for g in gs:
                    M.mbpt_vegas_iterate(ctx, [g], 1)
                    it += M.mbpt_ctx_last_timing(ctx)[0]
                with torch.cuda.stream(stream):
                    e1.record(stream)
                torch.cuda.synchronize()
                ms_it.append(it)
            else:
                M.mbpt_vegas_iterate(ctx, gs, 1)
                with torch.cuda.stream(stream):
                    e1.record(stream)
                torch.cuda.synchronize()
                ms_it.append(M.mbpt_ctx_last_timing(ctx)[0])
            ms_step.append(e0.elapsed_time(e1))
        return np.array(ms_it), np.array(ms_step)

    from paper_2603_24532_b300.autotune import autotune

    # ---- headline: batched, mixed precision, launch shape from the autotuner (untimed, states restored)
    gs, meta = build_integrals(M, ctx, M.MBPT_MIXED, seed_base=1 + rank, stream_base=10000 * rank)
    n_int = len(gs)
    tuned = autotune(ctx, gs, trials=1)["best"] if args.autotune else None
    timed_steps(gs, args.warmup)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms_it, ms_step = timed_steps(gs, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = slowest_rank_ms(dist, float(np.mean(ms_step)), dev)
    evals_step = n_int * SAMPLES
    value = job_value(world, evals_step, t_step)
    res_mixed = [M.mbpt_estimate(g) for g in gs]

    # live-sample fraction on the adapted grids (for the algorithmic FP64 work per sample)
    live = []
    for g in gs[:: max(1, n_int // 6)]:
        _, w = M.mbpt_dump_samples(g, 10 ** 6, 0, 1 << 15, 12, with_x=False)
        live.append(np.mean(w != 0))
    live_frac = float(np.mean(live))
    ops = FP64_OPS_LIVE * live_frac
    it_ms = float(np.mean(ms_it))
    achieved = ops * evals_step / (it_ms * 1e-3)

    # ---- e2e through the public API: per step H2D of the work table inside mbpt_vegas_iterate (a
    # 96-byte item and an 8-byte histogram pointer per integral, an 80-byte header) and a D2H read of
    # every integral's estimate with one synchronisation (80 bytes each, and the 4-byte error word)
    h2d = n_int * (96 + 8) + 80
    d2h = n_int * 80 + 4
    t0 = time.perf_counter()
    for _ in range(args.steps):
        M.mbpt_vegas_iterate(ctx, gs, 1)
        _ = [r.mean for r in M.mbpt_estimate_batch(gs)]
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_value = world * evals_step / e2e_s
    # ---- precision: mixed modes vs FP64 on identical counters and grids, paired over several
    # iterations (each trial restores the same grid and sets the iteration counter), per integral;
    # the scale of a near-zero diagram is 1e-3 of its order's sum
    imgs = [M.mbpt_get_state(g) for g in gs]
    twins = {}
    for name, prec in (("fp64", M.MBPT_FP64), ("map64", M.MBPT_MIXED_MAP64)):
        twins[name] = []
        for (kf, did) in meta:
            d = M.mbpt_generate(ORDER)[did]
            ph = M.physics(kF_n=kf, kF_p=0.0, K_max=kf + 6.0)
            sid = 10000 * rank + 100 * KF_SCAN.index(kf) + did
            twins[name].append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=SAMPLES, seed=1 + rank,
                                                                              stream_id=sid, precision=prec)))
    sets = {"mixed": gs, "fp64": twins["fp64"], "map64": twins["map64"]}
    trials = 6
    means = {k: np.zeros((trials, n_int)) for k in sets}
    t0_iter = 1000
    for k in range(trials):
        for name, arr in sets.items():
            for g, img in zip(arr, imgs):
                M.mbpt_set_state(g, M.state_with_iter(img, t0_iter + k))
            M.mbpt_vegas_iterate(ctx, arr, 1)
            means[name][k] = [r.last_mean for r in M.mbpt_estimate_batch(arr)]
    ref = means["fp64"]
    scale = np.zeros(n_int)
    for ki in range(len(KF_SCAN)):
        sl = slice(3 * ki, 3 * ki + 3)
        scale[sl] = np.maximum(np.abs(ref[:, sl]).mean(axis=0), 1e-3 * abs(np.sum(ref[:, sl].mean(axis=0))))
    precision_dev = {"definition": "paired over %d iterations on identical counters and grids: mean of "
                                   "(I_mode - I_fp64) / max(|I_fp64|, 1e-3 |order sum|) per integral" % trials}
    for name in ("mixed", "map64"):
        dif = (means[name] - ref) / scale
        mdif, se = dif.mean(axis=0), dif.std(axis=0, ddof=1) / np.sqrt(trials)
        precision_dev[name] = {"max_abs_mean": float(np.max(np.abs(mdif))),
                               "median_abs_mean": float(np.median(np.abs(mdif))),
                               "max_single_iteration": float(np.max(np.abs(dif))),
                               "max_abs_mean_over_se": float(np.max(np.abs(mdif) / np.maximum(se, 1e-300)))}
    for arr in twins.values():
        for g in arr:
            M.mbpt_destroy_diagram(g)
    for g in gs:
        M.mbpt_destroy_diagram(g)

    # ---- the same scan with the rotational reduction of the chord map (9D instead of 12D; NEXT row)
    grot, _ = build_integrals(M, ctx, M.MBPT_MIXED, seed_base=1 + rank, stream_base=10000 * rank, map_kind=1)
    timed_steps(grot, args.warmup)
    itrot, strot = timed_steps(grot, max(4, args.steps // 4))
    res_rot = M.mbpt_estimate_batch(grot)
    for g in grot:
        M.mbpt_destroy_diagram(g)
    vrot = world * evals_step / (float(np.mean(strot)) * 1e-3)

    # ---- fourth-order batch (all 39 diagrams x kF {1.0, 1.33, 1.6} x {PNM, SNM}, 2^24 samples each,
    # anomalous ones flagged and skipped): throughput of one batched iteration
    g4 = []
    for ki, kf in enumerate((1.0, 1.33, 1.6)):
        for mi, kfp in enumerate((0.0, kf)):
            ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0)
            for d in M.mbpt_generate(4):
                if d.anomalous:
                    continue
                g4.append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(
                    samples=1 << 24, seed=1 + rank, stream_id=10000 * rank + 1000 * mi + 100 * ki + d.diagram_id,
                    precision=M.MBPT_MIXED)))
    M.mbpt_vegas_iterate(ctx, g4, 1)
    torch.cuda.synchronize()
    it4, st4 = timed_steps(g4, 2)
    for g in g4:
        M.mbpt_destroy_diagram(g)
    v4 = world * len(g4) * (1 << 24) / (float(np.mean(st4)) * 1e-3)

    # ---- the same fourth-order workload as group integrals (Sec. III.A): per physics point one integral
    # per particle-hole group (4 groups of the 33 non-anomalous diagrams), 2^24 samples each, every
    # sample evaluating all members: the same member evaluations per iteration as the batch above
    gg, n_member_evals = [], 0
    for ki, kf in enumerate((1.0, 1.33, 1.6)):
        for mi, kfp in enumerate((0.0, kf)):
            ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0)
            by_key = {}
            for d in M.mbpt_generate(4):
                if not d.anomalous:
                    by_key.setdefault(M.mbpt_hole_chords(d), []).append(d)
            for key, ds in sorted(by_key.items()):
                gg.append(M.mbpt_create_group(ctx, ds, ph, M.vegas_cfg(
                    samples=1 << 24, seed=1 + rank, stream_id=10000 * rank + 1000 * mi + 100 * ki + 50 + key,
                    precision=M.MBPT_MIXED)))
                n_member_evals += len(ds) << 24
    M.mbpt_vegas_iterate(ctx, gg, 1)
    torch.cuda.synchronize()
    itg, stg = timed_steps(gg, 2)
    for g in gg:
        M.mbpt_destroy_diagram(g)
    vg = world * n_member_evals / (float(np.mean(stg)) * 1e-3)

    # ---- sixth order (Table I: 27300 diagrams, d = 21; the paper's proof-of-principle order): every
    # non-anomalous diagram, one integral per mirror pair (11269), PNM kF = 1.33, 2^16 samples each
    t6 = time.perf_counter()
    ph6 = M.physics(kF_n=1.33, K_max=7.33)
    g6 = [M.mbpt_create_diagram(ctx, d, ph6, M.vegas_cfg(samples=1 << 16, seed=1 + rank,
                                                         stream_id=100000 * rank + d.diagram_id,
                                                         precision=M.MBPT_MIXED))
          for d in M.mbpt_generate(6) if not d.anomalous and d.diagram_id <= d.mirror_id]
    create6_s = time.perf_counter() - t6
    M.mbpt_vegas_iterate(ctx, g6, 1)
    torch.cuda.synchronize()
    it6, st6 = timed_steps(g6, 2)
    for g in g6:
        M.mbpt_destroy_diagram(g)
    v6 = world * len(g6) * (1 << 16) / (float(np.mean(st6)) * 1e-3)

    # ---- FP64 batched, same workload (tuned the same way)
    g64, _ = build_integrals(M, ctx, M.MBPT_FP64, seed_base=1 + rank, stream_base=10000 * rank)
    tuned64 = autotune(ctx, g64, trials=1)["best"] if args.autotune else None
    timed_steps(g64, args.warmup)
    it64, st64 = timed_steps(g64, args.steps)
    res64 = [M.mbpt_estimate(g) for g in g64]
    for g in g64:
        M.mbpt_destroy_diagram(g)
    v64 = world * evals_step / (float(np.mean(st64)) * 1e-3)

    # ---- plain per-diagram FP64 loop: one launch per integral per iteration, default launch shape
    M.mbpt_ctx_set_kernel(ctx, 256, 2)
    for o in (2, 3, 4, 5):
        M.mbpt_ctx_set_launch(ctx, o, 32)
    gk0, _ = build_integrals(M, ctx, M.MBPT_FP64, seed_base=1 + rank, stream_base=10000 * rank)
    timed_steps(gk0, max(1, args.warmup // 2), per_diagram=True)
    itk0, stk0 = timed_steps(gk0, max(2, args.steps // 2), per_diagram=True)
    for g in gk0:
        M.mbpt_destroy_diagram(g)
    vk0 = world * evals_step / (float(np.mean(stk0)) * 1e-3)

    # ---- time to 0.1 % statistical error per integral, from each run's own variance
    def diags_per_s(results, rate):
        need = 0.0
        for r in results:
            if r.mean == 0.0 or r.sigma == 0.0:
                continue
            need += r.n_evals * (r.sigma / (1e-3 * abs(r.mean))) ** 2
        return len(results) / (need / rate) if need > 0 else None

    d_mixed = diags_per_s(res_mixed, value)
    d_rot = diags_per_s(res_rot, vrot)
    d_k0 = diags_per_s(res64, vk0)
    M.mbpt_ctx_destroy(ctx)
    del arena
    torch.cuda.synchronize()

    # ---- serving: a short Poisson stream of equation-of-state requests (p50/p99 latency)
    serving = None
    if args.serve_requests > 0:
        from paper_2603_24532_b300 import serve as S
        be = S.MbptBackend(device=local, arena_bytes=8 << 30)
        srv = S.Server(be, budget_bytes=6 << 30)
        trace = S.poisson_trace(args.serve_requests, 20.0, 7 + rank)
        t0 = time.perf_counter()
        done = srv.run(trace, realtime=True, time_limit=args.serve_seconds)
        wall = time.perf_counter() - t0
        st = S.latency_stats(done)
        met = [r for r in done if r.energy is not None and r.sigma is not None and r.sigma <= r.target * abs(r.energy)]
        serving = {"requests": len(trace), "completed": len(done), "wall_s": wall, "p50_s": st["p50_s"],
                   "p99_s": st["p99_s"], "target_met_fraction": len(met) / max(1, len(done)),
                   "workload": "Poisson 20/s, n ~ U[0.04, 0.20] fm^-3, delta {0..1}, order cap {2,3,4}, "
                               "target {1, 0.3, 0.1} %, seed 7 (+rank)"}
        be.close()
    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    cpu = cpu_baseline(budget_s=args.cpu_seconds) if world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "integrals": n_int, "samples_per_iter": SAMPLES,
                   "precision": "mixed (FP32 potentials, spin sum and sampling map; FP64 line momenta, Fermi steps, energy denominators, sums, grid)",
                   "step": "one batched VEGAS iteration over all integrals (sample, integrate, reduce, combine, refine)",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "launch": tuned},
        "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved / 1e9, "peak": FP64_PEAK_NOMINAL / 1e9,
                     "unit": "FP64 Gop/s (DADD-equivalents)", "frac": achieved / FP64_PEAK_NOMINAL,
                     "peak_kind": "nominal 1.25 TFLOP/s FP64 of the recipe at 2032 MHz",
                     "frac_of_measured_dfma": achieved / (FP64_PEAK_MEASURED * (clk.get("sm_mhz") or 2032.0)
                                                          / FP64_PEAK_MEASURED_MHZ),
                     "measured_dfma_note": "4.73e11 FP64 op/s at 1938 MHz, scaled to the median SM clock of the run",
                     "ops_per_sample": ops, "live_fraction": live_frac, "kernel": "k_iterate",
                     "kernel_ms": it_ms, "traffic": TRAFFIC_BYTES,
                     "traffic_note": "ncu dram read+write of one k_iterate launch on the 30 x 2^20 profiling case "
                                     "(grids and records; the 128 chunk slots per integral, as many as in this "
                                     "launch, stay in L2), not proportional to samples"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 5 * args.steps,   # per step: k_iterate parts (plain; regulated and group parts empty here), k_finalize
        "clocks": clk,
        "fp64_batched": {"value": v64, "unit": UNIT, "kernel_ms": float(np.mean(it64)), "launch": tuned64},
        "k0_plain_fp64_per_diagram": {"value": vk0, "unit": UNIT, "launches_per_step": 2 * n_int},
        "speedup_vs_k0": value / vk0,
        "mixed_vs_fp64_deviation": precision_dev,
        "diagrams_to_0p1pct_per_s": {"batched_mixed": d_mixed, "k0_plain_fp64": d_k0,
                                     "ratio": (d_mixed / d_k0) if (d_mixed and d_k0) else None,
                                     "batched_mixed_rotational_9d": d_rot},
        "fourth_order_batch": {"value": v4, "unit": UNIT, "integrals": len(g4), "samples_per_iter": 1 << 24,
                               "ms_per_iteration": float(np.mean(st4)),
                               "workload": "39 fourth-order diagrams (33 non-anomalous) x kF {1.0,1.33,1.6} x {PNM,SNM}, mixed"},
        "fourth_order_groups": {"value": vg, "unit": UNIT + " (member diagrams)", "integrals": len(gg),
                                "samples_per_iter": 1 << 24, "ms_per_iteration": float(np.mean(stg)),
                                "vs_per_diagram_batch": vg / v4,
                                "workload": "the fourth_order_batch diagrams as 4 particle-hole groups per physics "
                                            "point (24 group integrals), mixed"},
        "sixth_order_batch": {"value": v6, "unit": UNIT, "integrals": len(g6), "samples_per_iter": 1 << 16,
                              "ms_per_iteration": float(np.mean(st6)), "create_s": create6_s,
                              "workload": "27300 sixth-order diagrams, one integral per mirror pair of the 21572 "
                                          "non-anomalous ones, PNM kF 1.33, d = 21, mixed"},
        "rotational_9d": {"value": vrot, "unit": UNIT, "kernel_ms": float(np.mean(itrot)),
                          "note": "same scan with chord 0 along z and chord 1 in the xz plane (d = 9)"},
        "serving": serving,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return line


def cpu_baseline(budget_s=12.0, steps=None):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the same
    workload (every integral, the same number of samples each, uniform grid)."""
    import oracle as O

    Ds = O.enumerate_diagrams(ORDER)
    cores = os.cpu_count() or 1
    # calibrate on one integral
    po = O.Physics(kF_n=1.2, K_max=7.2)
    grid = O.uniform_grid(12, 50)
    m, dt = 1 << 14, 0.0
    while dt < 0.3 and m < (1 << 22):
        m *= 2
        t0 = time.perf_counter()
        for D in Ds:
            O.vegas_iteration(D, po, grid, 1, 0, 0, m, threads=cores)
        dt = time.perf_counter() - t0
    per = dt / (m * len(Ds))
    n = int(max(1024, min(1 << 22, budget_s / (per * len(KF_SCAN) * len(Ds)))))
    t0 = time.perf_counter()
    total = 0
    for ki, kf in enumerate(KF_SCAN):
        po = O.Physics(kF_n=kf, K_max=kf + 6.0)
        for D in Ds:
            O.vegas_iteration(D, po, grid, 1, 100 * ki + D.diagram_id, 0, n, threads=cores)
            total += n
    dt = time.perf_counter() - t0
    return {"value": total / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d samples of each of the 30 integrals (uniform grid, iteration 0), %.1f s" % (n, dt)}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    cb = None
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(budget_s=args.ref_seconds)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "integrals": 30, "samples_per_iter": SAMPLES,
                       "step": "bounded sample of one iteration of every integral on the host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--serve-requests", type=int, default=400, help="short serving run (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=40.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
