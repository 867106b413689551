#!/usr/bin/env python3
"""Benchmark on one B300.  Headline: one batched VEGAS iteration over every non-anomalous fifth-order
Hugenholtz diagram of pure neutron matter at kF in {1.0, 1.33, 1.6} fm^-1 (668 x 3 = 2004 integrals,
18 dimensions, 2^20 samples per integral per iteration), mixed precision.

A step is one VEGAS iteration over all 2004 integrals: Philox sampling, VEGAS map, integrand, per-chunk
sums and histograms, the fixed-order reduction, the combination of the iteration into each estimate and
the grid refinement, as one persistent launch per batch part plus the finalize launch, replayed from a
CUDA graph.  Beside it, from the same run: the same workload end to end through the C ABI, the time for
every fifth-order integral to reach 0.5 % (or an absolute floor for near-zero diagrams), the plain
per-diagram FP64 loop on a subset, the mixed-vs-FP64 deviation, the third-order density scan (with the
FP64 batched path and the plain loop), the fourth-order batch and its aligned groups, the sixth-order
batch, and the serving stream (p50/p99 latency, diagrams/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--profile-case fifth|third|sixth]
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
# fifth order (headline)
KF5 = (1.0, 1.33, 1.6)
SAMPLES5 = 1 << 20
ALPHA5 = 0.75
WORKLOAD = ("all 840 fifth-order Hugenholtz diagrams (668 non-anomalous; both members of every mirror pair "
            "evaluated) x kF {1.0, 1.33, 1.6} fm^-1, pure neutron matter, 18D, 2^20 samples/iteration, mixed")
# third order (density scan)
KF_SCAN = [round(0.8 + 0.1 * i, 2) for i in range(10)]
SAMPLES3 = 1 << 22
# nominal FP64 rate of the recipe (1.25 TFLOP/s, FMA = 2 flops) in FP64 instructions per second at 2032 MHz
FP64_PEAK_NOMINAL = 1.25e12 / 2.0
# FP64 thread operations (DADD + DMUL + DFMA, ncu) per sample of the profiled k_iterate launches
FP64_OPS_FILE = os.path.join(ROOT, "profiles", "fp64_ops_per_sample.txt")


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


def measured_counters(workload: str):
    """ncu counters of one k_iterate launch of a workload, from the committed summary (lines `<workload>
    <FP64 ops per sample> <samples per launch> <dadd> <dmul> <dfma> <dram read B> <dram write B> <warp
    instructions> <threads per block> <samples per thread> ...`): a dict, or None if the file has no such line."""
    try:
        with open(FP64_OPS_FILE) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 11 and not line.startswith("#") and parts[0] == workload:
                    return {"ops_per_sample": float(parts[1]), "samples": int(parts[2]),
                            "dram_bytes": int(parts[6]) + int(parts[7]), "warp_inst": int(parts[8]),
                            "chunk": int(parts[9]) * int(parts[10])}
    except (OSError, ValueError):
        pass
    return None


def measured_fp64_ops(workload: str):
    """FP64 thread operations per sample of a workload (measured_counters), or None."""
    c = measured_counters(workload)
    return c["ops_per_sample"] if c else None


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


# ---------------------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------------------
def fifth_order_integrals(M, ctx, precision, samples=SAMPLES5, seed=1, stream_base=0, every=1, map_kind=0, **cfg_kw):
    """The 2004 fifth-order integrals (or every `every`-th of them), with their (kF, descriptor); map_kind 1:
    the rotational reduction (15 dimensions)."""
    descs = [d for d in M.mbpt_generate(5) if not d.anomalous]
    gs, meta = [], []
    k = 0
    for ki, kf in enumerate(KF5):
        ph = M.physics(kF_n=kf, K_max=kf + 6.0, map_kind=map_kind)
        for d in descs:
            k += 1
            if (k - 1) % every:
                continue
            cfg = M.vegas_cfg(samples=samples, seed=seed, stream_id=stream_base + 1000 * ki + d.diagram_id,
                              precision=precision, alpha=ALPHA5, **cfg_kw)
            gs.append(M.mbpt_create_diagram(ctx, d, ph, cfg))
            meta.append((kf, d))
    return gs, meta


def third_order_integrals(M, ctx, precision, seed=1, stream_base=0, map_kind=0):
    descs = M.mbpt_generate(3)
    gs, meta = [], []
    for ki, kf in enumerate(KF_SCAN):
        ph = M.physics(kF_n=kf, kF_p=0.0, K_max=kf + 6.0, map_kind=map_kind)
        for d in descs:
            sid = stream_base + 100 * ki + d.diagram_id
            cfg = M.vegas_cfg(samples=SAMPLES3, seed=seed, stream_id=sid, precision=precision)
            gs.append(M.mbpt_create_diagram(ctx, d, ph, cfg))
            meta.append((kf, d.diagram_id))
    return gs, meta


def destroy(M, gs):
    for g in gs:
        M.mbpt_destroy_diagram(g)


def run_gpu(args):
    import torch

    from paper_2603_24532_b300 import mbpt as M
    from paper_2603_24532_b300 import run_fifth_order as RF
    from paper_2603_24532_b300.autotune import autotune

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    arena = torch.empty(32 << 30, dtype=torch.uint8, device=dev)   # room for the largest batch's chunk slots
    ctx = M.mbpt_ctx_create(local, arena.numel(), arena_ptr=arena.data_ptr())
    stream = torch.cuda.ExternalStream(M.mbpt_ctx_stream(ctx), device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)    # 256 MiB > 126 MB L2

    def timed_steps(gs, k, per_diagram=False):
        """k iterations; per step the k_iterate time (events inside the graph) and the step time (events
        around it on the context stream), with the L2 flushed before each step outside the events."""
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

    seed = 1 + rank
    sbase = 100000 * rank

    # ================= headline: fifth order, batched, mixed ==========================================
    # launch setting from the autotuner on every fourth integral (states restored), then the full batch
    tuned = None
    if args.autotune:
        sub, _ = fifth_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed, stream_base=sbase, every=4)
        M.mbpt_vegas_iterate(ctx, sub, 2)
        at = autotune(ctx, sub, trials=1)
        tuned = dict(at["launch"])
        tuned["search_ms"] = {"%dx%d spt%d" % (r["threads"], r["min_blocks"], r["spt"]): round(r["ms"], 2)
                              for r in at["table"]}
        tuned["search_ms"].update({"hist %d" % r["layout"]: round(r["ms"], 2) for r in at["layout_table"]})
        tuned["search_ms"].update({"spin %s" % ("fold" if r["spin_sum"] == M.MBPT_SPIN_FOLD else "table"):
                                   round(r["ms"], 2) for r in at["spin_table"]})
        tuned["search_batch"] = "every fourth fifth-order integral (501), one iteration each"
        destroy(M, sub)
    gs5, meta5 = fifth_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed, stream_base=sbase)
    n5 = len(gs5)
    timed_steps(gs5, args.warmup)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms_it, ms_step = timed_steps(gs5, args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = slowest_rank_ms(dist, float(np.mean(ms_step)), dev)
    evals_step = n5 * SAMPLES5
    value = job_value(world, evals_step, t_step)
    it_ms = float(np.mean(ms_it))

    # roofline of the dominant kernel: measured FP64 thread operations per sample (ncu) x samples per
    # launch / its CUDA-event time, against the FP64 rate measured here with the library's DFMA loop
    cnt5 = measured_counters("fifth_order_mixed")
    ops5 = cnt5["ops_per_sample"] if cnt5 else None
    fp64_rate = M.mbpt_fp64_rate(local, M.mbpt_ctx_stream(ctx))
    achieved = (ops5 * evals_step / (it_ms * 1e-3)) if ops5 else None
    # DRAM bytes of a launch of this shape: the counters come from a launch of the same kernel and integrals with
    # fewer samples per integral (2^18), whose traffic -- the chunk slots, written once per chunk -- grows with the
    # number of chunks, so it is scaled to the headline launch's chunks (its samples over its chunk size); and
    # the share of the SMs' instruction issue slots (4 warp instructions per SM per cycle) the launch uses
    tpb5, _, spt5 = M.mbpt_ctx_get_launch(ctx, 5)
    traffic5 = (cnt5["dram_bytes"] * (evals_step / (tpb5 * spt5)) / (cnt5["samples"] / cnt5["chunk"])) if cnt5 else None
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_frac = (cnt5["warp_inst"] / cnt5["samples"] * evals_step / (it_ms * 1e-3)
                  / (4.0 * n_sm * clk["sm_mhz"] * 1e6)) if cnt5 and clk.get("sm_mhz") else None

    # end to end through the public API: per step the work table goes up inside mbpt_vegas_iterate
    # (a WORK_ITEM_BYTES item and an 8-byte histogram pointer per integral, the work header), and
    # mbpt_estimate_batch sends the integrals' 8-byte state pointers and reads every integral's 80-byte
    # state head back in one copy, with one synchronisation
    h2d = n5 * (M.WORK_ITEM_BYTES + 8 + 8) + M.WORK_HEADER_BYTES
    d2h = n5 * M.RESULT_BYTES + 4
    t0 = time.perf_counter()
    for _ in range(args.steps):
        M.mbpt_vegas_iterate(ctx, gs5, 1)
        _ = [r.mean for r in M.mbpt_estimate_batch(gs5)]
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_value = world * evals_step / e2e_s

    # grids adapted by the timed iterations, for the paired precision check below
    grids5 = {}
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(n5, size=48, replace=False))
    for i in pick:
        grids5[i] = M.state_grid(M.mbpt_get_state(gs5[i]), 18, 50)
    destroy(M, gs5)

    # time for every fifth-order integral to reach 0.5 % relative error: 3 training iterations, then the
    # frozen-grid evaluation phase; a near-zero diagram's target is the absolute floor 0.5 % |E5| /
    # sqrt(668) of its kF (its share of a 0.5 % error of the order's sum); at most 40 iterations
    t0 = time.perf_counter()
    gsc, metac = fifth_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed + 100, stream_base=sbase, train_iters=3,
                                       combine=M.MBPT_COMBINE_POOLED, target_rel=0.005)
    M.mbpt_vegas_iterate(ctx, gsc, 3)
    rc = M.mbpt_estimate_batch(gsc)
    floors = {}
    for kf in KF5:
        idx = [i for i, (k, _) in enumerate(metac) if k == kf]
        floors[kf] = 0.005 * abs(sum(rc[i].last_mean for i in idx)) / math.sqrt(len(idx))
    for g, (kf, d) in zip(gsc, metac):
        cfg = M.vegas_cfg(samples=SAMPLES5, seed=seed + 100, stream_id=sbase + 1000 * KF5.index(kf) + d.diagram_id,
                          precision=M.MBPT_MIXED, alpha=ALPHA5, train_iters=3, combine=M.MBPT_COMBINE_POOLED,
                          target_rel=0.005, target_abs=floors[kf])
        M.mbpt_set_config(g, cfg)
    # adaptive samples per iteration (PVegas, Sec. III.C; run_fifth_order.converge): the integrals closest to
    # their targets get what they still need first (up to 2^22 per iteration), the rest 2^18, within 2^20
    # samples per unconverged integral per iteration
    def cfg5(i, n):
        kf, d = metac[i]
        return M.vegas_cfg(samples=n, seed=seed + 100, stream_id=sbase + 1000 * KF5.index(kf) + d.diagram_id,
                           precision=M.MBPT_MIXED, alpha=ALPHA5, train_iters=3, combine=M.MBPT_COMBINE_POOLED,
                           target_rel=0.005, target_abs=floors[kf])
    iters, ev, _ = RF.converge(M, ctx, gsc, lambda r, i: max(0.005 * abs(r.mean), floors[metac[i][0]]), cfg5,
                               lambda r: r.n_evals - 3 * SAMPLES5, base_samples=SAMPLES5, max_iters=40,
                               iters_done=3)
    conv_evals = 3 * len(gsc) * SAMPLES5 + ev
    rc = M.mbpt_estimate_batch(gsc)
    conv_s = time.perf_counter() - t0
    n_conv = int(sum(r.converged for r in rc))
    rel = [r.sigma / abs(r.mean) for r in rc if r.mean != 0.0]
    e5c = {}
    for kf in KF5:
        idx = [i for i, (k, _) in enumerate(metac) if k == kf]
        e5c[str(kf)] = {"E5": float(sum(rc[i].mean for i in idx)),
                        "sigma": float(math.sqrt(sum(rc[i].sigma ** 2 for i in idx))),
                        "floor": floors[kf]}
    destroy(M, gsc)

    # paired deviation of the mixed mode from FP64 (the FP64 path is parity-pinned to the oracle) on 48
    # integrals, on the grids the timed iterations adapted, identical counters: per integral
    # |I_mixed - I_fp64| / max(|I_fp64|, 1e-3 |E5 of its kF|), E5 from the evaluation phase above
    dev5, twins = [], []
    for i in pick:
        kf, d = meta5[i]
        ph = M.physics(kF_n=kf, K_max=kf + 6.0)
        pair = []
        for prec in (M.MBPT_FP64, M.MBPT_MIXED):
            g = M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=1 << 16, seed=seed, stream_id=7,
                                                              precision=prec, alpha=ALPHA5))
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grids5[i]))
            pair.append(g)
        twins.append((pair[0], pair[1], kf))
    M.mbpt_vegas_iterate(ctx, [g for t in twins for g in t[:2]], 1)
    r64 = M.mbpt_estimate_batch([t[0] for t in twins])
    rmx = M.mbpt_estimate_batch([t[1] for t in twins])
    for a, b, (_, _, kf) in zip(r64, rmx, twins):
        dev5.append(abs(b.last_mean - a.last_mean) / max(abs(a.last_mean), 1e-3 * abs(e5c[str(kf)]["E5"]), 1e-300))
    destroy(M, [g for t in twins for g in t[:2]])

    # E5 per kF from the 668 diagrams one by one vs from the five aligned particle-hole groups of the same
    # diagrams (Sec. III.A), at equal member evaluations (2^20 samples per integral and iteration; a group
    # sample evaluates each member once), 3 training + 6 evaluation iterations, pooled
    def e5_run(grouped, sd, map_kind=0):
        gs, keys = [], []
        descs = [d for d in M.mbpt_generate(5) if not d.anomalous]
        for ki, kf in enumerate(KF5):
            ph = M.physics(kF_n=kf, K_max=kf + 6.0, map_kind=map_kind)
            if grouped:
                by = {}
                for d in descs:
                    by.setdefault(M.mbpt_hole_chords(d), []).append(d)
                for key, mem in sorted(by.items()):
                    gs.append(M.mbpt_create_group(ctx, mem, ph, M.vegas_cfg(
                        samples=SAMPLES5, seed=sd, stream_id=sbase + 1000 * ki + 900 + key,
                        precision=M.MBPT_MIXED, alpha=ALPHA5, train_iters=3, combine=M.MBPT_COMBINE_POOLED)))
                    keys.append(kf)
            else:
                for d in descs:
                    gs.append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(
                        samples=SAMPLES5, seed=sd, stream_id=sbase + 1000 * ki + d.diagram_id,
                        precision=M.MBPT_MIXED, alpha=ALPHA5, train_iters=3, combine=M.MBPT_COMBINE_POOLED)))
                    keys.append(kf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.mbpt_vegas_iterate(ctx, gs, 13)
        rr = M.mbpt_estimate_batch(gs)
        dt = time.perf_counter() - t0
        out = {}
        for kf in KF5:
            idx = [i for i, k in enumerate(keys) if k == kf]
            out[str(kf)] = (float(sum(rr[i].mean for i in idx)), float(math.sqrt(sum(rr[i].sigma ** 2 for i in idx))))
        destroy(M, gs)
        return out, dt, len(gs)

    # two seeds each (single heavy-tailed samples make one seed's error estimate noisy)
    runs_sep = [e5_run(False, seed + 200 + j) for j in range(2)]
    runs_grp = [e5_run(True, seed + 200 + j) for j in range(2)]
    e5_sep = [r[0] for r in runs_sep]
    e5_grp = [r[0] for r in runs_grp]
    t_sep, n_sep = sum(r[1] for r in runs_sep), runs_sep[0][2]
    t_grp, n_grp = sum(r[1] for r in runs_grp), runs_grp[0][2]
    eff = [sum(e[k][1] ** 2 for e in e5_sep) * t_sep / (sum(e[k][1] ** 2 for e in e5_grp) * t_grp)
           for k in e5_sep[0] if all(e[k][1] > 0 for e in e5_grp)]
    # the rotational reduction (one chord on the z axis, one in the xz plane: 15 dimensions), the diagrams
    # one by one, the same seeds and iterations
    runs_rot = [e5_run(False, seed + 200 + j, map_kind=1) for j in range(2)]
    e5_rot = [r[0] for r in runs_rot]
    t_rot = sum(r[1] for r in runs_rot)
    eff_rot = [sum(e[k][1] ** 2 for e in e5_sep) * t_sep / (sum(e[k][1] ** 2 for e in e5_rot) * t_rot)
               for k in e5_sep[0] if all(e[k][1] > 0 for e in e5_rot)]
    g5r, _ = fifth_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed, stream_base=sbase, map_kind=1)
    timed_steps(g5r, 3)
    _, st5r = timed_steps(g5r, 5)
    v5r = world * len(g5r) * SAMPLES5 / (float(np.mean(st5r)) * 1e-3)
    destroy(M, g5r)

    # the plain per-diagram FP64 loop on every 20th fifth-order integral: one launch per integral and
    # iteration, default launch shape
    launch_now = {o: M.mbpt_ctx_get_launch(ctx, o) for o in (2, 3, 4, 5, 6)}
    layout_now = M.mbpt_ctx_get_hist_layout(ctx)
    spin_now = M.mbpt_ctx_get_spin_sum(ctx)
    M.mbpt_ctx_set_kernel(ctx, 256, 2)
    M.mbpt_ctx_set_hist_layout(ctx, M.MBPT_HIST_WARP_F32)
    for o in (2, 3, 4, 5, 6):
        M.mbpt_ctx_set_launch(ctx, o, 32)
    gk5, _ = fifth_order_integrals(M, ctx, M.MBPT_FP64, seed=seed, stream_base=sbase, every=20)
    timed_steps(gk5, 1, per_diagram=True)
    _, stk5 = timed_steps(gk5, 2, per_diagram=True)
    vk5 = world * len(gk5) * SAMPLES5 / (float(np.mean(stk5)) * 1e-3)
    destroy(M, gk5)
    M.mbpt_ctx_set_kernel(ctx, *launch_now[5][:2])
    M.mbpt_ctx_set_hist_layout(ctx, layout_now)
    M.mbpt_ctx_set_spin_sum(ctx, spin_now)
    for o, (_, _, spt) in launch_now.items():
        M.mbpt_ctx_set_launch(ctx, o, spt)

    # ================= third-order density scan (C2): mixed, FP64 batched, plain per-diagram loop ========
    g3, m3 = third_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed, stream_base=sbase)
    tuned3 = autotune(ctx, g3, trials=1)["launch"] if args.autotune else None
    n3 = len(g3)
    timed_steps(g3, 3)
    it3, st3 = timed_steps(g3, args.steps)
    v3 = world * n3 * SAMPLES3 / (float(np.mean(st3)) * 1e-3)
    ops3 = measured_fp64_ops("third_order_mixed")
    frac3 = (ops3 * n3 * SAMPLES3 / (float(np.mean(it3)) * 1e-3) / fp64_rate) if ops3 else None
    res3 = M.mbpt_estimate_batch(g3)
    live3 = []
    for g in g3[:: max(1, n3 // 6)]:
        _, w = M.mbpt_dump_samples(g, 10 ** 6, 0, 1 << 15, 12, with_x=False)
        live3.append(np.mean(w != 0))
    destroy(M, g3)
    g3r, _ = third_order_integrals(M, ctx, M.MBPT_MIXED, seed=seed, stream_base=sbase, map_kind=1)
    timed_steps(g3r, 3)
    _, st3r = timed_steps(g3r, max(4, args.steps // 4))
    v3r = world * n3 * SAMPLES3 / (float(np.mean(st3r)) * 1e-3)
    res3r = M.mbpt_estimate_batch(g3r)
    destroy(M, g3r)
    g64, _ = third_order_integrals(M, ctx, M.MBPT_FP64, seed=seed, stream_base=sbase)
    timed_steps(g64, 3)
    it64, st64 = timed_steps(g64, max(4, args.steps // 2))
    v64 = world * n3 * SAMPLES3 / (float(np.mean(st64)) * 1e-3)
    res64 = M.mbpt_estimate_batch(g64)
    destroy(M, g64)
    M.mbpt_ctx_set_kernel(ctx, 256, 2)
    M.mbpt_ctx_set_hist_layout(ctx, M.MBPT_HIST_WARP_F32)
    for o in (2, 3, 4, 5, 6):
        M.mbpt_ctx_set_launch(ctx, o, 32)
    gk0, _ = third_order_integrals(M, ctx, M.MBPT_FP64, seed=seed, stream_base=sbase)
    timed_steps(gk0, 2, per_diagram=True)
    _, stk0 = timed_steps(gk0, max(2, args.steps // 4), per_diagram=True)
    vk0 = world * n3 * SAMPLES3 / (float(np.mean(stk0)) * 1e-3)
    destroy(M, gk0)

    def diags_per_s(results, rate, rel_target=1e-3):
        """Integrals brought to rel_target per second at a throughput `rate`, from each run's own variance."""
        need = 0.0
        for r in results:
            if r.mean == 0.0 or r.sigma == 0.0:
                continue
            need += r.n_evals * (r.sigma / (rel_target * abs(r.mean))) ** 2
        return len(results) / (need / rate) if need > 0 else None

    d_mixed, d_rot, d_k0 = diags_per_s(res3, v3), diags_per_s(res3r, v3r), diags_per_s(res64, vk0)

    # ================= fourth order (C3): 198 live integrals x 2^24, and the aligned groups ===============
    M.mbpt_ctx_set_kernel(ctx, *launch_now[5][:2])
    M.mbpt_ctx_set_hist_layout(ctx, layout_now)
    M.mbpt_ctx_set_spin_sum(ctx, spin_now)
    for o, (_, _, spt) in launch_now.items():
        M.mbpt_ctx_set_launch(ctx, o, spt)
    g4, gg, member_evals = [], [], 0
    for ki, kf in enumerate((1.0, 1.33, 1.6)):
        for mi, kfp in enumerate((0.0, kf)):
            ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0)
            by_key = {}
            for d in M.mbpt_generate(4):
                if d.anomalous:
                    continue
                by_key.setdefault(M.mbpt_hole_chords(d), []).append(d)
                g4.append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(
                    samples=1 << 24, seed=seed, stream_id=sbase + 1000 * mi + 100 * ki + d.diagram_id,
                    precision=M.MBPT_MIXED, alpha=1.0)))
            for key, ds in sorted(by_key.items()):
                gg.append(M.mbpt_create_group(ctx, ds, ph, M.vegas_cfg(
                    samples=1 << 24, seed=seed, stream_id=sbase + 1000 * mi + 100 * ki + 50 + key,
                    precision=M.MBPT_MIXED, alpha=1.0)))
                member_evals += len(ds) << 24
    timed_steps(g4, 1)
    it4, st4 = timed_steps(g4, max(5, args.steps // 4))
    v4 = world * len(g4) * (1 << 24) / (float(np.mean(st4)) * 1e-3)
    timed_steps(gg, 1)
    _, stg = timed_steps(gg, max(5, args.steps // 4))
    vg = world * member_evals / (float(np.mean(stg)) * 1e-3)
    n4, ng = len(g4), len(gg)
    destroy(M, g4)
    destroy(M, gg)

    # ================= sixth order: every non-anomalous diagram, one integral per mirror pair ============
    t6 = time.perf_counter()
    ph6 = M.physics(kF_n=1.33, K_max=7.33)
    g6 = [M.mbpt_create_diagram(ctx, d, ph6, M.vegas_cfg(samples=1 << 16, seed=seed, stream_id=sbase + d.diagram_id,
                                                         precision=M.MBPT_MIXED, alpha=0.75))
          for d in M.mbpt_generate(6) if not d.anomalous and d.diagram_id <= d.mirror_id]
    create6_s = time.perf_counter() - t6
    timed_steps(g6, 1)
    _, st6 = timed_steps(g6, 3)
    v6 = world * len(g6) * (1 << 16) / (float(np.mean(st6)) * 1e-3)
    n6 = len(g6)
    destroy(M, g6)
    M.mbpt_ctx_destroy(ctx)
    del arena
    torch.cuda.synchronize()

    # ================= serving (C5): Poisson stream of equation-of-state requests ========================
    serving = None
    if args.serve_requests > 0:
        from paper_2603_24532_b300 import serve as S
        be = S.MbptBackend(device=local, arena_bytes=48 << 30)
        srv = S.Server(be, budget_bytes=40 << 30, round_samples=1 << 27, max_wait=2.0)
        trace = S.poisson_trace(args.serve_requests, 20.0, 7 + rank)
        t0 = time.perf_counter()
        done = srv.run(trace, realtime=True, time_limit=args.serve_seconds)
        wall = time.perf_counter() - t0
        fin = [r for r in done if r.energy is not None and math.isfinite(r.energy)]
        n_int = sum(len(r.integrals) for r in fin)
        n_diag = sum(it.mult for r in fin for it in r.integrals)
        serving = {"requests": len(trace), "completed": len(done), "wall_s": wall,
                   "latency_all": S.latency_stats(done), "latency_met": S.latency_stats(done, "met"),
                   "latency_capped": S.latency_stats(done, "capped"),
                   "p50_s": S.latency_stats(done)["p50_s"], "p99_s": S.latency_stats(done)["p99_s"],
                   "target_met_fraction": sum(r.met for r in done) / max(1, len(done)),
                   "capped_fraction": sum(r.capped for r in done) / max(1, len(done)),
                   "capped_by": {"cap": {str(c): sum(r.capped for r in done if r.cap == c) for c in (2, 3, 4)},
                                 "target": {str(t): sum(r.capped for r in done if r.target == t)
                                            for t in (0.01, 0.003, 0.001)},
                                 "delta": {str(d): sum(r.capped for r in done if r.delta == d)
                                           for d in (0.0, 0.25, 0.5, 0.75, 1.0)}},
                   "rounds_median": float(np.median([r.rounds for r in done])) if done else None,
                   "integrals_per_s": n_int / wall, "diagrams_per_s": n_diag / wall,
                   "evals_per_s": srv.evals / wall, "budget_bytes": srv.budget,
                   "max_iters": srv.max_iters, "max_samples_per_iter": srv.max_samples,
                   "workload": "Poisson 20/s, n ~ U[0.04, 0.20] fm^-3, delta {0..1}, order cap {2,3,4}, "
                               "target {1, 0.3, 0.1} %, seed 7 (+rank); 40 GB admission budget; rounds of at "
                               "most 2^27 samples, least work left first (a request waiting 2 s runs first); "
                               "adaptive samples per integral and iteration up to 2^25, at most 120 iterations; "
                               "diagrams/s counts a mirror-pair representative twice"}
        be.close()
    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    cpu = cpu_baseline(budget_s=args.cpu_seconds) if world == 1 else None
    sm_mhz = clk.get("sm_mhz") or 2032.0
    dev5 = np.array(dev5)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "integrals": n5, "samples_per_iter": SAMPLES5, "mirror_dedup": False,
                   "precision": "mixed (FP32 potentials, spin sum and sampling map; FP64 line momenta, Fermi "
                                "steps, energy denominators, sums, grid; FP64 map within 2^-7 kF^2 of a Fermi "
                                "surface)",
                   "vegas": {"bins": 50, "alpha": ALPHA5},
                   "step": "one batched VEGAS iteration over all integrals (sample, integrate, reduce, combine, "
                           "refine)",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "1 GPU", "launch": tuned},
        "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "k_iterate (order-2..5 plain part)",
                     "achieved": achieved / 1e9 if achieved else None, "peak": fp64_rate / 1e9,
                     "unit": "FP64 Gop/s (thread operations)",
                     "frac": achieved / fp64_rate if achieved else None,
                     "peak_kind": "FP64 DFMA rate measured in this run with the library's dependency-free DFMA "
                                  "loop (mbpt_fp64_rate)",
                     "frac_of_nominal": achieved / (FP64_PEAK_NOMINAL * sm_mhz / 2032.0) if achieved else None,
                     "nominal_note": "1.25 TFLOP/s FP64 of the recipe (FMA = 2) = 6.25e11 instructions/s at "
                                     "2032 MHz, scaled to the run's median SM clock",
                     "ops_per_sample": ops5, "ops_source": "ncu DADD + DMUL + DFMA thread instructions per "
                                                          "sample, profiles/fp64_ops_per_sample.txt",
                     "kernel_ms": it_ms, "traffic": traffic5, "traffic_unit": "bytes per launch",
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one launch of the same kernel "
                                     "and integrals at 2^18 samples each (ncu, profiles/fp64_ops_per_sample.txt), "
                                     "scaled by the number of chunks to this launch: the chunk slots written once "
                                     "(histogram and sums, 3.6 KB per chunk), records and grids; HBM is otherwise "
                                     "idle by design",
                     "issue_frac": issue_frac,
                     "issue_note": "warp instructions per sample (ncu sm__inst_executed.sum of the same launch "
                                   "shape) x samples / kernel time, over 4 issue slots per SM per cycle at the "
                                   "run's median SM clock: the kernel is bound by latency and issue, with the "
                                   "FP64 pipe about half busy"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,   # per step: the k_iterate kernel of the plain order-2..5 part, k_finalize
        "clocks": clk,
        "fifth_order_to_0p5pct": {"integrals": len(rc), "converged": n_conv, "wall_s": conv_s, "iterations": iters,
                                  "evals": conv_evals, "median_rel_err": float(np.median(rel)) if rel else None,
                                  "diagrams_per_s": n_conv / conv_s, "per_kF": e5c,
                                  "k0_diagrams_per_s": n_conv / (conv_evals / vk5),
                                  "definition": "3 training iterations of 2^20, then the frozen-grid evaluation "
                                                "phase with adaptive samples per iteration (the integrals closest to "
                                                "their targets first get what they still need, up to 2^22, the rest "
                                                "2^18, within 2^20 samples per unconverged integral per iteration); converged: sigma <= "
                                                "max(0.5 % |I|, 0.5 % |E5(kF)| / sqrt(668)); cap 40 iterations; "
                                                "k0: the same evaluations at the plain per-diagram FP64 loop's "
                                                "rate"},
        "fifth_order_rotational_15d": {"value": v5r, "unit": UNIT, "integrals": n5, "samples_per_iter": SAMPLES5,
                                       "per_kF": e5_rot, "wall_s": t_rot, "time_to_equal_error_ratio": eff_rot,
                                       "definition": "the headline's integrals with the rotational reduction "
                                                     "(d = 15; 5 timed steps); E5 +- sigma per kF and seed from 3 "
                                                     "training + 10 pooled iterations at 2^20 (two seeds, as "
                                                     "fifth_order_groups); ratio per kF = (sum of sigma^2) x "
                                                     "wall time, 18D over 15D"},
        "fifth_order_groups": {"per_kF_diagrams": e5_sep, "per_kF_groups": e5_grp, "wall_s_diagrams": t_sep,
                               "wall_s_groups": t_grp, "integrals": [n_sep, n_grp],
                               "time_to_equal_error_ratio": eff,
                               "definition": "E5 (MeV) +- sigma per kF and seed (two seeds) from the 668 diagrams "
                                             "one by one and from the 5 aligned particle-hole groups (hole loop "
                                             "momenta first), 3 training + 10 pooled iterations at 2^20 samples "
                                             "per integral each; ratio per kF = (sum over seeds of sigma^2) x "
                                             "wall time, diagrams over groups: the speed-up of the groups to a "
                                             "given error on E5"},
        "k0_plain_fp64_fifth_order": {"value": vk5, "unit": UNIT, "integrals": int(math.ceil(n5 / 20)),
                                      "note": "every 20th integral, one launch per integral and iteration"},
        "speedup_vs_k0": value / vk5,
        "mixed_vs_fp64_deviation": {"integrals": int(len(dev5)), "samples_each": 1 << 16,
                                    "max": float(dev5.max()), "median": float(np.median(dev5)),
                                    "frac_below_1e-4": float(np.mean(dev5 < 1e-4)),
                                    "definition": "same grid and counters: |I_mixed - I_fp64| / max(|I_fp64|, "
                                                  "1e-3 |E5 of the kF|), one iteration of 2^16 samples"},
        "third_order_scan": {"value": v3, "unit": UNIT, "integrals": n3, "samples_per_iter": SAMPLES3,
                             "kernel_ms": float(np.mean(it3)), "live_fraction": float(np.mean(live3)),
                             "roofline_frac": frac3, "ops_per_sample": ops3,
                             "launch": tuned3,
                             "fp64_batched": v64, "k0_plain_fp64_per_diagram": vk0, "speedup_vs_k0": v3 / vk0,
                             "rotational_9d": v3r,
                             "diagrams_to_0p1pct_per_s": {"batched_mixed": d_mixed, "k0_plain_fp64": d_k0,
                                                          "ratio": (d_mixed / d_k0) if (d_mixed and d_k0) else None,
                                                          "batched_mixed_rotational_9d": d_rot},
                             "workload": "3 third-order diagrams x kF 0.8..1.7 fm^-1 (10 points), PNM, 12D, "
                                         "2^22 samples/iteration, mixed"},
        "fourth_order_batch": {"value": v4, "unit": UNIT, "integrals": n4, "samples_per_iter": 1 << 24,
                               "ms_per_iteration": float(np.mean(st4)), "timed_steps": len(st4),
                               "workload": "39 fourth-order diagrams (33 non-anomalous) x kF {1.0,1.33,1.6} x "
                                           "{PNM,SNM}, mixed"},
        "fourth_order_groups": {"value": vg, "unit": UNIT + " (member diagrams)", "integrals": ng,
                                "samples_per_iter": 1 << 24, "ms_per_iteration": float(np.mean(stg)),
                                "vs_per_diagram_batch": vg / v4,
                                "workload": "the fourth_order_batch diagrams as 4 aligned particle-hole groups per "
                                            "physics point (24 group integrals), mixed"},
        "sixth_order_batch": {"value": v6, "unit": UNIT, "integrals": n6, "samples_per_iter": 1 << 16,
                              "ms_per_iteration": float(np.mean(st6)), "create_s": create6_s,
                              "workload": "27300 sixth-order diagrams, one integral per mirror pair of the 21572 "
                                          "non-anomalous ones, PNM kF 1.33, d = 21, mixed"},
        "serving": serving,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return line


# ---------------------------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------------------------------
def cpu_baseline(budget_s=12.0, stride=None, n=4096):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the headline workload -- every
    stride-th of the 2004 fifth-order integrals (in kF, then diagram order), n samples each, uniform grid.
    Without stride, the stride is calibrated on every 64th integral to take about budget_s seconds."""
    import oracle as O

    Ds = [D for D in O.enumerate_diagrams(5) if not O.is_anomalous(D)]
    cores = os.cpu_count() or 1
    grid = O.uniform_grid(18, 50)
    work = [(ki, kf, D) for ki, kf in enumerate(KF5) for D in Ds]

    need = []     # samples each integral would need for 0.1 % at its own per-sample variance

    def run(sel):
        need.clear()
        t0 = time.perf_counter()
        for ki, kf, D in sel:
            r = O.vegas_iteration(D, O.Physics(kF_n=kf, K_max=kf + 6.0), grid, 1, 1000 * ki + D.diagram_id, 0, n,
                                  threads=cores)
            mean = r.sum_w / n
            var = max(r.sum_w2 / n - mean * mean, 0.0)
            if mean != 0.0:
                need.append(var / (1e-3 * mean) ** 2)
        return time.perf_counter() - t0

    if stride is None:
        sel = work[::64]
        rate = len(sel) * n / run(sel)
        stride = max(1, int(math.ceil(len(work) * n / (rate * budget_s))))
    sel = work[::stride]
    dt = run(sel)
    rate = len(sel) * n / dt
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "stride": stride, "samples": len(sel) * n,
            "time_to_0p1pct_s": {"median": float(np.median(need)) / rate if need else None,
                                 "definition": "per sampled integral, its per-sample variance on the uniform grid "
                                               "over (0.1 % of its mean)^2 samples at the oracle's rate; median "
                                               "over the sampled integrals (no grid adaptation: an upper "
                                               "estimate)"},
            "sample": "%d samples of every %d-th of the %d fifth-order integrals (%d integrals, uniform grid, "
                      "iteration 0), %.1f s" % (n, stride, len(work), len(sel), dt)}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    cb = None
    times = []
    stride = cpu_baseline(budget_s=args.ref_seconds)["stride"]     # calibration, untimed
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(stride=stride)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = cb["samples"] / float(np.mean(times))      # oracle evaluations per second over the timed steps
    cb = dict(cb, value=value)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "integrals": 2004, "samples_per_iter": SAMPLES5,
                       "step": "bounded sample of one iteration of every integral on the host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def profile_case(args):
    """A small case of one workload for ncu captures of k_iterate: `fifth` (the 2004 fifth-order integrals),
    `third` (the 30 third-order integrals) or `sixth` (the 11269 sixth-order integrals, one per mirror
    pair, PNM kF 1.33), args.samples samples each, args.iters batched iterations, in an arena of
    args.arena_gb GiB."""
    from paper_2603_24532_b300 import mbpt as M
    ctx = M.mbpt_ctx_create(0, int(args.arena_gb * (1 << 30)))
    prec = M.MBPT_MIXED if args.precision == "mixed" else M.MBPT_FP64
    order = {"fifth": 5, "third": 3, "sixth": 6}[args.profile_case]
    if args.spt:
        M.mbpt_ctx_set_launch(ctx, order, args.spt)
    M.mbpt_ctx_set_spin_sum(ctx, M.MBPT_SPIN_FOLD if args.spin == "fold" else M.MBPT_SPIN_TABLE)
    if args.profile_case == "fifth":
        gs, _ = fifth_order_integrals(M, ctx, prec, samples=args.samples, near_band=args.near_band)
    elif args.profile_case == "sixth":
        ph = M.physics(kF_n=1.33, K_max=7.33)
        gs = [M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=args.samples, stream_id=d.diagram_id,
                                                            precision=prec, alpha=0.75))
              for d in M.mbpt_generate(6) if not d.anomalous and d.diagram_id <= d.mirror_id]
    else:
        descs = M.mbpt_generate(3)
        gs = []
        for ki, kf in enumerate(KF_SCAN):
            ph = M.physics(kF_n=kf, K_max=kf + 6.0)
            gs += [M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=args.samples, stream_id=100 * ki + d.diagram_id,
                                                                 precision=prec)) for d in descs]
    M.mbpt_vegas_iterate(ctx, gs, args.iters)
    r = M.mbpt_estimate(gs[0])
    it_ms, fin_ms = M.mbpt_ctx_last_timing(ctx)
    print("%s: integrals %d samples %d iters %d spin %s spt %d: k_iterate %.3f ms, k_finalize %.3f ms, first mean %.6g "
          "+- %.2g" % (args.profile_case, len(gs), args.samples, args.iters, args.spin,
             M.mbpt_ctx_get_launch(ctx, order)[2], it_ms, fin_ms, r.mean, r.sigma))
    M.mbpt_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--ref-seconds", type=float, default=6.0, help="reference arm: seconds per step")
    ap.add_argument("--serve-requests", type=int, default=1200, help="serving run (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=150.0)
    ap.add_argument("--profile-case", choices=["fifth", "third", "sixth"], default=None,
                    help="run only a small case of one workload (for ncu captures)")
    ap.add_argument("--samples", type=int, default=1 << 16, help="--profile-case: samples per integral")
    ap.add_argument("--iters", type=int, default=3, help="--profile-case: batched iterations")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed", help="--profile-case precision")
    ap.add_argument("--near-band", type=float, default=0.0, help="--profile-case: FP64-map band (0 = default)")
    ap.add_argument("--spt", type=int, default=0, help="--profile-case: samples per thread of a chunk (0 = default)")
    ap.add_argument("--spin", choices=["table", "fold"], default="table", help="--profile-case: Goldstone-sum strategy")
    ap.add_argument("--arena-gb", type=float, default=8.0, help="--profile-case: device arena (GiB)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
