"""Fifth-order workload: every fifth-order Hugenholtz diagram x kF in {1.0, 1.33, 1.6} fm^-1,
pure neutron matter, mixed precision, batched on one GPU until each integral reaches a relative
statistical error of 0.5 % (or the iteration cap), then the per-diagram deviation of the
mixed-precision evaluation from the FP64 oracle on a subset of samples.

    python -m paper_2603_24532_b300.run_fifth_order [--samples 2^20] [--max-iters 40] [--time-limit S]
        [--cap 2^22] [--budget N] [--target 0.005] [--oracle-integrals 48] [--oracle-samples 4096] [--map-kind 0]

Anomalous diagrams (zero at T = 0) are skipped.  Every integral trains its grid for `--train`
iterations (grid compression `--alpha`) and is then estimated on the frozen grid, every evaluation sample
weighted alike (pooled combination).  A near-zero diagram cannot reach a relative target; its absolute
target is 0.5 % of |sum over the order| / sqrt(number of integrals) at that density, from the last
training iteration.  The evaluation phase adapts each integral's samples per iteration to what it still
needs (`converge`, shared with bench.py).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import mbpt as M


def converge(M, ctx, gs, goals, cfg_for, done_evals, base_samples=1 << 20, min_samples=1 << 18,
             cap=1 << 22, budget=None, max_iters=40, iters_done=0, time_limit=None, progress=None):
    """Adaptive evaluation phase: iterate the unconverged integrals of gs until every one meets its target
    (sigma <= its goal), the iteration count reaches max_iters or time_limit seconds pass.

    PVegas' adaptive number of samples per iteration (Sec. III.C), read as: before each iteration, each live
    integral's remaining need is its per-sample variance over its goal squared, less the evaluation samples
    it already has; the integrals with the smallest need are served first with what they still need, rounded
    up to a power of two within [min_samples, cap], until the iteration's sample budget (by default
    base_samples per live integral; with `budget`, at least that many samples in all) is spent; the rest run
    min_samples.  goals(r, i) gives integral i's goal from its estimate r; cfg_for(i, samples) its
    configuration at that sample count (same seed, stream and targets); done_evals(r) the evaluation-phase
    samples an estimate already holds; progress(iterations, evaluations, seconds, live integrals), if
    given, is called before each iteration.  Returns (iterations, evaluations, seconds)."""
    t0 = time.perf_counter()
    cur = [base_samples] * len(gs)
    iters, evals = iters_done, 0
    while max_iters is None or iters < max_iters:
        if time_limit is not None and time.perf_counter() - t0 >= time_limit:
            break
        rc = M.mbpt_estimate_batch(gs)
        live = []
        for i, r in enumerate(rc):
            if r.converged:
                continue
            n_eval = done_evals(r)
            goal = goals(r, i)
            need = (r.sigma ** 2 * n_eval / goal ** 2 - n_eval) if (n_eval > 0 and math.isfinite(r.sigma)
                                                                  and goal > 0.0) else float(base_samples)
            live.append((max(need, 1.0), i))
        if progress is not None:
            progress(iters, evals, time.perf_counter() - t0, len(live))
        if not live:
            break
        live.sort()
        left = max(len(live) * base_samples, budget or 0)
        for need, i in live:
            nxt = min_samples
            if left > 0:
                nxt = 1 << int(math.ceil(math.log2(min(float(cap), max(float(min_samples), need)))))
            left -= nxt
            if nxt != cur[i]:
                M.mbpt_set_config(gs[i], cfg_for(i, nxt))
                cur[i] = nxt
        M.mbpt_vegas_iterate(ctx, [gs[i] for _, i in live], 1)
        evals += sum(cur[i] for _, i in live)
        iters += 1
    return iters, evals, time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--max-iters", type=int, default=40)
    ap.add_argument("--target", type=float, default=0.005)
    ap.add_argument("--oracle-integrals", type=int, default=48)
    ap.add_argument("--oracle-samples", type=int, default=1 << 16)
    ap.add_argument("--map-kind", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=0.75, help="grid compression exponent")
    ap.add_argument("--train", type=int, default=3, help="training iterations (grid refined, not combined)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "map64", "fp64"],
                    help="mixed: FP32 sampling map; map64: FP64 map, FP32 potentials and spin sums")
    ap.add_argument("--dedup-mirrors", action="store_true",
                    help="one integral per pair of mirror (complex-conjugate) diagrams, counted twice")
    ap.add_argument("--cap", type=int, default=1 << 22, help="most samples of one integral in one iteration")
    ap.add_argument("--budget", type=int, default=0,
                    help="samples per iteration in all, at least (0: --samples per unconverged integral)")
    ap.add_argument("--time-limit", type=float, default=0.0, help="seconds of evaluation phase (0: none)")
    a = ap.parse_args()
    prec = {"mixed": M.MBPT_MIXED, "map64": M.MBPT_MIXED_MAP64, "fp64": M.MBPT_FP64}[a.precision]
    ctx = M.mbpt_ctx_create(0, 16 << 30)
    descs = [d for d in M.mbpt_generate(5) if not d.anomalous]
    if a.dedup_mirrors:
        descs = [d for d in descs if d.diagram_id <= d.mirror_id]
    mult = {d.diagram_id: (2 if (a.dedup_mirrors and d.mirror_id != d.diagram_id) else 1) for d in descs}
    kfs = (1.0, 1.33, 1.6)
    gs, meta = [], []
    for ki, kf in enumerate(kfs):
        ph = M.physics(kF_n=kf, K_max=kf + 6.0, map_kind=a.map_kind)
        for d in descs:
            cfg = M.vegas_cfg(samples=a.samples, seed=1, stream_id=1000 * ki + d.diagram_id, precision=prec,
                              target_rel=a.target, alpha=a.alpha, train_iters=a.train,
                              combine=M.MBPT_COMBINE_POOLED)
            gs.append(M.mbpt_create_diagram(ctx, d, ph, cfg))
            meta.append((kf, d))
    t0 = time.perf_counter()
    # training iterations, then absolute floors for near-zero diagrams from the last one
    M.mbpt_vegas_iterate(ctx, gs, a.train)
    res = M.mbpt_estimate_batch(gs)
    floors = {}
    for ki, kf in enumerate(kfs):
        idx = [i for i, (k, _) in enumerate(meta) if k == kf]
        order_sum = abs(sum(mult[meta[i][1].diagram_id] * res[i].last_mean for i in idx))
        floors[kf] = a.target * order_sum / math.sqrt(sum(mult[meta[i][1].diagram_id] ** 2 for i in idx))

    def cfg_for(i, n):
        kf, d = meta[i]
        return M.vegas_cfg(samples=n, seed=1, stream_id=1000 * kfs.index(kf) + d.diagram_id, precision=prec,
                           target_rel=a.target, target_abs=floors[kf], alpha=a.alpha, train_iters=a.train,
                           combine=M.MBPT_COMBINE_POOLED)
    for i in range(len(gs)):
        M.mbpt_set_config(gs[i], cfg_for(i, a.samples))
    trace = []

    def report(it, ev, sec, n_live):
        if not trace or sec - trace[-1][2] >= 10.0 or n_live == 0:
            trace.append((it, ev, round(sec, 2), len(gs) - n_live))
    iters, ev, _ = converge(M, ctx, gs, lambda r, i: max(a.target * abs(r.mean), floors[meta[i][0]]), cfg_for,
                            lambda r: r.n_evals - a.train * a.samples, base_samples=a.samples,
                            min_samples=min(a.samples, 1 << 18), cap=max(a.cap, a.samples),
                            budget=a.budget or None, max_iters=a.max_iters or None, iters_done=a.train,
                            time_limit=a.time_limit or None, progress=report)
    evals = a.train * a.samples * len(gs) + ev
    res = M.mbpt_estimate_batch(gs)
    wall = time.perf_counter() - t0
    conv = sum(r.converged for r in res)
    rel = [r.sigma / abs(r.mean) for r in res if r.mean != 0.0]
    per_kf = {}
    for ki, kf in enumerate(kfs):
        idx = [i for i, (k, _) in enumerate(meta) if k == kf]
        per_kf[str(kf)] = {"E5_sum": float(sum(mult[meta[i][1].diagram_id] * res[i].mean for i in idx)),
                           "sigma": float(math.sqrt(sum((mult[meta[i][1].diagram_id] * res[i].sigma) ** 2
                                                        for i in idx)))}

    # per-diagram deviation of the mixed evaluation from the FP64 oracle on identical samples
    dev = None
    if a.oracle_integrals > 0:
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        rng = np.random.default_rng(5)
        pick = rng.choice(len(gs), size=min(a.oracle_integrals, len(gs)), replace=False)
        devs, l1, cancel = [], [], []
        Os = O.enumerate_diagrams(5)
        for i in pick:
            kf, d = meta[i]
            D = Os[d.diagram_id]
            po = O.Physics(kF_n=kf, K_max=kf + 6.0, map_kind=a.map_kind)
            img = M.mbpt_get_state(gs[i])
            dd = po.dim(D)
            grid = M.state_grid(img, dd, 50)
            _, wg = M.mbpt_dump_samples(gs[i], 99, 0, a.oracle_samples, dd, with_x=False)
            ref = O.vegas_iteration(D, po, grid, 1, 1000 * kfs.index(kf) + d.diagram_id, 99, a.oracle_samples)
            # sums of w/J-independent scale: E5 order sum per sample is mean(w) ~ E5/N_int
            _, _, _, wo = O.vegas_samples(0, D, po.array(), dd, grid, 1, 1000 * kfs.index(kf) + d.diagram_id, 99,
                                          0, a.oracle_samples, dump=True)
            scale = max(abs(ref.sum_w), 1e-3 * abs(per_kf[str(kf)]["E5_sum"]) * a.oracle_samples, 1e-300)
            devs.append(abs(np.sum(wg) - ref.sum_w) / scale)
            l1.append(np.sum(np.abs(wg - wo)) / max(np.sum(np.abs(wo)), 1e-300))
            cancel.append(np.sum(np.abs(wo)) / max(abs(ref.sum_w), 1e-300))
        devs = np.array(devs)
        worst = int(np.argmax(devs))
        dev = {"integrals": int(len(devs)), "samples_each": a.oracle_samples, "max": float(devs.max()),
               "median": float(np.median(devs)), "frac_below_1e-4": float(np.mean(devs < 1e-4)),
               "definition": "|sum w_mixed - sum w_oracle| / max(|sum w_oracle|, 1e-3 |E5 order sum| M), "
                             "same grid and counters",
               "l1_max": float(max(l1)), "l1_median": float(np.median(l1)),
               "l1_definition": "sum |w_mixed - w_oracle| / sum |w_oracle| per integral",
               "worst_cancellation": float(cancel[worst]),
               "cancellation_definition": "sum |w| / |sum w| of the integral with the largest deviation"}
    out = {"workload": "all 840 fifth-order diagrams (668 non-anomalous) x kF {1.0, 1.33, 1.6}, PNM, %s, "
                       "to %.2g relative or the floor (iteration cap %d)" % (a.precision, a.target, a.max_iters),
           "integrals": len(gs), "dedup_mirrors": a.dedup_mirrors, "samples_per_iter": a.samples,
           "adaptive": {"cap": a.cap, "budget": a.budget, "time_limit_s": a.time_limit}, "floors": floors,
           "map_kind": a.map_kind, "wall_s": wall,
           "trace": {"columns": ["iteration", "evaluation-phase samples", "seconds", "converged"], "rows": trace},
           "iterations": iters, "evals": evals, "evals_per_s": evals / wall, "converged": int(conv),
           "median_rel_err": float(np.median(rel)) if rel else None, "per_kF": per_kf,
           "oracle_deviation": dev}
    print(json.dumps(out))
    M.mbpt_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
