"""Serving benchmark: replay a Poisson stream of equation-of-state requests against the
continuous-batching server on one GPU and report latency percentiles and throughput.

    python -m paper_2603_24532_b300.bench_serve [--requests 1200] [--rate 20] [--seed 7]
        [--budget-gb 40] [--time-limit 300] [--warm-start] [--grouped]

Requests (seed 7, exponential gaps of mean 1/rate): n ~ U[0.04, 0.20] fm^-3, delta from
{0, 0.25, 0.5, 0.75, 1}, order cap from {2, 3, 4}, relative target from {1%, 0.3%, 0.1%};
admission by a fixed grid/accumulator memory budget.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import serve as S


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=1200)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--arena-gb", type=float, default=48.0)
    ap.add_argument("--time-limit", type=float, default=None)
    ap.add_argument("--max-iters", type=int, default=120)
    ap.add_argument("--max-samples", type=float, default=float(S.MAX_SAMPLES),
                    help="adaptive samples per iteration of one integral: at most this")
    ap.add_argument("--warm-start", action="store_true")
    ap.add_argument("--grouped", action="store_true", help="one integral per (order, particle-hole group)")
    ap.add_argument("--group-orders", default=None, help="with --grouped: only these orders, e.g. 4 or 3,4")
    ap.add_argument("--warm-blend", type=float, default=0.5, help="weight of the donor grid in a warm start")
    ap.add_argument("--warm-train", type=int, default=1, help="uncombined iterations after a warm start")
    ap.add_argument("--log", default=None, help="JSONL file: one record per finished integral and request")
    ap.add_argument("--round-samples", type=float, default=float(1 << 27),
                    help="samples per round (least work left first; 0: every active request every round)")
    ap.add_argument("--max-wait", type=float, default=2.0, help="with --round-samples: seconds before a request runs first")
    a = ap.parse_args()
    go = tuple(int(v) for v in a.group_orders.split(",")) if a.group_orders else None
    be = S.MbptBackend(arena_bytes=int(a.arena_gb * (1 << 30)), grouped=a.grouped, group_orders=go)
    logf = open(a.log, "w") if a.log else None
    srv = S.Server(be, budget_bytes=int(a.budget_gb * (1 << 30)), max_iters=a.max_iters, warm_start=a.warm_start,
                   warm_blend=a.warm_blend, warm_train=a.warm_train, log=logf,
                   round_samples=int(a.round_samples) if a.round_samples > 0 else None, max_wait=a.max_wait,
                   max_samples=int(a.max_samples))
    trace = S.poisson_trace(a.requests, a.rate, a.seed)
    t0 = time.perf_counter()
    done = srv.run(trace, realtime=True, time_limit=a.time_limit)
    wall = time.perf_counter() - t0
    st = S.latency_stats(done)
    n_int = sum(len(r.integrals) for r in done)
    caps = {c: sum(1 for r in done if r.cap == c) for c in (2, 3, 4)}
    met = [r for r in done if r.met]
    rounds = [r.rounds for r in done]
    out = {"workload": "EOS request stream, Poisson rate %.1f/s seed %d, %d requests" % (a.rate, a.seed, a.requests),
           "completed": len(done), "wall_s": wall, "latency": st, "latency_met": S.latency_stats(done, "met"),
           "latency_capped": S.latency_stats(done, "capped"),
           "capped_fraction": sum(r.capped for r in done) / max(1, len(done)),
           "capped_by_cap": {str(c): sum(r.capped for r in done if r.cap == c) for c in (2, 3, 4)},
           "capped_by_target": {str(t): sum(r.capped for r in done if r.target == t) for t in (0.01, 0.003, 0.001)},
           "group_orders": a.group_orders, "round_samples": a.round_samples, "max_wait": a.max_wait,
           "max_iters": a.max_iters, "max_samples": a.max_samples,
           "evals_per_request_median": {"cap%d target%g" % (c, t): float(np.median(
               [sum(it.evals for it in r.integrals) for r in done if r.cap == c and r.target == t] or [0]))
               for c in (2, 3, 4) for t in (0.01, 0.003, 0.001)},
           "diagrams_per_s": n_int / wall, "evals_per_s": srv.evals / wall, "rounds": srv.rounds,
           "completed_by_cap": caps, "budget_bytes": srv.budget,
           "target_met_fraction": len(met) / max(1, len(done)),
           "warm_start": a.warm_start, "warm_started_integrals": srv.warm_starts, "grouped": a.grouped,
           "warm_blend": a.warm_blend if a.warm_start else None, "warm_train": a.warm_train if a.warm_start else None,
           "rounds_per_request": {"median": float(sorted(rounds)[len(rounds) // 2]) if rounds else None,
                                  "max": max(rounds) if rounds else None},
           "example": [{"n": r.n_dens, "delta": r.delta, "cap": r.cap, "target": r.target, "E_corr": r.energy,
                        "sigma": r.sigma, "per_order": r.per_order, "latency_s": r.latency} for r in done[:3]]}
    print(json.dumps(out))
    if logf:
        logf.close()
    be.close()


if __name__ == "__main__":
    main()
