"""Sixth-order workload (Table I: 27300 diagrams, d = 21), which the paper implemented but evaluated
with low statistics only: every non-anomalous sixth-order diagram, one integral per mirror
(complex-conjugate) pair counted twice (Table I's N_diag^(eff) = 11269 integrals per density), pure
neutron matter, a fixed number of batched VEGAS iterations, then the sixth-order energy per density
and the deviation of the chosen precision from the FP64 oracle on a subset of integrals (same grid
and counters).

    python -m paper_2603_24532_b300.run_sixth_order [--kf 1.33] [--samples 2^18] [--iters 8]
        [--precision mixed] [--oracle-integrals 16] [--oracle-samples 4096] [--map-kind 0]

Prints one JSON line.
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kf", type=float, nargs="+", default=[1.33])
    ap.add_argument("--samples", type=int, default=1 << 18)
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "map64", "fp64"])
    ap.add_argument("--oracle-integrals", type=int, default=16)
    ap.add_argument("--oracle-samples", type=int, default=4096)
    ap.add_argument("--map-kind", type=int, default=0)
    a = ap.parse_args()
    prec = {"mixed": M.MBPT_MIXED, "map64": M.MBPT_MIXED_MAP64, "fp64": M.MBPT_FP64}[a.precision]
    t_gen = time.perf_counter()
    descs = [d for d in M.mbpt_generate(6) if not d.anomalous and d.diagram_id <= d.mirror_id]
    t_gen = time.perf_counter() - t_gen
    mult = {d.diagram_id: 2 if d.mirror_id != d.diagram_id else 1 for d in descs}
    ctx = M.mbpt_ctx_create(0, 24 << 30)
    gs, meta = [], []
    for ki, kf in enumerate(a.kf):
        ph = M.physics(kF_n=kf, K_max=kf + 6.0, map_kind=a.map_kind)
        for d in descs:
            cfg = M.vegas_cfg(samples=a.samples, seed=1, stream_id=100000 * ki + d.diagram_id, precision=prec)
            gs.append(M.mbpt_create_diagram(ctx, d, ph, cfg))
            meta.append((ki, kf, d))
    t0 = time.perf_counter()
    M.mbpt_vegas_iterate(ctx, gs, a.iters)
    res = M.mbpt_estimate_batch(gs)
    wall = time.perf_counter() - t0
    per_kf = {}
    for ki, kf in enumerate(a.kf):
        idx = [i for i, m in enumerate(meta) if m[0] == ki]
        chi2 = np.array([res[i].chi2_dof for i in idx])
        per_kf[str(kf)] = {
            "E6_sum": float(sum(mult[meta[i][2].diagram_id] * res[i].mean for i in idx)),
            "sigma": float(math.sqrt(sum((mult[meta[i][2].diagram_id] * res[i].sigma) ** 2 for i in idx))),
            "median_chi2_dof": float(np.median(chi2)), "frac_chi2_dof_above_3": float(np.mean(chi2 > 3.0)),
            "status_nonzero": int(sum(res[i].status != 0 for i in idx))}

    dev = None
    if a.oracle_integrals > 0:
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        Os = O.enumerate_diagrams(6)
        rng = np.random.default_rng(6)
        pick = rng.choice(len(gs), size=min(a.oracle_integrals, len(gs)), replace=False)
        devs, l1 = [], []
        for i in pick:
            ki, kf, d = meta[i]
            D = Os[d.diagram_id]
            po = O.Physics(kF_n=kf, K_max=kf + 6.0, map_kind=a.map_kind)
            dd = po.dim(D)
            grid = M.state_grid(M.mbpt_get_state(gs[i]), dd, 50)
            sid = 100000 * ki + d.diagram_id
            _, wg = M.mbpt_dump_samples(gs[i], 99, 0, a.oracle_samples, dd, with_x=False)
            _, _, _, wo = O.vegas_samples(0, D, po.array(), dd, grid, 1, sid, 99, 0, a.oracle_samples, dump=True)
            scale = max(abs(np.sum(wo)), 1e-3 * abs(per_kf[str(kf)]["E6_sum"]) * a.oracle_samples, 1e-300)
            devs.append(abs(np.sum(wg) - np.sum(wo)) / scale)
            l1.append(np.sum(np.abs(wg - wo)) / max(np.sum(np.abs(wo)), 1e-300))
        dev = {"integrals": int(len(devs)), "samples_each": a.oracle_samples, "max": float(np.max(devs)),
               "median": float(np.median(devs)), "frac_below_1e-4": float(np.mean(np.array(devs) < 1e-4)),
               "l1_max": float(np.max(l1)), "l1_median": float(np.median(l1)),
               "definition": "|sum w - sum w_oracle| / max(|sum w_oracle|, 1e-3 |E6 of the density| M), "
                             "same grid and counters; l1 = sum |w - w_oracle| / sum |w_oracle|"}
    evals = a.iters * a.samples * len(gs)
    out = {"workload": "27300 sixth-order diagrams (21572 non-anomalous, %d mirror-deduplicated integrals per "
                       "density) x kF %s, PNM, %s, %d iterations x %d samples"
                       % (len(descs), a.kf, a.precision, a.iters, a.samples),
           "integrals": len(gs), "generate_s": t_gen, "wall_s": wall, "evals": evals, "evals_per_s": evals / wall,
           "per_kF": per_kf, "oracle_deviation": dev}
    print(json.dumps(out))
    M.mbpt_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
