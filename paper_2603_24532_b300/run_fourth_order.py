"""Fourth-order workload: all 39 fourth-order diagrams x kF {1.0, 1.33, 1.6} fm^-1 x {neutron,
symmetric} matter = 234 integrals (the 36 anomalous ones are exactly zero and skipped), a fixed number
of batched VEGAS iterations -- `--train` training iterations, then the evaluation phase on the frozen
grid (pooled combination), grid compression alpha -- then the fourth-order energy per physics point
(from the diagrams one by one, and with --groups also from the four aligned particle-hole groups per
point) and the deviation of the chosen precision from the FP64 oracle on a subset of integrals (same grid
and counters).

    python -m paper_2603_24532_b300.run_fourth_order [--samples 2^24] [--iters 10] [--train 4]
        [--alpha 1.0] [--precision mixed] [--groups] [--oracle-integrals 24] [--oracle-samples 65536]
        [--map-kind 0]

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
    ap.add_argument("--samples", type=int, default=1 << 24)
    ap.add_argument("--iters", type=int, default=10, help="iterations in all (training + evaluation)")
    ap.add_argument("--train", type=int, default=4, help="training iterations (grid refined, not combined)")
    ap.add_argument("--alpha", type=float, default=1.0, help="grid compression exponent")
    ap.add_argument("--groups", action="store_true", help="also integrate the aligned particle-hole groups")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "map64", "fp64"])
    ap.add_argument("--oracle-integrals", type=int, default=24)
    ap.add_argument("--oracle-samples", type=int, default=1 << 16)
    ap.add_argument("--map-kind", type=int, default=0)
    a = ap.parse_args()
    prec = {"mixed": M.MBPT_MIXED, "map64": M.MBPT_MIXED_MAP64, "fp64": M.MBPT_FP64}[a.precision]
    ctx = M.mbpt_ctx_create(0, 16 << 30)
    descs = [d for d in M.mbpt_generate(4) if not d.anomalous]
    points = [(kf, kfp, mi, ki) for ki, kf in enumerate((1.0, 1.33, 1.6)) for mi, kfp in enumerate((0.0, kf))]
    gs, meta = [], []
    for kf, kfp, mi, ki in points:
        ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0, map_kind=a.map_kind)
        for d in descs:
            sid = 10000 * mi + 100 * ki + d.diagram_id
            gs.append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(
                samples=a.samples, seed=1, stream_id=sid, precision=prec, alpha=a.alpha, train_iters=a.train,
                combine=M.MBPT_COMBINE_POOLED)))
            meta.append((kf, kfp, sid, d))
    gg, gmeta = [], []
    if a.groups:
        for kf, kfp, mi, ki in points:
            ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0, map_kind=a.map_kind)
            by = {}
            for d in descs:
                by.setdefault(M.mbpt_hole_chords(d), []).append(d)
            for key, mem in sorted(by.items()):
                gg.append(M.mbpt_create_group(ctx, mem, ph, M.vegas_cfg(
                    samples=a.samples, seed=1, stream_id=10000 * mi + 100 * ki + 50 + key, precision=prec,
                    alpha=a.alpha, train_iters=a.train, combine=M.MBPT_COMBINE_POOLED)))
                gmeta.append((kf, kfp))
    t0 = time.perf_counter()
    M.mbpt_vegas_iterate(ctx, gs + gg, a.iters)
    res = M.mbpt_estimate_batch(gs)
    gres = M.mbpt_estimate_batch(gg) if gg else []
    wall = time.perf_counter() - t0
    per_point = {}
    for kf, kfp, mi, ki in points:
        idx = [i for i, m in enumerate(meta) if m[0] == kf and m[1] == kfp]
        rep = [i for i in idx if meta[i][3].repeated_denominator]
        rest = [i for i in idx if not meta[i][3].repeated_denominator]
        per_point["%s kF=%.2f" % ("SNM" if kfp else "PNM", kf)] = {
            "E4": float(sum(res[i].mean for i in idx)),
            "sigma": float(math.sqrt(sum(res[i].sigma ** 2 for i in idx))),
            "max_chi2_dof": float(max(res[i].chi2_dof for i in idx)),
            "repeated_denominator": {"integrals": len(rep), "sum": float(sum(res[i].mean for i in rep)),
                                     "sigma": float(math.sqrt(sum(res[i].sigma ** 2 for i in rep))),
                                     "max_chi2_dof": float(max(res[i].chi2_dof for i in rep))},
            "groups": ({"E4": float(sum(r.mean for r, m in zip(gres, gmeta) if m == (kf, kfp))),
                        "sigma": float(math.sqrt(sum(r.sigma ** 2 for r, m in zip(gres, gmeta) if m == (kf, kfp))))}
                       if gg else None),
            "others": {"integrals": len(rest), "sum": float(sum(res[i].mean for i in rest)),
                       "sigma": float(math.sqrt(sum(res[i].sigma ** 2 for i in rest))),
                       "max_chi2_dof": float(max(res[i].chi2_dof for i in rest)),
                       "median_chi2_dof": float(np.median([res[i].chi2_dof for i in rest]))}}

    dev = None
    if a.oracle_integrals > 0:
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        rng = np.random.default_rng(4)
        pick = rng.choice(len(gs), size=min(a.oracle_integrals, len(gs)), replace=False)
        Os = O.enumerate_diagrams(4)
        devs, l1 = [], []
        for i in pick:
            kf, kfp, sid, d = meta[i]
            D = Os[d.diagram_id]
            po = O.Physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0, map_kind=a.map_kind)
            dd = po.dim(D)
            grid = M.state_grid(M.mbpt_get_state(gs[i]), dd, 50)
            _, wg = M.mbpt_dump_samples(gs[i], 99, 0, a.oracle_samples, dd, with_x=False)
            _, _, _, wo = O.vegas_samples(0, D, po.array(), dd, grid, 1, sid, 99, 0, a.oracle_samples, dump=True)
            key = "%s kF=%.2f" % ("SNM" if kfp else "PNM", kf)
            scale = max(abs(np.sum(wo)), 1e-3 * abs(per_point[key]["E4"]) * a.oracle_samples, 1e-300)
            devs.append(abs(np.sum(wg) - np.sum(wo)) / scale)
            l1.append(np.sum(np.abs(wg - wo)) / max(np.sum(np.abs(wo)), 1e-300))
        dev = {"integrals": int(len(devs)), "samples_each": a.oracle_samples, "max": float(np.max(devs)),
               "median": float(np.median(devs)), "frac_below_1e-4": float(np.mean(np.array(devs) < 1e-4)),
               "l1_max": float(np.max(l1)), "l1_median": float(np.median(l1)),
               "definition": "|sum w - sum w_oracle| / max(|sum w_oracle|, 1e-3 |E4 of the point| M), "
                             "same grid and counters; l1 = sum |w - w_oracle| / sum |w_oracle|"}
    evals = a.iters * a.samples * len(gs)
    out = {"workload": "39 fourth-order diagrams (33 non-anomalous) x kF {1.0, 1.33, 1.6} x {PNM, SNM}, %s, "
                       "%d iterations (%d training) x %d samples, alpha %g" % (a.precision, a.iters, a.train,
                                                                              a.samples, a.alpha),
           "integrals": len(gs), "wall_s": wall, "evals": evals, "evals_per_s": evals / wall,
           "per_point": per_point, "oracle_deviation": dev}
    print(json.dumps(out))
    M.mbpt_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
