"""Denominator-regulator study (Sec. III.A): every fourth-order diagram of neutron (or symmetric) matter at one density,
integrated with three energy-denominator shifts and their quadratic extrapolation to zero shift beside
the unregulated estimate, on identical samples.  Mirror partners (equal integrals by symmetry) measure
how far each estimate can be trusted: their difference in units of the combined error.

    python -m paper_2603_24532_b300.run_regulator_study [--kf 1.33] [--samples 2^20] [--iters 10]
        [--shifts 1 2 3] [--precision mixed]

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import mbpt as M


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kf", type=float, default=1.33)
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--shifts", type=float, nargs=3, default=(1.0, 2.0, 3.0))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--map-kind", type=int, default=0)
    ap.add_argument("--snm", action="store_true", help="symmetric matter (kF_p = kF_n) instead of neutron matter")
    a = ap.parse_args()
    prec = M.MBPT_MIXED if a.precision == "mixed" else M.MBPT_FP64
    ctx = M.mbpt_ctx_create(0, 4 << 30)
    ph = M.physics(kF_n=a.kf, kF_p=a.kf if a.snm else 0.0, K_max=a.kf + 6.0, map_kind=a.map_kind)
    descs = [d for d in M.mbpt_generate(4) if not d.anomalous]
    gs = [M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=a.samples, seed=7, stream_id=d.diagram_id,
                                                        precision=prec, shifts=a.shifts, train_iters=2))
          for d in descs]
    M.mbpt_vegas_iterate(ctx, gs, a.iters)
    res = M.mbpt_estimate_batch(gs)
    rows = {}
    for d, g, r in zip(descs, gs, res):
        mean, sig = M.mbpt_estimate_shifts(g)
        rows[d.diagram_id] = {"mirror": d.mirror_id, "mean": r.mean, "sigma": r.sigma, "chi2": r.chi2_dof,
                              "shifted": [float(v) for v in mean[:3]], "shifted_sigma": [float(v) for v in sig[:3]],
                              "extrapolated": float(mean[3]), "extrapolated_sigma": float(sig[3])}
    pairs = []
    for i, row in rows.items():
        j = row["mirror"]
        if i < j and j in rows:
            o = rows[j]
            z0 = (row["mean"] - o["mean"]) / max(math.hypot(row["sigma"], o["sigma"]), 1e-300)
            ze = (row["extrapolated"] - o["extrapolated"]) / max(math.hypot(row["extrapolated_sigma"],
                                                                            o["extrapolated_sigma"]), 1e-300)
            zs = (row["shifted"][0] - o["shifted"][0]) / max(math.hypot(row["shifted_sigma"][0],
                                                                        o["shifted_sigma"][0]), 1e-300)
            pairs.append({"pair": [i, j], "z_unregulated": z0, "z_smallest_shift": zs, "z_extrapolated": ze})
    tot = {k: float(sum(r[k] for r in rows.values())) for k in ("mean", "extrapolated")}
    tot_sig = {"mean": float(math.sqrt(sum(r["sigma"] ** 2 for r in rows.values()))),
               "extrapolated": float(math.sqrt(sum(r["extrapolated_sigma"] ** 2 for r in rows.values())))}
    chi2 = [r["chi2"] for r in rows.values()]
    out = {"workload": "33 non-anomalous fourth-order diagrams, %s kF %.2f, %s, %d x %d samples (2 training), "
                       "shifts %s MeV" % ("SNM" if a.snm else "PNM", a.kf, a.precision, a.iters, a.samples,
                                          list(a.shifts)),
           "E4_unregulated": tot["mean"], "sigma_unregulated": tot_sig["mean"],
           "E4_extrapolated": tot["extrapolated"], "sigma_extrapolated": tot_sig["extrapolated"],
           "E4_shifted": [float(sum(r["shifted"][k] for r in rows.values())) for k in range(3)],
           "max_chi2_unregulated": float(np.max(chi2)), "median_chi2_unregulated": float(np.median(chi2)),
           "mirror_pairs": len(pairs),
           "max_abs_z_unregulated": float(max(abs(p["z_unregulated"]) for p in pairs)),
           "max_abs_z_smallest_shift": float(max(abs(p["z_smallest_shift"]) for p in pairs)),
           "max_abs_z_extrapolated": float(max(abs(p["z_extrapolated"]) for p in pairs)),
           "pairs": pairs}
    print(json.dumps(out))
    M.mbpt_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
