"""Small profiling case: a few batched VEGAS iterations of the third-order
neutron-matter density scan (3 diagrams x 10 Fermi momenta) with fewer samples
than the benchmark, for ncu captures of k_iterate.

    python -m paper_2603_24532_b300.profile_case [--samples N] [--iters K] [--precision mixed|fp64] [--order 3]
"""
import argparse

from . import mbpt as M


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=1 << 18)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--order", type=int, default=3)
    a = ap.parse_args()
    prec = M.MBPT_MIXED if a.precision == "mixed" else M.MBPT_FP64
    ctx = M.mbpt_ctx_create(0, 4 << 30)
    gs = []
    for ki in range(10):
        kf = 0.8 + 0.1 * ki
        ph = M.physics(kF_n=kf, K_max=kf + 6.0)
        for d in M.mbpt_generate(a.order):
            if d.anomalous:
                continue
            gs.append(M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=a.samples, stream_id=100 * ki + d.diagram_id,
                                                                   precision=prec)))
    M.mbpt_vegas_iterate(ctx, gs, a.iters)
    r = M.mbpt_estimate(gs[0])
    it_ms, fin_ms = M.mbpt_ctx_last_timing(ctx)
    print("integrals %d samples %d iters %d: k_iterate %.3f ms, k_finalize %.3f ms, first mean %.6g +- %.2g"
          % (len(gs), a.samples, a.iters, it_ms, fin_ms, r.mean, r.sigma))
    M.mbpt_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
