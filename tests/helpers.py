"""Shared helpers for the GPU tests: oracle-built descriptors, matched physics
points, random VEGAS grids and the per-sample tolerance."""
import numpy as np

import oracle as O
from paper_2603_24532_b300 import mbpt as M

EPS = np.finfo(np.float64).eps


def make_desc(D: O.Diagram) -> M.mbpt_diagram_desc:
    """Product descriptor built from the oracle's own enumeration (no product code involved)."""
    return M.mbpt_diagram_desc.from_lists(D.n, D.lines, D.ports, D.chords, D.coef(), diagram_id=D.diagram_id,
                                          flags=M.FLAG_ANOMALOUS if O.is_anomalous(D) else 0)


def phys_pair(kF_n=1.0, kF_p=0.0, **kw):
    po = O.Physics(kF_n=kF_n, kF_p=kF_p, **kw)
    pm = M.physics(kF_n=kF_n, kF_p=kF_p, hbar2_over_m=po.hbar2_over_m, C_S=po.C_S, C_Y=po.C_Y, m_pi=po.m_pi,
                   Lam=po.Lam, reg_power=po.reg_power, K_max=po.K_max, map_kind=po.map_kind,
                   spectrum=po.spectrum)
    return po, pm


MATTER = {
    "pnm": dict(kF_n=1.0, kF_p=0.0),
    "snm": dict(kF_n=1.33, kF_p=1.33),
    "asym": dict(kF_n=1.2, kF_p=0.85),
}


def matter_pair(name, map_kind=0, **kw):
    args = dict(MATTER[name])
    args.update(kw)
    kmax = max(args["kF_n"], args["kF_p"]) + 6.0
    return phys_pair(K_max=kmax, map_kind=map_kind, **args)


def random_grid(d, nb, rng, strength=0.9):
    """A valid, strongly non-uniform VEGAS grid (monotone, 0 .. 1)."""
    g = np.zeros((d, nb + 1))
    for a in range(d):
        w = rng.random(nb) ** 3 + (1 - strength) * 0.05
        e = np.concatenate([[0.0], np.cumsum(w)])
        e /= e[-1]
        e[-1] = 1.0
        g[a] = e
    return g


def oracle_dump(D, po, grid, seed, sid, t, first, count):
    sums, hist, x, w = O.vegas_samples(0, D, po.array(), grid.shape[0], grid, seed, sid, t, first, first + count,
                                       dump=True)
    return x, w


def near_surface(D, po, x, rel=1e-9):
    """(mixed precision places samples with an FP32 map: compare with rel ~ 1e-5 there)"""
    # True where some line momentum sits within rel*kF^2 of a Fermi surface.
    kf2 = [k * k for k in (po.kF_n, po.kF_p) if k > 0]
    out = np.zeros(len(x), dtype=bool)
    for i in range(len(x)):
        u = O.line_ksq(D, po, x[i])
        out[i] = any(np.min(np.abs(u - k2)) < rel * k2 for k2 in kf2)
    return out


def fp64_tol(D, po, x, w_oracle):
    """Per-sample tolerance for the FP64 path: 1e-12 relative, widened by the
    rounding amplification of the sample (64 ulps times the oracle's condition
    number: sum_m sum_{l in cut m} eps_l / |D_m| for the energy denominators plus
    sum |spin-sum terms| / |spin sum| for the cancellation between direct and
    exchange terms).  Callers add an absolute floor of 1e-15 times the mean |w| of
    the sample set: weights that far below the scale of the integral (products of
    regulators near the FP64 underflow range) cannot move the estimate."""
    tol = np.zeros(len(x))
    for i in range(len(x)):
        if w_oracle[i] == 0.0:
            continue
        f, cond = O.integrand(D, po, x[i], with_cond=True)
        tol[i] = (1e-12 + 64 * EPS * cond) * abs(w_oracle[i])
    return tol
