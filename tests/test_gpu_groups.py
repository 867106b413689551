"""Grouped evaluation (Sec. III.A): one integral over the sum of same-order diagrams, every member
through its own chord map at the shared sampled point.  The CUDA path against the oracle's group
integrand (the plain sum of the members' integrands) per sample and per iteration, exact identities
of the group machinery, and its combination with the denominator regulator."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from helpers import EPS, fp64_tol, make_desc, matter_pair, near_surface, oracle_dump, random_grid
from paper_2603_24532_b300 import mbpt as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = M.mbpt_ctx_create(0, 2 << 30)
    yield c
    M.mbpt_ctx_destroy(c)


def _group(n, key, k, scales=None):
    G = O.groups(n)[key]
    members = G.members[:k]
    return O.Group(members, list(scales) if scales is not None else [1.0] * len(members))


def _create(ctx, G, pm, cfg):
    return M.mbpt_create_group(ctx, [make_desc(D) for D in G.members], pm, cfg, scales=G.scales)


@pytest.mark.parametrize("n,key,matter,mapk", [(3, 3, "pnm", 0), (4, 4, "snm", 0), (4, 3, "asym", 1),
                                               (5, 5, "pnm", 0)])
def test_group_per_sample_fp64(ctx, n, key, matter, mapk):
    """Dumped group weights equal the scaled sum of the oracle's member weights at every sample,
    within the sum of the members' FP64 tolerances."""
    rng = np.random.default_rng(70 + n + key + mapk)
    po, pm = matter_pair(matter, map_kind=mapk)
    G = _group(n, key, 4, scales=(1.0, 2.0, 0.5, 1.0))
    G = O.Group(G.members, G.scales[:len(G.members)])
    d = po.dim(G)
    cfg = M.vegas_cfg(samples=1 << 16, seed=99, stream_id=17, precision=M.MBPT_FP64)
    g = _create(ctx, G, pm, cfg)
    try:
        grid = random_grid(d, 50, rng)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        t, first, count = 2, 777, 1536
        xg, wg = M.mbpt_dump_samples(g, t, first, count, d)
        tol = np.zeros(count)
        wo = np.zeros(count)
        ok = np.ones(count, dtype=bool)
        for D, c in zip(G.members, G.scales):
            xo, w = oracle_dump(D, po, grid, 99, 17, t, first, count)
            assert np.max(np.abs(xg - xo)) <= 4 * EPS
            ok &= ~near_surface(D, po, xo)
            wo += c * w
            tol += abs(c) * (fp64_tol(D, po, xo, w) + 1e-15 * np.mean(np.abs(w)))
        assert (~ok).sum() <= 2
        assert np.all(np.abs(wg - wo)[ok] <= tol[ok])
        assert (wo != 0).sum() > 0
    finally:
        M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_FP64, M.MBPT_MIXED])
def test_group_one_iteration_vs_oracle(ctx, prec):
    """One iteration of a fourth-order group on a ragged sample count: sum w, sum w^2 and the
    histogram against the oracle's group iteration on the same grid and counters; the refined grid
    against the oracle's refinement of the GPU histogram."""
    rng = np.random.default_rng(8)
    po, pm = matter_pair("pnm")
    G = _group(4, 4, 6, scales=(1.0, -1.0, 2.0, 1.0, 1.0, 0.25))
    M_s = 20000 + 37
    g = _create(ctx, G, pm, M.vegas_cfg(samples=M_s, seed=5, stream_id=23, precision=prec))
    try:
        grid = random_grid(G.d, 50, rng, strength=0.5)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = M.mbpt_estimate(g)
        img = M.mbpt_get_state(g)
        ref = O.vegas_iteration(G, po, grid, 5, 23, 0, M_s)
        parts = [abs(c) * abs(O.vegas_iteration(D, po, grid, 5, 23, 0, M_s).sum_w) for D, c in
                 zip(G.members, G.scales)]
        rel = 1e-11 if prec == M.MBPT_FP64 else 1e-4
        assert r.n_evals == M_s
        assert abs(r.last_mean * M_s - ref.sum_w) <= rel * max(abs(ref.sum_w), sum(parts))
        assert r.last_sigma == pytest.approx(np.sqrt(ref.var_of_mean), rel=10 * rel)
        h = M.state_last_hist(img, G.d, 50)
        hn, rn = h / h.sum(axis=1, keepdims=True), ref.hist / ref.hist.sum(axis=1, keepdims=True)
        assert np.max(np.abs(hn - rn)) < (1e-5 if prec == M.MBPT_FP64 else 1e-3)
        assert np.max(np.abs(M.state_grid(img, G.d, 50) - O.refine(grid, h))) < 1e-12
    finally:
        M.mbpt_destroy_diagram(g)


def test_group_of_a_repeated_member_is_twice_the_diagram(ctx):
    """The group [a, a] doubles every weight exactly: it equals the group [a, a] with scales (2, 0)
    bit for bit over several iterations (same loop, same grids), and after one iteration on the
    uniform grid its estimate is twice that of diagram a (whose loop sums in another order)."""
    po, pm = matter_pair("snm")
    D = O.enumerate_diagrams(4)[11]
    assert not O.is_anomalous(D)
    cfg = M.vegas_cfg(samples=50000, seed=2, stream_id=31, precision=M.MBPT_MIXED_MAP64)
    a = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
    g1 = M.mbpt_create_group(ctx, [make_desc(D), make_desc(D)], pm, cfg)
    g2 = M.mbpt_create_group(ctx, [make_desc(D), make_desc(D)], pm, cfg, scales=[2.0, 0.0])
    try:
        M.mbpt_vegas_iterate(ctx, [a, g1, g2], 1)
        ra, r1 = M.mbpt_estimate(a), M.mbpt_estimate(g1)
        assert r1.last_mean == pytest.approx(2.0 * ra.last_mean, rel=1e-12)
        assert r1.last_sigma == pytest.approx(2.0 * ra.last_sigma, rel=1e-10)
        M.mbpt_vegas_iterate(ctx, [g1, g2], 2)
        r1, r2 = M.mbpt_estimate(g1), M.mbpt_estimate(g2)
        assert (r1.mean, r1.sigma, r1.chi2_dof) == (r2.mean, r2.sigma, r2.chi2_dof)
        assert np.array_equal(M.state_grid(M.mbpt_get_state(g1), D.d, 50),
                              M.state_grid(M.mbpt_get_state(g2), D.d, 50))
    finally:
        for h in (a, g1, g2):
            M.mbpt_destroy_diagram(h)


def test_group_alone_equals_group_in_a_mixed_batch(ctx):
    po, pm = matter_pair("pnm", map_kind=1)
    G = _group(5, 4, 3)
    cfg = M.vegas_cfg(samples=30000, seed=4, stream_id=8, precision=M.MBPT_MIXED)
    g1 = _create(ctx, G, pm, cfg)
    g2 = _create(ctx, G, pm, cfg)
    others = [M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=40000, stream_id=i))
              for i, D in enumerate(O.enumerate_diagrams(3))]
    try:
        M.mbpt_vegas_iterate(ctx, [g1], 2)
        M.mbpt_vegas_iterate(ctx, others[:2] + [g2] + others[2:], 2)
        r1, r2 = M.mbpt_estimate(g1), M.mbpt_estimate(g2)
        assert (r1.mean, r1.sigma, r1.n_evals) == (r2.mean, r2.sigma, r2.n_evals)
        assert M.mbpt_get_state(g1) == M.mbpt_get_state(g2)
    finally:
        for h in [g1, g2] + others:
            M.mbpt_destroy_diagram(h)


def test_group_with_regulator_components(ctx):
    """Group and regulator together: each shifted component of the group after one iteration equals
    the oracle's group iteration with that shift."""
    rng = np.random.default_rng(14)
    po, pm = matter_pair("pnm")
    G = _group(4, 3, 3)
    shifts = (2.0, 5.0, 8.0)
    M_s = 9000 + 5
    g = _create(ctx, G, pm, M.vegas_cfg(samples=M_s, seed=6, stream_id=3, precision=M.MBPT_FP64, shifts=shifts))
    try:
        grid = random_grid(G.d, 50, rng, strength=0.4)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        mean, sigma = M.mbpt_estimate_shifts(g)
        refs = [O.vegas_iteration(G, dataclasses.replace(po, shift=s), grid, 6, 3, 0, M_s) for s in shifts]
        for k in range(3):
            assert mean[k] == pytest.approx(refs[k].mean, rel=1e-11)
            assert sigma[k] == pytest.approx(np.sqrt(refs[k].var_of_mean), rel=1e-10)
        r0 = O.vegas_iteration(G, po, grid, 6, 3, 0, M_s)
        assert M.mbpt_estimate(g).last_mean == pytest.approx(r0.mean, rel=1e-11)
    finally:
        M.mbpt_destroy_diagram(g)


def test_group_errors(ctx):
    po, pm = matter_pair("pnm")
    d3 = make_desc(O.enumerate_diagrams(3)[0])
    d4 = make_desc(O.enumerate_diagrams(4)[0])
    cfg = M.vegas_cfg(samples=1000)
    with pytest.raises(M.MbptError):
        M.mbpt_create_group(ctx, [d3, d4], pm, cfg)             # mixed orders
    with pytest.raises(M.MbptError):
        M.mbpt_create_group(ctx, [], pm, cfg)                   # no members
    with pytest.raises(M.MbptError):
        M.mbpt_create_group(ctx, [d3, d3], pm, cfg, scales=[1.0, float("nan")])
    g = M.mbpt_create_group(ctx, [d3], pm, cfg)                 # one member: a plain integral
    M.mbpt_destroy_diagram(g)


def test_group_with_hartree_fock_spectrum_and_regulator(ctx):
    """The three options together: a group integral in the Hartree-Fock spectrum with denominator
    shifts; its plain estimate and each shifted component after one iteration equal the oracle's
    group iteration with the same spectrum and shift (FP64)."""
    rng = np.random.default_rng(21)
    po, pm = matter_pair("snm", spectrum=1)
    G = _group(3, 3, 2)
    shifts = (1.5, 3.0, 4.5)
    M_s = 8000 + 3
    g = _create(ctx, G, pm, M.vegas_cfg(samples=M_s, seed=8, stream_id=41, precision=M.MBPT_FP64, shifts=shifts))
    try:
        grid = random_grid(G.d, 50, rng, strength=0.4)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        assert M.mbpt_estimate(g).last_mean == pytest.approx(O.vegas_iteration(G, po, grid, 8, 41, 0, M_s).mean,
                                                             rel=1e-11)
        mean, _ = M.mbpt_estimate_shifts(g)
        for k, s in enumerate(shifts):
            ref = O.vegas_iteration(G, dataclasses.replace(po, shift=s), grid, 8, 41, 0, M_s)
            assert mean[k] == pytest.approx(ref.mean, rel=1e-11)
    finally:
        M.mbpt_destroy_diagram(g)
