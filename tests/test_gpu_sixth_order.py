"""Sixth order on the device (Table I: 27300 diagrams, d = 21; evaluated by the paper with low
statistics only): per-sample parity with the FP64 oracle on shared grids, the mixed modes on
identical samples, one batched iteration against the oracle's (single diagrams, a group, the
denominator regulator), anomalous diagrams, and the shared-memory bin limit at d = 21."""
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


@pytest.fixture(scope="module")
def diagrams():
    return O.enumerate_diagrams(6)


def _pick(Ds, k, rng, anomalous=False):
    pool = [D for D in Ds if O.is_anomalous(D) == anomalous]
    return [pool[i] for i in sorted(rng.choice(len(pool), size=k, replace=False))]


@pytest.mark.parametrize("matter,k,mapk,count", [("pnm", 3, 0, 1536), ("pnm", 2, 1, 1536), ("snm", 1, 0, 512),
                                                 ("asym", 1, 0, 512)])
def test_per_sample_parity_fp64(ctx, diagrams, matter, k, mapk, count):
    rng = np.random.default_rng(600 + len(matter) + 7 * mapk)
    po, pm = matter_pair(matter, map_kind=mapk)
    for D in _pick(diagrams, k, rng):
        cfg = M.vegas_cfg(samples=1 << 16, seed=4242, stream_id=D.diagram_id + 3, precision=M.MBPT_FP64)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
        try:
            grid = random_grid(po.dim(D), 50, rng)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            t, first = 2, 333
            xg, wg = M.mbpt_dump_samples(g, t, first, count, po.dim(D))
            xo, wo = oracle_dump(D, po, grid, 4242, D.diagram_id + 3, t, first, count)
            assert np.max(np.abs(xg - xo)) <= 4 * EPS
            ok = ~near_surface(D, po, xo)
            assert (~ok).sum() <= 2
            assert np.array_equal(wg[ok] == 0.0, wo[ok] == 0.0)
            assert (wo != 0).sum() > 0
            tol = fp64_tol(D, po, xo, wo) + 1e-15 * np.mean(np.abs(wo))
            err = np.abs(wg - wo)
            assert not (ok & (err > tol)).any(), (D.diagram_id, np.max(err[ok] / np.maximum(np.abs(wo[ok]), 1e-300)))
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_MIXED, M.MBPT_MIXED_MAP64])
@pytest.mark.parametrize("matter,k", [("pnm", 3), ("snm", 1)])
def test_mixed_precision_deviation(ctx, diagrams, matter, k, prec):
    """64-term spin sums in FP32 (difference form): deviation from the FP64 oracle on identical
    samples below 1e-4 of the summed |w|."""
    rng = np.random.default_rng(61 + len(matter))
    po, pm = matter_pair(matter)
    count = 2048 if matter == "pnm" else 512
    for D in _pick(diagrams, k, rng):
        cfg = M.vegas_cfg(samples=1 << 16, seed=17, stream_id=D.diagram_id, precision=prec)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
        try:
            grid = random_grid(po.dim(D), 50, rng, strength=0.5)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            xg, wg = M.mbpt_dump_samples(g, 0, 0, count, po.dim(D))
            xo, wo = oracle_dump(D, po, grid, 17, D.diagram_id, 0, 0, count)
            assert np.max(np.abs(xg - xo)) <= (4 * EPS if prec == M.MBPT_MIXED_MAP64 else 2e-7)
            ok = ~near_surface(D, po, xo, rel=1e-5 if prec == M.MBPT_MIXED else 1e-9)
            l1 = np.sum(np.abs(wg[ok] - wo[ok])) / max(np.sum(np.abs(wo[ok])), 1e-300)
            assert l1 < 1e-4, l1
            assert abs(np.sum(wg[ok]) - np.sum(wo[ok])) <= 1e-4 * np.sum(np.abs(wo[ok]))
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_FP64, M.MBPT_MIXED])
def test_one_iteration_against_the_oracle(ctx, diagrams, prec):
    """One batched iteration (ragged sample count, several chunks): sum w and sum w^2 against the
    oracle's iteration on the same grid, and the refined grid against the oracle's refinement of the
    GPU histogram."""
    rng = np.random.default_rng(66)
    po, pm = matter_pair("pnm")
    D = _pick(diagrams, 1, rng)[0]
    M_s = 20000 + 77
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=M_s, seed=8, stream_id=5, precision=prec))
    try:
        grid = random_grid(D.d, 50, rng, strength=0.5)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = M.mbpt_estimate(g)
        img = M.mbpt_get_state(g)
        ref = O.vegas_iteration(D, po, grid, 8, 5, 0, M_s)
        rel = 1e-11 if prec == M.MBPT_FP64 else 1e-4
        assert r.n_iter == 1 and r.n_evals == M_s and r.status == 0
        assert r.last_mean == pytest.approx(ref.mean, rel=rel)
        assert r.last_sigma == pytest.approx(np.sqrt(ref.var_of_mean), rel=10 * rel)
        h = M.state_last_hist(img, D.d, 50)
        new_grid = M.state_grid(img, D.d, 50)
        assert np.max(np.abs(new_grid - O.refine(grid, h))) < 1e-12
    finally:
        M.mbpt_destroy_diagram(g)


def test_anomalous_sixth_order_integrals_are_zero(ctx, diagrams):
    rng = np.random.default_rng(67)
    po, pm = matter_pair("asym")
    for D in _pick(diagrams, 4, rng, anomalous=True):
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=8192, precision=M.MBPT_MIXED))
        try:
            _, w = M.mbpt_dump_samples(g, 0, 0, 4096, po.dim(D), with_x=False)
            assert np.all(w == 0.0)
            M.mbpt_vegas_iterate(ctx, [g], 2)
            r = M.mbpt_estimate(g)
            assert r.mean == 0.0 and r.sigma == 0.0 and r.status == 0
        finally:
            M.mbpt_destroy_diagram(g)


def test_bins_limited_by_shared_memory_at_d21(ctx, diagrams):
    """d x n_bins <= MBPT_MAX_GRID_CELLS: 54 bins at d = 21, 64 at d = 18 (rotational map)."""
    D = diagrams[1234]
    _, pm = matter_pair("pnm")
    with pytest.raises(M.MbptError) as e:
        M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=4096, n_bins=55))
    assert e.value.status == M.MBPT_EINVAL
    for nb, mapk in ((54, 0), (64, 1)):
        _, pm = matter_pair("pnm", map_kind=mapk)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=4096, n_bins=nb))
        try:
            M.mbpt_vegas_iterate(ctx, [g], 2)
            assert M.mbpt_estimate(g).status == 0
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_FP64, M.MBPT_MIXED])
def test_sixth_order_group_one_iteration(ctx, diagrams, prec):
    """A group of three sixth-order diagrams of one particle-hole composition (scales 1, -1, 2): one
    iteration against the oracle's group iteration on the same grid and counters."""
    po, pm = matter_pair("pnm")
    key = sorted(O.groups(6))[2]
    members = O.groups(6)[key].members[:3]
    G = O.Group(members, [1.0, -1.0, 2.0])
    rng = np.random.default_rng(68)
    M_s = 12000 + 11
    g = M.mbpt_create_group(ctx, [make_desc(D) for D in G.members], pm,
                            M.vegas_cfg(samples=M_s, seed=2, stream_id=31, precision=prec), scales=G.scales)
    try:
        grid = random_grid(G.d, 50, rng, strength=0.5)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = M.mbpt_estimate(g)
        ref = O.vegas_iteration(G, po, grid, 2, 31, 0, M_s)
        parts = [abs(c) * abs(O.vegas_iteration(D, po, grid, 2, 31, 0, M_s).sum_w) for D, c in
                 zip(G.members, G.scales)]
        rel = 1e-11 if prec == M.MBPT_FP64 else 1e-4
        assert r.n_evals == M_s and r.status == 0
        assert abs(r.last_mean * M_s - ref.sum_w) <= rel * max(abs(ref.sum_w), sum(parts))
    finally:
        M.mbpt_destroy_diagram(g)


def test_sixth_order_regulator_components(ctx, diagrams):
    """Denominator regulator at sixth order (five shifted denominators per sample): each component
    of one iteration against the oracle's iteration with that shift."""
    import dataclasses
    po, pm = matter_pair("pnm")
    rng = np.random.default_rng(69)
    D = _pick(diagrams, 1, rng)[0]
    shifts = (2.0, 4.0, 6.0)
    M_s = 12000 + 5
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=M_s, seed=6, stream_id=41,
                                                                 precision=M.MBPT_FP64, shifts=shifts))
    try:
        grid = random_grid(D.d, 50, rng, strength=0.4)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        mean, sigma = M.mbpt_estimate_shifts(g)
        for k, sh in enumerate(shifts):
            ref = O.vegas_iteration(D, dataclasses.replace(po, shift=sh), grid, 6, 41, 0, M_s)
            assert mean[k] == pytest.approx(ref.mean, rel=1e-11)
            assert sigma[k] == pytest.approx(np.sqrt(ref.var_of_mean), rel=1e-10)
    finally:
        M.mbpt_destroy_diagram(g)
