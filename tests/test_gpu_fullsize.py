"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (autotuned shape): sampled outputs against the oracle one by one,
and the batched kernel's sum over 2^22 (or 2^24) samples against the sum of every
sample re-evaluated individually (a property that holds at any size)."""
import numpy as np
import pytest

import oracle as O
from helpers import fp64_tol, make_desc, near_surface, oracle_dump
from paper_2603_24532_b300 import autotune as A
from paper_2603_24532_b300 import mbpt as M

pytestmark = pytest.mark.gpu

KF_SCAN = [round(0.8 + 0.1 * i, 2) for i in range(10)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = M.mbpt_ctx_create(0, 8 << 30)
    yield c
    M.mbpt_ctx_destroy(c)


def _pair(kf_n, kf_p):
    po = O.Physics(kF_n=kf_n, kF_p=kf_p, K_max=max(kf_n, kf_p) + 6.0)
    pm = M.physics(kF_n=kf_n, kF_p=kf_p, K_max=max(kf_n, kf_p) + 6.0)
    return po, pm


def _sampled_indices(n_samples, k, rng):
    idx = np.unique(np.concatenate([rng.integers(0, n_samples, size=k - 2), [0, n_samples - 1]]))
    return idx


def _run_and_check(ctx, specs, samples, prec, check_sum_of, check_samples_of, rng, tuned=True):
    """specs: list of (oracle diagram, oracle physics, product physics, stream id)."""
    gs = [M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=samples, seed=1, stream_id=sid,
                                                                   precision=prec))
          for D, po, pm, sid in specs]
    try:
        if tuned:
            A.autotune(ctx, gs, spts=(32, 64), trials=1)
        pre = [M.mbpt_get_state(g) for g in gs]
        M.mbpt_vegas_iterate(ctx, gs, 1)
        res = M.mbpt_estimate_batch(gs)
        for i in check_sum_of:
            D = specs[i][0]
            post = M.mbpt_get_state(gs[i])
            M.mbpt_set_state(gs[i], pre[i])                  # the grid iteration 0 used
            _, w = M.mbpt_dump_samples(gs[i], 0, 0, samples, D.d, with_x=False)
            M.mbpt_set_state(gs[i], post)
            s_all = float(np.sum(w))
            assert s_all / samples == pytest.approx(res[i].last_mean, rel=1e-11, abs=1e-300)
        for i in check_samples_of:
            D, po, pm, sid = specs[i]
            M.mbpt_set_state(gs[i], pre[i])
            grid = O.uniform_grid(D.d, 50)
            idx = _sampled_indices(samples, 96, rng)
            wg = np.concatenate([M.mbpt_dump_samples(gs[i], 0, int(j), 1, D.d, with_x=False)[1] for j in idx])
            od = [oracle_dump(D, po, grid, 1, sid, 0, int(j), 1) for j in idx]
            xo = np.concatenate([o[0] for o in od])
            wo = np.concatenate([o[1] for o in od])
            ok = ~near_surface(D, po, xo, rel=1e-9 if prec == M.MBPT_FP64 else 1e-5)
            # a sample outside the Fermi-sea steps is zero on both sides; in mixed precision a weight
            # below the FP32 range of the regulator (|w| ~ 1e-100) may also round to zero
            assert np.all(wg[ok & (wo == 0)] == 0)
            if prec == M.MBPT_FP64:
                assert np.array_equal(wg[ok] == 0, wo[ok] == 0)
                tol = fp64_tol(D, po, xo, wo) + 1e-15 * np.mean(np.abs(wo))
                assert np.all(np.abs(wg - wo)[ok] <= tol[ok])
            else:
                assert np.sum(np.abs(wg - wo)[ok]) <= 1e-4 * np.sum(np.abs(wo[ok])) + 1e-300
        return res
    finally:
        for g in gs:
            M.mbpt_destroy_diagram(g)


def test_third_order_scan_full_size(ctx):
    """Benchmark workload: 3 third-order diagrams x 10 Fermi momenta, 2^22 samples each."""
    rng = np.random.default_rng(21)
    specs = []
    for ki, kf in enumerate(KF_SCAN):
        po, pm = _pair(kf, 0.0)
        for D in O.enumerate_diagrams(3):
            specs.append((D, po, pm, 100 * ki + D.diagram_id))
    res = _run_and_check(ctx, specs, 1 << 22, M.MBPT_MIXED, check_sum_of=[0, 14, 29], check_samples_of=[1, 15, 28],
                         rng=rng)
    assert all(r.n_evals == 1 << 22 for r in res)
    # the same three integrals in FP64: per-sample parity at 1e-12
    _run_and_check(ctx, [specs[1], specs[15], specs[28]], 1 << 22, M.MBPT_FP64, check_sum_of=[1],
                   check_samples_of=[0, 1, 2], rng=rng, tuned=False)


def test_fourth_order_pnm_snm_full_size(ctx):
    """All 39 fourth-order diagrams x kF {1.0, 1.33, 1.6} x {PNM, SNM} = 234 integrals,
    2^24 samples each, one batched launch per iteration."""
    rng = np.random.default_rng(4)
    specs = []
    for ki, kf in enumerate((1.0, 1.33, 1.6)):
        for mi, kfp in enumerate((0.0, kf)):
            po, pm = _pair(kf, kfp)
            for D in O.enumerate_diagrams(4):
                specs.append((D, po, pm, 10000 * mi + 100 * ki + D.diagram_id))
    live = [i for i, s in enumerate(specs) if not O.is_anomalous(s[0])]
    snm = [i for i in live if specs[i][1].kF_p > 0]
    res = _run_and_check(ctx, specs, 1 << 24, M.MBPT_MIXED, check_sum_of=[live[3], snm[-1]],
                         check_samples_of=[live[0], live[40], snm[5], snm[60]], rng=rng)
    for i, s in enumerate(specs):
        if O.is_anomalous(s[0]):
            assert res[i].last_mean == 0.0


def test_fifth_order_all_diagrams_shape(ctx):
    """Every fifth-order diagram x kF {1.0, 1.33, 1.6}, neutron matter, mixed precision, in one
    batch (2520 integrals, 2^15 samples each): sampled per-sample parity on a spread of
    diagrams, exact zeros for the anomalous ones."""
    rng = np.random.default_rng(5)
    specs = []
    for ki, kf in enumerate((1.0, 1.33, 1.6)):
        po, pm = _pair(kf, 0.0)
        for D in O.enumerate_diagrams(5):
            specs.append((D, po, pm, 1000 * ki + D.diagram_id))
    live = [i for i, s in enumerate(specs) if not O.is_anomalous(s[0])]
    pick = [live[j] for j in rng.choice(len(live), size=12, replace=False)]
    res = _run_and_check(ctx, specs, 1 << 15, M.MBPT_MIXED, check_sum_of=[pick[0]], check_samples_of=pick,
                         rng=rng, tuned=False)
    for i, s in enumerate(specs):
        if O.is_anomalous(s[0]):
            assert res[i].last_mean == 0.0 and res[i].last_sigma == 0.0
        assert np.isfinite(res[i].last_mean)


@pytest.mark.parametrize("prec", [M.MBPT_MIXED, M.MBPT_MIXED_MAP64, M.MBPT_FP64])
def test_batched_sum_equals_every_sample_dumped(ctx, prec):
    """The batched iteration (FP32 pre-test, compacted evaluation) against the sum of every sample
    evaluated individually (no pre-test), for all 33 live fourth-order diagrams of symmetric matter at
    kF = 1.6 on adapted grids: a live sample the pre-test wrongly dropped would show here."""
    po, pm = _pair(1.6, 1.6)
    Ds = [D for D in O.enumerate_diagrams(4) if not O.is_anomalous(D)]
    n = 1 << 18
    gs = [M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=n, seed=3, stream_id=70 + D.diagram_id,
                                                                   precision=prec)) for D in Ds]
    try:
        M.mbpt_vegas_iterate(ctx, gs, 4)                    # adapt the grids
        pre = [M.mbpt_get_state(g) for g in gs]
        M.mbpt_vegas_iterate(ctx, gs, 1)
        res = M.mbpt_estimate_batch(gs)
        for g, D, img, r in zip(gs, Ds, pre, res):
            post = M.mbpt_get_state(g)
            M.mbpt_set_state(g, img)
            _, w = M.mbpt_dump_samples(g, 4, 0, n, D.d, with_x=False)
            M.mbpt_set_state(g, post)
            s = float(np.sum(w))
            assert s / n == pytest.approx(r.last_mean, rel=1e-10, abs=1e-12 * float(np.sum(np.abs(w))) / n), D.diagram_id
    finally:
        for g in gs:
            M.mbpt_destroy_diagram(g)


def test_fifth_order_mixed_deviation_48_integrals(ctx):
    """The headline mode at fifth order (FP32 sampling map, FP64 map near a Fermi surface) against the FP64
    mode on identical grids and counters: on 48 fifth-order integrals with grids adapted by three training
    iterations, one iteration of 2^16 samples deviates by at most 1e-4 of max(|I_fp64|, 1e-3 |E5|) per
    integral (the scale of a near-zero diagram is 1e-3 of the order's sum, E5 here from the evaluation
    phase of all 668 integrals: an inverse-variance combination of few iterations can underestimate |E5|
    badly at this order)."""
    kf = 1.33
    ph = M.physics(kF_n=kf, K_max=kf + 6.0)
    descs = [d for d in M.mbpt_generate(5) if not d.anomalous]
    gs = [M.mbpt_create_diagram(ctx, d, ph, M.vegas_cfg(samples=1 << 17, seed=3, stream_id=d.diagram_id,
                                                         precision=M.MBPT_MIXED, alpha=0.75, train_iters=3,
                                                         combine=M.MBPT_COMBINE_POOLED)) for d in descs]
    twins = []
    try:
        M.mbpt_vegas_iterate(ctx, gs, 6)
        e5 = abs(sum(r.mean for r in M.mbpt_estimate_batch(gs)))
        pick = np.random.default_rng(8).choice(len(descs), size=48, replace=False)
        for i in pick:
            grid = M.state_grid(M.mbpt_get_state(gs[i]), 18, 50)
            pair = []
            for prec in (M.MBPT_FP64, M.MBPT_MIXED):
                g = M.mbpt_create_diagram(ctx, descs[i], ph, M.vegas_cfg(samples=1 << 16, seed=3, stream_id=9,
                                                                          precision=prec, alpha=0.75))
                M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
                pair.append(g)
            twins.append(pair)
        M.mbpt_vegas_iterate(ctx, [g for p in twins for g in p], 1)
        devs = []
        for (g64, gmx) in twins:
            a, b = M.mbpt_estimate(g64).last_mean, M.mbpt_estimate(gmx).last_mean
            devs.append(abs(b - a) / max(abs(a), 1e-3 * e5))
        assert max(devs) <= 1e-4, (max(devs), np.median(devs))
    finally:
        for g in gs + [g for p in twins for g in p]:
            M.mbpt_destroy_diagram(g)


def test_fifth_order_mixed_vs_oracle_on_host_grids(ctx):
    """The same bound directly against the oracle on strongly non-uniform grids made on the host: eight
    fifth-order integrals, 4096 samples each, sum of the mixed weights vs the oracle's sum."""
    from helpers import random_grid
    rng = np.random.default_rng(12)
    po, pm = _pair(1.33, 0.0)
    Ds = [D for D in O.enumerate_diagrams(5) if not O.is_anomalous(D)]
    for j in rng.choice(len(Ds), size=8, replace=False):
        D = Ds[j]
        grid = random_grid(D.d, 50, rng, strength=0.5)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=4096, seed=6, stream_id=D.diagram_id,
                                                                      precision=M.MBPT_MIXED))
        try:
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            _, wg = M.mbpt_dump_samples(g, 2, 0, 4096, D.d, with_x=False)
        finally:
            M.mbpt_destroy_diagram(g)
        _, wo = oracle_dump(D, po, grid, 6, D.diagram_id, 2, 0, 4096)
        l1 = float(np.sum(np.abs(wg - wo)) / max(np.sum(np.abs(wo)), 1e-300))
        assert l1 <= 1e-4, (D.diagram_id, l1)
