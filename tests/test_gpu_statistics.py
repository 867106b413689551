"""Statistics of the estimates (Sec. III.C: PVegas' training and evaluation phases; Sec. III.A: grouped
evaluation).  The evaluation-phase combination against the oracle's pooled combination on one grid,
the frozen grid, and at fourth order -- where single weights are heavy-tailed -- the scatter of
independent runs against their own errors: eight seeds of the per-diagram sums and of the aligned group
sums must scatter as their errors say, the two must agree, and mirror partners must agree; the same
scatter test for E5 at fifth order."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import make_desc, matter_pair, random_grid
from paper_2603_24532_b300 import mbpt as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = M.mbpt_ctx_create(0, 8 << 30)
    yield c
    M.mbpt_ctx_destroy(c)


def _chi2dof(vals, sig):
    vals, sig = np.asarray(vals, dtype=float), np.asarray(sig, dtype=float)
    w = 1.0 / sig ** 2
    m = float(np.sum(w * vals) / np.sum(w))
    return float(np.sum((vals - m) ** 2 * w) / (len(vals) - 1)), m, float(1.0 / math.sqrt(np.sum(w)))


@pytest.mark.parametrize("matter", ["pnm", "asym"])
def test_pooled_combination_vs_oracle(ctx, matter):
    """On a grid handed to both sides and frozen (no training iterations), the evaluation-phase estimate,
    error and chi^2 of three FP64 iterations of unequal size equal the oracle's pooled combination of its
    own iteration sums, and the grid is not refined."""
    rng = np.random.default_rng(21)
    D = O.enumerate_diagrams(3)[2]
    po, pm = matter_pair(matter)
    d = po.dim(D)
    grid = random_grid(d, 50, rng, strength=0.6)
    cfg = M.vegas_cfg(samples=6000, seed=4, stream_id=17, combine=M.MBPT_COMBINE_POOLED)
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
    M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
    s1, s2, cnt = [], [], []
    for t, m in enumerate((6000, 3001, 4500)):
        cfg.samples_per_iter = m
        M.mbpt_set_config(g, cfg)
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = O.vegas_iteration(D, po, grid, 4, 17, t, m)
        s1.append(r.sum_w)
        s2.append(r.sum_w2)
        cnt.append(m)
    res = M.mbpt_estimate(g)
    mean, sigma, chi2 = O.combine_pooled(s1, s2, cnt)
    scale = sum(abs(a) for a in s1) / sum(cnt) + abs(mean)
    assert abs(res.mean - mean) <= 1e-10 * scale
    assert res.sigma == pytest.approx(sigma, rel=1e-8)
    assert res.chi2_dof == pytest.approx(chi2, rel=1e-6, abs=1e-9)
    assert res.n_iter == 3 and res.n_evals == sum(cnt)
    assert np.array_equal(M.state_grid(M.mbpt_get_state(g), d, 50), grid)
    M.mbpt_destroy_diagram(g)


def test_training_iterations_then_frozen_grid(ctx):
    """With train_iters = 3 the grid is refined after the three training iterations and then kept; the
    estimate combines the evaluation iterations only (before the first one it has infinite error)."""
    D = O.enumerate_diagrams(2)[0]
    po, pm = matter_pair("pnm")
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=1 << 15, seed=2, stream_id=1,
                                                                  combine=M.MBPT_COMBINE_POOLED, train_iters=3,
                                                                  precision=M.MBPT_MIXED))
    grids = []
    for it in range(6):
        M.mbpt_vegas_iterate(ctx, [g], 1)
        grids.append(M.state_grid(M.mbpt_get_state(g), 9, 50))
        r = M.mbpt_estimate(g)
        if it < 3:
            assert math.isinf(r.sigma)
        else:
            assert 0.0 < r.sigma < math.inf
    assert not np.array_equal(grids[0], grids[1]) and not np.array_equal(grids[1], grids[2])
    assert np.array_equal(grids[2], grids[3]) and np.array_equal(grids[3], grids[5])
    img = M.mbpt_get_state(g)
    T = 6
    hm = np.frombuffer(img, dtype=np.float64, count=T, offset=M.STATE_HEADER_BYTES + 80)
    r = M.mbpt_estimate(g)
    assert r.mean == pytest.approx(float(np.mean(hm[3:])), rel=1e-12)   # equal sizes: the plain average
    M.mbpt_destroy_diagram(g)


# ---- fourth order: scatter of independent runs --------------------------------------------------------
SEEDS = range(1, 9)
TRAIN, EVAL, SAMPLES = 6, 10, 1 << 22
POINTS = {"PNM kF=1.33": (1.33, 0.0), "SNM kF=1.6": (1.6, 1.6)}


def _cfg(seed, sid):
    return M.vegas_cfg(samples=SAMPLES, seed=seed, stream_id=sid, precision=M.MBPT_MIXED, alpha=1.0,
                       train_iters=TRAIN, combine=M.MBPT_COMBINE_POOLED)


def _run(ctx, gs):
    M.mbpt_vegas_iterate(ctx, gs, TRAIN + EVAL)
    res = M.mbpt_estimate_batch(gs)
    for g in gs:
        M.mbpt_destroy_diagram(g)
    return res


@pytest.fixture(scope="module")
def fourth_order_runs(ctx):
    """Per physics point and seed: the sum of the 33 non-anomalous fourth-order diagrams integrated one by
    one, and the sum of the four aligned group integrals (the same diagrams by number of hole loop
    momenta); 6 training iterations, then 10 frozen-grid iterations of 2^22 samples each."""
    descs = [d for d in M.mbpt_generate(4) if not d.anomalous]
    groups = {}
    for d in descs:
        groups.setdefault(M.mbpt_hole_chords(d), []).append(d)
    out = {}
    for name, (kf, kfp) in POINTS.items():
        ph = M.physics(kF_n=kf, kF_p=kfp, K_max=kf + 6.0)
        per, grp, diag = [], [], []
        for seed in SEEDS:
            r = _run(ctx, [M.mbpt_create_diagram(ctx, d, ph, _cfg(seed, d.diagram_id)) for d in descs])
            per.append((sum(x.mean for x in r), math.sqrt(sum(x.sigma ** 2 for x in r))))
            diag.append([(x.mean, x.sigma) for x in r])
            r = _run(ctx, [M.mbpt_create_group(ctx, mem, ph, _cfg(seed, 500 + key))
                           for key, mem in sorted(groups.items())])
            grp.append((sum(x.mean for x in r), math.sqrt(sum(x.sigma ** 2 for x in r))))
        out[name] = {"per": per, "grp": grp, "diag": diag, "descs": descs}
    return out


@pytest.mark.parametrize("name", list(POINTS))
def test_fourth_order_seed_scatter(fourth_order_runs, name):
    """Eight independent seeds: the per-diagram sums and the group sums each scatter consistently with
    their errors (chi^2/dof <= 2 over 7 degrees of freedom), and the eight-seed mean of the group sums
    agrees with that of the per-diagram sums (3.4e8 samples per diagram) within 3 sigma."""
    R = fourth_order_runs[name]
    c_per, m_per, s_per = _chi2dof(*zip(*R["per"]))
    c_grp, m_grp, s_grp = _chi2dof(*zip(*R["grp"]))
    assert c_per <= 2.0, (c_per, R["per"])
    assert c_grp <= 2.0, (c_grp, R["grp"])
    assert abs(m_grp - m_per) <= 3.0 * math.hypot(s_grp, s_per), (m_grp, s_grp, m_per, s_per)
    # the aligned groups are at least as precise as the diagrams integrated one by one at equal member
    # evaluations (every group sample evaluates each of its members once)
    assert s_grp <= 1.1 * s_per, (s_grp, s_per)


@pytest.mark.parametrize("name", list(POINTS))
def test_fourth_order_mirror_pairs_agree(fourth_order_runs, name):
    """Mirror (complex-conjugate) partners have equal integrals for a real symmetric potential: their
    eight-seed estimates, integrated independently, agree within 3 sigma."""
    R = fourth_order_runs[name]
    descs = R["descs"]
    pos = {d.diagram_id: i for i, d in enumerate(descs)}
    pairs = [(pos[d.diagram_id], pos[d.mirror_id]) for d in descs
             if d.mirror_id != d.diagram_id and d.diagram_id < d.mirror_id and d.mirror_id in pos]
    assert len(pairs) >= 3
    for i, j in pairs:
        _, mi, si = _chi2dof([R["diag"][k][i][0] for k in range(len(SEEDS))], [R["diag"][k][i][1] for k in range(len(SEEDS))])
        _, mj, sj = _chi2dof([R["diag"][k][j][0] for k in range(len(SEEDS))], [R["diag"][k][j][1] for k in range(len(SEEDS))])
        assert abs(mi - mj) <= 3.0 * math.hypot(si, sj), (descs[i].diagram_id, mi, si, mj, sj)


FIFTH_SEEDS = range(11, 19)
FIFTH_POINTS = (1.0, 1.33)


@pytest.fixture(scope="module")
def fifth_order_runs(ctx):
    """Per Fermi momentum (PNM) and seed: E5 as the sum of the 668 non-anomalous fifth-order diagrams
    integrated one by one, and as the sum of the five aligned group integrals; 3 training iterations, then
    10 frozen-grid iterations of 2^20 samples each, alpha 0.75 (about 1 min on one B300)."""
    descs = [d for d in M.mbpt_generate(5) if not d.anomalous]
    groups = {}
    for d in descs:
        groups.setdefault(M.mbpt_hole_chords(d), []).append(d)

    def cfg(seed, sid):
        return M.vegas_cfg(samples=1 << 20, seed=seed, stream_id=sid, precision=M.MBPT_MIXED, alpha=0.75,
                           train_iters=3, combine=M.MBPT_COMBINE_POOLED)

    out = {}
    for kf in FIFTH_POINTS:
        ph = M.physics(kF_n=kf, K_max=kf + 6.0)
        per, grp = [], []
        for seed in FIFTH_SEEDS:
            gs = [M.mbpt_create_diagram(ctx, d, ph, cfg(seed, d.diagram_id)) for d in descs]
            M.mbpt_vegas_iterate(ctx, gs, 13)
            r = M.mbpt_estimate_batch(gs)
            per.append((sum(x.mean for x in r), math.sqrt(sum(x.sigma ** 2 for x in r))))
            for g in gs:
                M.mbpt_destroy_diagram(g)
            gg = [M.mbpt_create_group(ctx, mem, ph, cfg(seed, 5000 + key)) for key, mem in sorted(groups.items())]
            M.mbpt_vegas_iterate(ctx, gg, 13)
            r = M.mbpt_estimate_batch(gg)
            grp.append((sum(x.mean for x in r), math.sqrt(sum(x.sigma ** 2 for x in r))))
            for g in gg:
                M.mbpt_destroy_diagram(g)
        out[kf] = {"per": per, "grp": grp}
    return out


@pytest.mark.parametrize("kf", FIFTH_POINTS)
def test_fifth_order_seed_scatter(fifth_order_runs, kf):
    """E5 at fifth order, where single weights are heaviest-tailed: over eight independent seeds the
    per-diagram sums and the aligned group sums each scatter consistently with their errors (chi^2/dof <= 2
    over 7 degrees of freedom), their eight-seed means agree within 3 sigma, and the groups are at least as
    precise at equal member evaluations."""
    R = fifth_order_runs[kf]
    c_per, m_per, s_per = _chi2dof(*zip(*R["per"]))
    c_grp, m_grp, s_grp = _chi2dof(*zip(*R["grp"]))
    assert c_per <= 2.0, (c_per, R["per"])
    assert c_grp <= 2.0, (c_grp, R["grp"])
    assert abs(m_grp - m_per) <= 3.0 * math.hypot(s_grp, s_per), (m_grp, s_grp, m_per, s_per)
    assert s_grp <= 1.1 * s_per, (s_grp, s_per)


def test_histogram_layouts_agree(ctx):
    """The block-shared FP64 histogram layout gives the same sums as the warp-private FP32 one (sums do not
    depend on the histogram) and histograms equal to FP32 rounding."""
    D = O.enumerate_diagrams(4)[7]
    po, pm = matter_pair("pnm")
    imgs, res = [], []
    for layout in (M.MBPT_HIST_WARP_F32, M.MBPT_HIST_BLOCK_F64):
        M.mbpt_ctx_set_hist_layout(ctx, layout)
        assert M.mbpt_ctx_get_hist_layout(ctx) == layout
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=1 << 18, seed=3, stream_id=2,
                                                                      precision=M.MBPT_MIXED))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        res.append(M.mbpt_estimate(g))
        imgs.append(M.state_last_hist(M.mbpt_get_state(g), po.dim(D), 50))
        M.mbpt_destroy_diagram(g)
    M.mbpt_ctx_set_hist_layout(ctx, M.MBPT_HIST_WARP_F32)
    assert res[0].mean == res[1].mean and res[0].sigma == res[1].sigma
    assert np.allclose(imgs[0], imgs[1], rtol=1e-5, atol=1e-6 * float(np.max(imgs[0])))
    with pytest.raises(M.MbptError):
        M.mbpt_ctx_set_hist_layout(ctx, 7)
