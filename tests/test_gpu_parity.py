"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Per-sample parity hands the same VEGAS grid to both sides;
FP64 mode must match to 1e-12 relative (widened only by the conditioning of the
energy denominators), mixed mode is reported against FP64 with a 1e-4 bound."""
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


def _pick(n, k, rng):
    Ds = O.enumerate_diagrams(n)
    if len(Ds) <= k:
        return Ds
    idx = sorted(rng.choice(len(Ds), size=k, replace=False))
    return [Ds[i] for i in idx]


def test_philox_device_matches_oracle(ctx):
    rng = np.random.default_rng(1)
    for _ in range(4):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, size=4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, size=2)]
        got = M.mbpt_philox_device(ctx, ctr, key, 300)
        for i in (0, 1, 77, 299):
            want = O.philox4x32_10([(ctr[0] + i) & 0xFFFFFFFF, ctr[1], ctr[2], ctr[3]], key)
            assert list(got[i]) == want


CASES = [(2, "pnm", 1, 0), (2, "snm", 1, 0), (3, "pnm", 3, 0), (3, "snm", 3, 0), (3, "asym", 3, 0),
         (4, "pnm", 8, 0), (4, "snm", 5, 0), (4, "asym", 5, 0), (5, "pnm", 8, 0), (5, "asym", 3, 0),
         (2, "pnm", 1, 1), (3, "snm", 3, 1), (4, "asym", 4, 1), (5, "pnm", 5, 1)]


@pytest.mark.parametrize("n,matter,k,mapk", CASES)
def test_per_sample_parity_fp64(ctx, n, matter, k, mapk):
    rng = np.random.default_rng(1000 * n + len(matter) + 7 * mapk)
    po, pm = matter_pair(matter, map_kind=mapk)
    count = 1536 if n >= 5 else 3072
    for D in _pick(n, k, rng):
        cfg = M.vegas_cfg(samples=1 << 16, seed=12345, stream_id=D.diagram_id + 7, precision=M.MBPT_FP64)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
        try:
            grid = random_grid(po.dim(D), 50, rng)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            t, first = 3, 1021          # ragged offset, non-zero iteration counter
            xg, wg = M.mbpt_dump_samples(g, t, first, count, po.dim(D))
            xo, wo = oracle_dump(D, po, grid, 12345, D.diagram_id + 7, t, first, count)
            assert np.max(np.abs(xg - xo)) <= 4 * EPS
            ns = near_surface(D, po, xo)
            assert ns.sum() <= 2, "too many samples on a Fermi surface"
            ok = ~ns
            # exact zeros agree
            assert np.array_equal(wg[ok] == 0.0, wo[ok] == 0.0)
            tol = fp64_tol(D, po, xo, wo) + 1e-15 * np.mean(np.abs(wo))
            err = np.abs(wg - wo)
            bad = ok & (err > tol)
            assert not bad.any(), (D.diagram_id, np.max(err[ok] / np.maximum(np.abs(wo[ok]), 1e-300)))
            if O.is_anomalous(D):
                assert not wg.any()
            else:
                assert (wo != 0).sum() > 0
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_MIXED, M.MBPT_MIXED_MAP64])
@pytest.mark.parametrize("n,matter,mapk", [(3, "pnm", 0), (4, "snm", 0), (5, "pnm", 0), (4, "asym", 0),
                                           (3, "pnm", 1), (5, "pnm", 1)])
def test_mixed_precision_deviation(ctx, n, matter, mapk, prec):
    """Mixed modes (FP32 potentials and spin sum; FP32 or FP64 sampling map) on identical
    samples: aggregate deviation from the FP64 oracle below 1e-4 relative."""
    rng = np.random.default_rng(7 * n + mapk)
    po, pm = matter_pair(matter, map_kind=mapk)
    for D in _pick(n, 3, rng):
        if O.is_anomalous(D):
            continue
        cfg = M.vegas_cfg(samples=1 << 16, seed=99, stream_id=D.diagram_id, precision=prec)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
        try:
            grid = random_grid(po.dim(D), 50, rng, strength=0.5)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            xg, wg = M.mbpt_dump_samples(g, 0, 0, 2048, po.dim(D))
            xo, wo = oracle_dump(D, po, grid, 99, D.diagram_id, 0, 0, 2048)
            assert np.max(np.abs(xg - xo)) <= (4 * EPS if prec == M.MBPT_MIXED_MAP64 else 2e-7)
            ok = ~near_surface(D, po, xo, rel=1e-5 if prec == M.MBPT_MIXED else 1e-9)
            l1 = np.sum(np.abs(wg[ok] - wo[ok])) / max(np.sum(np.abs(wo[ok])), 1e-300)
            assert l1 < 1e-4, l1
            s_o = np.sum(wo[ok])
            assert abs(np.sum(wg[ok]) - s_o) <= 1e-4 * np.sum(np.abs(wo[ok]))
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("n,matter,mapk", [(3, "pnm", 0), (4, "snm", 1), (4, "asym", 0), (5, "pnm", 0)])
def test_mixed_map_near_fermi_surfaces_is_the_fp64_map(ctx, n, matter, mapk):
    """Mixed mode places a live sample with a line within ~1e-3 kF^2 of a Fermi surface with the FP64
    map (the oracle's point to rounding), and decides every Fermi step as the FP64 oracle does: zero
    patterns agree except for weights below the FP32 range of the potentials."""
    rng = np.random.default_rng(300 + 7 * n + mapk)
    po, pm = matter_pair(matter, map_kind=mapk)
    kf2 = [k * k for k in (po.kF_n, po.kF_p) if k > 0]
    for D in _pick(n, 2, rng):
        if O.is_anomalous(D):
            continue
        cfg = M.vegas_cfg(samples=1 << 16, seed=5, stream_id=D.diagram_id, precision=M.MBPT_MIXED)
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
        try:
            grid = random_grid(po.dim(D), 50, rng, strength=0.5)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            xg, wg = M.mbpt_dump_samples(g, 1, 0, 4096, po.dim(D))
            xo, wo = oracle_dump(D, po, grid, 5, D.diagram_id, 1, 0, 4096)
            dist = np.array([min(np.min(np.abs(O.line_ksq(D, po, x) - k2)) / k2 for k2 in kf2) for x in xo])
            band = (dist < 5e-4) & (wo != 0)
            assert band.sum() > 0
            assert np.max(np.abs(xg[band] - xo[band])) <= 4 * EPS
            ok = dist > 1e-9
            mism = ok & ((wg == 0) != (wo == 0))
            assert np.all(wg[mism] == 0) and np.all(np.abs(wo[mism]) < 1e-20 * np.max(np.abs(wo)))
        finally:
            M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("n,matter,mapk", [(2, "pnm", 0), (3, "snm", 1), (4, "pnm", 0), (5, "snm", 0)])
def test_hartree_fock_spectrum_per_sample(ctx, n, matter, mapk):
    """Hartree-Fock single-particle energies (Eq. (7)) in the energy denominators: FP64 per-sample
    parity with the oracle's own tabulation and spline (tolerance widened by the conditioning of
    each denominator, kinetic and self-energy parts counted separately), and the mixed modes within
    the aggregate 1e-4 bound."""
    rng = np.random.default_rng(900 + n + mapk)
    po, pm = matter_pair(matter, map_kind=mapk, spectrum=1)
    for D in _pick(n, 2, rng):
        if O.is_anomalous(D):
            continue
        grid = random_grid(po.dim(D), 50, rng, strength=0.5)
        xo, wo = oracle_dump(D, po, grid, 11, D.diagram_id, 2, 333, 1536)
        ns = near_surface(D, po, xo)
        for prec in (M.MBPT_FP64, M.MBPT_MIXED, M.MBPT_MIXED_MAP64):
            cfg = M.vegas_cfg(samples=1 << 16, seed=11, stream_id=D.diagram_id, precision=prec)
            g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
            try:
                M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
                xg, wg = M.mbpt_dump_samples(g, 2, 333, 1536, po.dim(D))
                if prec == M.MBPT_FP64:
                    ok = ~ns
                    assert np.array_equal(wg[ok] == 0.0, wo[ok] == 0.0)
                    tol = fp64_tol(D, po, xo, wo) + 1e-15 * np.mean(np.abs(wo))
                    assert np.all(np.abs(wg - wo)[ok] <= tol[ok])
                    assert (wo != 0).sum() > 0
                else:
                    ok = ~near_surface(D, po, xo, rel=1e-5)
                    l1 = np.sum(np.abs(wg[ok] - wo[ok])) / max(np.sum(np.abs(wo[ok])), 1e-300)
                    assert l1 < 1e-4, l1
            finally:
                M.mbpt_destroy_diagram(g)


def test_hartree_fock_spectrum_changes_the_integrand_and_rejects_asymmetric_matter(ctx):
    po0, pm0 = matter_pair("pnm")
    po1, pm1 = matter_pair("pnm", spectrum=1)
    D = O.enumerate_diagrams(3)[1]
    cfg = M.vegas_cfg(samples=1 << 14, seed=3)
    g0 = M.mbpt_create_diagram(ctx, make_desc(D), pm0, cfg)
    g1 = M.mbpt_create_diagram(ctx, make_desc(D), pm1, cfg)
    try:
        _, w0 = M.mbpt_dump_samples(g0, 0, 0, 512, D.d, with_x=False)
        _, w1 = M.mbpt_dump_samples(g1, 0, 0, 512, D.d, with_x=False)
        assert np.array_equal(w0 == 0, w1 == 0) and np.any(w0 != w1)
    finally:
        M.mbpt_destroy_diagram(g0)
        M.mbpt_destroy_diagram(g1)
    _, pa = matter_pair("asym", spectrum=1)
    with pytest.raises(M.MbptError):
        M.mbpt_create_diagram(ctx, make_desc(D), pa, cfg)


@pytest.mark.parametrize("prec", [M.MBPT_FP64, M.MBPT_MIXED, M.MBPT_MIXED_MAP64])
def test_one_iteration_sums_histogram_and_refinement(ctx, prec):
    """One batched iteration on a ragged sample count: sum w, sum w^2 against the
    oracle on the same grid; the histogram (FP32 accumulation) to 1e-5; the refined
    grid against the oracle's refinement of the GPU histogram to 1e-12."""
    rng = np.random.default_rng(5)
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(3)[1]
    M_s = 40000 + 123
    cfg = M.vegas_cfg(samples=M_s, seed=3, stream_id=11, precision=prec)
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
    try:
        grid = random_grid(D.d, 50, rng, strength=0.5)
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = M.mbpt_estimate(g)
        img = M.mbpt_get_state(g)
        ref = O.vegas_iteration(D, po, grid, 3, 11, 0, M_s)
        rel = 1e-11 if prec == M.MBPT_FP64 else 1e-4
        assert r.n_iter == 1 and r.n_evals == M_s
        assert r.last_mean == pytest.approx(ref.mean, rel=rel)
        assert r.last_sigma == pytest.approx(np.sqrt(ref.var_of_mean), rel=10 * rel)
        h = M.state_last_hist(img, D.d, 50)
        hn, rn = h / h.sum(axis=1, keepdims=True), ref.hist / ref.hist.sum(axis=1, keepdims=True)
        assert np.max(np.abs(hn - rn)) < (1e-5 if prec == M.MBPT_FP64 else 1e-3)
        new_grid = M.state_grid(img, D.d, 50)
        assert np.max(np.abs(new_grid - O.refine(grid, h))) < 1e-12
    finally:
        M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("n,matter", [(2, "pnm"), (3, "snm"), (4, "pnm"), (5, "pnm"), (5, "snm"), (6, "pnm")])
def test_spin_sum_fold_equals_table(ctx, n, matter):
    """The vertex-by-vertex fold of the Goldstone table (MBPT_SPIN_FOLD) evaluates the polynomial that the
    product table does: one mixed-precision iteration on a ragged sample count, same grid and counters,
    gives a sum of weights within FP32 rounding of the spin sum (1e-5 of sum |w|) of the table's, and
    both are within the mixed tolerance (1e-4 of sum |w|) of the FP64 oracle's sum over the same samples."""
    rng = np.random.default_rng(60 + n)
    po, pm = matter_pair(matter)
    M_s = (2048 if n == 6 else 8192) + 77
    for D in _pick(n, 2, rng):
        if O.is_anomalous(D):
            continue
        d = po.dim(D)
        grid = random_grid(d, 50, rng, strength=0.4)
        _, _, _, wo = O.vegas_samples(0, D, po.array(), d, grid, 8, 31, 0, 0, M_s, dump=True)
        s_o, l1_o = float(np.sum(wo)), float(np.sum(np.abs(wo)))
        sums = {}
        for strat in (M.MBPT_SPIN_TABLE, M.MBPT_SPIN_FOLD):
            M.mbpt_ctx_set_spin_sum(ctx, strat)
            assert M.mbpt_ctx_get_spin_sum(ctx) == strat
            g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=M_s, seed=8, stream_id=31,
                                                                          precision=M.MBPT_MIXED))
            try:
                M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
                M.mbpt_vegas_iterate(ctx, [g], 1)
                sums[strat] = M.mbpt_estimate(g).last_mean * M_s
            finally:
                M.mbpt_destroy_diagram(g)
                M.mbpt_ctx_set_spin_sum(ctx, M.MBPT_SPIN_TABLE)
        assert l1_o > 0.0
        assert abs(sums[M.MBPT_SPIN_FOLD] - sums[M.MBPT_SPIN_TABLE]) <= 1e-5 * l1_o, (D.diagram_id, sums, l1_o)
        for strat, v in sums.items():
            assert abs(v - s_o) <= 1e-4 * l1_o, (D.diagram_id, strat, v, s_o, l1_o)


@pytest.mark.parametrize("mapk", [0, 1])
def test_second_order_estimate_config1(ctx, mapk):
    """Config 1: one second-order diagram, neutron matter kF = 1, 10 x 2^18 samples,
    FP64: the GPU estimate agrees with the oracle's own VEGAS run and with the
    deterministic quadrature of Eq. (2) within 3 combined standard errors."""
    import quad_pins as Q
    po, pm = matter_pair("pnm", map_kind=mapk)
    pm.K_max = 7.0
    po.K_max = 7.0
    (D,) = O.enumerate_diagrams(2)
    cfg = M.vegas_cfg(samples=1 << 18, seed=1, stream_id=0, precision=M.MBPT_FP64)
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)
    try:
        M.mbpt_vegas_iterate(ctx, [g], 10)
        r = M.mbpt_estimate(g)
    finally:
        M.mbpt_destroy_diagram(g)
    mo, so, chi, _ = O.vegas(D, po, 10, 1 << 18, seed=1, sid=0)
    quad = Q.second_order(1.0, 2, 41.47, -50.0, -200.0, 0.7, 2.0, n_rad=10, n_ang=10)
    assert r.n_iter == 10 and r.n_evals == 10 * (1 << 18)
    assert abs(r.mean - mo) <= 3 * np.hypot(r.sigma, so)
    assert abs(r.mean - quad) <= 3 * r.sigma
    assert r.sigma < 3e-3 * abs(quad)


def _run(ctx, specs, iters):
    gs = [M.mbpt_create_diagram(ctx, d, p, c) for d, p, c in specs]
    try:
        M.mbpt_vegas_iterate(ctx, gs, iters)
        return [M.mbpt_estimate(g).as_dict() for g in gs], [M.mbpt_get_state(g) for g in gs]
    finally:
        for g in gs:
            M.mbpt_destroy_diagram(g)


def _specs():
    po, pm = matter_pair("pnm")
    ps, pms = matter_pair("snm")
    out = []
    for n, k in ((2, 1), (3, 3), (4, 2)):
        for D in O.enumerate_diagrams(n)[:k]:
            out.append((make_desc(D), pm, M.vegas_cfg(samples=50000 + 17 * D.diagram_id, seed=5,
                                                       stream_id=100 * n + D.diagram_id, precision=M.MBPT_MIXED)))
    D = O.enumerate_diagrams(3)[2]
    out.append((make_desc(D), pms, M.vegas_cfg(samples=30001, seed=5, stream_id=999, precision=M.MBPT_FP64)))
    return out


def test_deterministic_and_alone_equals_mix(ctx):
    specs = _specs()
    a, sa = _run(ctx, specs, 3)
    b, sb = _run(ctx, specs, 3)
    assert a == b and sa == sb          # run to run: bit for bit
    for i in (0, 3, len(specs) - 1):
        alone, salone = _run(ctx, [specs[i]], 3)
        assert alone[0] == a[i] and salone[0] == sa[i]


def test_batched_estimate_equals_single_estimates(ctx):
    """mbpt_estimate_batch (the states' heads gathered on the device and read back in one copy) returns
    exactly what mbpt_estimate returns integral by integral: for a batch, for a larger batch that grows
    the gather buffers, and for a subset in reverse order."""
    descs = M.mbpt_generate(3)
    gs = []
    for i in range(120):
        kf = 0.8 + 0.01 * i
        cfg = M.vegas_cfg(samples=1 << 14, seed=3, stream_id=i, precision=M.MBPT_MIXED)
        gs.append(M.mbpt_create_diagram(ctx, descs[i % 3], M.physics(kF_n=kf, K_max=kf + 6.0), cfg))
    try:
        M.mbpt_vegas_iterate(ctx, gs, 2)
        for batch in (gs[:37], gs, gs[::-3]):
            got = [r.as_dict() for r in M.mbpt_estimate_batch(batch)]
            want = [M.mbpt_estimate(g).as_dict() for g in batch]
            assert len(got) == len(want)
            for a, b in zip(got, want):
                assert all(a[k] == b[k] or (a[k] != a[k] and b[k] != b[k]) for k in a), (a, b)
            assert all(r["n_iter"] == 2 and r["n_evals"] == 2 << 14 for r in got)
    finally:
        for g in gs:
            M.mbpt_destroy_diagram(g)


def test_checkpoint_restore_continues_bitwise(ctx):
    d, p, c = _specs()[2]
    g = M.mbpt_create_diagram(ctx, d, p, c)
    M.mbpt_vegas_iterate(ctx, [g], 2)
    ck = M.mbpt_get_state(g)
    M.mbpt_vegas_iterate(ctx, [g], 2)
    ra = M.mbpt_estimate(g).as_dict()
    M.mbpt_destroy_diagram(g)
    h = M.mbpt_create_diagram(ctx, d, p, c)
    M.mbpt_set_state(h, ck)
    M.mbpt_vegas_iterate(ctx, [h], 2)
    rb = M.mbpt_estimate(h).as_dict()
    M.mbpt_destroy_diagram(h)
    assert ra == rb and ra["n_iter"] == 4


def test_anomalous_integral_is_exactly_zero(ctx):
    po, pm = matter_pair("pnm")
    D = next(D for D in O.enumerate_diagrams(4) if O.is_anomalous(D))
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=20000, target_rel=1e-3))
    try:
        M.mbpt_vegas_iterate(ctx, [g], 5)
        r = M.mbpt_estimate(g)
        # every sample is exactly zero; with a target the integral converges after two iterations
        assert r.mean == 0.0 and r.sigma == 0.0 and r.n_iter == 2 and r.converged == 1
    finally:
        M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("mapk", [0, 1])
def test_anomalous_diagrams_in_asymmetric_matter_are_zero(ctx, mapk):
    """A hole and a particle forced to equal momentum can pass their steps for different species
    in asymmetric matter; the spin sum is then exactly zero and so is the weight (no 0/0)."""
    po, pm = matter_pair("asym", map_kind=mapk)
    rng = np.random.default_rng(33)
    for D in [D for D in O.enumerate_diagrams(4) if O.is_anomalous(D)] + \
             [D for D in O.enumerate_diagrams(5) if O.is_anomalous(D)][:20]:
        g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=4096, precision=M.MBPT_MIXED))
        try:
            grid = random_grid(po.dim(D), 50, rng)
            M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
            _, w = M.mbpt_dump_samples(g, 0, 0, 4096, po.dim(D), with_x=False)
            assert np.all(w == 0.0)
            M.mbpt_vegas_iterate(ctx, [g], 2)
            r = M.mbpt_estimate(g)
            assert r.mean == 0.0 and r.sigma == 0.0 and r.status == 0
        finally:
            M.mbpt_destroy_diagram(g)


def test_targets_stop_iterating(ctx):
    po, pm = matter_pair("pnm")
    (D,) = O.enumerate_diagrams(2)
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=1 << 16, target_rel=0.05))
    try:
        M.mbpt_vegas_iterate(ctx, [g], 20)
        r = M.mbpt_estimate(g)
        assert r.converged == 1 and r.n_iter < 20 and r.sigma <= 0.05 * abs(r.mean)
    finally:
        M.mbpt_destroy_diagram(g)


def test_training_iterations_are_not_combined(ctx):
    """With train_iters = 2 the first two iterations refine the grid but do not enter the
    combined estimate (oracle combination with skip = 2 on the recorded history)."""
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(3)[2]
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=1 << 15, train_iters=2))
    try:
        M.mbpt_vegas_iterate(ctx, [g], 1)
        assert np.isinf(M.mbpt_estimate(g).sigma)
        M.mbpt_vegas_iterate(ctx, [g], 4)
        r = M.mbpt_estimate(g)
        img = M.mbpt_get_state(g)
        hm = np.frombuffer(img, dtype=np.float64, count=5, offset=M.STATE_HEADER_BYTES + 7 * 8 + 8 + 16)
        hv = np.frombuffer(img, dtype=np.float64, count=5,
                           offset=M.STATE_HEADER_BYTES + 7 * 8 + 8 + 16 + 8 * M.MAX_ITERS)
        m, s, chi = O.combine(hm, hv, skip=2)
        assert r.n_iter == 5 and r.mean == pytest.approx(m, rel=1e-12) and r.sigma == pytest.approx(s, rel=1e-12)
    finally:
        M.mbpt_destroy_diagram(g)


@pytest.mark.parametrize("prec", [M.MBPT_FP64, M.MBPT_MIXED])
def test_denominator_regulator_components(ctx, prec):
    """Regulator of Sec. III.A: each sample also evaluates the integrand with every energy
    denominator D_m replaced by D_m - s_k; after one iteration each component's mean and error
    match the oracle's iteration with that shift (same grid, same counters), the fourth component
    is the quadratic extrapolation sum_k L_k I_k to s = 0, and the main estimate is unchanged."""
    import dataclasses
    rng = np.random.default_rng(12)
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(4)[7]
    shifts = (3.0, 6.0, 9.0)
    M_s = 30000 + 77
    grid = random_grid(D.d, 50, rng, strength=0.4)
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=M_s, seed=4, stream_id=21, precision=prec,
                                                                 shifts=shifts))
    g0 = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=M_s, seed=4, stream_id=21, precision=prec))
    try:
        for h in (g, g0):
            M.mbpt_set_state(h, M.state_with_grid(M.mbpt_get_state(h), grid))
        M.mbpt_vegas_iterate(ctx, [g, g0], 1)
        r, r0 = M.mbpt_estimate(g), M.mbpt_estimate(g0)
        assert r.last_mean == r0.last_mean and r.last_sigma == r0.last_sigma
        mean, sigma = M.mbpt_estimate_shifts(g)
        rel = 1e-11 if prec == M.MBPT_FP64 else 1e-4
        refs = [O.vegas_iteration(D, dataclasses.replace(po, shift=s), grid, 4, 21, 0, M_s) for s in shifts]
        for k in range(3):
            assert mean[k] == pytest.approx(refs[k].mean, rel=rel)
            assert sigma[k] == pytest.approx(np.sqrt(refs[k].var_of_mean), rel=10 * rel)
        lag = [np.prod([(0.0 - shifts[j]) / (shifts[k] - shifts[j]) for j in range(3) if j != k]) for k in range(3)]
        ext = sum(L * ref.mean for L, ref in zip(lag, refs))
        scale = sum(abs(L * ref.mean) for L, ref in zip(lag, refs))
        assert abs(mean[3] - ext) <= rel * scale
        # shifts move every denominator away from zero: each component smaller than the last
        assert abs(refs[2].mean) < abs(refs[1].mean) < abs(refs[0].mean)
        with pytest.raises(M.MbptError):
            M.mbpt_estimate_shifts(g0)
        M.mbpt_vegas_iterate(ctx, [g], 3)
        mean, sigma = M.mbpt_estimate_shifts(g)
        assert np.all(np.isfinite(mean)) and np.all(sigma > 0) and np.all(np.isfinite(sigma))
    finally:
        M.mbpt_destroy_diagram(g)
        M.mbpt_destroy_diagram(g0)


def test_denominator_regulator_rejects_bad_shifts(ctx):
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(3)[0]
    for sh in ((0.0, 1.0, 2.0), (1.0, 1.0, 2.0), (-1.0, 1.0, 2.0)):
        with pytest.raises(M.MbptError):
            M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=1000, shifts=sh))
    cfg = M.vegas_cfg(samples=1000, shifts=(1.0, 2.0, 3.0))
    cfg.n_shifts = 2
    with pytest.raises(M.MbptError):
        M.mbpt_create_diagram(ctx, make_desc(D), pm, cfg)


def test_freeze_keeps_grid(ctx):
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(3)[0]
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=20000, freeze_after=2))
    try:
        M.mbpt_vegas_iterate(ctx, [g], 2)
        g2 = M.state_grid(M.mbpt_get_state(g), D.d, 50)
        M.mbpt_vegas_iterate(ctx, [g], 2)
        g4 = M.state_grid(M.mbpt_get_state(g), D.d, 50)
        assert np.array_equal(g2, g4)
    finally:
        M.mbpt_destroy_diagram(g)


def test_edge_cases_and_errors(ctx):
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(3)[1]
    good = make_desc(D)
    M.mbpt_vegas_iterate(ctx, [], 3)                       # empty batch is a no-op
    # smallest sample count
    g = M.mbpt_create_diagram(ctx, good, pm, M.vegas_cfg(samples=2))
    M.mbpt_vegas_iterate(ctx, [g], 1)
    assert M.mbpt_estimate(g).n_evals == 2
    with pytest.raises(M.MbptError):
        M.mbpt_vegas_iterate(ctx, [g, g], 1)               # same integral twice
    with pytest.raises(M.MbptError):
        M.mbpt_set_state(g, b"\0" * 16)
    M.mbpt_destroy_diagram(g)
    bad = make_desc(D)
    bad.line_coef[D.n + 1][0] = 1 - bad.line_coef[D.n + 1][0]   # break momentum conservation
    bad2 = make_desc(D)
    bad2.vtx_out[0][0] = bad2.vtx_in[0][0]
    bad3 = make_desc(D)
    bad3.order = 6
    for d in (bad, bad2, bad3):
        with pytest.raises(M.MbptError) as e:
            M.mbpt_create_diagram(ctx, d, pm, M.vegas_cfg())
        assert e.value.status == M.MBPT_EINVAL
    for kw in (dict(kF_n=0.0, kF_p=0.0), dict(reg_power=3), dict(K_max=0.5)):
        p = M.physics(**kw)
        with pytest.raises(M.MbptError) as e:
            M.mbpt_create_diagram(ctx, good, p, M.vegas_cfg())
        assert e.value.status == M.MBPT_EINVAL
    with pytest.raises(M.MbptError) as e:
        M.mbpt_create_diagram(ctx, good, pm, M.vegas_cfg(samples=1))
    assert e.value.status == M.MBPT_EINVAL


def test_arena_exhaustion_is_enomem():
    small = M.mbpt_ctx_create(0, 1 << 20)
    try:
        po, pm = matter_pair("pnm")
        D = O.enumerate_diagrams(5)[10]
        made = []
        with pytest.raises(M.MbptError) as e:
            for _ in range(1000):
                made.append(M.mbpt_create_diagram(small, make_desc(D), pm, M.vegas_cfg()))
        assert e.value.status == M.MBPT_ENOMEM and len(made) > 10
        for g in made:
            M.mbpt_destroy_diagram(g)
        used, free = M.mbpt_ctx_mem(small)
        assert used == 0
    finally:
        M.mbpt_ctx_destroy(small)


def test_more_iterations_than_the_history_holds(ctx):
    """The per-iteration history keeps 512 entries; an integral that runs longer keeps combining and
    reports a finite estimate with every evaluation counted.  In the pooled evaluation phase the 526
    small iterations on the frozen grid (2^13 samples each) are one long run: the estimate agrees with the
    oracle's own pooled estimate within 3 sigma (inverse-variance weights of so many small iterations
    are biased towards the iterations that missed the tail of the weights)."""
    po, pm = matter_pair("pnm")
    D = O.enumerate_diagrams(2)[0]
    g = M.mbpt_create_diagram(ctx, make_desc(D), pm, M.vegas_cfg(samples=8192, seed=9, train_iters=4,
                                                                  combine=M.MBPT_COMBINE_POOLED))
    try:
        M.mbpt_vegas_iterate(ctx, [g], 100)
        r100 = M.mbpt_estimate(g)
        M.mbpt_vegas_iterate(ctx, [g], 430)
        r = M.mbpt_estimate(g)
        assert r.n_iter == 530 and r.n_evals == 530 * 8192
        assert np.isfinite(r.mean) and np.isfinite(r.sigma) and 0 < r.sigma < r100.sigma and r.status == 0
        q = O.vegas(D, po, 8, 1 << 15, seed=1, train_iters=4, pooled=True)
        assert abs(r.mean - q[0]) <= 3.0 * np.hypot(r.sigma, q[1]), (r.mean, r.sigma, q[0], q[1])
    finally:
        M.mbpt_destroy_diagram(g)
