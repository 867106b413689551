"""Pins of the oracle's integrand and VEGAS against closed forms, independent
quadratures, exact symmetries and scaling laws (arXiv:2603.24532 Sec. II,
Eqs. (1)-(6); VEGAS per Lepage 1978)."""
import math

import numpy as np
import pytest

import oracle as O
import quad_pins as Q
from helpers import random_grid


def within(est, sig, ref, k=3.0):
    return abs(est - ref) <= k * sig


# --- first order (Eq. (1) potential term) -----------------------------------------------

@pytest.mark.parametrize("g,kfp", [(2, 0.0), (4, 1.0)])
def test_first_order_contact_closed_form(g, kfp):
    """Unregulated contact: E/N = C_S n (g - 1)/(2g) (= C_S n/4 for neutrons)."""
    ph = O.Physics(kF_n=1.0, kF_p=kfp, C_S=-50.0, C_Y=0.0, Lam=1e6)
    ref = Q.first_order_contact(1.0, g, -50.0)
    if g == 2:
        assert ref == pytest.approx(-0.42217, abs=1e-5)
    m, s, chi, _ = O.vegas(None, ph, 8, 1 << 15, seed=3, kind=1, d=6)
    assert within(m, s, ref)
    assert s < 2e-3 * abs(ref)


@pytest.mark.parametrize("g,kfp", [(2, 0.0), (4, 1.0)])
def test_first_order_full_potential_quadrature(g, kfp):
    ph = O.Physics(kF_n=1.0, kF_p=kfp)
    ref = Q.first_order_full_v(1.0, g, ph.C_S, ph.C_Y, ph.m_pi, ph.Lam)
    m, s, chi, _ = O.vegas(None, ph, 8, 1 << 15, seed=5, kind=1, d=6)
    assert within(m, s, ref)
    assert s < 2e-3 * abs(ref)


# --- second order (Eq. (2)) ---------------------------------------------------------------

_Q2 = {}


def q2(CY, g=2):
    if (CY, g) not in _Q2:
        _Q2[(CY, g)] = Q.second_order(1.0, g, 41.47, -50.0, CY, 0.7, 2.0, n_rad=10, n_ang=10)
    return _Q2[(CY, g)]


@pytest.mark.parametrize("CY", [0.0, -200.0])
def test_second_order_vs_gauss_legendre(CY):
    (D,) = O.enumerate_diagrams(2)
    ph = O.Physics(C_Y=CY)
    m, s, chi, _ = O.vegas(D, ph, 10, 1 << 16, seed=1)
    assert within(m, s, q2(CY))
    assert s < 5e-3 * abs(q2(CY))


def test_second_order_snm_vs_gauss_legendre():
    (D,) = O.enumerate_diagrams(2)
    ph = O.Physics(kF_n=1.0, kF_p=1.0)
    m, s, chi, _ = O.vegas(D, ph, 10, 1 << 15, seed=2)
    assert within(m, s, q2(-200.0, g=4))


def test_shifted_denominator_second_order_vs_quadrature():
    """Denominator regulator (Sec. III.A): with D -> D - s the oracle's second-order VEGAS estimate
    matches the relative-coordinate quadrature with the same shift; the shift only moves D away from
    its pole (|E(s)| < |E(0)|); and the quadratic through three shifts, evaluated at s = 0, lands much
    closer to the unshifted energy than the smallest shift does."""
    (D,) = O.enumerate_diagrams(2)
    shifts = (2.0, 4.0, 6.0)
    qs = [Q.second_order(1.0, 2, 41.47, -50.0, -200.0, 0.7, 2.0, n_rad=10, n_ang=10, shift=s) for s in shifts]
    q0 = q2(-200.0)
    assert abs(qs[0]) < abs(q0) and abs(qs[2]) < abs(qs[1]) < abs(qs[0])
    m, s, chi, _ = O.vegas(D, O.Physics(shift=shifts[1]), 10, 1 << 16, seed=1)
    assert within(m, s, qs[1])
    assert s < 5e-3 * abs(qs[1])
    lag = [np.prod([(0.0 - shifts[j]) / (shifts[k] - shifts[j]) for j in range(3) if j != k]) for k in range(3)]
    ext = float(np.dot(lag, qs))
    assert abs(ext - q0) < 0.2 * abs(qs[0] - q0)


def test_shifted_denominator_per_sample():
    """At every sample the shifted integrand is the unshifted one times D/(D - s) for the single
    second-order cut: same sign, smaller magnitude (D < 0 on the whole domain)."""
    (D,) = O.enumerate_diagrams(2)
    rng = np.random.default_rng(8)
    ph0, ph1 = O.Physics(), O.Physics(shift=5.0)
    nz = 0
    for _ in range(400):
        x = rng.random(D.d)
        f0, f1 = O.integrand(D, ph0, x), O.integrand(D, ph1, x)
        if f0 == 0.0:
            assert f1 == 0.0
            continue
        nz += 1
        assert np.sign(f1) == np.sign(f0) and abs(f1) < abs(f0)
    assert nz > 20


def test_group_iteration_is_the_sum_of_member_iterations():
    """A group's integrand is the sum of its members' integrands at the same point (Sec. III.A):
    on one grid and one set of counters its sum of weights is the scaled sum of the members' sums."""
    rng = np.random.default_rng(3)
    G = O.groups(4)[4]
    G = O.Group(G.members[:5], [1.0, 2.0, 0.5, 1.0, 3.0])
    ph = O.Physics(kF_n=1.2)
    grid = random_grid(G.d, 50, rng, strength=0.5)
    r = O.vegas_iteration(G, ph, grid, 7, 3, 2, 3000)
    parts = [O.vegas_iteration(D, ph, grid, 7, 3, 2, 3000).sum_w for D in G.members]
    ref = float(np.dot(G.scales, parts))
    assert r.sum_w == pytest.approx(ref, rel=1e-12, abs=1e-12 * float(np.sum(np.abs(parts))))
    x = rng.random(G.d)
    assert O.group_integrand(G, ph, x) == pytest.approx(
        sum(c * O.integrand(D, ph, x) for D, c in zip(G.members, G.scales)), rel=1e-15)


def test_third_order_group_estimate_matches_members():
    """The third-order group of diagrams with three hole loop momenta (hh and ph ladders/ring)
    integrated as one integrand agrees with the sum of the separately integrated members within the
    combined error."""
    G = O.groups(3)[3]
    assert len(G.members) == 2
    ph = O.Physics()
    mg, sg, _, _ = O.vegas(G, ph, 8, 1 << 15, seed=2, sid=5)
    ms = [O.vegas(D, ph, 8, 1 << 15, seed=2, sid=6 + i)[:2] for i, D in enumerate(G.members)]
    tot = sum(m for m, _ in ms)
    st = math.sqrt(sum(s * s for _, s in ms))
    assert within(mg, math.hypot(sg, st), tot)


# --- Hartree-Fock spectrum (Eq. (7)) ---------------------------------------------------------

def test_gauss_legendre_rule():
    x = np.zeros(12)
    w = np.zeros(12)
    O.lib().oracle_gauss_legendre(12, O._dp(x), O._dp(w))
    assert np.sum(w) == pytest.approx(2.0, rel=1e-14)
    for deg in (2, 10, 22):                       # exact to degree 2n - 1 = 23
        assert np.sum(w * x ** deg) == pytest.approx(2.0 / (deg + 1), rel=1e-13)


@pytest.mark.parametrize("kfp", [0.0, 1.0])
def test_hf_self_energy_contact_closed_form(kfp):
    """Unregulated contact: Sigma(k) = C_S n (g - 1)/g for every k (C_S n/2 in neutron matter)."""
    ph = O.Physics(kF_n=1.0, kF_p=kfp, C_Y=0.0, Lam=1e6)
    g = 4 if kfp else 2
    for k in (0.0, 0.4, 1.3, 3.0):
        assert O.hf_self_energy(ph, k) == pytest.approx(-50.0 * ph.density * (g - 1) / g, rel=1e-12)


@pytest.mark.parametrize("kfp", [0.0, 1.0])
def test_hf_self_energy_integrates_to_first_order(kfp):
    """(g/2n) sum over the Fermi sea of Sigma is the first-order energy per particle, pinned
    independently by the 1D reduction over the relative momentum."""
    ph = O.Physics(kF_n=1.0, kF_p=kfp, spectrum=1)
    g = 4 if kfp else 2
    ref = Q.first_order_full_v(1.0, g, ph.C_S, ph.C_Y, ph.m_pi, ph.Lam)
    direct = Q.first_order_from_sigma(1.0, g, np.vectorize(lambda k: O.hf_self_energy(ph, k)), n=48)
    spline = Q.first_order_from_sigma(1.0, g, np.vectorize(lambda k: O.sp_energy(ph, k) - 0.5 * 41.47 * k * k),
                                      n=48)
    assert direct == pytest.approx(ref, rel=1e-10)
    assert spline == pytest.approx(ref, rel=1e-7)


def test_hf_spline_between_knots():
    """The tabulated spectrum: between knots the spline is within 1e-7 MeV of the direct quadrature,
    and it is the cubic spline with zero slope at k = 0 and zero curvature at the end (an independent
    spline construction on the same knots agrees to rounding)."""
    from scipy.interpolate import CubicSpline
    ph = O.Physics(spectrum=1)
    y, m, h = O.hf_table(ph)
    ks = (np.arange(0, 400, 7) + 0.5) * h
    sp = np.array([O.sp_energy(ph, k) - 0.5 * ph.hbar2_over_m * k * k for k in ks])
    dq = np.array([O.hf_self_energy(ph, k) for k in ks])
    assert np.max(np.abs(sp - dq)) < 1e-7
    cs = CubicSpline(np.arange(len(y)) * h, y, bc_type=((1, 0.0), (2, 0.0)))
    assert np.max(np.abs(sp - cs(ks))) < 1e-12
    assert O.sp_energy(ph, 2.0 * ph.K_max + 0.1) == pytest.approx(0.5 * ph.hbar2_over_m * (2 * ph.K_max + 0.1) ** 2)


def test_hf_second_order_vs_quadrature():
    """Eq. (2) with Hartree-Fock single-particle energies in the denominator: the oracle's VEGAS
    estimate against the relative-coordinate quadrature with the same spectrum (an independent
    spline of the oracle's knot values), and clearly apart from the free-spectrum value."""
    from scipy.interpolate import CubicSpline
    (D,) = O.enumerate_diagrams(2)
    ph = O.Physics(spectrum=1)
    y, m, h = O.hf_table(ph)
    cs = CubicSpline(np.arange(len(y)) * h, y, bc_type=((1, 0.0), (2, 0.0)))
    kend = (len(y) - 1) * h
    sig = lambda k: np.where(k < kend, cs(np.minimum(k, kend)), 0.0)
    ref = Q.second_order(1.0, 2, 41.47, -50.0, -200.0, 0.7, 2.0, n_rad=10, n_ang=10, sigma=sig)
    mm, ss, _, _ = O.vegas(D, ph, 10, 1 << 16, seed=1)
    assert within(mm, ss, ref)
    assert ss < 5e-3 * abs(ref)
    assert abs(ref - q2(-200.0)) > 5 * ss


def test_rotational_reduction_second_order_vs_quadrature():
    """Chord map 1 (chord 0 along z, chord 1 in the xz plane, 4 pi x 2 pi integrated out; Sec. III.C)
    integrates the same Eq. (2) in 6 instead of 9 dimensions."""
    (D,) = O.enumerate_diagrams(2)
    ph = O.Physics(map_kind=1)
    assert ph.dim(D) == 6
    m, s, chi, _ = O.vegas(D, ph, 10, 1 << 16, seed=1)
    assert within(m, s, q2(-200.0))
    assert s < 3e-3 * abs(q2(-200.0))


@pytest.mark.parametrize("i", [0, 2])
def test_rotational_reduction_third_order_matches_full_map(i):
    D = O.enumerate_diagrams(3)[i]
    m0, s0, _, _ = O.vegas(D, O.Physics(map_kind=0), 12, 1 << 16, seed=11)
    m1, s1, _, _ = O.vegas(D, O.Physics(map_kind=1), 12, 1 << 16, seed=12)
    assert abs(m0 - m1) <= 3.0 * math.hypot(s0, s1)


def test_planted_spin_sum_error_is_caught():
    """Dropping the direct-exchange cross term of the spin sum (a plausible
    mistake) moves the reference far outside the oracle's error bar."""
    (D,) = O.enumerate_diagrams(2)
    m, s, chi, _ = O.vegas(D, O.Physics(), 10, 1 << 16, seed=1)
    wrong = Q.second_order(1.0, 2, 41.47, -50.0, -200.0, 0.7, 2.0, n_rad=8, n_ang=8, cross=False)
    assert not within(m, s, wrong, k=10)


# --- exact symmetries and scaling laws (per sample) -----------------------------------

def _valid_point(D, ph, rng, tries=2000):
    for _ in range(tries):
        x = rng.random(D.d)
        f = O.integrand(D, ph, x)
        if f != 0.0:
            return x, f
    raise RuntimeError("no non-zero sample")


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_coupling_and_mass_scaling(n):
    """E_G(lambda C_S, lambda C_Y) = lambda^n E_G; E_G(s hbar^2/m) = s^-(n-1) E_G."""
    rng = np.random.default_rng(100 + n)
    ph = O.Physics()
    for D in O.enumerate_diagrams(n)[:: max(1, len(O.enumerate_diagrams(n)) // 6)]:
        if O.is_anomalous(D):
            continue
        x, f = _valid_point(D, ph, rng)
        lam, s = 1.7, 0.6
        f1 = O.integrand(D, O.Physics(C_S=lam * ph.C_S, C_Y=lam * ph.C_Y), x)
        f2 = O.integrand(D, O.Physics(hbar2_over_m=s * ph.hbar2_over_m), x)
        assert f1 == pytest.approx(lam ** n * f, rel=1e-12)
        assert f2 == pytest.approx(s ** (-(n - 1)) * f, rel=1e-12)


@pytest.mark.parametrize("n", [4, 5])
def test_anomalous_diagrams_vanish(n):
    rng = np.random.default_rng(n)
    ph = O.Physics()
    for D in O.enumerate_diagrams(n):
        if not O.is_anomalous(D):
            continue
        for _ in range(20):
            assert O.integrand(D, ph, rng.random(D.d)) == 0.0


def _valid_chords(D, ph, rng, tries=20000):
    """Random chord momenta (hole chords in the Fermi ball, particle chords in a
    shell) at which the integrand is non-zero."""
    kfs = [k for k in (ph.kF_n, ph.kF_p) if k > 0]
    for _ in range(tries):
        ck = np.zeros((D.n + 1, 3))
        for c, l in enumerate(D.chords):
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            r = rng.uniform(0.0, max(kfs)) if D.hole(l) else rng.uniform(min(kfs), 3.0)
            ck[c] = r * v
        f = O.integrand_momenta(D, ph, ck)
        if f != 0.0:
            return ck, f
    raise RuntimeError("no non-zero configuration")


@pytest.mark.parametrize("n,matter", [(3, "pnm"), (4, "pnm"), (4, "snm"), (5, "pnm"), (4, "asym")])
def test_mirror_pairs_equal_per_sample(n, matter):
    """Time reversal + arrow reversal maps a diagram to its complex-conjugate
    partner; with a real symmetric V the two integrands agree when every line
    carries the same momentum."""
    rng = np.random.default_rng(7 * n)
    ph = {"pnm": O.Physics(), "snm": O.Physics(kF_n=1.0, kF_p=1.0), "asym": O.Physics(kF_n=1.2, kF_p=0.9)}[matter]
    Ds = O.enumerate_diagrams(n)
    idx = {D.A: k for k, D in enumerate(Ds)}
    checked = 0
    for D in Ds[:: max(1, len(Ds) // 25)]:
        if O.is_anomalous(D):
            continue
        M = Ds[idx[O.mirror_matrix(D.A)]]
        # mirror line of (u -> v) is (n-1-v -> n-1-u); equivalent lines are interchangeable
        img, used = {}, set()
        for l, (u, v) in enumerate(D.lines):
            for lm, st in enumerate(M.lines):
                if st == (n - 1 - v, n - 1 - u) and lm not in used:
                    used.add(lm)
                    img[lm] = l
                    break
        for _ in range(3):
            ck, f = _valid_chords(D, ph, rng)
            kl = O.line_momenta(D, ck)
            mk = np.array([kl[img[lm]] for lm in M.chords])
            fm = O.integrand_momenta(M, ph, mk)
            assert fm == pytest.approx(f, rel=1e-12, abs=0.0)
            checked += 1
    assert checked > 0


# --- VEGAS on test integrands (Lepage 1978) -----------------------------------------------

def test_vegas_separable_gaussian():
    d = 4
    ref = math.erf(0.5 / (0.1 * math.sqrt(2))) ** d
    m, s, chi, grid = O.vegas(None, np.array([0.5, 0.1]), 10, 1 << 14, seed=9, kind=2, d=d)
    assert within(m, s, ref)
    assert s < 3e-3
    # the adapted grid concentrates its bins around the peak
    w = np.diff(grid[0])
    assert w[24] < 0.5 / 50 and w[0] > 2.0 / 50


def test_vegas_product_of_sines():
    m, s, chi, grid = O.vegas(None, np.array([0.0, 0.0]), 10, 1 << 14, seed=4, kind=3, d=9)
    assert within(m, s, 1.0)


def test_refine_keeps_uniform_grid_and_endpoints():
    g = O.uniform_grid(3, 50)
    h = np.ones((3, 50))
    g2 = O.refine(g, h)
    assert np.allclose(g2, g, atol=1e-14)
    rng = np.random.default_rng(0)
    h = rng.random((3, 50)) ** 4
    g3 = O.refine(g, h)
    assert np.all(np.diff(g3, axis=1) > 0)
    assert np.all(g3[:, 0] == 0.0) and np.all(g3[:, -1] == 1.0)
    # all-zero histogram keeps the grid
    assert np.array_equal(O.refine(g3, np.zeros((3, 50))), g3)


def test_combination_weighted_mean():
    m, s, chi = O.combine([1.0, 3.0], [1.0, 1.0])
    assert m == 2.0 and s == pytest.approx(1 / math.sqrt(2)) and chi == pytest.approx(2.0)


# --- evaluation phase of PVegas (Sec. III.C): pooled combination on a frozen grid ---------------------

def test_pooled_combination_is_one_long_run():
    """combine_pooled of per-iteration sums equals the plain Monte Carlo mean and standard error of all
    the iterations' samples taken together (numpy on the dumped weights), for iterations of unequal
    size; the inverse-variance mean of the same iterations differs from it."""
    rng = np.random.default_rng(11)
    grid = random_grid(4, 50, rng, strength=0.6)
    ws, s1, s2, cnt, means, vars_ = [], [], [], [], [], []
    for t, m in ((0, 3000), (1, 2000), (2, 4096)):
        sums, _, _, w = O.vegas_samples(2, None, np.array([0.5, 0.1]), 4, grid, 9, 0, t, 0, m, dump=True)
        ws.append(w)
        s1.append(sums[0])
        s2.append(sums[1])
        cnt.append(m)
        means.append(sums[0] / m)
        vars_.append((sums[1] / m - (sums[0] / m) ** 2) / (m - 1))
    allw = np.concatenate(ws)
    mean, sigma, chi2 = O.combine_pooled(s1, s2, cnt)
    assert mean == pytest.approx(float(np.mean(allw)), rel=1e-12)
    assert sigma == pytest.approx(float(np.std(allw, ddof=1)) / math.sqrt(len(allw)), rel=1e-9)
    ref_chi2 = sum((mi - mean) ** 2 / vi for mi, vi in zip(means, vars_)) / 2
    assert chi2 == pytest.approx(ref_chi2, rel=1e-9)
    assert O.combine(means, vars_)[0] != pytest.approx(mean, rel=1e-12)


def test_pooled_vegas_freezes_grid_after_training():
    """With the pooled combination the grid is refined after the training iterations only (the final grid
    is the one three refinements give) and the estimate of a known integral lies within 3 sigma."""
    d = 4
    ref = math.erf(0.5 / (0.1 * math.sqrt(2))) ** d
    par = np.array([0.5, 0.1])
    m, s, chi, grid = O.vegas(None, par, 8, 1 << 14, seed=9, kind=2, d=d, train_iters=3, pooled=True)
    _, _, _, g3 = O.vegas(None, par, 3, 1 << 14, seed=9, kind=2, d=d)
    assert np.array_equal(grid, g3)
    assert within(m, s, ref) and s < 3e-3


def test_generator_lists_hole_chords_first():
    """The canonical chord order (hole chords first, each kind in line order): at orders 2..5 every
    diagram's chord list starts with its hole chords, and diagrams with equal numbers of hole chords
    therefore share the radial ranges of the loop-momentum map."""
    for n in (2, 3, 4, 5):
        for D in O.enumerate_diagrams(n):
            holes = [D.hole(l) for l in D.chords]
            k = O.hole_chords(D)
            assert holes == [True] * k + [False] * (len(holes) - k)
            assert D.chords[:k] == sorted(D.chords[:k]) and D.chords[k:] == sorted(D.chords[k:])
