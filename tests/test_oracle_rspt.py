"""Pin of the diagram rules at orders 2-6: in a finite single-particle space the
sum over all generated diagrams, evaluated with unrestricted discrete label
sums and the oracle's sign, weight and cut rules, equals the exact
Rayleigh-Schroedinger coefficient of H0 + lambda W_N (linked-diagram theorem;
textbook references of Sec. II)."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("seed,nh,np_", [(11, 3, 3), (5, 2, 4)])
def test_diagram_sum_equals_rspt(seed, nh, np_):
    rng = np.random.default_rng(seed)
    N = nh + np_
    w = O.random_antisymmetric_w(N, rng, 0.3)
    eps = np.concatenate([rng.uniform(-3.0, -1.0, nh), rng.uniform(1.0, 3.0, np_)])
    E, WN, ref = O.rspt_coefficients(w, eps, nh, 5)
    assert abs(E[0]) < 1e-14                      # W_N has no reference expectation value
    for n in (2, 3, 4, 5):
        s = sum(O.discrete_diagram(D, nh, np_, w, eps) for D in O.enumerate_diagrams(n))
        assert s == pytest.approx(E[n - 1], rel=1e-10, abs=1e-14), n


@pytest.mark.parametrize("seed", [11, 4])
def test_sixth_order_diagram_sum_equals_rspt(seed):
    """The same sum rule over all 27300 sixth-order diagrams (two holes, two particles)."""
    rng = np.random.default_rng(seed)
    nh, np_ = 2, 2
    w = O.random_antisymmetric_w(nh + np_, rng, 0.3)
    eps = np.concatenate([rng.uniform(-3.0, -1.0, nh), rng.uniform(1.0, 3.0, np_)])
    E, _, _ = O.rspt_coefficients(w, eps, nh, 6)
    s = sum(O.discrete_diagram(D, nh, np_, w, eps) for D in O.enumerate_diagrams(6))
    assert abs(E[5]) > 1e-8
    assert s == pytest.approx(E[5], rel=1e-10, abs=1e-16)


def test_planted_sign_error_is_caught():
    """A plausible mistake (dropping the (-1)^l0 factor) breaks the sum rule."""
    rng = np.random.default_rng(3)
    nh, np_ = 3, 3
    w = O.random_antisymmetric_w(nh + np_, rng, 0.3)
    eps = np.concatenate([rng.uniform(-3.0, -1.0, nh), rng.uniform(1.0, 3.0, np_)])
    E, _, _ = O.rspt_coefficients(w, eps, nh, 4)
    wrong = 0.0
    for D in O.enumerate_diagrams(4):
        v = O.discrete_diagram(D, nh, np_, w, eps)
        wrong += v * (-1) ** D.l0
    assert abs(wrong - E[3]) > 1e-6 * abs(E[3])
