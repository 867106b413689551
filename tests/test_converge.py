"""Adaptive evaluation phase (run_fifth_order.converge) on a fake library: host logic only, no GPU."""
import math

from paper_2603_24532_b300 import run_fifth_order as RF


class _Res:
    def __init__(self, mean, sigma, n_evals, converged):
        self.mean, self.sigma, self.n_evals, self.converged = mean, sigma, n_evals, converged


class FakeLib:
    """Integral i has mean m_i and per-sample standard deviation s_i; after n evaluation samples its error
    is s_i / sqrt(n); it is converged once that error is at most its goal.  `train` training samples
    count in n_evals but not in the error, as in the library's pooled evaluation phase."""

    def __init__(self, means, sds, goals, train):
        self.means, self.sds, self.goals, self.train = means, sds, goals, train
        self.n = [0] * len(means)
        self.samples = [None] * len(means)
        self.calls = []

    def mbpt_estimate_batch(self, gs):
        out = []
        for i in gs:
            n = self.n[i]
            sig = self.sds[i] / math.sqrt(n) if n > 0 else math.inf
            out.append(_Res(self.means[i], sig, self.train + n, sig <= self.goals[i]))
        return out

    def mbpt_set_config(self, g, cfg):
        self.samples[g] = cfg

    def mbpt_vegas_iterate(self, ctx, gs, k):
        assert k == 1
        self.calls.append(list(gs))
        for g in gs:
            self.n[g] += self.samples[g]


def run(lib, gs, **kw):
    return RF.converge(lib, None, gs, lambda r, i: lib.goals[i], lambda i, n: n,
                       lambda r: r.n_evals - lib.train, **kw)


def test_every_integral_reaches_its_goal_and_the_loop_stops():
    # needs (s/goal)^2: 1e4, 1e6, 4e6, 1.6e7 samples
    sds, goals = [1.0, 10.0, 20.0, 40.0], [0.01] * 4
    lib = FakeLib([1.0] * 4, sds, goals, train=0)
    lib.samples = [1 << 16] * 4
    iters, evals, _ = run(lib, list(range(4)), base_samples=1 << 16, min_samples=1 << 10, cap=1 << 22,
                          max_iters=200)
    res = lib.mbpt_estimate_batch(range(4))
    assert all(r.converged for r in res)
    assert iters < 200 and evals == sum(lib.n)
    # converged integrals are not iterated again
    assert lib.calls[-1] == [3]


def test_smallest_need_first_within_the_budget():
    # after a pilot of 1000 samples each, needs are 9e3, 9.9e5, 9.9e7 samples; the budget is 2^12 per live
    # integral: the first gets its need rounded up to a power of two (2^14), the others the minimum
    sds, goals = [1.0, 10.0, 100.0], [0.01] * 3
    lib = FakeLib([1.0] * 3, sds, goals, train=0)
    lib.n = [1000] * 3
    lib.samples = [1 << 12] * 3
    run(lib, [0, 1, 2], base_samples=1 << 12, min_samples=1 << 8, cap=1 << 20, max_iters=1)
    assert lib.samples == [1 << 14, 1 << 8, 1 << 8]
    # with a larger total budget the second is served too, capped per iteration
    lib2 = FakeLib([1.0] * 3, sds, goals, train=0)
    lib2.n = [1000] * 3
    lib2.samples = [1 << 12] * 3
    run(lib2, [0, 1, 2], base_samples=1 << 12, min_samples=1 << 8, cap=1 << 18, budget=1 << 19, max_iters=1)
    assert lib2.samples == [1 << 14, 1 << 18, 1 << 18]


def test_iteration_and_time_limits():
    lib = FakeLib([1.0], [1e3], [1e-6], train=0)
    lib.samples = [1 << 10]
    iters, evals, _ = run(lib, [0], base_samples=1 << 10, max_iters=5, iters_done=3)
    assert iters == 5 and len(lib.calls) == 2
    lib = FakeLib([1.0], [1e3], [1e-6], train=0)
    lib.samples = [1 << 10]
    iters, evals, _ = run(lib, [0], base_samples=1 << 10, max_iters=None, time_limit=0.0)
    assert iters == 0 and evals == 0 and not lib.calls
