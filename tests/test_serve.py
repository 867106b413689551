"""Serving loop (continuous batching of EOS requests): scheduling logic on CPU with a
deterministic fake backend; a GPU test that a request's result is the same alone and
in a mix of concurrent requests."""
import math

import numpy as np
import pytest

from paper_2603_24532_b300 import serve as S


class FakeDesc:
    def __init__(self, order, i):
        self.order = order
        self.diagram_id = i
        self.anomalous = False


class FakeBackend:
    """Integral i converges like sigma0/sqrt(iterations) around a value fixed by its
    stream id; memory 25 kB per integral; an optional arena limit raises MemoryError."""

    COUNTS = {2: 1, 3: 3, 4: 33, 5: 668}

    def __init__(self, arena_limit=None):
        self.live = {}
        self.next = 0
        self.arena_limit = arena_limit
        self.iterated = []

    def diagrams(self, order):
        return [FakeDesc(order, i) for i in range(self.COUNTS[order])]

    def physics(self, kn, kp):
        return (kn, kp)

    def cfg(self, samples, sid, seed, order=2):
        return (samples, sid, seed)

    def nbytes(self, d, cfg):
        return 25_000

    def create(self, d, phys, cfg):
        if self.arena_limit is not None and len(self.live) >= self.arena_limit:
            raise MemoryError("arena")
        h = self.next
        self.next += 1
        sid = cfg[1]
        self.live[h] = {"sid": sid, "it": 0, "val": -0.5 / d.order ** 2 * (1 + (sid % 7) / 10.0)}
        return h

    def iterate(self, handles):
        self.iterated.append(len(handles))
        for h in handles:
            self.live[h]["it"] += 1

    def estimate(self, h):
        s = self.live[h]
        it = s["it"]
        rng = np.random.default_rng(s["sid"] * 1000 + it)
        sigma = 0.05 * abs(s["val"]) / math.sqrt(it)
        return s["val"] + 0.1 * sigma * rng.standard_normal(), sigma, it

    def destroy(self, h):
        del self.live[h]


def test_grid_cache_nearest_within_window():
    c = S.GridCache(window=0.02)
    c.put(4, 7, 0.5, 0.10, "g10")
    c.put(4, 7, 0.5, 0.13, "g13")
    c.put(4, 7, 0.25, 0.11, "other-delta")
    c.put(3, 7, 0.5, 0.11, "other-order")
    assert c.get(4, 7, 0.5, 0.105) == "g10"
    assert c.get(4, 7, 0.5, 0.125) == "g13"
    assert c.get(4, 7, 0.5, 0.16) is None          # outside the window
    assert c.get(4, 8, 0.5, 0.10) is None          # other diagram
    small = S.GridCache(max_entries=2)
    for i in range(3):
        small.put(2, 0, 0.0, 0.05 + i, i)
    assert len(small.entries) == 2 and small.get(2, 0, 0.0, 0.05) is None


def test_fermi_momenta():
    kn, kp = S.fermi_momenta(0.16, 0.0)
    assert kn == pytest.approx(kp) and kn == pytest.approx((3 * math.pi ** 2 * 0.08) ** (1 / 3))
    kn, kp = S.fermi_momenta(0.1, 1.0)
    assert kp == 0.0 and kn == pytest.approx((3 * math.pi ** 2 * 0.1) ** (1 / 3))


def test_trace_is_deterministic_and_in_range():
    a = S.poisson_trace(200)
    b = S.poisson_trace(200)
    assert [(r.arrival, r.n_dens, r.delta, r.cap, r.target) for r in a] == \
           [(r.arrival, r.n_dens, r.delta, r.cap, r.target) for r in b]
    assert all(0.04 <= r.n_dens <= 0.2 and r.cap in (2, 3, 4) and r.target in (0.01, 0.003, 0.001) for r in a)
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert 0.03 < np.mean(gaps) < 0.07          # mean 1/20 s


def test_all_requests_complete_and_memory_is_released():
    be = FakeBackend()
    srv = S.Server(be, budget_bytes=10 ** 9, min_iters=2, max_iters=50, clock=iter(range(10 ** 6)).__next__)
    trace = S.poisson_trace(30)
    done = srv.run(trace, realtime=False)
    assert len(done) == 30 and all(r.energy is not None and np.isfinite(r.energy) for r in done)
    assert srv.used_bytes == 0 and srv.n_integrals == 0 and not be.live
    for r in done:
        assert r.sigma <= r.target * abs(r.energy) * 1.5 or r.rounds >= 50


def test_admission_respects_memory_budget_and_fifo():
    be = FakeBackend()
    # room for 40 integrals: a cap-4 request (37 integrals) blocks the next one until it completes
    srv = S.Server(be, budget_bytes=40 * 25_000, min_iters=2, clock=iter(range(10 ** 6)).__next__)
    reqs = [S.Request(0.1, 0.0, 4, 0.01, rid=0), S.Request(0.1, 0.0, 4, 0.01, rid=1),
            S.Request(0.1, 0.0, 2, 0.01, rid=2)]
    for r in reqs:
        srv.submit(r)
    srv.step()
    assert [r.rid for r in srv.active] == [0] and len(srv.waiting) == 2
    assert max(be.iterated) <= 40
    while srv.step():
        assert srv.used_bytes <= 40 * 25_000
    assert [r.rid for r in srv.done] == [0, 1, 2]   # FIFO: the small request does not overtake


def test_oversized_request_is_rejected_not_blocking():
    be = FakeBackend()
    srv = S.Server(be, budget_bytes=10 * 25_000, clock=iter(range(10 ** 6)).__next__)
    big, small = S.Request(0.1, 0.0, 4, 0.01, rid=0), S.Request(0.1, 0.0, 2, 0.01, rid=1)
    srv.submit(big)
    srv.submit(small)
    while srv.step():
        pass
    assert math.isnan(big.energy) and np.isfinite(small.energy)


def test_arena_refusal_rolls_back():
    be = FakeBackend(arena_limit=5)
    srv = S.Server(be, budget_bytes=10 ** 9, clock=iter(range(10 ** 6)).__next__)
    srv.submit(S.Request(0.1, 0.0, 3, 0.01, rid=0))   # 4 integrals
    srv.submit(S.Request(0.1, 0.0, 3, 0.01, rid=1))   # would need 8 > 5
    srv.step()
    assert len(be.live) == 4 and len(srv.waiting) == 1
    while srv.step():
        pass
    assert len(srv.done) == 2


def test_arena_refusal_with_nothing_running_completes_unfittable():
    """An arena that refuses a request while no other request holds memory can never take it: the
    request completes as unfittable (energy NaN) instead of waiting forever, and the queue moves on."""
    be = FakeBackend(arena_limit=3)
    srv = S.Server(be, budget_bytes=10 ** 9, clock=iter(range(10 ** 6)).__next__)
    big = S.Request(0.1, 0.0, 3, 0.01, rid=0)       # 4 integrals > 3
    small = S.Request(0.1, 0.0, 2, 0.01, rid=1)     # 1 integral
    done = srv.run([big, small], realtime=False)
    assert [r.rid for r in done] == [0, 1]
    assert math.isnan(big.energy) and not big.met and np.isfinite(small.energy)
    assert not be.live and srv.used_bytes == 0


def test_latency_split_by_outcome():
    """Requests stopped by the iteration cap are flagged and reported apart from those that met
    their target."""
    be = FakeBackend()
    srv = S.Server(be, min_iters=2, max_iters=3, clock=iter(range(10 ** 6)).__next__)
    reqs = [S.Request(0.1, 0.0, 2, 0.5, rid=0), S.Request(0.1, 0.0, 2, 1e-6, rid=1)]
    done = srv.run(reqs, realtime=False)
    by = {r.rid: r for r in done}
    assert by[0].met and not by[0].capped
    assert by[1].capped and not by[1].met
    assert S.latency_stats(done, "met")["n"] == 1 and S.latency_stats(done, "capped")["n"] == 1
    assert S.latency_stats(done)["n"] == 2


def test_result_same_alone_and_in_mix_fake():
    trace = S.poisson_trace(12)
    be = FakeBackend()
    mix = {r.rid: r.energy for r in S.Server(be, clock=iter(range(10 ** 6)).__next__).run(trace, realtime=False)}
    for rid in (0, 5, 11):
        r0 = S.poisson_trace(12)[rid]
        alone = S.Server(FakeBackend(), clock=iter(range(10 ** 6)).__next__).run([r0], realtime=False)
        assert alone[0].energy == mix[rid]


@pytest.mark.gpu
def test_result_same_alone_and_in_mix_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    full = S.poisson_trace(40)
    trace = [r for r in full if r.cap == 4][:2] + [r for r in full if r.cap <= 3][:4]   # fourth order included
    for r in trace:
        r.target = 0.01
    small = {2: 1 << 15, 3: 1 << 16, 4: 1 << 16}
    be = S.MbptBackend(arena_bytes=2 << 30)
    try:
        mix = S.Server(be, samples_by_order=small, max_iters=30).run([S.Request(**_req(r)) for r in trace],
                                                                     realtime=False)
        mixd = {r.rid: (r.energy, r.sigma, dict(r.per_order)) for r in mix}
        assert len(mixd) == len(trace)
        for r in trace[:2] + trace[2:3]:
            alone = S.Server(be, samples_by_order=small, max_iters=30).run([S.Request(**_req(r))], realtime=False)
            assert (alone[0].energy, alone[0].sigma, dict(alone[0].per_order)) == mixd[r.rid]
            assert alone[0].energy < 0.0
    finally:
        be.close()


class MirrorDesc:
    def __init__(self, order, i, mirror):
        self.order, self.diagram_id, self.mirror_id = order, i, mirror


class MirrorBackend(FakeBackend):
    """Fake whose integrals depend only on the mirror orbit (pairs have equal values), with a
    deterministic error sigma0/sqrt(iterations); grouping support like the real backend."""

    MIRROR = {2: [0], 3: [0, 1, 2], 4: [0, 1, 2, 5, 4, 3, 6, 8, 7, 9]}

    def __init__(self, dedup, grouped=False):
        super().__init__()
        self.dedup, self.grouped = dedup, grouped

    def diagrams(self, order):
        ds = [MirrorDesc(order, i, m) for i, m in enumerate(self.MIRROR[order])]
        return [d for d in ds if d.diagram_id <= d.mirror_id] if self.dedup else ds

    def multiplicity(self, d):
        return 2 if (self.dedup and d.mirror_id != d.diagram_id) else 1

    def create(self, d, phys, cfg):
        h = super().create(d, phys, cfg)
        orbit = min(d.diagram_id, d.mirror_id)
        self.live[h]["val"] = -0.01 * (1 + orbit) / d.order ** 2
        return h

    def estimate(self, h):
        s = self.live[h]
        return s["val"], 1e-4 * abs(s["val"]) / math.sqrt(s["it"]), s["it"]


def test_mirror_dedup_bookkeeping_fake():
    """One representative per mirror pair, counted twice in the request's sum and (squared) in its
    error budget and error, reproduces the full diagram sum when pair members are equal."""
    req = dict(n_dens=0.16, delta=0.0, cap=4, target=0.01, arrival=0.0, rid=3)
    clock = iter(range(10 ** 6)).__next__
    a = S.Server(MirrorBackend(dedup=False), clock=clock).run([S.Request(**req)], realtime=False)[0]
    b = S.Server(MirrorBackend(dedup=True), clock=clock).run([S.Request(**req)], realtime=False)[0]
    assert len(a.integrals) == 1 + 3 + 10 and len(b.integrals) == 1 + 3 + 8
    assert b.energy == pytest.approx(a.energy, rel=1e-14)
    for o in (2, 3, 4):
        assert b.per_order[o] == pytest.approx(a.per_order[o], rel=1e-14)
    assert sum(it.mult for it in b.integrals if it.order == 4) == 10
    assert b.sigma == pytest.approx(math.sqrt(sum((it.mult * it.sigma) ** 2 for it in b.integrals)), rel=1e-14)


@pytest.mark.gpu
def test_mirror_dedup_and_groups_run_on_gpu():
    """Per-diagram, mirror-deduplicated and grouped backends on one cap-4 request: the expected integral
    counts (1 + 3 + 33, 1 + 3 + 27, 1 + 2 + 4), finite energies, each energy the multiplicity-weighted
    sum of its integrals, and the three energies within 3 sigma of each other (one representative per
    mirror pair counted twice equals the full sum; the aligned groups equal the sum of their members).
    The evaluation phase on frozen grids keeps the errors of the heavy-tailed fourth-order weights
    honest enough for this comparison."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    small = {2: 1 << 15, 3: 1 << 16, 4: 1 << 16}
    req = dict(n_dens=0.16, delta=0.0, cap=4, target=0.01, arrival=0.0, rid=3)
    counts = {(False, False): 37, (True, False): 31, (True, True): 7}
    got = {}
    for (dedup, grouped), n in counts.items():
        be = S.MbptBackend(arena_bytes=1 << 30, dedup_mirrors=dedup, grouped=grouped)
        try:
            r = S.Server(be, samples_by_order=small, max_iters=20).run([S.Request(**req)], realtime=False)[0]
            assert len(r.integrals) == n
            assert np.isfinite(r.energy) and r.energy < 0.0 and np.isfinite(r.sigma)
            assert r.energy == pytest.approx(sum(it.mult * it.mean for it in r.integrals), rel=1e-14)
            if grouped:
                assert sorted(u.key for u in be.units(4)) == [2, 3, 4, 5]
                assert sum(sum(u.scales) for u in be.units(4)) == 33
            got[(dedup, grouped)] = (r.energy, r.sigma)
        finally:
            be.close()
    (e0, s0), (e1, s1), (e2, s2) = got[(False, False)], got[(True, False)], got[(True, True)]
    assert abs(e1 - e0) <= 3.0 * math.hypot(s0, s1), got
    assert abs(e2 - e0) <= 3.0 * math.hypot(s0, s2), got


@pytest.mark.gpu
def test_warm_start_seeds_grid_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    be = S.MbptBackend(arena_bytes=1 << 30)
    try:
        small = {2: 1 << 15, 3: 1 << 16, 4: 1 << 16}
        cold = S.Server(be, samples_by_order=small, max_iters=40)
        r_cold = cold.run([S.Request(0.121, 0.5, 3, 0.003, rid=2)], realtime=False)[0]
        srv = S.Server(be, samples_by_order=small, max_iters=40, warm_start=True)
        srv.run([S.Request(0.110, 0.5, 3, 0.003, rid=1)], realtime=False)
        r_warm = srv.run([S.Request(0.121, 0.5, 3, 0.003, rid=2)], realtime=False)[-1]
        assert srv.warm_starts == 4                       # 1 + 3 integrals seeded from n = 0.110
        assert abs(r_warm.energy - r_cold.energy) <= 3 * math.hypot(r_warm.sigma, r_cold.sigma)
        assert r_warm.sigma <= r_warm.target * abs(r_warm.energy) * 1.2
    finally:
        be.close()


def _req(r):
    return dict(n_dens=r.n_dens, delta=r.delta, cap=r.cap, target=r.target, arrival=0.0, rid=r.rid)


def test_cancel_frees_slots_and_logs():
    """A cancelled request leaves the queue or releases its integrals' bytes; the JSONL log records
    finished integrals, finished requests and the cancellation."""
    import io
    import json as _json
    log = io.StringIO()
    be = FakeBackend()
    srv = S.Server(be, clock=iter(range(10 ** 6)).__next__, log=log)
    trace = S.poisson_trace(4)
    for r in trace:
        srv.submit(r)
    srv.step()                                   # admits all four, one round
    used = srv.used_bytes
    victim = srv.active[1]
    n_int = len(victim.integrals)
    assert srv.cancel(victim.rid)
    assert srv.used_bytes == used - 25_000 * n_int and len(be.live) == sum(len(r.integrals) for r in srv.active)
    assert not srv.cancel(victim.rid) and not srv.cancel(999)
    while srv.step():
        pass
    done = {r.rid: r for r in srv.done}
    assert done[victim.rid].cancelled and done[victim.rid].energy is None
    assert all(r.energy is not None for k, r in done.items() if k != victim.rid)
    recs = [_json.loads(line) for line in log.getvalue().splitlines()]
    kinds = [r["event"] for r in recs]
    assert kinds.count("request") == 3 and kinds.count("cancelled") == 1
    assert kinds.count("integral") == sum(len(r.integrals) for k, r in done.items() if k != victim.rid)


def test_round_scheduling_keeps_results_and_bounds_rounds():
    """With a round sample limit the server runs the requests with the least work left first (and any
    request that has waited too long); a request that sits out rounds keeps its state, so every result
    equals the unscheduled run's, and no round exceeds the limit unless a single request does."""
    be0 = FakeBackend()
    srv0 = S.Server(be0, clock=iter(range(10 ** 6)).__next__)
    ref = {r.rid: (r.energy, r.sigma) for r in srv0.run(S.poisson_trace(20), realtime=False)}
    be = FakeBackend()
    srv = S.Server(be, clock=iter(range(10 ** 6)).__next__, round_samples=40 * (1 << 16), max_wait=50)
    done = srv.run(S.poisson_trace(20), realtime=False)
    assert {r.rid: (r.energy, r.sigma) for r in done} == ref
    biggest = max(sum(1 for _ in r.integrals) for r in done)
    assert max(be.iterated) <= max(40, biggest)
    assert max(be0.iterated) > 40 and srv.rounds > srv0.rounds   # smaller, more rounds than unscheduled


class DriftBackend(FakeBackend):
    """As FakeBackend, but each integral's estimate drifts towards zero by up to 40 % over its first
    iterations, so the request's error goal (target x |energy|) shrinks after some integrals retired."""

    def estimate(self, h):
        m, sigma, it = super().estimate(h)
        return m * (0.6 + 0.4 / it), sigma, it


def test_every_request_ends_met_or_capped():
    """A request whose integrals each met their share of the error budget when they retired, but whose
    total error is above the goal of its final estimate, reopens the integrals above their current share:
    every completed request either meets its target or was stopped by the iteration cap."""
    done = S.Server(DriftBackend(), clock=iter(range(10 ** 6)).__next__).run(S.poisson_trace(40), realtime=False)
    assert len(done) == 40
    assert all(r.met or r.capped for r in done), [(r.rid, r.sigma, r.target * abs(r.energy)) for r in done
                                                  if not (r.met or r.capped)]
    assert sum(r.met for r in done) >= 10
