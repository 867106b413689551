"""Continuous-batching server for equation-of-state requests.

A request asks for the correlation energy per particle sum_{k=2}^{cap} E^(k)/N of nucleon
matter at density n (fm^-3) and isospin asymmetry delta, to a relative statistical error
`target`.  It expands into one integral per non-anomalous Hugenholtz diagram of orders
2..cap at kF_n = (3 pi^2 n (1 + delta)/2)^(1/3), kF_p = (3 pi^2 n (1 - delta)/2)^(1/3)
(Sec. II; a species with zero density is absent).  With a grouped backend an order expands
instead into one integral per particle-hole group of its diagrams (Sec. III.A).

The loop (one "round" per VEGAS iteration of every resident integral):
  1. admit waiting requests in arrival order while the device arena holds their integrals
     (memory admission: state bytes from mbpt_diag_bytes, budget in bytes) and the slot
     limit allows;
  2. run one batched iteration of all resident, unfinished integrals (one graph replay);
  3. read the estimates; the request's summed estimate E_sum sets its error goal target |E_sum|,
     shared among its integrals in proportion to the square roots of their per-sample variances
     (the Neyman allocation, the cheapest split of the goal); integrals that reach their share
     (after at least `min_iters` iterations) retire and stop consuming samples, the others get
     the samples their share still needs;
  4. a request completes when all its integrals have retired (or hit `max_iters`), or earlier,
     once the error of its sum, sqrt(sum sigma_G^2), meets target |E_sum|; its integrals are
     destroyed, freeing arena memory for waiting requests.

With the GPU backend every integral trains its VEGAS grid for a few iterations and then
estimates on the frozen grid, every evaluation sample carrying the same weight (PVegas'
training and evaluation phases, Sec. III.C); its error is the standard error of all its
evaluation samples, which stays honest for the heavy-tailed weights of fourth-order diagrams.

Requests that arrive while others are on the GPU join the next round: their integrals run in
the same persistent launch as everything else.  Each integral's random stream is keyed by
(request id, order, diagram id), and every quantity that decides its iterations is local to
its request, so a request's result is the same alone and in a mix.
"""
from __future__ import annotations

import bisect
import json
import math
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

HBAR2_OVER_M = 41.47


def fermi_momenta(n_dens: float, delta: float):
    """kF_n, kF_p of matter with total density n and asymmetry delta = (n_n - n_p)/n."""
    nn = 0.5 * n_dens * (1.0 + delta)
    npr = 0.5 * n_dens * (1.0 - delta)
    kn = (3.0 * math.pi ** 2 * nn) ** (1.0 / 3.0) if nn > 0 else 0.0
    kp = (3.0 * math.pi ** 2 * npr) ** (1.0 / 3.0) if npr > 1e-15 else 0.0
    return kn, kp


@dataclass
class Request:
    n_dens: float
    delta: float
    cap: int
    target: float
    arrival: float = 0.0
    rid: int = -1
    # filled by the server
    admitted: Optional[float] = None
    completed: Optional[float] = None
    energy: Optional[float] = None
    sigma: Optional[float] = None
    per_order: Dict[int, float] = field(default_factory=dict)
    integrals: list = field(default_factory=list)
    budget: Optional[float] = None
    rounds: int = 0
    cancelled: bool = False
    capped: bool = False      # some integral stopped at the iteration cap before reaching its error budget
    remaining: float = 0.0    # estimated samples still to run (scheduling priority)
    last_run: float = 0.0     # clock of its last round

    @property
    def met(self) -> bool:
        """Finished with a finite energy whose error meets the requested relative target."""
        return (self.energy is not None and self.sigma is not None and math.isfinite(self.energy)
                and self.sigma <= self.target * abs(self.energy))

    @property
    def latency(self) -> Optional[float]:
        if self.completed is None:
            return None
        return self.completed - self.arrival


@dataclass
class Integral:
    req: Request
    order: int
    diagram_id: int
    handle: object
    bytes: int
    cfg: object = None
    samples: int = 0
    evals: int = 0
    warm: bool = False
    mult: int = 1
    mean: float = 0.0
    sigma: float = float("inf")
    n_iter: int = 0
    done: bool = False
    n_train: int = 0          # leading training iterations (no estimate of the error yet)
    eval_samples: int = 0     # samples of the evaluation iterations so far
    need: float = 0.0         # evaluation samples its error share still needs (Neyman allocation)


class GroupUnit:
    """The diagrams of one order sharing a particle-hole composition (number of hole loop momenta),
    integrated as one integrand (Sec. III.A); member scales carry mirror multiplicities."""

    def __init__(self, order: int, key: int, descs, scales):
        self.order = order
        self.key = key
        self.diagram_id = 1000 + key      # unit id within the order (stream ids, grid cache)
        self.mirror_id = self.diagram_id
        self.descs = list(descs)
        self.scales = list(scales)


# VEGAS grid compression by order (measured: at fourth and fifth order Lepage's alpha = 1.5 concentrates
# the bins so strongly that rare samples in the wide bins dominate the variance) and training iterations
ALPHA_BY_ORDER = {2: 1.5, 3: 1.5, 4: 1.0, 5: 0.75, 6: 0.75}
TRAIN_BY_ORDER = {2: 2, 3: 2, 4: 3, 5: 3, 6: 3}


class MbptBackend:
    """The C ABI as the server's backend (all work on the GPU).  With grouped=True each order of a
    request is a handful of group integrals (Table I's N_grp) instead of one integral per diagram;
    group_orders limits that to some orders (e.g. (4,): fourth order in aligned groups, orders 2-3
    diagram by diagram).
    Integrals train their grid for TRAIN_BY_ORDER iterations and are then estimated on the frozen grid
    (MBPT_COMBINE_POOLED), with grid compression ALPHA_BY_ORDER."""

    def __init__(self, device: int = 0, arena_bytes: int = 8 << 30, arena_ptr: int = 0, stream: int = 0,
                 precision: Optional[int] = None, map_kind: int = 1, dedup_mirrors: bool = True,
                 grouped: bool = False, group_orders=None):
        from . import mbpt as M
        self.M = M
        self.map_kind = map_kind
        self.dedup_mirrors = dedup_mirrors
        self.grouped = grouped
        self.group_orders = None if group_orders is None else set(group_orders)
        self._units = {}
        self.ctx = M.mbpt_ctx_create(device, arena_bytes, arena_ptr=arena_ptr, stream=stream)
        self.precision = M.MBPT_MIXED if precision is None else precision
        self._descs = {}

    def diagrams(self, order: int):
        """Non-anomalous diagrams; with mirror deduplication one representative per pair of
        complex-conjugate (time- and arrow-reversed) diagrams, whose integrands are equal sample by
        sample for a real symmetric potential, each with its multiplicity (1 or 2): the N_eff
        diagrams of Table I."""
        if order not in self._descs:
            ds = [d for d in self.M.mbpt_generate(order) if not d.anomalous]
            if self.dedup_mirrors:
                ds = [d for d in ds if d.diagram_id <= d.mirror_id]
            self._descs[order] = ds
        return self._descs[order]

    def units(self, order: int):
        """What one order of a request expands into: diagrams, or groups of them."""
        if not self.grouped or (self.group_orders is not None and order not in self.group_orders):
            return self.diagrams(order)
        if order not in self._units:
            by_key = {}
            for d in self.diagrams(order):
                by_key.setdefault(self.M.mbpt_hole_chords(d), []).append(d)
            self._units[order] = [GroupUnit(order, k, ds, [self._mult(d) for d in ds])
                                  for k, ds in sorted(by_key.items())]
        return self._units[order]

    def _mult(self, desc) -> int:
        if not self.dedup_mirrors:
            return 1
        return 1 if desc.mirror_id == desc.diagram_id else 2

    def multiplicity(self, unit) -> int:
        return 1 if isinstance(unit, GroupUnit) else self._mult(unit)

    def physics(self, kF_n: float, kF_p: float):
        return self.M.physics(kF_n=kF_n, kF_p=kF_p, K_max=max(kF_n, kF_p) + 6.0, map_kind=self.map_kind)

    def train_iters(self, order: int) -> int:
        return TRAIN_BY_ORDER[order]

    def cfg(self, samples: int, stream_id: int, seed: int, order: int = 2):
        return self.M.vegas_cfg(samples=samples, seed=seed, stream_id=stream_id, precision=self.precision,
                                alpha=ALPHA_BY_ORDER[order], train_iters=TRAIN_BY_ORDER[order],
                                combine=self.M.MBPT_COMBINE_POOLED)

    def nbytes(self, desc, cfg) -> int:
        if isinstance(desc, GroupUnit):
            return self.M.mbpt_group_bytes(desc.descs, cfg)
        return self.M.mbpt_diag_bytes(desc, cfg)

    def create(self, desc, phys, cfg):
        try:
            if isinstance(desc, GroupUnit):
                return self.M.mbpt_create_group(self.ctx, desc.descs, phys, cfg, scales=desc.scales)
            return self.M.mbpt_create_diagram(self.ctx, desc, phys, cfg)
        except self.M.MbptError as e:
            if e.status == self.M.MBPT_ENOMEM:
                raise MemoryError(str(e)) from e
            raise

    def iterate(self, handles: Sequence):
        self.M.mbpt_vegas_iterate(self.ctx, list(handles), 1)

    def estimate(self, h):
        r = self.M.mbpt_estimate(h)
        return r.mean, r.sigma, r.n_iter

    def estimate_many(self, handles: Sequence):
        return [(r.mean, r.sigma, r.n_iter) for r in self.M.mbpt_estimate_batch(list(handles))]

    def get_grid(self, h):
        img = self.M.mbpt_get_state(h)
        d = int(np.frombuffer(img, dtype=np.int32, count=2, offset=8)[0])
        nb = int(np.frombuffer(img, dtype=np.int32, count=2, offset=8)[1])
        return self.M.state_grid(img, d, nb)

    def set_grid(self, h, grid):
        self.M.mbpt_set_state(h, self.M.state_with_grid(self.M.mbpt_get_state(h), grid))

    def set_train(self, h, cfg, iters: int):
        cfg.train_iters = int(iters)
        self.M.mbpt_set_config(h, cfg)

    def set_samples(self, h, cfg, samples: int):
        cfg.samples_per_iter = int(samples)
        self.M.mbpt_set_config(h, cfg)

    def destroy(self, h):
        self.M.mbpt_destroy_diagram(h)

    def close(self):
        self.M.mbpt_ctx_destroy(self.ctx)


class GridCache:
    """Trained VEGAS grids of finished integrals, keyed by (order, diagram, asymmetry), for warm
    starts at neighbouring densities (Sec. III.C: importance-sampling distributions propagate in
    density for changes up to about 0.02 fm^-3).  Each key keeps its densities sorted, so a lookup
    is a bisection; the oldest entries are evicted beyond max_entries."""

    def __init__(self, window: float = 0.02, max_entries: int = 50000):
        self.window = window
        self.max_entries = max_entries
        self.entries: "OrderedDict[tuple, np.ndarray]" = OrderedDict()    # insertion order, for eviction
        self._by_key: Dict[tuple, List[float]] = {}

    def put(self, order: int, did: int, delta: float, n_dens: float, grid) -> None:
        if grid is None:
            return
        k = (order, did, round(delta, 6))
        n = round(n_dens, 6)
        key = k + (n,)
        if key not in self.entries:
            bisect.insort(self._by_key.setdefault(k, []), n)
        self.entries[key] = grid
        self.entries.move_to_end(key)
        while len(self.entries) > self.max_entries:
            old, _ = self.entries.popitem(last=False)
            lst = self._by_key[old[:3]]
            lst.pop(bisect.bisect_left(lst, old[3]))

    def get(self, order: int, did: int, delta: float, n_dens: float):
        k = (order, did, round(delta, 6))
        lst = self._by_key.get(k)
        if not lst:
            return None
        i = bisect.bisect_left(lst, n_dens)
        best, best_d = None, None
        for j in (i - 1, i):
            if 0 <= j < len(lst):
                dist = abs(lst[j] - n_dens)
                if dist <= self.window and (best_d is None or dist < best_d):
                    best, best_d = lst[j], dist
        return None if best is None else self.entries[k + (best,)]


SAMPLES_BY_ORDER = {2: 1 << 16, 3: 1 << 16, 4: 1 << 17, 5: 1 << 17}   # training iterations
# adaptive samples per iteration of one integral: between these.  Measured on the 1200-request stream (cap
# at 120 iterations): at most 2^25 leaves 0.8 % of the requests short of their target at the cap, against
# 3.6 % with at most 2^23 (6.5 % with a 60-iteration cap), at a p99 latency of 55 s instead of 22 s (6 s):
# the requests that need 10^9 samples or more then finish instead of stopping early
MIN_SAMPLES, MAX_SAMPLES = 1 << 16, 1 << 25


class Server:
    def __init__(self, backend, budget_bytes: int = 40 << 30, max_integrals: int = 1 << 16,
                 samples_by_order: Optional[Dict[int, int]] = None, min_iters: int = 3, max_iters: int = 120,
                 seed: int = 1, clock: Callable[[], float] = time.perf_counter, adaptive: bool = True,
                 warm_start: bool = False, warm_window: float = 0.02, warm_blend: float = 0.5,
                 warm_train: int = 1, log=None, round_samples: Optional[int] = None, max_wait: float = 2.0,
                 max_samples: int = MAX_SAMPLES):
        self.b = backend
        self.max_samples = max_samples        # adaptive samples per iteration of one integral: at most this
        self.log = log                        # optional text stream: one JSON record per finished integral / request
        # round scheduling: with round_samples set, a round runs the requests with the least estimated work
        # left first, up to that many samples (at least one request), and any request that has not run for
        # max_wait seconds before the others; a request that sits out a round keeps its state, so its
        # result does not depend on the schedule
        self.round_samples = round_samples
        self.max_wait = max_wait
        self.adaptive = adaptive
        self.cache = GridCache(warm_window) if warm_start else None
        self.warm_blend = warm_blend          # weight of the donor grid (rest: uniform bins)
        self.warm_train = warm_train          # leading iterations of a warm-started integral not combined
        self.warm_starts = 0
        self.budget = budget_bytes
        self.max_integrals = max_integrals
        self.samples = dict(SAMPLES_BY_ORDER if samples_by_order is None else samples_by_order)
        self.min_iters = min_iters
        self.max_iters = max_iters
        self.seed = seed
        self.clock = clock
        self.waiting: List[Request] = []
        self.active: List[Request] = []
        self.done: List[Request] = []
        self.used_bytes = 0
        self.n_integrals = 0
        self.rounds = 0
        self.evals = 0
        self._next_id = 0

    # ---- request bookkeeping ------------------------------------------------------------
    def submit(self, req: Request) -> int:
        if req.rid < 0:
            req.rid = self._next_id
        self._next_id = max(self._next_id, req.rid + 1)
        if req.cap < 2:
            raise ValueError("order cap must be >= 2")
        self.waiting.append(req)
        return req.rid

    def _plan(self, req: Request):
        kn, kp = fermi_momenta(req.n_dens, req.delta)
        phys = self.b.physics(kn, kp)
        plan = []
        for order in range(2, req.cap + 1):
            for d in (self.b.units(order) if hasattr(self.b, "units") else self.b.diagrams(order)):
                sid = (req.rid * 8 + order) * 1024 + d.diagram_id
                cfg = self.b.cfg(self.samples[order], sid & 0xFFFFFFFF, self.seed, order=order)
                plan.append((order, d, phys, cfg, self.b.nbytes(d, cfg)))
        return plan

    def _admit(self, now: float):
        while self.waiting:
            req = self.waiting[0]
            plan = self._plan(req)
            need = sum(p[4] for p in plan)
            if need > self.budget:
                # can never fit: reject rather than block the queue
                self.waiting.pop(0)
                req.completed = now
                req.energy = float("nan")
                self.done.append(req)
                continue
            if self.used_bytes + need > self.budget or self.n_integrals + len(plan) > self.max_integrals:
                return
            created = []
            try:
                for order, d, phys, cfg, nb in plan:
                    h = self.b.create(d, phys, cfg)
                    it = Integral(req, order, d.diagram_id, h, nb, cfg, self.samples[order],
                                  mult=self.b.multiplicity(d) if hasattr(self.b, "multiplicity") else 1,
                                  n_train=self.b.train_iters(order) if hasattr(self.b, "train_iters") else 0)
                    created.append(it)
                    if self.cache is not None and hasattr(self.b, "set_grid"):
                        g = self.cache.get(order, d.diagram_id, req.delta, req.n_dens)
                        if g is not None:
                            # the donor's bin structure blended with uniform bins, plus warm_train
                            # training iterations that are not combined (abbreviated retraining)
                            u = np.linspace(0.0, 1.0, g.shape[1])[None, :]
                            self.b.set_grid(h, self.warm_blend * g + (1.0 - self.warm_blend) * u)
                            if self.warm_train and hasattr(self.b, "set_train"):
                                self.b.set_train(h, it.cfg, self.warm_train)
                            it.warm = True
            except MemoryError:
                # the arena refused (its scratch competes with integral state): roll back and retry once
                # running requests have freed memory; with nothing running nothing will be freed, so the
                # request can never fit and is completed as unfittable instead of blocking the queue
                for it in created:
                    self.b.destroy(it.handle)
                if self.active:
                    return
                self.waiting.pop(0)
                req.completed = now
                req.energy = float("nan")
                self.done.append(req)
                self._log({"event": "unfittable", "rid": req.rid})
                continue
            self.waiting.pop(0)
            req.admitted = now
            req.last_run = now
            req.remaining = float(sum(it.samples * (it.n_train + 2) for it in created))
            req.integrals = created
            self.used_bytes += need
            self.n_integrals += len(plan)
            self.active.append(req)

    def cancel(self, rid: int) -> bool:
        """Withdraw a request: waiting, it leaves the queue; admitted, its integrals are destroyed
        and their arena bytes return to the budget.  It completes with energy None.  False if the
        request is unknown or already finished."""
        for q in (self.waiting, self.active):
            for req in q:
                if req.rid == rid:
                    q.remove(req)
                    for it in req.integrals:
                        self.b.destroy(it.handle)
                        self.used_bytes -= it.bytes
                    self.n_integrals -= len(req.integrals)
                    req.integrals = []
                    req.energy = None
                    req.completed = self.clock()
                    req.cancelled = True
                    self.done.append(req)
                    self._log({"event": "cancelled", "rid": rid})
                    return True
        return False

    def _log(self, rec: dict) -> None:
        if self.log is not None:
            self.log.write(json.dumps(rec) + "\n")

    def _retire_and_complete(self, now: float, batch=None):
        batch = self.active if batch is None else batch
        live = [it for req in batch for it in req.integrals if not it.done]
        if hasattr(self.b, "estimate_many"):
            ests = self.b.estimate_many([it.handle for it in live])
        else:
            ests = [self.b.estimate(it.handle) for it in live]
        for it, e in zip(live, ests):
            it.mean, it.sigma, it.n_iter = e
        finished = set()
        for req in batch:
            req.rounds += 1
            req.last_run = now
            e_sum = sum(it.mult * it.mean for it in req.integrals)
            goal = req.target * abs(e_sum)     # the request's error target, from its current estimate
            req.budget = goal
            for it in req.integrals:
                if not it.done:
                    it.evals += it.samples
                    if it.n_iter > it.n_train:
                        it.eval_samples += it.samples
            trained = all(it.n_iter >= max(self.min_iters, it.n_train + 1) and math.isfinite(it.sigma)
                          for it in req.integrals)
            if trained and math.sqrt(sum((it.mult * it.sigma) ** 2 for it in req.integrals)) <= goal:
                # the request's own target is met: every integral retires with it
                for it in req.integrals:
                    it.done = True
            # Neyman allocation of the error budget: with per-sample variances v_i = sigma_i^2 N_i (N_i the
            # evaluation samples), the evaluation samples that reach a total error `goal` at the least total
            # cost are N_i = mult_i sqrt(v_i) S / goal^2, S = sum_j mult_j sqrt(v_j); integral i's share of the
            # error is then sigma_i^2 = sqrt(v_i) goal^2 / (mult_i S).  Integrals still training have no v_i yet.
            v = {id(it): it.sigma ** 2 * it.eval_samples for it in req.integrals
                 if math.isfinite(it.sigma) and it.eval_samples > 0}
            S = sum(it.mult * math.sqrt(v[id(it)]) for it in req.integrals if id(it) in v)
            n_eff = sum(it.mult ** 2 for it in req.integrals)
            shares = {}
            for it in req.integrals:
                if id(it) in v and S > 0.0:
                    shares[id(it)] = goal * math.sqrt(math.sqrt(v[id(it)]) / (it.mult * S))
                else:
                    shares[id(it)] = goal / math.sqrt(n_eff)
            for it in req.integrals:
                if it.done:
                    continue
                share = shares[id(it)]
                if it.n_iter >= self.min_iters and it.sigma <= share:
                    it.done = True
                elif it.n_iter >= self.max_iters:
                    it.done = True
                    req.capped = True
                elif (self.adaptive and hasattr(self.b, "set_samples") and id(it) in v and share > 0.0):
                    # evaluation samples still needed for the share, spread over a few iterations
                    need = v[id(it)] / share ** 2 - it.eval_samples
                    it.need = max(0.0, need)
                    left = max(1, self.min_iters - it.n_iter, 3)
                    nxt = int(min(self.max_samples, max(MIN_SAMPLES, need / left)))
                    nxt = 1 << max(0, int(round(math.log2(nxt))))
                    if nxt != it.samples:
                        self.b.set_samples(it.handle, it.cfg, nxt)
                        it.samples = nxt
            if (all(it.done for it in req.integrals) and not req.capped
                    and math.sqrt(sum((it.mult * it.sigma) ** 2 for it in req.integrals)) > goal):
                # every integral met the share it had when it retired, but the goal and the shares have moved
                # with the estimate since: reopen those above their current share (at least the largest term)
                above = [it for it in req.integrals if it.sigma > shares[id(it)]]
                for it in above or [max(req.integrals, key=lambda x: x.mult * x.sigma)]:
                    it.done = False
            if all(it.done for it in req.integrals):
                req.energy = e_sum
                req.sigma = math.sqrt(sum((it.mult * it.sigma) ** 2 for it in req.integrals))
                for order in range(2, req.cap + 1):
                    req.per_order[order] = sum(it.mult * it.mean for it in req.integrals if it.order == order)
                req.completed = now
                for it in req.integrals:
                    self._log({"event": "integral", "rid": req.rid, "order": it.order, "diagram": it.diagram_id,
                               "mult": it.mult, "mean": it.mean, "sigma": it.sigma, "iterations": it.n_iter,
                               "evals": it.evals, "warm": it.warm})
                self._log({"event": "request", "rid": req.rid, "n": req.n_dens, "delta": req.delta, "cap": req.cap,
                           "target": req.target, "energy": req.energy, "sigma": req.sigma,
                           "per_order": req.per_order, "rounds": req.rounds, "latency_s": req.latency})
                for it in req.integrals:
                    if self.cache is not None and hasattr(self.b, "get_grid"):
                        self.cache.put(it.order, it.diagram_id, req.delta, req.n_dens, self.b.get_grid(it.handle))
                    self.warm_starts += int(it.warm)
                    self.b.destroy(it.handle)
                    self.used_bytes -= it.bytes
                self.n_integrals -= len(req.integrals)
                self.done.append(req)
                finished.add(id(req))
            else:
                # estimated samples still to run: the next iteration's samples of every unfinished integral,
                # or the samples its share still needs if that is more
                req.remaining = float(sum(max(it.samples, it.need) for it in req.integrals if not it.done))
        self.active = [r for r in self.active if id(r) not in finished]

    def _schedule(self, now: float):
        """The requests of this round (all of them without a round sample limit)."""
        if self.round_samples is None:
            return list(self.active)
        order = sorted(self.active, key=lambda r: (0 if now - r.last_run > self.max_wait else 1, r.remaining,
                                                   r.arrival, r.rid))
        batch, total = [], 0
        for r in order:
            need = sum(it.samples for it in r.integrals if not it.done)
            if batch and total + need > self.round_samples:
                continue
            batch.append(r)
            total += need
        return batch

    def step(self) -> bool:
        """One round; returns False when there is nothing to run."""
        now = self.clock()
        self._admit(now)
        batch = self._schedule(now)
        handles = [it.handle for req in batch for it in req.integrals if not it.done]
        if not handles:
            return False
        self.b.iterate(handles)
        self.evals += sum(it.samples for req in batch for it in req.integrals if not it.done)
        self.rounds += 1
        self._retire_and_complete(self.clock(), batch)
        return True

    def run(self, trace: Sequence[Request], realtime: bool = True, time_limit: Optional[float] = None):
        """Replay a trace: request i becomes visible at t0 + trace[i].arrival (wall clock when
        realtime, else all at once in order).  Returns the completed requests."""
        pending = sorted(trace, key=lambda r: r.arrival)
        t0 = self.clock()
        k = 0
        while k < len(pending) or self.waiting or self.active:
            now = self.clock() - t0
            while k < len(pending) and (not realtime or pending[k].arrival <= now):
                r = pending[k]
                r.arrival = t0 + r.arrival if realtime else self.clock()
                self.submit(r)
                k += 1
            ran = self.step()
            if not ran and k < len(pending) and realtime:
                wait = pending[k].arrival - (self.clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            if time_limit is not None and self.clock() - t0 > time_limit:
                break
        return self.done


def poisson_trace(n_requests: int, rate: float = 20.0, seed: int = 7) -> List[Request]:
    """Synthetic EOS request stream: exponential inter-arrival gaps (mean 1/rate), and per
    request, in this draw order: n ~ U[0.04, 0.20] fm^-3, delta from {0, .25, .5, .75, 1},
    order cap from {2, 3, 4}, target from {1 %, 0.3 %, 0.1 %}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n = rng.uniform(0.04, 0.20)
        delta = [0.0, 0.25, 0.5, 0.75, 1.0][rng.integers(0, 5)]
        cap = [2, 3, 4][rng.integers(0, 3)]
        target = [0.01, 0.003, 0.001][rng.integers(0, 3)]
        out.append(Request(n_dens=n, delta=delta, cap=cap, target=target, arrival=t, rid=i))
    return out


def latency_stats(done: Sequence[Request], which: str = "all"):
    """Latency percentiles of finished requests with a finite energy: all of them, only those whose
    error met the target ("met"), or only those stopped by the iteration cap ("capped")."""
    sel = [r for r in done if r.latency is not None and r.energy is not None and np.isfinite(r.energy)]
    if which == "met":
        sel = [r for r in sel if r.met]
    elif which == "capped":
        sel = [r for r in sel if r.capped]
    elif which != "all":
        raise ValueError(which)
    lat = np.array([r.latency for r in sel])
    if len(lat) == 0:
        return {"p50_s": None, "p99_s": None, "n": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "n": int(len(lat))}
