"""Host logic of the continuous-batching loop, on the CPU with a fake pool backend and a
virtual clock: admission in arrival order under the HBM budget, requests of one problem
packed into shared pools, joins only between steps, every request's window of sweeps, pool
closing, and the latency report."""
import numpy as np
import pytest

from paper_2106_00712_gb300.serving import (Request, Server, poisson_stream, report,
                                            request_observables)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances virtual time
        return self.t


class FakePoolBackend:
    """A pool step costs `cost` virtual seconds per sweep whatever its size; footprint =
    slots x L^4 bytes. Records what the loop asks for."""

    def __init__(self, clock, cost=1e-3):
        self.clock, self.cost = clock, cost
        self.in_use = 0
        self.max_in_use = 0
        self.opened = []
        self.joins = []       # (pool id, sweeps done by the pool, [(slot, rid)])
        self.collected = {}   # rid -> (pool id, slot, first row)

    def footprint(self, r, slots, max_sweeps):
        return slots * r.L ** 4

    def open(self, r, slots):
        h = {"id": len(self.opened), "key": r.key, "slots": slots, "busy_until": 0.0,
             "sweeps": 0, "bytes": self.footprint(r, slots, 0)}
        self.opened.append(h)
        self.in_use += h["bytes"]
        self.max_in_use = max(self.max_in_use, self.in_use)
        return h

    def join(self, h, placements):
        assert self.idle(h) and h["sweeps"] % 2 == 0
        for _, r in placements:
            assert r.key == h["key"]
        self.joins.append((h["id"], h["sweeps"], [(s, r.rid) for s, r in placements]))

    def step(self, h, n):
        assert self.idle(h)
        h["busy_until"] = self.clock.t + n * self.cost
        h["sweeps"] += n

    def idle(self, h):
        return self.clock.t >= h["busy_until"]

    def collect(self, h, slot, r, first_row):
        assert first_row + r.n_meas <= h["sweeps"]
        self.collected[r.rid] = (h["id"], slot, first_row)
        return {"energy": -1.0 - 0.01 * (r.rid % 7)}

    def close(self, h):
        self.in_use -= h["bytes"]
        return {"max_drift": 0.0, "error": None}


def test_admission_packs_pools_within_budget_and_everything_completes():
    clock = FakeClock()
    be = FakePoolBackend(clock)
    reqs = poisson_stream(60, rate=400.0, seed=3, lattices=(4, 6), betas=(2.0,), Us=(4.0,),
                          chains=2, n_warm=3, n_meas=4)
    budget = 6 * 8 * 6 ** 4
    srv = Server(be, budget, max_slots=4, clock=clock, idle_sleep=0.0)
    results, makespan = srv.run(reqs)
    assert set(results) == {r.rid for r in reqs}
    assert be.max_in_use <= budget and be.in_use == 0
    # requests of one problem share pools: fewer pools than requests, several per pool
    assert len(be.opened) < len(reqs)
    assert max(p["served"] for p in srv.pool_log) > 1
    assert sum(p["served"] for p in srv.pool_log) == len(reqs)
    # each request joined once, between steps, and its measuring window follows its own
    # warm-up inside its pool
    joined = {}
    for pid, sweeps, places in be.joins:
        for slot, rid in places:
            assert rid not in joined
            joined[rid] = (pid, slot, sweeps)
    for r in reqs:
        pid, slot, row = joined[r.rid]
        assert be.collected[r.rid] == (pid, slot, row + r.n_warm)
        res = results[r.rid]
        assert res.admitted >= r.arrival - 1e-9
        assert res.done - res.admitted >= r.sweeps * be.cost - 1e-9
    rep = report(results, reqs, makespan)
    assert rep["p50_latency_s"] <= rep["p99_latency_s"]
    assert rep["n_requests"] == 60


def test_slots_are_reused_only_after_their_request_is_done():
    clock = FakeClock()
    be = FakePoolBackend(clock)
    reqs = [Request(i, 4, 1.0, 4.0, arrival=0.0001 * i, chains=2, n_warm=2, n_meas=2)
            for i in range(6)]
    srv = Server(be, 2 * 4 ** 4, max_slots=2, clock=clock, idle_sleep=0.0)  # one pool of 2
    results, _ = srv.run(reqs)
    assert len(results) == 6
    spans = {}
    for pid, sweeps, places in be.joins:
        for slot, rid in places:
            spans[rid] = (pid, slot, sweeps, sweeps + reqs[rid].sweeps)
    for a in spans.values():
        for b in spans.values():
            if a is not b and a[:2] == b[:2]:
                assert a[3] <= b[2] or b[3] <= a[2]   # no overlap in one slot


def test_oversize_request_is_rejected():
    clock = FakeClock()
    srv = Server(FakePoolBackend(clock), 100, clock=clock, idle_sleep=0.0)
    with pytest.raises(ValueError):
        srv.run([Request(0, 8, 1.0, 4.0)])


def test_request_observables_are_window_ratios_then_chain_means():
    rng = np.random.default_rng(0)
    ser = rng.uniform(0.5, 1.5, size=(5, 3, 8))
    got = request_observables(ser, 3)
    per = ser[:, :, 0].sum(axis=0) / ser[:, :, 5].sum(axis=0)
    assert got["energy"] == pytest.approx(per.mean(), rel=1e-14)
    assert got["energy_err"] == pytest.approx(per.std(ddof=1) / np.sqrt(3), rel=1e-12)


def test_poisson_stream_is_seeded_and_mixed():
    a = poisson_stream(200, rate=10.0, seed=1)
    b = poisson_stream(200, rate=10.0, seed=1)
    assert [(r.L, r.beta, r.U, r.seed, r.arrival) for r in a] == \
           [(r.L, r.beta, r.U, r.seed, r.arrival) for r in b]
    assert {r.L for r in a} == {6, 8, 10, 12}
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert 0.07 < sum(gaps) / len(gaps) < 0.14
