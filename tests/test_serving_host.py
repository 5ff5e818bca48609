"""Host logic of the continuous-batching loop, on the CPU with a fake backend and a
virtual clock: admission in arrival order under the HBM budget, work kept in flight for
every active request, completion and the latency report."""
import pytest

from paper_2106_00712_gb300.serving import Request, Server, poisson_stream, report


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances virtual time
        return self.t


class FakeBackend:
    """A request costs `cost` virtual seconds per sweep; footprint = L^4 bytes."""

    def __init__(self, clock, cost=1e-3):
        self.clock, self.cost = clock, cost
        self.in_use = 0
        self.max_in_use = 0
        self.concurrent = 0
        self.max_concurrent = 0

    def footprint(self, r):
        return r.L ** 4

    def start(self, r):
        self.in_use += self.footprint(r)
        self.max_in_use = max(self.max_in_use, self.in_use)
        return {"r": r, "busy_until": 0.0, "sweeps": 0}

    def enqueue(self, h, n, measure):
        h["busy_until"] = self.clock.t + n * self.cost
        h["sweeps"] += n

    def idle(self, h):
        return self.clock.t >= h["busy_until"]

    def finish(self, h):
        r = h["r"]
        self.in_use -= self.footprint(r)
        assert h["sweeps"] == r.n_warm + r.n_meas
        return {"energy": -1.0 - 0.01 * r.seed % 7}


def test_admission_respects_budget_and_everything_completes():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = poisson_stream(40, rate=200.0, seed=3, lattices=(4, 6, 8), chains=2, n_warm=3,
                          n_meas=4)
    budget = 3 * 8 ** 4
    srv = Server(be, budget, chunk=2, clock=clock, idle_sleep=0.0)
    results, makespan = srv.run(reqs)
    assert set(results) == {r.rid for r in reqs}
    assert be.max_in_use <= budget
    assert srv.peak_active >= 2                 # several requests in flight at once
    for r in reqs:
        res = results[r.rid]
        assert res.admitted >= r.arrival - 1e-9
        assert res.done - res.admitted >= (r.n_warm + r.n_meas) * be.cost - 1e-9
    rep = report(results, reqs, makespan)
    assert rep["p50_latency_s"] <= rep["p99_latency_s"]
    assert rep["n_requests"] == 40


def test_oversize_request_is_rejected():
    clock = FakeClock()
    srv = Server(FakeBackend(clock), 100, clock=clock, idle_sleep=0.0)
    with pytest.raises(ValueError):
        srv.run([Request(0, 8, 1.0, 4.0)])


def test_poisson_stream_is_seeded_and_mixed():
    a = poisson_stream(200, rate=10.0, seed=1)
    b = poisson_stream(200, rate=10.0, seed=1)
    assert [(r.L, r.beta, r.U, r.seed, r.arrival) for r in a] == \
           [(r.L, r.beta, r.U, r.seed, r.arrival) for r in b]
    assert {r.L for r in a} == {6, 8, 10, 12}
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert 0.07 < sum(gaps) / len(gaps) < 0.14
