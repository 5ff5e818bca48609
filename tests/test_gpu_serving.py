"""Continuous batching on the GPU: requests packed into shared pools give each request the
result it gets alone.

Library level: chains started afresh inside a running context (nmc_restart_chains) follow
exactly the trajectory of the same global chains in a fresh context -- and the oracle's --
while the other chains of the context continue undisturbed. Serving level: eight requests
(three sharing a problem) run (a) one at a time and (b) together through the pooled loop;
every request's observables agree exactly, whichever pool and slot it landed in."""
import numpy as np
import pytest

from oracle.dqmc import Chain, Model, initial_fields
from paper_2106_00712_gb300.serving import GpuPoolBackend, Request, Server, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def backend():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return GpuPoolBackend(precision=2)


@pytest.mark.parametrize("prec", [0, 2])
def test_restarted_chains_follow_fresh_chains(backend, prec):
    from paper_2106_00712_gb300 import nmc
    model = Model(4, 4, 1.0, 4.0, 1.0, 0.1, 5, seed=77)

    def ctx(n):
        c = nmc.Context(4, 4, 1.0, 4.0, 1.0, 0.1, 5, seed=77, n_chains=n, precision=prec)
        c.generate()
        return c

    with ctx(4) as a, ctx(2) as b, ctx(4) as c:
        a.sweep(4, measure=1)
        with pytest.raises(nmc.NmcError):     # only between sweep pairs
            a.sweep(1, measure=1)
            a.restart_chains([1], [9])
        a.sweep(1, measure=1)                 # back to an even phase (6 sweeps)
        a.restart_chains([1, 2], [50, 51])
        b.restart_chains([0, 1], [50, 51])
        a.sweep(4, measure=1)
        b.sweep(4, measure=1)
        c.sweep(10, measure=1)
        fa, fb, fc = a.fields(), b.fields(), c.fields()
        np.testing.assert_array_equal(fa[1:3], fb)            # restarted = fresh
        np.testing.assert_array_equal(fa[[0, 3]], fc[[0, 3]])  # the others undisturbed
        for k in range(2):
            for sp in (0, 1):
                np.testing.assert_array_equal(a.green(1 + k, sp), b.green(k, sp))
        np.testing.assert_array_equal(a.series_range(6, 4)[:, 1:3], b.series_range(0, 4))
        np.testing.assert_array_equal(a.green(3, 1), c.green(3, 1))
        # the fresh global chains are the oracle's chains 50 and 51
        for k, gid in enumerate((50, 51)):
            ref = Chain(model, initial_fields(model, gid), gid)
            for _ in range(4):
                ref.sweep(True)
            np.testing.assert_array_equal(fb[k], ref.s)


def _requests():
    mix = [(4, 1.0, 2.0), (6, 2.0, 4.0), (4, 1.0, 2.0), (8, 1.0, 8.0), (6, 1.0, 2.0),
           (4, 1.0, 2.0), (10, 1.0, 4.0), (6, 2.0, 8.0)]
    return [Request(i, L, b, U, arrival=0.002 * i, chains=4, n_warm=2, n_meas=4, n_wrap=5)
            for i, (L, b, U) in enumerate(mix)]


def test_results_same_alone_and_in_the_mix(backend):
    reqs = _requests()
    alone = {}
    for r in reqs:
        srv = Server(backend, hbm_budget=1 << 40, max_slots=4)
        res, _ = srv.run([r], realtime=False)
        alone[r.rid] = res[r.rid].obs
    srv = Server(backend, hbm_budget=1 << 40, max_slots=4)
    mixed, makespan = srv.run(reqs, realtime=False)
    assert srv.peak_active >= 4
    assert max(p["served"] for p in srv.pool_log) >= 3     # the three 4x4 requests share a pool
    for r in reqs:
        for k in ("energy", "double_occ", "s_pipi", "density"):
            assert mixed[r.rid].obs[k] == alone[r.rid][k], (r.rid, k)
    assert max(p["max_drift"] for p in srv.pool_log) <= 1e-5
    rep = report(mixed, reqs, makespan)
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0


def test_budget_limits_pools(backend):
    reqs = [Request(i, 6, 1.0, 4.0, chains=4, n_warm=1, n_meas=3, n_wrap=5) for i in range(4)]
    one = backend.footprint(reqs[0], 1, 2000)
    srv = Server(backend, hbm_budget=one, max_slots=1)
    res, _ = srv.run(reqs, realtime=False)
    assert srv.peak_pools == 1 and len(res) == 4


def test_concurrent_contexts_match_alone_large_lattices(backend):
    """Eight contexts of N = 100 and N = 144 (G in global memory in the flip kernel, QR and
    solve workspaces in global memory) advancing together on separate streams, three times:
    every result equals the context run alone. Concurrent kernels on the same SMs shift warp
    timing, which is what exposed a barrier race in the flip kernels' accept flag."""
    import torch
    from paper_2106_00712_gb300 import nmc

    def mk(L, seed, stream=None):
        c = nmc.Context(L, L, 1.0, 4.0, 2.0, 0.1, 5, seed=seed, n_chains=4, precision=2,
                        drift_tol=1e300, stream=stream.cuda_stream if stream else None)
        c.generate()
        return c

    def done(c):
        c.sync()
        e = c.measure().energy.mean
        c.close()
        return e

    sizes = [10, 12] * 4
    ref = []
    for k, L in enumerate(sizes):
        c = mk(L, 100 + k)
        c.sweep(2, 0)
        c.sweep(3, 1)
        ref.append(done(c))
    for _ in range(3):
        ctxs = [mk(L, 100 + k, torch.cuda.Stream()) for k, L in enumerate(sizes)]
        left = [[2, 3] for _ in sizes]
        while any(a or b for a, b in left):
            for k, c in enumerate(ctxs):
                if (left[k][0] or left[k][1]) and c.idle():
                    meas = 0 if left[k][0] else 1
                    c.sweep_async(1, meas)
                    left[k][meas] -= 1
        got = [done(c) for c in ctxs]
        assert all(abs(a - b) < 1e-12 for a, b in zip(ref, got)), (ref, got)
