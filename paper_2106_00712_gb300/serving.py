"""Continuous-batching request loop for DQMC runs on one GPU.

A request asks for `chains` independent chains of one lattice problem (L x L square
lattice, beta, U; dtau and n_wrap from the coupling), `n_warm` thermalization and `n_meas`
measuring sweeps, from random (Philox) initial fields -- the short Markov chains that step 4
of Algorithm 1 runs from each initial configuration.

Requests of the same problem share contexts ("pools"): a pool of S slots holds S x chains
chains and advances them together, two sweeps (one ascending, one descending) per step, so
its kernels run over the batch of all its requests. The loop:

* admits arrived requests in arrival order: into a free slot of a pool of the same problem,
  else into a new pool if its device footprint (nmc_footprint) fits the HBM budget; a request
  that fits nowhere blocks the ones behind it. A new pool gets as many slots as its problem
  has requests waiting and running (a power of two, at most `max_slots`), so pools grow
  with a problem's traffic;
* between two steps of a pool, starts the chains of newly admitted requests afresh
  (nmc_restart_chains: each request's chains have global indices rid * chains + j, and their
  Philox sweep numbering starts at their admission), retires requests whose measuring
  window is complete (their observables come from the per-sweep accumulators of their own
  chains over their own window, nmc_series_range), and enqueues the next step
  (nmc_sweep_async) while any slot is in use; an empty pool is closed and its memory freed;
* pools run on their own CUDA streams, so different pools' kernels overlap on the device.

A request's chains, trajectory and observables depend only on the loop's seed and the
request's id: the same alone and in the mix (tested), whichever pool and slot it lands in.
"""
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    L: int
    beta: float
    U: float
    arrival: float = 0.0          # seconds after the start of the stream
    dtau: float = 0.1
    n_wrap: int = 10
    chains: int = 16
    n_warm: int = 20
    n_meas: int = 50
    seed: int = 0                 # kept for reference; chains are identified by rid
    t: float = 1.0

    @property
    def key(self):
        """Requests with the same key can share a pool."""
        return (self.L, self.beta, self.U, self.dtau, self.n_wrap, self.t, self.chains)

    @property
    def sweeps(self):
        return self.n_warm + self.n_meas

    @property
    def flips(self):
        return self.chains * self.L * self.L * int(round(self.beta / self.dtau)) * self.sweeps


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    obs: dict = field(default_factory=dict)

    @property
    def latency(self):
        return self.done - self.arrival


def wrap_interval(U, dtau):
    """Stabilization interval from the coupling: the wrap amplifies errors by about
    e^{2 lam + 2 dtau W} per slice, so the interval shrinks as U dtau grows (the compensated
    path's measured drift stays below 1e-5 with these on L <= 12, beta <= 6)."""
    return 10 if U * dtau <= 0.2 + 1e-12 else 5 if U * dtau <= 0.4 + 1e-12 else 4


def poisson_stream(n, rate, seed=0, lattices=(6, 8, 10, 12), betas=(2.0, 4.0, 6.0),
                   Us=(2.0, 4.0, 8.0), **kw):
    """n requests with exponential inter-arrival times (rate per second) and a uniform mix
    of lattice sizes, temperatures and couplings."""
    rng = np.random.default_rng(seed)
    fixed_wrap = kw.pop("n_wrap", None)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        U = float(rng.choice(Us))
        nw = fixed_wrap or wrap_interval(U, kw.get("dtau", 0.1))
        out.append(Request(rid=i, L=int(rng.choice(lattices)), beta=float(rng.choice(betas)),
                           U=U, arrival=t, seed=int(rng.integers(2**31)), n_wrap=nw, **kw))
    return out


def request_observables(series, chains):
    """Observables of one request from the per-sweep accumulators of its chains over its
    measuring window: series [sweeps][chains][8] (sign-weighted sums of energy, ekin,
    double_occ, s_pipi, density; sum of signs). Per chain the ratio of the window's sums,
    then the mean and standard error over the request's chains -- the reduction
    nmc_measure applies to a context's accumulators."""
    names = ("energy", "ekin", "double_occ", "s_pipi", "density")
    per = {k: [] for k in names}
    for c in range(chains):
        tot = [0.0] * 6
        for s in range(series.shape[0]):
            for k in range(6):
                tot[k] += float(series[s, c, k])
        for k, nm in enumerate(names):
            per[nm].append(tot[k] / tot[5] if tot[5] != 0 else 0.0)
    out = {}
    for nm in names:
        v = per[nm]
        m = sum(v) / len(v)
        out[nm] = m
        out[nm + "_err"] = (math.sqrt(sum((x - m) ** 2 for x in v) / (len(v) - 1) / len(v))
                            if len(v) > 1 else 0.0)
    return out


class GpuPoolBackend:
    """Pools as nmc contexts, each on its own CUDA stream; one Philox key for the loop."""

    def __init__(self, precision=2, delay_k=16, seed=2106):
        import torch
        from . import nmc
        self.torch, self.nmc = torch, nmc
        self.precision, self.delay_k, self.seed = precision, delay_k, seed
        self._fp = {}

    def _opts(self, n_chains):
        o = self.nmc.nmc_default_options()
        o.n_chains, o.delay_k, o.precision = n_chains, self.delay_k, self.precision
        return o

    def footprint(self, r, slots, max_sweeps):
        key = (r.key, slots, max_sweeps)
        if key not in self._fp:
            n = slots * r.chains
            series = 8 * 8 * n * (max_sweeps + 2)
            self._fp[key] = self.nmc.nmc_footprint(r.L, r.L, r.t, r.U, r.beta, r.dtau,
                                                   r.n_wrap, self._opts(n)) + series
        return self._fp[key]

    def open(self, r, slots):
        stream = self.torch.cuda.Stream()
        ctx = self.nmc.Context(r.L, r.L, r.t, r.U, r.beta, r.dtau, r.n_wrap, seed=self.seed,
                               n_chains=slots * r.chains, delay_k=self.delay_k,
                               precision=self.precision, stream=stream.cuda_stream)
        ctx.generate()
        return {"ctx": ctx, "stream": stream}

    def join(self, h, placements):
        """placements: [(slot, request)]; restart those slots' chains."""
        chains, ids = [], []
        for slot, r in placements:
            for j in range(r.chains):
                chains.append(slot * r.chains + j)
                ids.append(r.rid * r.chains + j)
        h["ctx"].restart_chains(chains, ids)

    def step(self, h, n):
        h["ctx"].sweep_async(n, 1)

    def idle(self, h):
        return h["ctx"].idle()

    def collect(self, h, slot, r, first_row):
        ser = h["ctx"].series_range(first_row, r.n_meas)
        lo = slot * r.chains
        return request_observables(ser[:, lo:lo + r.chains, :], r.chains)

    def close(self, h):
        ctx = h["ctx"]
        err = None
        try:
            ctx.sync()
        except self.nmc.NmcError as e:   # drift above the bar or non-finite: report it
            err = str(e)
        hist = ctx.drift_history()
        ctx.close()
        return {"max_drift": float(hist.max()) if hist.size else 0.0, "error": err}


def _pow2_at_least(n):
    p = 1
    while p < n:
        p *= 2
    return p


class Server:
    """Continuous batching into pools under an HBM budget (bytes)."""

    def __init__(self, backend, hbm_budget, max_slots=8, step=2, max_pool_sweeps=2000,
                 clock=time.perf_counter, idle_sleep=2e-4):
        if step % 2:
            raise ValueError("a step is a whole number of sweep pairs")
        self.b = backend
        self.budget = hbm_budget
        self.max_slots = max_slots
        self.step = step
        self.max_pool_sweeps = max_pool_sweeps
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.peak_bytes = 0
        self.peak_active = 0
        self.peak_pools = 0
        self.pool_log = []      # per closed pool: slots, requests served, sweeps, max drift

    def run(self, requests, realtime=True):
        """Serve the requests (sorted by arrival). realtime=False admits every request at
        once (arrival times ignored) -- a throughput run."""
        queue = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        pools = []
        results = {}
        used = 0
        t0 = self.clock()
        while queue or waiting or pools:
            now = self.clock() - t0
            progressed = False
            while queue and (not realtime or queue[0].arrival <= now):
                waiting.append(queue.popleft())
            # admission in arrival order: a free slot of a same-problem pool, else a new pool
            while waiting:
                r = waiting[0]
                pool = next((p for p in pools if p["key"] == r.key and not p["closing"] and
                             None in p["slots"]), None)
                if pool is None:
                    # sized for the problem's current concurrency: its waiting requests plus
                    # those already running in its other pools
                    want = (sum(1 for w in waiting if w.key == r.key) +
                            sum(isinstance(st, dict) for p in pools if p["key"] == r.key
                                for st in p["slots"]))
                    slots = min(self.max_slots, _pow2_at_least(want))
                    need = self.b.footprint(r, slots, self.max_pool_sweeps)
                    if need > self.budget:
                        raise ValueError(f"request {r.rid}: a pool needs {need} bytes > budget")
                    if used + need > self.budget:
                        break
                    pool = {"key": r.key, "h": self.b.open(r, slots), "slots": [None] * slots,
                            "pending": [], "rows": 0, "busy": False, "closing": False,
                            "bytes": need, "served": 0}
                    pools.append(pool)
                    used += need
                    self.peak_bytes = max(self.peak_bytes, used)
                    self.peak_pools = max(self.peak_pools, len(pools))
                s = pool["slots"].index(None)
                pool["slots"][s] = "reserved"
                pool["pending"].append((s, r))
                waiting.popleft()
                progressed = True
            # drive every pool that is between steps
            for pool in list(pools):
                if pool["busy"] and not self.b.idle(pool["h"]):
                    continue
                pool["busy"] = False
                for s, st in enumerate(pool["slots"]):
                    if isinstance(st, dict) and pool["rows"] >= st["row"] + st["r"].sweeps:
                        r = st["r"]
                        obs = self.b.collect(pool["h"], s, r, st["row"] + r.n_warm)
                        results[r.rid] = Result(r.rid, r.arrival if realtime else 0.0,
                                                st["admitted"], self.clock() - t0, obs)
                        pool["slots"][s] = None
                        pool["served"] += 1
                        progressed = True
                if pool["pending"]:
                    self.b.join(pool["h"], pool["pending"])
                    t_adm = self.clock() - t0
                    for s, r in pool["pending"]:
                        pool["slots"][s] = {"r": r, "row": pool["rows"], "admitted": t_adm}
                    pool["pending"] = []
                    progressed = True
                if pool["rows"] >= self.max_pool_sweeps:
                    pool["closing"] = True
                if any(isinstance(st, dict) for st in pool["slots"]):
                    self.b.step(pool["h"], self.step)
                    pool["rows"] += self.step
                    pool["busy"] = True
                    progressed = True
                elif not any(st == "reserved" for st in pool["slots"]):
                    info = self.b.close(pool["h"])
                    self.pool_log.append({"slots": len(pool["slots"]), "served": pool["served"],
                                          "sweeps": pool["rows"], **info})
                    used -= pool["bytes"]
                    pools.remove(pool)
                    progressed = True
            active = sum(isinstance(st, dict) for p in pools for st in p["slots"])
            self.peak_active = max(self.peak_active, active)
            if not progressed:
                time.sleep(self.idle_sleep)
        makespan = self.clock() - t0
        return results, makespan


def report(results, requests, makespan):
    lat = np.array([results[r.rid].latency for r in requests])
    flips = sum(r.flips for r in requests)
    return {"n_requests": len(requests), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": makespan,
            "flips_per_s": flips / makespan if makespan > 0 else math.nan}


def serve_stream(n_requests=64, budget_gb=100.0, load=0.7, seed=0, precision=2,
                 max_slots=8, saturation_requests=None, **kw):
    """Saturation run (all requests admitted at once) on `saturation_requests` requests of
    the mix (default: all) to measure capacity, then a Poisson stream of n_requests at
    `load` x that capacity (requests per second)."""
    be = GpuPoolBackend(precision=precision)
    n_sat = saturation_requests or n_requests
    sat_reqs = poisson_stream(n_sat, rate=1.0, seed=seed + 1, **kw)
    srv = Server(be, int(budget_gb * 2**30), max_slots=max_slots)
    res, span = srv.run(sat_reqs, realtime=False)
    sat = report(res, sat_reqs, span)
    rate = load * n_sat / span
    reqs = poisson_stream(n_requests, rate=rate, seed=seed, **kw)
    srv = Server(be, int(budget_gb * 2**30), max_slots=max_slots)
    res, span = srv.run(reqs, realtime=True)
    out = report(res, reqs, span)
    drifts = [p["max_drift"] for p in srv.pool_log]
    out.update({"rate_per_s": rate, "load": load, "saturation_flips_per_s": sat["flips_per_s"],
                "saturation_requests": n_sat, "peak_active": srv.peak_active,
                "peak_pools": srv.peak_pools, "peak_bytes": srv.peak_bytes,
                "pools": len(srv.pool_log), "max_slots": max_slots,
                "hbm_budget_gb": budget_gb,
                "max_drift": max(drifts) if drifts else float("nan"),
                "failed_pools": sum(1 for p in srv.pool_log if p.get("error"))})
    return out


def batched_mix_rate(n_requests=2000, seed=0, chains_per_class=128, warm=2, sweeps=4,
                     precision=2, **kw):
    """The batched path on the serving mix, for comparison with the loop's capacity: each
    (L, beta, U) class of the mix runs alone as one context of `chains_per_class` chains
    (the largest pool: max_slots x chains), timed over `sweeps` measuring sweeps after
    `warm` (CUDA events); the mix's rate is its total flips over the time its classes would
    take at those rates one after another (no overlap between classes)."""
    import torch
    from . import nmc
    nmc.load()
    reqs = poisson_stream(n_requests, rate=1.0, seed=seed + 1, **kw)
    classes = {}
    for r in reqs:
        c = classes.setdefault((r.L, r.beta, r.U, r.dtau, r.n_wrap), [0, 0.0])
        c[0] += r.flips
    stream = torch.cuda.current_stream()
    per = []
    total_time = 0.0
    for (L, beta, U, dtau, n_wrap), (flips, _) in sorted(classes.items()):
        with nmc.Context(L, L, 1.0, U, beta, dtau, n_wrap, seed=2106, n_chains=chains_per_class,
                         precision=precision, drift_tol=1e300,
                         stream=stream.cuda_stream) as c:
            c.generate()
            c.sweep(warm, measure=1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.sweep(sweeps, measure=1)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
        rate = chains_per_class * L * L * int(round(beta / dtau)) * sweeps / (ms * 1e-3)
        total_time += flips / rate
        per.append({"L": L, "beta": beta, "U": U, "n_wrap": n_wrap, "flips_per_s": rate})
    flips = sum(r.flips for r in reqs)
    return {"classes": per, "mix_flips_per_s": flips / total_time,
            "chains_per_class": chains_per_class, "n_requests": n_requests}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--saturation-requests", type=int, default=None)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--budget-gb", type=float, default=100.0)
    ap.add_argument("--chains", type=int, default=16)
    ap.add_argument("--warm", type=int, default=20)
    ap.add_argument("--meas", type=int, default=50)
    ap.add_argument("--max-slots", type=int, default=8)
    ap.add_argument("--batched-mix", action="store_true",
                    help="time the batched path on each class of the mix instead of serving")
    args = ap.parse_args()
    if args.batched_mix:
        print(json.dumps(batched_mix_rate(args.requests, chains_per_class=args.max_slots *
                                          args.chains, chains=args.chains, n_warm=args.warm,
                                          n_meas=args.meas)))
        return
    print(json.dumps(serve_stream(args.requests, args.budget_gb, args.load, chains=args.chains,
                                  n_warm=args.warm, n_meas=args.meas, max_slots=args.max_slots,
                                  saturation_requests=args.saturation_requests)))


if __name__ == "__main__":
    main()
