"""Network-initialized Monte Carlo end to end on the paper's Hubbard point (Algorithm 1;
Table 2: honeycomb L = 6, 72 sites, U/t = 3.83, beta = 6, dtau = 0.1).

1. Training samples: n_train chains from random fields run n_short sweeps (unthermalized);
   per configuration S(Gamma) and E_k at slice 0 (nmc_gen_observables).
2. Train the generator of SM Sec. II on those observables with the Eq. 4 loss (Adam,
   lr 1e-3, batch 3, 15 epochs as in SM Sec. II; weights = inverse target variances).
3. Generate n_gen configurations (input stream 1): "NN" values measured directly on
   x = 2p - 1, and Bernoulli +-1 fields for the chains.
4. DQMC chains from the generated fields (NIMC), from random fields and from the training
   configurations: per-sweep E_k and S(Gamma) over chains (nmc_series).

The chains run in FP64 (particle-hole single spin) with n_wrap = 5: generated
configurations can be more ordered than random or Markov-chain ones, and at n_wrap = 10
their stabilization drift exceeded the bars (1e-5 compensated FP32, 1e-6 FP64). Training
bounds each step's gradient norm (clip = 1): single-configuration estimators are
unbounded, and without a bound one configuration's gradient (norm > 1e19) overflowed
Adam's second moment and froze the generator.

Usage: python -m paper_2106_00712_gb300.nimc_run [--train 1000] [--short 10] [--epochs 15]
       [--batch 3] [--gen 1000] [--sweeps 60]
Prints one JSON object.
"""
import argparse
import json
import sys
import time

import numpy as np

from . import nmc
from .workloads import HONEYCOMB_6x6

# long-run reference of the same library (1024 chains, 200 + 200 sweeps, FP32X2 ph)
REFERENCE = {"ekin": (-1.35713, 0.00013), "s_gamma": (0.71756, 0.00299)}


def _log(out, *keys):
    print(json.dumps({k: out[k] for k in keys}), file=sys.stderr, flush=True)


def _stat(v):
    v = np.asarray(v, dtype=np.float64)
    return [float(v.mean()), float(v.std(ddof=1) / np.sqrt(len(v)))]


def _ctx(wl, chains, seed, precision, ph):
    return nmc.Context(wl.Lx, wl.Ly, wl.t, wl.U, wl.beta, wl.dtau, wl.n_wrap, seed=seed,
                       n_chains=chains, delay_k=wl.delay_k, precision=precision,
                       ph_symmetric=ph, lattice=wl.lattice)


def _curve(ctx, sweeps):
    ctx.sweep(sweeps, measure=1)
    ser = ctx.series()                      # [sweeps][chains][5]
    return {"ekin": [_stat(ser[k, :, 1]) for k in range(ser.shape[0])],
            "s_gamma": [_stat(ser[k, :, 3]) for k in range(ser.shape[0])]}


def _converged_at(curve, key, ref, nsig=2.0):
    """First sweep from which every later per-sweep mean is within nsig combined errors."""
    m = np.array([c[0] for c in curve[key]])
    e = np.array([c[1] for c in curve[key]])
    ok = np.abs(m - ref[0]) <= nsig * np.sqrt(e * e + ref[1] ** 2)
    for k in range(len(ok)):
        if ok[k:].all():
            return k + 1
    return None


def run(n_train=1000, n_short=10, epochs=15, batch=3, lr=1e-3, n_gen=1000, sweeps=60,
        precision=nmc.NMC_FP64, ph=1, wl=HONEYCOMB_6x6.with_(n_wrap=5), seed=2106, clip=1.0):
    import torch
    out = {"workload": "hubbard-honeycomb-L6-U3.83-beta6", "n_train": n_train,
           "n_short": n_short, "epochs": epochs, "batch": batch, "lr": lr, "n_gen": n_gen,
           "sweeps": sweeps, "n_wrap": wl.n_wrap, "clip": clip}
    t0 = time.perf_counter()
    # 1. training samples
    with _ctx(wl, n_train, seed + 1, precision, ph) as c:
        c.generate()
        c.sweep(n_short, measure=0)
        train_fields = c.fields()
    gen = nmc.Generator(wl.Lx, wl.Ly, wl.t, wl.U, wl.beta, wl.dtau, wl.n_wrap, seed=seed,
                        max_batch=64, lattice=wl.lattice)
    gen.set_clip(clip)
    d_x = torch.from_numpy(train_fields.astype(np.float64)).cuda()
    d_o = torch.empty((n_train, 2), dtype=torch.float64, device="cuda")
    gen.observables(d_x.data_ptr(), n_train, d_o.data_ptr())
    targets = d_o.cpu().numpy()
    del d_x
    out["train"] = {"s_gamma": _stat(targets[:, 0]), "ekin": _stat(targets[:, 1])}
    out["t_samples_s"] = time.perf_counter() - t0
    _log(out, "train")
    # 2. training
    t1 = time.perf_counter()
    d_o0 = torch.empty((n_gen, 2), dtype=torch.float64, device="cuda")
    gen.generated_observables(0, n_gen, 1, d_o0.data_ptr())
    nn0 = d_o0.cpu().numpy()
    out["nn_untrained"] = {"s_gamma": _stat(nn0[:, 0]), "ekin": _stat(nn0[:, 1])}
    hist = gen.train(targets, epochs=epochs, batch=batch, lr=lr)
    out["epoch_loss"] = [float(v) for v in hist]
    out["t_train_s"] = time.perf_counter() - t1
    out["adam_steps"] = int(gen.steps())
    _log(out, "epoch_loss", "t_train_s", "nn_untrained")
    # 3. generated configurations measured directly
    gen.generated_observables(0, n_gen, 1, d_o0.data_ptr())
    nn = d_o0.cpu().numpy()
    out["nn"] = {"s_gamma": _stat(nn[:, 0]), "ekin": _stat(nn[:, 1])}
    _log(out, "nn")
    # 4. chains from generated, random and training configurations
    t2 = time.perf_counter()
    curves = {}
    with _ctx(wl, n_gen, seed + 2, precision, ph) as c:
        c.generate(mode=1, model=gen)
        curves["nimc"] = _curve(c, sweeps)
    with _ctx(wl, n_gen, seed + 3, precision, ph) as c:
        c.generate()
        curves["random"] = _curve(c, sweeps)
    with _ctx(wl, min(n_gen, n_train), seed + 4, precision, ph) as c:
        c.set_fields(train_fields[:min(n_gen, n_train)])
        curves["train"] = _curve(c, sweeps)
    gen.close()
    out["t_chains_s"] = time.perf_counter() - t2
    out["reference"] = REFERENCE
    out["converged_at_sweep"] = {
        k: {key: _converged_at(v, key, REFERENCE[key]) for key in ("ekin", "s_gamma")}
        for k, v in curves.items()}
    out["curves"] = curves
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1000)
    ap.add_argument("--short", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=15)
    ap.add_argument("--batch", type=int, default=3)
    ap.add_argument("--gen", type=int, default=1000)
    ap.add_argument("--sweeps", type=int, default=60)
    ap.add_argument("--clip", type=float, default=1.0)
    a = ap.parse_args()
    print(json.dumps(run(a.train, a.short, a.epochs, a.batch, n_gen=a.gen, sweeps=a.sweeps,
                         clip=a.clip)))


if __name__ == "__main__":
    main()
