"""Network-initialized Monte Carlo end to end (Algorithm 1).

1. Training samples: n_train chains from random fields run n_short sweeps (unthermalized);
   per configuration the observables at slice 0 (nmc_gen_observables): S (S(Gamma) on the
   honeycomb, S(pi,pi) on the square lattice) and E_k.
2. Train the generator (SM Sec. II structure) on those observables with the Eq. 4 loss
   (Adam, lr 1e-3, batch 3, 15 epochs as in SM Sec. II; weights = inverse target variances).
3. Generate n_gen configurations (input stream 1): "NN" values measured directly on
   x = 2p - 1, and Bernoulli +-1 fields for the chains.
4. DQMC chains from the generated fields (NIMC), from random fields and from the training
   configurations: per-sweep means over chains of E, E_k, D and S (nmc_series), and the
   first sweep from which each stays at equilibrium.

Workloads: "honeycomb" -- the paper's Hubbard point (Table 2: L = 6, 72 sites, U/t = 3.83,
beta = 6, dtau = 0.1) with the paper's network (10x2x2 -> 20 x 16x6x3 -> 36x6x3); "square8" --
the 8x8 square lattice at U = 4, beta = 4 (L_tau = 40) with a network of the same structure
sized to 40x8x8 (10x2x2 -> 20 x 11x4x4 -> 21x4x4); convergence of energy and double occupancy.
The equilibrium reference is the paper's printed values for the honeycomb (our long run) and
a long run of random starts (200 + 200 sweeps) for the square lattice.

Convergence criterion (the paper gives none in numbers): the first sweep s whose mean over
chains is within 1 combined standard error of the reference while every later sweep stays
within 3.

The chains run in FP64 (particle-hole single spin) with n_wrap = 5: generated
configurations can be more ordered than random or Markov-chain ones, and at n_wrap = 10
their stabilization drift exceeded the bars (1e-5 compensated FP32, 1e-6 FP64). Training
bounds each step's gradient norm (clip = 1): single-configuration estimators are
unbounded, and without a bound one configuration's gradient (norm > 1e19) overflowed
Adam's second moment and froze the generator.

"square8-ml" -- the convolutional generator of include/nmc_cgen.h on the same 8x8 lattice,
trained by maximum likelihood on 20000 DQMC fields (one every 10 sweeps), judged the same way
(run_ml).

Usage: python -m paper_2106_00712_gb300.nimc_run [--workload honeycomb|square8|square8-ml]
       [--train 1000] [--short 10] [--epochs 15] [--batch 3] [--gen N] [--sweeps 60]
Prints one JSON object.
"""
import argparse
import json
import sys
import time

import numpy as np

from . import nmc
from .workloads import HONEYCOMB_6x6, SQUARE_8x8

KEYS = ("energy", "ekin", "double_occ", "s_pipi")   # nmc_series columns 0..3

WORKLOADS = {
    "honeycomb": dict(wl=HONEYCOMB_6x6.with_(n_wrap=5), arch=None, n_gen=1000,
                      # library long run (1024 chains, 200 + 200 sweeps, FP32X2 ph)
                      reference={"ekin": (-1.35713, 0.00013), "s_pipi": (0.71756, 0.00299)},
                      converge_on=("ekin", "s_pipi")),
    "square8": dict(wl=SQUARE_8x8.with_(n_wrap=5), arch=dict(k1=(11, 4, 4), k2=(21, 4, 4)),
                    n_gen=4096, reference=None, converge_on=("energy", "double_occ")),
}


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
    return {k: [_stat(ser[s, :, i]) for s in range(ser.shape[0])] for i, k in enumerate(KEYS)}


def _converged_at(curve, key, ref):
    m = np.array([c[0] for c in curve[key]])
    e = np.array([c[1] for c in curve[key]])
    z = np.abs(m - ref[0]) / np.sqrt(e * e + ref[1] ** 2)
    for k in range(len(z)):
        if z[k] <= 1.0 and np.all(z[k:] <= 3.0):
            return k + 1
    return None


def _reference(wl, seed, precision, ph, chains=1024, warm=200, meas=200):
    with _ctx(wl, chains, seed, precision, ph) as c:
        c.generate()
        c.sweep(warm, measure=0)
        c.sweep(meas, measure=1)
        o = c.measure()
    return {k: (getattr(o, k).mean, getattr(o, k).err) for k in KEYS}


def run(workload="honeycomb", n_train=1000, n_short=10, epochs=15, batch=3, lr=1e-3,
        n_gen=None, sweeps=60, precision=nmc.NMC_FP64, ph=1, seed=2106, clip=1.0):
    import torch
    spec = WORKLOADS[workload]
    wl = spec["wl"]
    n_gen = n_gen or spec["n_gen"]
    out = {"workload": workload, "lattice": f"{wl.lattice} {wl.Lx}x{wl.Ly}", "U": wl.U,
           "beta": wl.beta, "dtau": wl.dtau, "n_train": n_train, "n_short": n_short,
           "epochs": epochs, "batch": batch, "lr": lr, "n_gen": n_gen, "sweeps": sweeps,
           "n_wrap": wl.n_wrap, "clip": clip}
    t0 = time.perf_counter()
    # 1. training samples
    with _ctx(wl, n_train, seed + 1, precision, ph) as c:
        c.generate()
        c.sweep(n_short, measure=0)
        train_fields = c.fields()
    arch = nmc.gen_arch(**spec["arch"]) if spec["arch"] else nmc.gen_arch()
    out["arch"] = {"z": list(arch.z), "c1": arch.c1, "k1": list(arch.k1), "k2": list(arch.k2)}
    gen = nmc.Generator(wl.Lx, wl.Ly, wl.t, wl.U, wl.beta, wl.dtau, wl.n_wrap, arch=arch,
                        seed=seed, max_batch=64, lattice=wl.lattice)
    gen.set_clip(clip)
    d_x = torch.from_numpy(train_fields.astype(np.float64)).cuda()
    d_o = torch.empty((n_train, 2), dtype=torch.float64, device="cuda")
    gen.observables(d_x.data_ptr(), n_train, d_o.data_ptr())
    targets = d_o.cpu().numpy()
    del d_x
    out["train"] = {"s_pipi": _stat(targets[:, 0]), "ekin": _stat(targets[:, 1])}
    out["t_samples_s"] = time.perf_counter() - t0
    _log(out, "train")
    # 2. training
    t1 = time.perf_counter()
    d_o0 = torch.empty((n_gen, 2), dtype=torch.float64, device="cuda")
    gen.generated_observables(0, n_gen, 1, d_o0.data_ptr())
    nn0 = d_o0.cpu().numpy()
    out["nn_untrained"] = {"s_pipi": _stat(nn0[:, 0]), "ekin": _stat(nn0[:, 1])}
    hist = gen.train(targets, epochs=epochs, batch=batch, lr=lr)
    out["epoch_loss"] = [float(v) for v in hist]
    out["t_train_s"] = time.perf_counter() - t1
    out["adam_steps"] = int(gen.steps())
    _log(out, "epoch_loss", "t_train_s", "nn_untrained")
    # 3. generated configurations measured directly
    gen.generated_observables(0, n_gen, 1, d_o0.data_ptr())
    nn = d_o0.cpu().numpy()
    out["nn"] = {"s_pipi": _stat(nn[:, 0]), "ekin": _stat(nn[:, 1])}
    _log(out, "nn")
    # reference
    t2 = time.perf_counter()
    ref = spec["reference"] or _reference(wl, seed + 5, precision, ph)
    out["reference"] = ref
    # 4. chains from generated, random and training configurations
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
    out["converged_at_sweep"] = {
        k: {key: _converged_at(v, key, ref[key]) for key in spec["converge_on"] if key in ref}
        for k, v in curves.items()}
    out["curves"] = curves
    return out


def run_ml(n_fields=20000, every=10, warm=100, chains=256, channels=32, epochs=3, batch=64,
           lr=1e-3, n_gen=4096, sweeps=60, precision=nmc.NMC_FP64, ph=1, seed=2106):
    """The convolutional generator (include/nmc_cgen.h) on the 8x8 lattice at U = 4, beta = 4
    (fields of shape L_tau x 8 x 8 = 40 x 8 x 8):
    1. training fields: `chains` DQMC chains (SPLIT_BF16) from random fields, `warm` sweeps,
       then one field per chain every `every` sweeps until n_fields are collected;
    2. maximum-likelihood training (Adam, lr, batches of `batch` fields with fresh noise);
    3. the thermalization test: n_gen chains from generated fields and n_gen from random
       fields, per-sweep means of E and D, and the first sweep from which each stays at
       equilibrium (the reference: a long run of random starts).
    With noise independent of the fields the likelihood's optimum is a constant logit per
    entry, the log-odds of its mean occupation (oracle.cgen.optimal_bias), so the test is
    expected to find generated starts no better than random ones; the run measures it, with
    a second set of random starts (another seed) to show how far the convergence sweep moves
    between two draws of one start distribution."""
    import torch
    wl = SQUARE_8x8.with_(n_wrap=5)
    out = {"workload": "square8-ml", "lattice": f"{wl.lattice} {wl.Lx}x{wl.Ly}", "U": wl.U,
           "beta": wl.beta, "L_tau": wl.L_tau, "n_fields": n_fields, "every": every,
           "warm": warm, "chains": chains, "channels": channels, "epochs": epochs,
           "batch": batch, "lr": lr, "n_gen": n_gen, "sweeps": sweeps}
    t0 = time.perf_counter()
    fields = []
    with _ctx(wl, chains, seed + 11, nmc.NMC_SPLIT_BF16, 0) as c:
        c.generate()
        c.sweep(warm, measure=0)
        while sum(len(f) for f in fields) < n_fields:
            c.sweep(every, measure=0)
            fields.append(c.fields())
    data = np.concatenate(fields)[:n_fields]                  # [n][L_tau][N], +-1
    out["data_mean_occupation"] = float(((1 + data) / 2).mean())
    out["t_fields_s"] = time.perf_counter() - t0
    _log(out, "data_mean_occupation", "t_fields_s")
    t1 = time.perf_counter()
    rng = np.random.default_rng(seed)
    gen = nmc.ConvGenerator(wl.Lx, wl.Ly, wl.L_tau, channels=channels, seed=seed,
                            max_batch=batch)
    d_data = torch.from_numpy(data.astype(np.int8)).cuda()
    epoch_loss, sample = [], 0
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(n_fields)).cuda()
        tot, cnt = 0.0, 0
        for k in range(0, n_fields - batch + 1, batch):
            xb = d_data[order[k:k + batch]].contiguous()
            tot += gen.train_step(xb.data_ptr(), batch, sample, lr)
            sample += batch
            cnt += 1
        epoch_loss.append(tot / cnt)
    out["epoch_loss"] = epoch_loss
    y = out["data_mean_occupation"]
    out["loss_at_ml_optimum"] = float(-(y * np.log(y) + (1 - y) * np.log(1 - y)))
    out["t_train_s"] = time.perf_counter() - t1
    _log(out, "epoch_loss", "loss_at_ml_optimum", "t_train_s")
    # generated fields
    d_gen = torch.empty((n_gen, wl.L_tau, wl.N), dtype=torch.int8, device="cuda")
    d_log = torch.empty((batch, wl.L_tau, wl.N), dtype=torch.float32, device="cuda")
    lstats = []
    for k in range(0, n_gen, batch):
        m = min(batch, n_gen - k)
        gen.sample(k, m, d_gen[k:k + m].data_ptr(), d_log.data_ptr())
        lstats.append(d_log[:m].double().cpu().numpy())
    lg = np.concatenate(lstats)
    out["generated"] = {"mean_occupation": float(((1 + d_gen.double()) / 2).mean().item()),
                        "logit_mean": float(lg.mean()), "logit_std_over_noise": float(
                            lg.std(axis=0).mean()), "logit_std_over_entries": float(
                            lg.mean(axis=0).std())}
    gen.close()
    _log(out, "generated")
    t2 = time.perf_counter()
    ref = _reference(wl, seed + 5, precision, ph)
    out["reference"] = ref
    torch.cuda.synchronize()
    curves = {}
    with _ctx(wl, n_gen, seed + 2, precision, ph) as c:
        nmc.nmc_set_fields_device(c.ctx, d_gen.data_ptr(), d_gen.numel())
        curves["generated"] = _curve(c, sweeps)
    with _ctx(wl, n_gen, seed + 3, precision, ph) as c:
        c.generate()
        curves["random"] = _curve(c, sweeps)
    # a second, independent set of random starts: the spread of the convergence sweep
    # between two draws of the same start distribution
    with _ctx(wl, n_gen, seed + 4, precision, ph) as c:
        c.generate()
        curves["random_2"] = _curve(c, sweeps)
    out["t_chains_s"] = time.perf_counter() - t2
    out["converged_at_sweep"] = {
        k: {key: _converged_at(v, key, ref[key]) for key in ("energy", "double_occ")}
        for k, v in curves.items()}
    out["first_sweep"] = {k: {key: v[key][0] for key in ("energy", "double_occ")}
                          for k, v in curves.items()}
    out["curves"] = curves
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="honeycomb", choices=sorted(WORKLOADS) + ["square8-ml"])
    ap.add_argument("--train", type=int, default=1000)
    ap.add_argument("--short", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=15)
    ap.add_argument("--batch", type=int, default=3)
    ap.add_argument("--gen", type=int, default=None)
    ap.add_argument("--sweeps", type=int, default=60)
    ap.add_argument("--clip", type=float, default=1.0)
    ap.add_argument("--epochs-ml", type=int, default=3)
    a = ap.parse_args()
    if a.workload == "square8-ml":
        print(json.dumps(run_ml(epochs=a.epochs_ml, n_gen=a.gen or 4096, sweeps=a.sweeps)))
        return
    print(json.dumps(run(a.workload, a.train, a.short, a.epochs, a.batch, n_gen=a.gen,
                         sweeps=a.sweeps, clip=a.clip)))


if __name__ == "__main__":
    main()
