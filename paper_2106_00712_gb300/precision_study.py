"""Precision study of the propagation arithmetic on the 16x16 workload.

Half-filled Hubbard model, periodic 16x16 lattice (N=256), t=1, beta=8, dtau=0.05
(L_tau=160), n_wrap=8, delay k=32, 32 chains, U in {2, 4, 8}. For each U and each
reduced-precision mode:

* replay: the mode follows the FP64 GPU run's accept decisions (nmc_sweep_replay), so both
  see the same fields; the library records, at every stabilization, the maximum over
  chains of |G_propagated - G_recomputed| where G_recomputed is the FP64 recompute from the
  FP64 UDV stacks of those fields -- i.e. max |G - G_fp64| before each stabilization;
* free running: the mode runs its own chain from the same initial fields, and the pooled
  energy, double occupancy and S(pi,pi) are compared with the FP64 run in units of the
  combined standard error (across chains).

Usage: python -m paper_2106_00712_gb300.precision_study [--sweeps 8] [--warm 2]
                                                       [--U 2,4,8] [--modes fp32,split_bf16]
Prints one JSON object.
"""
import argparse
import json
import math
import time

import numpy as np

from . import nmc
from .workloads import SQUARE_16x16

MODES = {"fp32": nmc.NMC_FP32, "split_bf16": nmc.NMC_SPLIT_BF16, "fp32x2": nmc.NMC_FP32X2}


def _ctx(wl, U, prec):
    return nmc.Context(wl.Lx, wl.Ly, wl.t, U, wl.beta, wl.dtau, wl.n_wrap, seed=wl.seed,
                       n_chains=wl.n_chains, delay_k=wl.delay_k, precision=prec,
                       drift_tol=1e300)


def _obs(o):
    return {k: (getattr(o, k).mean, getattr(o, k).err)
            for k in ("energy", "double_occ", "s_pipi")}


def study_one(wl, U, n_warm, n_meas, modes=tuple(MODES)):
    out = {"U": U}
    t0 = time.perf_counter()
    ref = _ctx(wl, U, nmc.NMC_FP64)
    ref.generate()
    fields = [ref.fields()]
    for s in range(n_warm + n_meas):
        ref.sweep(1, measure=int(s >= n_warm))
        fields.append(ref.fields())
    o64 = ref.measure()
    out["fp64"] = {"max_drift": o64.max_drift, "obs": _obs(o64),
                   "drift_history_max": float(ref.drift_history().max())}
    ref.close()
    accepts = [(fields[s + 1] != fields[s]).astype(np.uint8) for s in range(len(fields) - 1)]
    for name in modes:
        prec = MODES[name]
        row = {}
        c = _ctx(wl, U, prec)
        c.generate()
        try:
            for s, acc in enumerate(accepts):
                c.sweep_replay(acc, measure=int(s >= n_warm))
            h = c.drift_history()
            o = c.measure()
            row["replay"] = {"max_drift": float(h.max()), "median_drift": float(np.median(h)),
                             "stabilizations": int(h.size), "disagreements": o.n_disagree,
                             "meets_1e-5": bool(h.max() <= 1e-5)}
        except nmc.NmcError as e:
            row["replay"] = {"error": str(e)}
        c.close()
        c = _ctx(wl, U, prec)
        c.generate()
        try:
            c.sweep(n_warm, measure=0)
            c.sweep(n_meas, measure=1)
            o = _obs(c.measure())
            dev = {}
            for k, (m, e) in o.items():
                m64, e64 = out["fp64"]["obs"][k]
                s = math.sqrt(e * e + e64 * e64)
                dev[k] = (m - m64) / s if s > 0 else float("nan")
            row["free"] = {"obs": o, "deviation_sigma": dev}
        except nmc.NmcError as e:
            row["free"] = {"error": str(e)}
        c.close()
        out[name] = row
    out["seconds"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweeps", type=int, default=6)
    ap.add_argument("--warm", type=int, default=2)
    ap.add_argument("--U", default="2,4,8")
    ap.add_argument("--modes", default=",".join(MODES),
                    help="reduced-precision modes to compare with the FP64 run")
    args = ap.parse_args()
    modes = [m for m in args.modes.split(",") if m]
    wl = SQUARE_16x16
    report = {"workload": "hubbard-16x16-beta8-dtau0.05-nwrap8-k32-32chains",
              "sweeps": args.sweeps, "warm": args.warm,
              "modes": modes,
              "results": [study_one(wl, float(U), args.warm, args.sweeps, modes)
                          for U in args.U.split(",")]}
    print(json.dumps(report))


if __name__ == "__main__":
    main()
