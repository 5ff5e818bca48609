"""Physics check of the honeycomb run against the paper's reference DQMC values.

Table 2 of the paper lists, for the half-filled Hubbard model on the L = 6 honeycomb
lattice (72 sites) at U/t = 3.83, beta = 6, dtau = 0.1, the kinetic energy
E_k = -1.358(1) and the antiferromagnetic structure factor S(Gamma) = 3.00(4) from a long
DQMC run ("Good DQMC", 10000 configurations in 1000 bins). This module runs the library's
sweep on that point with many independent chains from random fields and prints both
estimators with their standard errors (across chains), together with the plain
rescalings of S that other normalizations of Eq. 4 would give (spin operator n_up - n_dn
instead of (n_up - n_dn)/2: x4; 1/N_cells instead of 1/N_sites: x2).

Usage: python -m paper_2106_00712_gb300.honeycomb_check [--chains 1024] [--warm 200]
       [--meas 200] [--precision 2] [--ph 1]
Prints one JSON object.
"""
import argparse
import json
import time

from . import nmc
from .workloads import HONEYCOMB_6x6

TABLE2 = {"ekin": (-1.358, 0.001), "s_gamma": (3.00, 0.04)}


def run(wl=HONEYCOMB_6x6, chains=None, warm=None, meas=None, precision=nmc.NMC_SPLIT_BF16, ph=1,
        stream=None):
    chains = chains or wl.n_chains
    warm = wl.n_warm if warm is None else warm
    meas = wl.n_meas if meas is None else meas
    t0 = time.perf_counter()
    with nmc.Context(wl.Lx, wl.Ly, wl.t, wl.U, wl.beta, wl.dtau, wl.n_wrap, seed=wl.seed,
                     n_chains=chains, delay_k=wl.delay_k, precision=precision,
                     ph_symmetric=ph, lattice=wl.lattice, stream=stream) as c:
        c.generate()
        c.sweep(warm, measure=0)
        c.sweep(meas, measure=1)
        o = c.measure()
    secs = time.perf_counter() - t0
    s, se = o.s_pipi.mean, o.s_pipi.err
    return {"workload": wl.name, "chains": chains, "warm": warm, "meas": meas,
            "precision": precision, "ph_symmetric": ph, "seconds": secs,
            "ekin": [o.ekin.mean, o.ekin.err], "energy": [o.energy.mean, o.energy.err],
            "double_occ": [o.double_occ.mean, o.double_occ.err],
            "density": [o.density.mean, o.density.err],
            "s_gamma": [s, se], "s_gamma_x2": [2 * s, 2 * se], "s_gamma_x4": [4 * s, 4 * se],
            "accept": o.accept, "max_drift": o.max_drift, "table2_good_dqmc": TABLE2}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=None)
    ap.add_argument("--warm", type=int, default=None)
    ap.add_argument("--meas", type=int, default=None)
    ap.add_argument("--precision", type=int, default=nmc.NMC_SPLIT_BF16)
    ap.add_argument("--ph", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(chains=a.chains, warm=a.warm, meas=a.meas, precision=a.precision,
                         ph=a.ph)))


if __name__ == "__main__":
    main()
