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


def spin_structure_factors(Gt_up, Gt_dn, p):
    """S_zz(Q) and S_xx(Q) of one configuration from its symmetric-Trotter Green's functions
    G~_ij = <c_i c_j^+> (per spin) and the pattern p (sublattice signs for Gamma on the
    honeycomb): S_aa = (1/N) sum_ij p_i p_j <s^a_i s^a_j>, s = sigma / 2, by Wick's theorem
        <s^z_i s^z_j> = 1/4 sum_{sigma sigma'} sigma sigma' <n_i sigma n_j sigma'>,
          same spin <n_i n_j> = (1 - G_ii)(1 - G_jj) + (delta_ij - G_ji) G_ij,
          other spin <n_i^ n_jv> = (1 - G^_ii)(1 - Gv_jj);
        <s^x_i s^x_j> = 1/4 [(delta_ij - G^_ji) Gv_ij + (delta_ij - Gv_ji) G^_ij]
    (the two spin-flip terms of s^x_i s^x_j; the others vanish in a sigma-conserving
    configuration). For an SU(2)-symmetric ensemble the two agree; the spin-channel
    Hubbard-Stratonovich decoupling breaks SU(2) at finite dtau, so at a fixed dtau they
    differ by its Trotter error."""
    import numpy as np
    N = Gt_up.shape[0]
    eye = np.eye(N)
    nu, nd = 1.0 - np.diag(Gt_up), 1.0 - np.diag(Gt_dn)
    same_u = np.outer(nu, nu) + (eye - Gt_up.T) * Gt_up
    same_d = np.outer(nd, nd) + (eye - Gt_dn.T) * Gt_dn
    cross = np.outer(nu, nd)
    szsz = 0.25 * (same_u + same_d - cross - cross.T)
    sxsx = 0.25 * ((eye - Gt_up.T) * Gt_dn + (eye - Gt_dn.T) * Gt_up)
    return float(p @ szsz @ p) / N, float(p @ sxsx @ p) / N


def run_su2(wl=HONEYCOMB_6x6, chains=1024, warm=200, samples=20, every=10,
            precision=nmc.NMC_SPLIT_BF16, ph=1):
    """The Table 2 point with both spin components: after `warm` sweeps, `samples` times
    (every `every` sweeps) the Green's functions of every chain are read, and S_zz(Gamma),
    S_xx(Gamma) are formed on G~ (the estimator position of the library's own S), so that
    the zz estimator the paper's Eq. 4 names can be set beside the SU(2) average
    (S_zz + 2 S_xx) / 3 at the same dtau."""
    import numpy as np
    t0 = time.perf_counter()
    p = np.array([1.0 if i % 2 == 0 else -1.0 for i in range(wl.N)])
    Eph = nmc.nmc_expk(wl.Lx, wl.Ly, wl.t, wl.dtau / 2, wl.lattice)
    Emh = nmc.nmc_expk(wl.Lx, wl.Ly, wl.t, -wl.dtau / 2, wl.lattice)
    zz, xx = [], []
    with nmc.Context(wl.Lx, wl.Ly, wl.t, wl.U, wl.beta, wl.dtau, wl.n_wrap, seed=wl.seed,
                     n_chains=chains, delay_k=wl.delay_k, precision=precision,
                     ph_symmetric=ph, lattice=wl.lattice) as c:
        c.generate()
        c.sweep(warm, measure=0)
        for _ in range(samples):
            c.sweep(every, measure=1)
            for ch in range(chains):
                gu = Eph @ c.green(ch, 0) @ Emh
                gd = Eph @ c.green(ch, 1) @ Emh
                a, b = spin_structure_factors(gu, gd, p)
                zz.append(a)
                xx.append(b)
        o = c.measure()
    zz, xx = np.array(zz).reshape(samples, chains), np.array(xx).reshape(samples, chains)
    su2 = (zz + 2 * xx) / 3

    def stat(v):   # mean over samples per chain, then the error across chains
        m = v.mean(axis=0)
        return [float(4 * m.mean()), float(4 * m.std(ddof=1) / np.sqrt(len(m)))]
    return {"workload": wl.name, "chains": chains, "warm": warm, "samples": samples,
            "every": every, "precision": precision, "ph_symmetric": ph,
            "four_s_zz": stat(zz), "four_s_xx": stat(xx), "four_s_su2": stat(su2),
            "four_s_library": [4 * o.s_pipi.mean, 4 * o.s_pipi.err],
            "ekin": [o.ekin.mean, o.ekin.err], "table2_good_dqmc": TABLE2,
            "seconds": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=None)
    ap.add_argument("--warm", type=int, default=None)
    ap.add_argument("--meas", type=int, default=None)
    ap.add_argument("--precision", type=int, default=nmc.NMC_SPLIT_BF16)
    ap.add_argument("--ph", type=int, default=1)
    ap.add_argument("--su2", action="store_true",
                    help="S_zz, S_xx and their SU(2) average from the Green's functions")
    ap.add_argument("--samples", type=int, default=20)
    a = ap.parse_args()
    if a.su2:
        print(json.dumps(run_su2(chains=a.chains or 1024, warm=a.warm or 200,
                                 samples=a.samples, precision=a.precision, ph=a.ph)))
        return
    print(json.dumps(run(chains=a.chains, warm=a.warm, meas=a.meas, precision=a.precision,
                         ph=a.ph)))


if __name__ == "__main__":
    main()
