"""Seeded synthetic workloads for the DQMC sweep (shared by tests and the benchmark).

This module holds input recipes only -- lattice/parameter sets and seeded +-1 fields --
and none of the method's arithmetic. The paper's Hubbard workload is the honeycomb
lattice at the critical coupling (Sec. "Models", Table 2: L = 6, i.e. 72 sites, U = 3.83,
beta = 6, dtau = 0.1); the square-lattice sets are the benchmark shapes. Fields are
i.i.d. uniform +-1, the shape the sweep sees from a random or generated start.
"""
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    Lx: int
    Ly: int
    t: float
    U: float
    beta: float
    dtau: float
    n_wrap: int
    n_chains: int
    delay_k: int
    n_warm: int
    n_meas: int
    seed: int = 0
    lattice: str = "square"

    @property
    def N(self):
        return self.Lx * self.Ly * (2 if self.lattice == "honeycomb" else 1)

    @property
    def L_tau(self):
        return int(round(self.beta / self.dtau))

    def with_(self, **kw):
        return replace(self, **kw)


# 4x4, U=4, beta=2, dtau=0.1, n_wrap=10, 1 chain, 200 sweeps (first 50 warm-up).
SQUARE_4x4 = Workload("hubbard-4x4-U4-beta2-1chain", 4, 4, 1.0, 4.0, 2.0, 0.1, 10,
                      1, 16, 50, 150)
# 8x8, U=4, beta=4, dtau=0.1 (L_tau=40), n_wrap=10, 256 chains, k=16, 100 + 400 sweeps.
SQUARE_8x8 = Workload("hubbard-8x8-U4-beta4-256chains", 8, 8, 1.0, 4.0, 4.0, 0.1, 10,
                      256, 16, 100, 400)
# 16x16, U in {2,4,8}, beta=8, dtau=0.05 (L_tau=160), n_wrap=8, 32 chains, k=32.
SQUARE_16x16 = Workload("hubbard-16x16-U4-beta8-32chains", 16, 16, 1.0, 4.0, 8.0, 0.05, 8,
                        32, 32, 50, 200)

# Honeycomb, 6x6 cells (72 sites), U=3.83, beta=6, dtau=0.1 (L_tau=60), n_wrap=10,
# 1024 chains, k=16, 200 + 200 sweeps: the paper's Hubbard point (Table 2).
HONEYCOMB_6x6 = Workload("hubbard-honeycomb-L6-U3.83-beta6-1024chains", 6, 6, 1.0, 3.83, 6.0,
                         0.1, 10, 1024, 16, 200, 200, seed=2106, lattice="honeycomb")

WORKLOADS = {w.name: w for w in (SQUARE_4x4, SQUARE_8x8, SQUARE_16x16, HONEYCOMB_6x6)}


def random_fields(n_chains, L_tau, N, seed):
    """i.i.d. uniform +-1 fields, int8 [n_chains][L_tau][N], from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=(n_chains, L_tau, N), dtype=np.int8)
    return (1 - 2 * bits).astype(np.int8)
