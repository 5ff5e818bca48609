"""Fock-space (second-quantized) reference for tiny Hubbard clusters.

Independent of oracle/: builds the Hamiltonian of Eq. 3 from fermion operators
(Jordan-Wigner), with the bond list given explicitly, and evaluates traces directly in
the 4^N-dimensional Fock space. Used to pin the oracle's weight, Green's functions and
estimators, which are written in the single-particle (determinant) language.
"""
import numpy as np
import scipy.linalg


def fermion_ops(n_modes):
    """Annihilation operators c_m (dense, 2^n x 2^n) with Jordan-Wigner strings."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for m in range(n_modes):
        mats = [z] * m + [a] + [eye] * (n_modes - m - 1)
        op = mats[0]
        for x in mats[1:]:
            op = np.kron(op, x)
        ops.append(op)
    return ops


class Cluster:
    """Hubbard cluster: sites 0..N-1, explicit bond list, hopping t, interaction U."""

    def __init__(self, n_sites, bonds, t, U):
        self.N = n_sites
        c = fermion_ops(2 * n_sites)
        self.c_up = c[:n_sites]
        self.c_dn = c[n_sites:]
        dim = 2 ** (2 * n_sites)
        self.dim = dim
        Hk = np.zeros((dim, dim))
        for (i, j) in bonds:
            for cs in (self.c_up, self.c_dn):
                hop = cs[i].T @ cs[j]
                Hk += -t * (hop + hop.T)
        self.n_up = [o.T @ o for o in self.c_up]
        self.n_dn = [o.T @ o for o in self.c_dn]
        I = np.eye(dim)
        HU = np.zeros((dim, dim))
        for i in range(n_sites):
            HU += U * (self.n_up[i] - 0.5 * I) @ (self.n_dn[i] - 0.5 * I)
        self.Hk, self.HU, self.H = Hk, HU, Hk + HU

    def observables(self, signs):
        """Operators per site count N: H/N, H_k/N, double occupancy, S(pi,pi), density."""
        N = self.N
        D = sum(self.n_up[i] @ self.n_dn[i] for i in range(N)) / N
        sz = [0.5 * (self.n_up[i] - self.n_dn[i]) for i in range(N)]
        stag = sum(signs[i] * sz[i] for i in range(N))
        S = stag @ stag / N
        dens = sum(self.n_up[i] + self.n_dn[i] for i in range(N)) / N
        return dict(energy=self.H / N, ekin=self.Hk / N, double_occ=D, s_pipi=S,
                    density=dens)

    def trotter_symmetric(self, dtau, L):
        """Single-slice symmetric Trotter propagator e^{-dtau Hk/2} e^{-dtau HU} e^{-dtau Hk/2}."""
        h = scipy.linalg.expm(-0.5 * dtau * self.Hk)
        u = scipy.linalg.expm(-dtau * self.HU)
        return np.linalg.matrix_power(h @ u @ h, L)

    def z_trotter(self, dtau, L):
        """Tr[(e^{-dtau Hk} e^{-dtau HU})^L] (SM Sec. I.2 Trotter split)."""
        k = scipy.linalg.expm(-dtau * self.Hk)
        u = scipy.linalg.expm(-dtau * self.HU)
        return float(np.trace(np.linalg.matrix_power(k @ u, L)))

    def expect_trotter(self, dtau, L, signs):
        rho = self.trotter_symmetric(dtau, L)
        Z = np.trace(rho)
        return {k: float(np.trace(rho @ O) / Z) for k, O in self.observables(signs).items()}

    def expect_exact(self, beta, signs):
        rho = scipy.linalg.expm(-beta * self.H)
        Z = np.trace(rho)
        return {k: float(np.trace(rho @ O) / Z) for k, O in self.observables(signs).items()}
