"""FP64 CPU DQMC oracle: one Markov chain over the discrete Hubbard-Stratonovich field of
the half-filled Hubbard model on a periodic Lx x Ly square lattice.

TEST INFRASTRUCTURE ONLY (see the package docstring). Plain numpy/scipy in float64.
No blocking, no delayed updates, no fusion: every step is the definition or the
algorithm step written out, in the order below.

Paper passages (arXiv 2106.00712):
* Eq. 3: H = -t sum_<ij>,s (c+_is c_js + h.c.) + U sum_i (n_i^ - 1/2)(n_iv - 1/2).
* SM Sec. I.2: Trotter split Z = Tr prod_l e^{-dtau H_k} e^{-dtau H_U} + O(dtau^2);
  discrete HS transform e^{-dtau U (n^-1/2)(nv-1/2)} = 1/2 e^{-U dtau/4} sum_s e^{nu s (n^-nv)}
  with cosh nu = e^{U dtau/2}; trace-determinant identity; the weight
  Z = (1/2 e^{-U dtau/4})^{N L} sum_s prod_sigma Det[I + B^sigma(L,L-1)...B^sigma(1,0)].
* Eq. 4 text / SM Sec. I.1: S(Q) = (1/N) sum_ij e^{-iQ(r_i-r_j)} <s^z_i s^z_j>,
  s^z = (n^ - nv)/2.
* SM Sec. I.3: a sweep is one flip attempt on every auxiliary spin.

Readings where the paper is silent (the same readings bind the CUDA library):
R1 lattice: square, periodic; K_ij = -t for each nearest-neighbour pair, set (not summed),
   so a length-2 direction has one bond and a length-1 direction none. The honeycomb
   lattice of the paper's Hubbard runs ("Models"; SM Sec. II.1: L x L cells, 2 sites per
   cell) is the option lattice="honeycomb": site i = 2 (x + Lx y) + sub, A(x,y) bonded to
   B(x,y), B(x-1,y), B(x,y-1) (periodic), sublattice sign +1 (A), -1 (B).
R2 B order: B_l = e^{-dtau K} e^{V_l}, V_l = sigma*lam*diag(s(.,l)), lam = acosh(e^{dtau U/2}).
   The paper writes e^{V} e^{-dtau T}; the two cyclic products are similar matrices, so the
   weight and every flip ratio are unchanged.
R3 G at slice l (0-based l = 0..L-1): G_l = (I + B_{l-1}...B_0 B_{L-1}...B_l)^{-1}.
R4 Flip of s(i,l): Delta^sigma = e^{-2 sigma lam s(i,l)} - 1, R^sigma = 1 + Delta^sigma (1 - G_ii),
   R = R^up R^dn; u = x0 * 2^-32 from Philox counter (l*N+i, sweep, chain, 0);
   accept iff u < |R| (Metropolis); on accept G <- G - (Delta/R^sigma)(e_i - G[:,i]) G[i,:]
   (Sherman-Morrison), s -> -s, sign *= sign(R).
R5 Sweep order: sweeps alternate direction, up (l = 0..L-1) on even phase, down on odd;
   sites i = 0..N-1 ascending within a slice. Up: flip slice l, then wrap
   G_{l+1} = B_l G_l B_l^{-1}. Down: wrap G_l = B_l^{-1} G_{l+1} B_l, then flip slice l.
R6 Stabilization every n_wrap slices (block j = slices j*w..j*w+w-1): UDV stacks by
   Householder QR with column pivoting; the right product R_j = B_{jw-1}...B_0 is stored as
   U D T, the left product L_j = B_{L-1}...B_{jw} as L_j^T = U D T. After block j of an up
   sweep R_{j+1} is rebuilt and G_{(j+1)w} = (I + R_{j+1} L_{j+1})^{-1} recomputed; after
   block j of a down sweep L_j is rebuilt and G_{jw} = (I + R_j L_j)^{-1} recomputed. The
   recomputed G replaces the propagated one; max|G_prop - G_new| is the drift.
R7 Measurement at each stabilization point of a measuring sweep, on the symmetric-Trotter
   G~ = e^{dtau K/2} G e^{-dtau K/2}.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg

from .philox import flip_uniforms, init_fields as _philox_init_fields

SIGMAS = (+1, -1)  # spin up, spin down


@dataclass(frozen=True)
class Model:
    """Parameters of one DQMC problem (Eq. 3 and SM Sec. I.2)."""
    Lx: int
    Ly: int
    t: float
    U: float
    beta: float
    dtau: float
    n_wrap: int
    seed: int = 0
    lattice: str = "square"

    @property
    def N(self):
        return self.Lx * self.Ly * (2 if self.lattice == "honeycomb" else 1)

    @property
    def L_tau(self):
        return int(round(self.beta / self.dtau))

    @property
    def n_blocks(self):
        return self.L_tau // self.n_wrap


# ----------------------------------------------------------------------------- model

def hopping_matrix(Lx, Ly, t):
    """Kinetic matrix of Eq. 3 on the periodic Lx x Ly square lattice (reading R1).

    Site index i = x + Lx*y. K_ij = -t for nearest neighbours (set, not accumulated).
    """
    N = Lx * Ly
    K = np.zeros((N, N))
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                j = (x + dx) % Lx + Lx * ((y + dy) % Ly)
                if j != i:
                    K[i, j] = -t
    return K


def honeycomb_hopping(Lx, Ly, t):
    """Kinetic matrix of Eq. 3 on the periodic honeycomb lattice of Lx x Ly cells (reading R1):
    A(x,y) - B(x,y), A(x,y) - B(x-1,y), A(x,y) - B(x,y-1); set, not accumulated."""
    N = 2 * Lx * Ly
    K = np.zeros((N, N))
    for y in range(Ly):
        for x in range(Lx):
            a = 2 * (x + Lx * y)
            for (bx, by) in ((x, y), ((x - 1) % Lx, y), (x, (y - 1) % Ly)):
                b = 2 * (bx + Lx * by) + 1
                K[a, b] = K[b, a] = -t
    return K


def lattice_hopping(model):
    if model.lattice == "honeycomb":
        return honeycomb_hopping(model.Lx, model.Ly, model.t)
    return hopping_matrix(model.Lx, model.Ly, model.t)


def expm_sym(K, c):
    """e^{cK} for symmetric K by its eigendecomposition."""
    w, V = np.linalg.eigh(K)
    return (V * np.exp(c * w)) @ V.T


def hs_lambda(U, dtau):
    """HS coupling: cosh(lam) = e^{U dtau / 2} (SM Sec. I.2, discrete HS transform)."""
    return float(np.arccosh(np.exp(dtau * U / 2.0)))


class Propagators:
    """e^{-dtau K}, e^{+dtau K}, e^{-dtau K/2}, e^{+dtau K/2} for one lattice."""

    def __init__(self, model):
        self.K = lattice_hopping(model)
        self.expK_m = expm_sym(self.K, -model.dtau)
        self.expK_p = expm_sym(self.K, +model.dtau)
        self.expK_mh = expm_sym(self.K, -model.dtau / 2)
        self.expK_ph = expm_sym(self.K, +model.dtau / 2)
        self.lam = hs_lambda(model.U, model.dtau)


def v_diag(lam, sigma, s_l):
    """Diagonal of V_l^sigma = sigma * lam * s(., l)."""
    return sigma * lam * s_l.astype(np.float64)


def b_matrix(P, sigma, s_l):
    """B_l^sigma = e^{-dtau K} e^{V_l^sigma} (reading R2; SM Sec. I.2 B(l2,l1))."""
    return P.expK_m * np.exp(v_diag(P.lam, sigma, s_l))[None, :]


def weight_prefactor(model):
    """(1/2 e^{-U dtau/4})^{N L_tau} (SM Sec. I.2, determinant form of Z)."""
    return (0.5 * np.exp(-model.U * model.dtau / 4.0)) ** (model.N * model.L_tau)


def product_from(P, fields, sigma, l):
    """Plain (unstabilized) A_l = B_{l-1}...B_0 B_{L-1}...B_l (reading R3). Small beta only."""
    L = fields.shape[0]
    A = np.eye(fields.shape[1])
    for k in range(L):
        A = b_matrix(P, sigma, fields[(l + k) % L]) @ A
    return A


def green_naive(P, fields, sigma, l=0):
    """G_l = (I + A_l)^{-1} by direct inversion. Small beta only."""
    A = product_from(P, fields, sigma, l)
    return np.linalg.inv(np.eye(A.shape[0]) + A)


# ----------------------------------------------------------------------------- UDV

class UDT:
    """A matrix held as U diag(D) T: U orthogonal, D > 0, T well conditioned."""

    def __init__(self, U, D, T):
        self.U, self.D, self.T = U, D, T

    @staticmethod
    def identity(N):
        return UDT(np.eye(N), np.ones(N), np.eye(N))

    def matrix(self):
        return (self.U * self.D[None, :]) @ self.T


def qrp_udt(M):
    """Householder QR with column pivoting, M P = Q R (LAPACK geqp3 via scipy).

    Returns (Q, D, T) with M = Q diag(D) T, D = |diag(R)|, T = diag(D)^{-1} R P^T.
    """
    Q, R, piv = scipy.linalg.qr(M, pivoting=True)
    D = np.abs(np.diag(R))
    T = np.empty_like(R)
    T[:, piv] = R / D[:, None]
    return Q, D, T


def right_update(P, fields, sigma, block, n_wrap, Rst):
    """R_{j+1} = B_{(j+1)w-1}...B_{jw} R_j as UDT (reading R6).

    Multiply the slices of block j onto U_R diag(D_R), then QRP, then T <- T' T_R.
    """
    X = Rst.U * Rst.D[None, :]
    for l in range(block * n_wrap, (block + 1) * n_wrap):
        X = P.expK_m @ (np.exp(v_diag(P.lam, sigma, fields[l]))[:, None] * X)
    Q, D, Tp = qrp_udt(X)
    return UDT(Q, D, Tp @ Rst.T)


def left_update(P, fields, sigma, block, n_wrap, Lst):
    """L_j = L_{j+1} B_{(j+1)w-1}...B_{jw}, held as L_j^T = U D T (reading R6).

    L_j^T = B_{jw}^T ... B_{(j+1)w-1}^T L_{j+1}^T with B_l^T = e^{V_l} e^{-dtau K}; the slices
    of block j are applied from the highest down, then QRP, then T <- T' T_L.
    """
    X = Lst.U * Lst.D[None, :]
    for l in range((block + 1) * n_wrap - 1, block * n_wrap - 1, -1):
        X = np.exp(v_diag(P.lam, sigma, fields[l]))[:, None] * (P.expK_m @ X)
    Q, D, Tp = qrp_udt(X)
    return UDT(Q, D, Tp @ Lst.T)


def green_from_stacks(Rst, Lst):
    """G = (I + R L)^{-1} from R = U_R D_R T_R and L^T = U_L D_L T_L (reading R6).

    With D = Db Ds, Db = max(D, 1), Ds = min(D, 1):
      G = U_L Db_L^{-1} X^{-1} Db_R^{-1} U_R^T,
      X = Db_R^{-1} (U_R^T U_L) Db_L^{-1} + Ds_R (T_R T_L^T) Ds_L,
    X solved by LU with partial pivoting (numpy.linalg.solve).
    """
    DbR, DsR = np.maximum(Rst.D, 1.0), np.minimum(Rst.D, 1.0)
    DbL, DsL = np.maximum(Lst.D, 1.0), np.minimum(Lst.D, 1.0)
    X = (Rst.U.T @ Lst.U) / DbR[:, None] / DbL[None, :] \
        + DsR[:, None] * (Rst.T @ Lst.T.T) * DsL[None, :]
    Y = np.linalg.solve(X, Rst.U.T / DbR[:, None])
    return (Lst.U / DbL[None, :]) @ Y


def green_scratch(P, fields, sigma, l, n_wrap):
    """G_l from the fields alone by a stabilized product over all slices starting at l.

    A_l = B_{l-1}...B_0 B_{L-1}...B_l is built as U D T with a QRP every n_wrap slices,
    then G = (I + A_l)^{-1} by green_from_stacks with L = I.
    """
    L, N = fields.shape
    A = UDT.identity(N)
    X = A.U * A.D[None, :]
    for k in range(L):
        sl = fields[(l + k) % L]
        X = P.expK_m @ (np.exp(v_diag(P.lam, sigma, sl))[:, None] * X)
        if (k + 1) % n_wrap == 0 or k == L - 1:
            Q, D, Tp = qrp_udt(X)
            A = UDT(Q, D, Tp @ A.T)
            X = A.U * A.D[None, :]
    return green_from_stacks(A, UDT.identity(N))


# ----------------------------------------------------------------------------- measure

def staggered_signs(Lx, Ly, lattice="square"):
    """Square: p_i = (-1)^{x_i + y_i} = e^{-i (pi,pi) . r_i}. Honeycomb: the sublattice sign
    (+1 on A, -1 on B), the antiferromagnetic pattern whose structure factor the paper calls
    S(Gamma)."""
    if lattice == "honeycomb":
        return np.array([1.0 if i % 2 == 0 else -1.0 for i in range(2 * Lx * Ly)])
    return np.array([(-1.0) ** (x + y) for y in range(Ly) for x in range(Lx)])


def measure(P, model, G_up, G_dn):
    """Equal-time estimators on one field configuration (reading R7).

    G_ij = <c_i c_j^+> per spin; G~ = e^{dtau K/2} G e^{-dtau K/2}.
    Returns dict: energy (<H>/N from Eq. 3), ekin, double_occ, s_pipi, density.
    S(pi,pi) = (1/N) sum_ij p_i p_j <s^z_i s^z_j> (Eq. 4 definition) with
    <s^z_i s^z_j> = 1/4 sum_{sigma,sigma'} sigma sigma' <n_i,sigma n_j,sigma'> and Wick:
      same spin:  <n_i n_j> = (1 - G_ii)(1 - G_jj) + (delta_ij - G_ji) G_ij,
      other spin: <n_i^ n_jv> = (1 - G^_ii)(1 - Gv_jj).
    """
    N = model.N
    Gt = [P.expK_ph @ G @ P.expK_mh for G in (G_up, G_dn)]
    ekin = -sum(np.trace(P.K @ g) for g in Gt) / N
    du, dd = np.diag(Gt[0]), np.diag(Gt[1])
    epot = model.U * np.sum((0.5 - du) * (0.5 - dd)) / N
    docc = np.sum((1.0 - du) * (1.0 - dd)) / N
    dens = np.sum((1.0 - du) + (1.0 - dd)) / N
    p = staggered_signs(model.Lx, model.Ly, model.lattice)
    eye = np.eye(N)
    nn = {}
    for a, sa in enumerate(SIGMAS):
        for b, sb in enumerate(SIGMAS):
            na = 1.0 - np.diag(Gt[a])
            nb = 1.0 - np.diag(Gt[b])
            m = np.outer(na, nb)
            if a == b:
                m = m + (eye - Gt[a].T) * Gt[a]
            nn[(sa, sb)] = m
    szsz = 0.25 * sum(sa * sb * nn[(sa, sb)] for sa in SIGMAS for sb in SIGMAS)
    s_pipi = float(p @ szsz @ p) / N
    return dict(energy=ekin + epot, ekin=ekin, double_occ=docc, s_pipi=s_pipi, density=dens)


OBS_KEYS = ("energy", "ekin", "double_occ", "s_pipi", "density", "sign")


# ----------------------------------------------------------------------------- chain

class Chain:
    """One DQMC Markov chain (readings R3-R7). State: fields, G per spin, UDV stack
    entries, sweep counter (Philox counter word 1), direction phase, sign, accumulators."""

    def __init__(self, model, fields, chain_index=0, sweep_index=0, P=None):
        self.model = model
        self.P = P if P is not None else Propagators(model)
        self.s = np.array(fields, dtype=np.int8).reshape(model.L_tau, model.N).copy()
        if not np.all(np.abs(self.s) == 1):
            raise ValueError("fields must be +-1")
        if model.L_tau % model.n_wrap:
            raise ValueError("L_tau must be a multiple of n_wrap")
        self.chain = chain_index
        self.sweep_index = sweep_index
        self.phase = 0
        self.sign = 1.0
        self.attempts = 0
        self.accepts = 0
        self.max_drift = 0.0
        self.n_meas = 0
        self.sums = {k: 0.0 for k in OBS_KEYS}
        self.sweep_means = []          # per measuring sweep: mean of its measurements
        self.decisions = []            # per sweep: uint8 [L_tau][N] accept flags
        self._init_stacks()

    # -- stacks -----------------------------------------------------------------
    def _init_stacks(self):
        """Build L_j for j = nb..0 (L_nb = I) and G_0 = (I + L_0)^{-1} (reading R6)."""
        m = self.model
        nb, w, N = m.n_blocks, m.n_wrap, m.N
        self.slots = [[None] * (nb + 1) for _ in SIGMAS]
        self.G = [None, None]
        for a, sigma in enumerate(SIGMAS):
            Lst = UDT.identity(N)
            for j in range(nb - 1, -1, -1):
                Lst = left_update(self.P, self.s, sigma, j, w, Lst)
                if j >= 1:
                    self.slots[a][j] = Lst
            self.G[a] = green_from_stacks(UDT.identity(N), Lst)

    def _right(self, a, j):
        return UDT.identity(self.model.N) if j == 0 else self.slots[a][j]

    def _left(self, a, j):
        return UDT.identity(self.model.N) if j == self.model.n_blocks else self.slots[a][j]

    # -- local update -------------------------------------------------------------
    def _flip_slice(self, l, dec):
        """Metropolis flip attempts at slice l, sites in ascending order (reading R4)."""
        m, P = self.model, self.P
        u = flip_uniforms(m.seed, l, m.N, self.sweep_index, self.chain)
        for i in range(m.N):
            s = float(self.s[l, i])
            deltas, ratios = [], []
            for a, sigma in enumerate(SIGMAS):
                d = np.exp(-2.0 * sigma * P.lam * s) - 1.0
                deltas.append(d)
                ratios.append(1.0 + d * (1.0 - self.G[a][i, i]))
            R = ratios[0] * ratios[1]
            self.attempts += 1
            if u[i] < abs(R):
                for a in range(2):
                    G = self.G[a]
                    col = -G[:, i].copy()
                    col[i] += 1.0                      # e_i - G[:, i]
                    row = G[i, :].copy()
                    self.G[a] = G - (deltas[a] / ratios[a]) * np.outer(col, row)
                self.s[l, i] = -self.s[l, i]
                self.sign *= np.sign(R)
                self.accepts += 1
                dec[l, i] = 1

    def _wrap_up(self, l):
        """G_{l+1} = B_l G_l B_l^{-1} = e^{-dtau K} e^{V} G e^{-V} e^{dtau K}."""
        P = self.P
        for a, sigma in enumerate(SIGMAS):
            ev = np.exp(v_diag(P.lam, sigma, self.s[l]))
            self.G[a] = P.expK_m @ (ev[:, None] * self.G[a] / ev[None, :]) @ P.expK_p

    def _wrap_down(self, l):
        """G_l = B_l^{-1} G_{l+1} B_l = e^{-V} e^{dtau K} G e^{-dtau K} e^{V}."""
        P = self.P
        for a, sigma in enumerate(SIGMAS):
            ev = np.exp(v_diag(P.lam, sigma, self.s[l]))
            self.G[a] = (P.expK_p @ self.G[a] @ P.expK_m) / ev[:, None] * ev[None, :]

    def _replace(self, a, G_new):
        self.max_drift = max(self.max_drift, float(np.max(np.abs(self.G[a] - G_new))))
        self.G[a] = G_new

    def _measure(self, acc):
        obs = measure(self.P, self.model, self.G[0], self.G[1])
        for k in OBS_KEYS[:-1]:
            acc[k] += obs[k] * self.sign
        acc["sign"] += self.sign

    # -- sweeps -----------------------------------------------------------------
    def sweep(self, measure_on=True):
        """One sweep: every s(i,l) gets one flip attempt (SM Sec. I.3; reading R5)."""
        m = self.model
        nb, w = m.n_blocks, m.n_wrap
        dec = np.zeros((m.L_tau, m.N), dtype=np.uint8)
        acc = {k: 0.0 for k in OBS_KEYS}
        n_meas = 0
        if self.phase % 2 == 0:                       # up sweep
            for j in range(nb):
                for l in range(j * w, (j + 1) * w):
                    self._flip_slice(l, dec)
                    self._wrap_up(l)
                for a, sigma in enumerate(SIGMAS):
                    Rn = right_update(self.P, self.s, sigma, j, w, self._right(a, j))
                    G_new = green_from_stacks(Rn, self._left(a, j + 1))
                    if j + 1 < nb:
                        self.slots[a][j + 1] = Rn
                    self._replace(a, G_new)
                if measure_on:
                    self._measure(acc)
                    n_meas += 1
        else:                                         # down sweep
            for j in range(nb - 1, -1, -1):
                for l in range((j + 1) * w - 1, j * w - 1, -1):
                    self._wrap_down(l)
                    self._flip_slice(l, dec)
                for a, sigma in enumerate(SIGMAS):
                    Ln = left_update(self.P, self.s, sigma, j, w, self._left(a, j + 1))
                    G_new = green_from_stacks(self._right(a, j), Ln)
                    if j >= 1:
                        self.slots[a][j] = Ln
                    self._replace(a, G_new)
                if measure_on:
                    self._measure(acc)
                    n_meas += 1
        if n_meas:
            for k in OBS_KEYS:
                self.sums[k] += acc[k]
            self.n_meas += n_meas
            self.sweep_means.append({k: acc[k] / n_meas for k in OBS_KEYS})
        self.decisions.append(dec)
        self.phase += 1
        self.sweep_index += 1

    def means(self):
        """Per-chain means of the sign-weighted estimators: <O s> / <s>."""
        if self.n_meas == 0:
            return None
        out = {k: self.sums[k] / self.sums["sign"] for k in OBS_KEYS[:-1]}
        out["sign"] = self.sums["sign"] / self.n_meas
        out["accept"] = self.accepts / max(self.attempts, 1)
        return out


def initial_fields(model, chain_index):
    """Philox-generated initial field for one chain (counter tag 1)."""
    return _philox_init_fields(model.seed, model.L_tau, model.N, chain_index)


def run_chain(model, fields=None, chain_index=0, n_warm=0, n_meas=0):
    """Convenience: create a chain, n_warm non-measuring then n_meas measuring sweeps."""
    if fields is None:
        fields = initial_fields(model, chain_index)
    ch = Chain(model, fields, chain_index)
    for _ in range(n_warm):
        ch.sweep(False)
    for _ in range(n_meas):
        ch.sweep(True)
    return ch
