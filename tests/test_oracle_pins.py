"""Pins of the FP64 oracle against results the paper and mathematics fix.

None of these compares the oracle with itself: each reference below is an independent
construction (Fock-space traces, closed forms, full determinants, direct inversion,
exact enumeration of the field sum, an independent generator implementation).
"""
import ctypes
import ctypes.util
import itertools

import numpy as np
import pytest

from oracle import dqmc
from oracle.dqmc import Chain, Model, Propagators, initial_fields
from oracle.philox import init_fields, philox4x32_10, seed_key
from tests._fock import Cluster

DIMER_BONDS = [(0, 1)]
DIMER_SIGNS = [1, -1]
PLAQ_BONDS = [(0, 1), (2, 3), (0, 2), (1, 3)]       # 2x2, site = x + 2y
PLAQ_SIGNS = [1, -1, -1, 1]


# ----------------------------------------------------------------------- Philox

def _curand():
    for name in ("libcurand.so.10", "libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator emits block j = Philox(counter (0,0,j,0),
    key = seed). Independent implementation; runs on the CPU."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n_blocks = 4096
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
        lib.curandDestroyGenerator(gen)
        k0, k1 = seed_key(seed)
        j = np.arange(n_blocks, dtype=np.uint64)
        words = philox4x32_10(0, 0, j, 0, k0, k1)
        mine = np.stack([w.astype(np.uint32) for w in words], axis=1).reshape(-1)
        np.testing.assert_array_equal(mine, out)


def test_philox_words_are_used_and_fields_balanced():
    """Every counter word and key word changes the output; initial fields are +-1 and
    balanced (binomial bound) -- guards against a dropped word in the counter."""
    base = [int(x[0]) for x in philox4x32_10([5], [6], [7], [8], 9, 10)]
    for pos in range(6):
        args = [5, 6, 7, 8, 9, 10]
        args[pos] += 1
        other = [int(x) for x in philox4x32_10(*args)]
        assert other != base
    s = init_fields(0, 40, 64, 3)
    assert set(np.unique(s)) == {-1, 1}
    assert abs(int(s.sum())) < 5 * np.sqrt(s.size)


# ----------------------------------------------------------------------- lattice / K

def test_hopping_matrix_spectrum_and_bonds():
    """Periodic 4x4 square lattice: four neighbours per site and eigenvalues
    -2t(cos kx + cos ky), k = 2 pi n / L (plane waves)."""
    t = 1.3
    K = dqmc.hopping_matrix(4, 4, t)
    assert np.allclose(K, K.T)
    assert np.all((K != 0).sum(axis=1) == 4)
    ks = 2 * np.pi * np.arange(4) / 4
    eps = np.sort([-2 * t * (np.cos(a) + np.cos(b)) for a in ks for b in ks])
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), eps, atol=1e-13)
    # 2-site dimer (length-2 direction: one bond) and 2x2 plaquette
    assert np.array_equal(dqmc.hopping_matrix(2, 1, 1.0), -np.array([[0, 1], [1, 0.0]]))
    Kp = dqmc.hopping_matrix(2, 2, 1.0)
    ref = np.zeros((4, 4))
    for i, j in PLAQ_BONDS:
        ref[i, j] = ref[j, i] = -1.0
    assert np.array_equal(Kp, ref)


def _honeycomb_bloch_energies(Lx, Ly, t):
    """+-t |1 + e^{i k1} + e^{i k2}|, k_a = 2 pi n_a / L_a: the two bands of the honeycomb
    lattice (two-site cell, three bonds per A site along 0, -a1, -a2)."""
    out = []
    for n1 in range(Lx):
        for n2 in range(Ly):
            g = abs(1 + np.exp(2j * np.pi * n1 / Lx) + np.exp(2j * np.pi * n2 / Ly))
            out += [-t * g, t * g]
    return np.sort(out)


@pytest.mark.parametrize("Lx,Ly", [(3, 3), (6, 6), (4, 2)])
def test_honeycomb_hopping_spectrum_and_bonds(Lx, Ly):
    """Honeycomb (SM Sec. II.1, 2 L^2 sites): three neighbours per site, all on the other
    sublattice (P K P = -K), and the Bloch band energies +-t|gamma_k|."""
    t = 0.9
    model = Model(Lx, Ly, t, 0.0, 1.0, 0.1, 10, lattice="honeycomb")
    K = dqmc.lattice_hopping(model)
    assert K.shape == (2 * Lx * Ly, 2 * Lx * Ly) and np.allclose(K, K.T)
    assert np.all((K != 0).sum(axis=1) == 3)
    p = dqmc.staggered_signs(Lx, Ly, "honeycomb")
    assert np.array_equal(p[:, None] * K * p[None, :], -K)
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), _honeycomb_bloch_energies(Lx, Ly, t),
                       atol=1e-13)


def test_hs_lambda_values():
    """cosh(lam) = e^{U dtau/2}; spot values for the workloads' (U, dtau)."""
    for U, dt, lam in ((4, 0.1, 0.65373), (2, 0.05, 0.31887), (4, 0.05, 0.45470),
                       (8, 0.05, 0.65373), (8, 0.1, 0.95508)):
        assert abs(dqmc.hs_lambda(U, dt) - lam) < 5e-6
        assert abs(np.cosh(dqmc.hs_lambda(U, dt)) - np.exp(U * dt / 2)) < 1e-14


# ----------------------------------------------------------------------- weight and estimators

def _enumerate(model):
    """Sum over all 2^(N L) fields of W(s) and of W(s) * O(s) with the oracle's pieces."""
    P = Propagators(model)
    N, L = model.N, model.L_tau
    pref = dqmc.weight_prefactor(model)
    Z = 0.0
    acc = {}
    for bits in itertools.product((1, -1), repeat=N * L):
        s = np.array(bits, dtype=np.int8).reshape(L, N)
        Gs, w = [], pref
        for sigma in dqmc.SIGMAS:
            A = dqmc.product_from(P, s, sigma, 0)
            w *= np.linalg.det(np.eye(N) + A)
            Gs.append(np.linalg.inv(np.eye(N) + A))
        assert w > 0                       # half filling, bipartite: no sign problem
        obs = dqmc.measure(P, model, Gs[0], Gs[1])
        Z += w
        for k, v in obs.items():
            acc[k] = acc.get(k, 0.0) + w * v
    return Z, {k: v / Z for k, v in acc.items()}


@pytest.mark.parametrize("case", ["dimer", "plaquette", "honeycomb_ring"])
def test_field_sum_equals_fock_trotter(case):
    """sum_s W(s) = Tr[(e^{-dtau Hk} e^{-dtau HU})^L] and the symmetric-Trotter estimators
    equal Fock-space traces with the operator between half kinetic steps (SM Sec. I.2:
    Trotter split, HS transform and trace-determinant identity are exact per slice)."""
    if case == "dimer":
        model = Model(2, 1, 1.0, 4.0, 1.0, 0.25, 2)
        cl = Cluster(2, DIMER_BONDS, 1.0, 4.0)
        signs = DIMER_SIGNS
    elif case == "plaquette":
        model = Model(2, 2, 1.0, 3.0, 0.9, 0.3, 3)
        cl = Cluster(4, PLAQ_BONDS, 1.0, 3.0)
        signs = PLAQ_SIGNS
    else:
        # 2 x 1 honeycomb cells: A0=0, B0=1, A1=2, B1=3; bonds A0-B0, A0-B1 (x-1), A1-B1,
        # A1-B0 (the y-1 bond repeats the first of each cell): a four-site ring in the
        # honeycomb site order, sublattice signs (+,-,+,-)
        model = Model(2, 1, 1.0, 3.5, 0.8, 0.2, 2, lattice="honeycomb")
        cl = Cluster(4, [(0, 1), (0, 3), (2, 3), (2, 1)], 1.0, 3.5)
        signs = [1, -1, 1, -1]
    Z, obs = _enumerate(model)
    Zf = cl.z_trotter(model.dtau, model.L_tau)
    assert abs(Z / Zf - 1) < 1e-11
    ref = cl.expect_trotter(model.dtau, model.L_tau, signs)
    for k in ("energy", "ekin", "double_occ", "s_pipi", "density"):
        assert abs(obs[k] - ref[k]) < 1e-11, (k, obs[k], ref[k])


def test_trotter_error_is_second_order():
    """Symmetric Trotter values converge to exact diagonalization as O(dtau^2)
    (SM Sec. I.2: error O(dtau^2)); dimer, beta = 2, U = 4."""
    cl = Cluster(2, DIMER_BONDS, 1.0, 4.0)
    beta = 2.0
    exact = cl.expect_exact(beta, DIMER_SIGNS)
    errs = []
    for L in (8, 16, 32):
        v = cl.expect_trotter(beta / L, L, DIMER_SIGNS)
        errs.append(abs(v["double_occ"] - exact["double_occ"]))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# ----------------------------------------------------------------------- U = 0

def test_u0_closed_form():
    """lam = 0: G_0 = (I + e^{-beta K})^{-1} exactly, every flip is accepted, and the
    estimators equal momentum-space sums over f(eps) = 1/(1 + e^{beta eps})."""
    t, beta = 1.0, 2.0
    model = Model(4, 4, t, 0.0, beta, 0.1, 10, seed=3)
    ch = Chain(model, initial_fields(model, 0))
    K = dqmc.hopping_matrix(4, 4, t)
    w, V = np.linalg.eigh(K)
    G_exact = V @ np.diag(1 / (1 + np.exp(-beta * w))) @ V.T
    for _ in range(2):
        ch.sweep(True)
        assert ch.accepts == ch.attempts
        for a in range(2):
            assert np.max(np.abs(ch.G[a] - G_exact)) < 1e-11
    ks = 2 * np.pi * np.arange(4) / 4
    eps = np.array([-2 * t * (np.cos(a) + np.cos(b)) for b in ks for a in ks])
    f = 1 / (1 + np.exp(beta * eps))
    N = 16
    ekin = 2 * np.sum(eps * f) / N
    s_pipi = np.sum((1 - f) ** 2) / (2 * N)
    mm = ch.means()
    assert abs(mm["ekin"] - ekin) < 1e-11
    assert abs(mm["energy"] - ekin) < 1e-11
    assert abs(mm["double_occ"] - 0.25) < 1e-12
    assert abs(mm["s_pipi"] - s_pipi) < 1e-11
    assert abs(mm["density"] - 1.0) < 1e-12


def test_u0_closed_form_honeycomb():
    """Honeycomb, lam = 0: every flip accepted and the estimators equal sums over the Bloch
    bands; with P K P = -K, P G P = I - G, so S(Gamma) = (1/2N) sum (1 - f)^2 too."""
    t, beta = 1.0, 3.0
    model = Model(3, 3, t, 0.0, beta, 0.1, 10, seed=4, lattice="honeycomb")
    ch = Chain(model, initial_fields(model, 1), 1)
    for _ in range(2):
        ch.sweep(True)
        assert ch.accepts == ch.attempts
    eps = _honeycomb_bloch_energies(3, 3, t)
    f = 1 / (1 + np.exp(beta * eps))
    N = 18
    mm = ch.means()
    assert abs(mm["ekin"] - 2 * np.sum(eps * f) / N) < 1e-11
    assert abs(mm["s_pipi"] - np.sum((1 - f) ** 2) / (2 * N)) < 1e-11
    assert abs(mm["double_occ"] - 0.25) < 1e-12
    assert abs(mm["density"] - 1.0) < 1e-12


# ----------------------------------------------------------------------- ratio / updates

def _model_4x4():
    return Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=11)


def test_ratio_equals_determinant_ratio():
    """R^sigma = 1 + Delta (1 - G_ii) equals det(I + A')/det(I + A) for a flipped field."""
    model = _model_4x4()
    P = Propagators(model)
    rng = np.random.default_rng(5)
    s = np.where(rng.random((model.L_tau, model.N)) < 0.5, -1, 1).astype(np.int8)
    for (l, i) in ((0, 0), (7, 3), (19, 15)):
        s2 = s.copy()
        s2[l, i] = -s2[l, i]
        for sigma in dqmc.SIGMAS:
            G = dqmc.green_naive(P, s, sigma, l)
            delta = np.exp(-2 * sigma * P.lam * s[l, i]) - 1
            R = 1 + delta * (1 - G[i, i])
            A = dqmc.product_from(P, s, sigma, l)
            A2 = dqmc.product_from(P, s2, sigma, l)
            d1 = np.linalg.slogdet(np.eye(16) + A)
            d2 = np.linalg.slogdet(np.eye(16) + A2)
            assert abs(R - d2[0] * d1[0] * np.exp(d2[1] - d1[1])) < 1e-10 * abs(R)


def test_fast_update_and_wrap_equal_direct_inversion():
    """After the flips of one slice (Sherman-Morrison) and after each wrap, G equals the
    direct inverse (I + A_l)^{-1} for the current field."""
    model = _model_4x4()
    ch = Chain(model, initial_fields(model, 0))
    dec = np.zeros((model.L_tau, model.N), dtype=np.uint8)
    for l in range(3):
        ch._flip_slice(l, dec)
        for a, sigma in enumerate(dqmc.SIGMAS):
            Gd = dqmc.green_naive(ch.P, ch.s, sigma, l)
            assert np.max(np.abs(ch.G[a] - Gd)) < 1e-10
        ch._wrap_up(l)
        for a, sigma in enumerate(dqmc.SIGMAS):
            Gd = dqmc.green_naive(ch.P, ch.s, sigma, l + 1)
            assert np.max(np.abs(ch.G[a] - Gd)) < 1e-10
    assert dec.sum() > 0
    # wrap down returns to the previous slice
    ch._wrap_down(2)
    for a, sigma in enumerate(dqmc.SIGMAS):
        assert np.max(np.abs(ch.G[a] - dqmc.green_naive(ch.P, ch.s, sigma, 2))) < 1e-10


def test_qrp_udt_is_a_pivoted_udt_decomposition():
    """The stabilization's decomposition M = U diag(D) T against its definition (reading R6),
    on columns graded over 24 decades as a UDV chain makes them: U orthogonal, D the moduli
    of R's diagonal in non-increasing order (column pivoting), T P upper triangular with a
    unit-modulus diagonal, the product reconstructing M column by column, and the first
    pivot the column of largest norm (ties to the lowest index, checked on an exact tie)."""
    rng = np.random.default_rng(7)
    N = 24
    M = rng.normal(size=(N, N)) * np.logspace(-12, 12, N)[rng.permutation(N)][None, :]
    U, D, T = dqmc.qrp_udt(M)
    assert np.max(np.abs(U.T @ U - np.eye(N))) < 1e-13
    assert np.all(D > 0) and np.all(np.diff(D) <= 0)
    # T's column order: T P = R / D is upper triangular with |diagonal| = 1, so pivot k is
    # the column whose last nonzero entry is in row k
    norms = np.linalg.norm(M, axis=0)
    last = [int(np.nonzero(T[:, c])[0].max()) for c in range(N)]
    assert sorted(last) == list(range(N))
    piv = [last.index(k) for k in range(N)]
    TP = T[:, piv]
    assert np.max(np.abs(np.tril(TP, -1))) == 0.0
    assert np.allclose(np.abs(np.diag(TP)), 1.0, atol=1e-12)
    assert piv[0] == int(np.argmax(norms))
    rec = U @ (D[:, None] * T)
    assert np.max(np.abs(rec - M) / norms[None, :]) < 1e-13
    # an exact tie of the largest norms (both exactly 5) goes to the lower index
    Mt = rng.normal(size=(6, 6)) * 0.1
    Mt[:, 1] = [3.0, 4.0, 0.0, 0.0, 0.0, 0.0]
    Mt[:, 4] = [0.0, 0.0, 5.0, 0.0, 0.0, 0.0]
    _, Dt, Tt = dqmc.qrp_udt(Mt)
    assert Dt[0] == 5.0
    assert abs(abs(Tt[0, 1]) - 1.0) < 1e-15 and np.all(Tt[1:, 1] == 0.0)


def test_stabilized_green_vs_scratch_and_naive():
    """Stack-recomputed G agrees with a from-scratch stabilized product (8x8, beta=4,
    cond(A) ~ 1e9) and with direct inversion at small beta."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=2)
    ch = Chain(model, initial_fields(model, 1), chain_index=1)
    for _ in range(2):
        ch.sweep(False)
        l = 0  # after an even number of sweeps, G sits at slice 0
        for a, sigma in enumerate(dqmc.SIGMAS):
            Gs = dqmc.green_scratch(ch.P, ch.s, sigma, l, model.n_wrap)
            assert np.max(np.abs(ch.G[a] - Gs)) < 1e-10
    assert ch.max_drift < 1e-7
    m2 = Model(4, 4, 1.0, 4.0, 1.0, 0.1, 5, seed=2)
    ch2 = Chain(m2, initial_fields(m2, 0))
    ch2.sweep(False)
    for a, sigma in enumerate(dqmc.SIGMAS):   # odd sweep count: G at slice 0 again
        assert np.max(np.abs(ch2.G[a] - dqmc.green_naive(ch2.P, ch2.s, sigma, 0))) < 1e-12


def test_particle_hole_invariants():
    """Bipartite lattice, mu = 0: G^dn = I - P (G^up)^T P with P = diag((-1)^{x+y}),
    G~^up_ii + G~^dn_ii = 1 on every site, R^dn = R^up e^{2 lam s}, sign stays +."""
    model = _model_4x4()
    ch = Chain(model, initial_fields(model, 0))
    p = dqmc.staggered_signs(4, 4)
    Pm = np.diag(p)
    for _ in range(3):
        ch.sweep(True)
        Gu, Gd = ch.G
        assert np.max(np.abs(Gd - (np.eye(16) - Pm @ Gu.T @ Pm))) < 1e-10
        Gtu = ch.P.expK_ph @ Gu @ ch.P.expK_mh
        Gtd = ch.P.expK_ph @ Gd @ ch.P.expK_mh
        assert np.max(np.abs(np.diag(Gtu) + np.diag(Gtd) - 1)) < 1e-10
        for i in range(16):
            s = ch.s[0, i]
            ru = 1 + (np.exp(-2 * ch.P.lam * s) - 1) * (1 - Gu[i, i])
            rd = 1 + (np.exp(+2 * ch.P.lam * s) - 1) * (1 - Gd[i, i])
            assert abs(rd - ru * np.exp(2 * ch.P.lam * s)) < 1e-10 * abs(rd)
    assert ch.sign == 1.0
    assert abs(ch.means()["density"] - 1) < 1e-12


# ----------------------------------------------------------------------- Metropolis

def test_metropolis_samples_the_determinant_weight():
    """Dimer, L_tau = 4: the chain's visited fields follow W(s)/Z (total variation) and its
    observables agree with the exact field sum within 4 sigma (binned errors)."""
    model = Model(2, 1, 1.0, 4.0, 1.0, 0.25, 2, seed=7)
    P = Propagators(model)
    N, L = model.N, model.L_tau
    pref = dqmc.weight_prefactor(model)
    weights = np.zeros(2 ** (N * L))
    for idx in range(weights.size):
        bits = [(idx >> b) & 1 for b in range(N * L)]
        s = np.array([1 - 2 * x for x in bits], dtype=np.int8).reshape(L, N)
        w = pref
        for sigma in dqmc.SIGMAS:
            w *= np.linalg.det(np.eye(N) + dqmc.product_from(P, s, sigma, 0))
        weights[idx] = w
    p_exact = weights / weights.sum()
    Z, exact = _enumerate(model)

    ch = Chain(model, initial_fields(model, 0))
    n_sweeps = 16000
    counts = np.zeros_like(weights)
    pow2 = 2 ** np.arange(N * L)
    for _ in range(n_sweeps):
        ch.sweep(True)
        bits = (1 - ch.s.reshape(-1)) // 2
        counts[int(bits @ pow2)] += 1
    tv = 0.5 * np.sum(np.abs(counts / n_sweeps - p_exact))
    # finite-sample scale: total variation of i.i.d. draws of the same size from W/Z;
    # the chain's samples are mildly correlated, hence the factor 1.5 on the 99th pct.
    rng = np.random.default_rng(0)
    tv_iid = [0.5 * np.sum(np.abs(rng.multinomial(n_sweeps, p_exact) / n_sweeps - p_exact))
              for _ in range(200)]
    assert tv < 1.5 * np.quantile(tv_iid, 0.99), (tv, np.quantile(tv_iid, 0.99))
    nb = 20
    for k in ("double_occ", "energy", "s_pipi"):
        series = np.array([m[k] for m in ch.sweep_means]).reshape(nb, -1).mean(axis=1)
        err = series.std(ddof=1) / np.sqrt(nb)
        assert abs(series.mean() - exact[k]) < 4 * err + 1e-12, (k, series.mean(), exact[k], err)
