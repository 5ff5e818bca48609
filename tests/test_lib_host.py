"""CPU-only checks of the C-ABI library: it loads, exports every symbol include/nmc.h
declares, validates arguments, and its host-side set-up (Philox, e^{cK}) agrees with the
oracle. No device compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import dqmc
from oracle.philox import philox4x32_10

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc as m
    return m


def test_exports_every_declared_symbol(nmc):
    header = open(os.path.join(ROOT, "include", "nmc.h")).read()
    declared = set(re.findall(r"\b(nmc_[a-z_]+)\s*\(", header))
    assert declared == set(nmc.EXPORTED), declared ^ set(nmc.EXPORTED)
    lib = ctypes.CDLL(nmc.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert "sm_103a" in nmc.nmc_version()


def test_exports_every_conv_generator_symbol(nmc):
    header = open(os.path.join(ROOT, "include", "nmc_cgen.h")).read()
    declared = set(re.findall(r"\b(nmc_cgen_[a-z_]+)\s*\(", header))
    assert declared == set(nmc.EXPORTED_CGEN), declared ^ set(nmc.EXPORTED_CGEN)
    lib = ctypes.CDLL(nmc.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_conv_generator_rejects_bad_sizes_without_gpu_work(nmc):
    lib = nmc.load()
    h = ctypes.c_void_p()
    for args in ((0, 8, 40, 32), (8, 8, 40, 0), (8, 8, 40, 65), (8, 8, 0, 32)):
        assert lib.nmc_cgen_create(*args, 0, 4, None, ctypes.byref(h)) == nmc.NMC_EINVAL
    assert lib.nmc_cgen_create(8, 8, 40, 32, 0, 0, None, ctypes.byref(h)) == nmc.NMC_EINVAL


def test_exports_every_generator_symbol(nmc):
    header = open(os.path.join(ROOT, "include", "nmc_gen.h")).read()
    declared = set(re.findall(r"\b(nmc_gen_[a-z_]+)\s*\(", header))
    assert declared == set(nmc.EXPORTED_GEN), declared ^ set(nmc.EXPORTED_GEN)
    lib = ctypes.CDLL(nmc.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    a = nmc.gen_arch()
    assert (tuple(a.z), a.c1, tuple(a.k1), tuple(a.k2)) == ((10, 2, 2), 20, (16, 6, 3), (36, 6, 3))


def test_create_validates_arguments(nmc):
    good = dict(Lx=4, Ly=4, t=1.0, U=4.0, beta=2.0, dtau=0.1, n_wrap=10, seed=0)
    ctx = nmc.nmc_create(**good)
    assert nmc.nmc_get_dims(ctx)[:2] == (16, 20)
    nmc.nmc_destroy(ctx)
    bad = [dict(Lx=3), dict(Lx=1, Ly=1), dict(t=0.0), dict(U=-1.0), dict(beta=0.0),
           dict(dtau=-0.1), dict(dtau=0.3), dict(n_wrap=3), dict(n_wrap=0), dict(Lx=64, Ly=32)]
    for b in bad:
        with pytest.raises(nmc.NmcError) as e:
            nmc.nmc_create(**{**good, **b})
        assert e.value.status == nmc.NMC_EINVAL, b
    # 1 x 2 chain and the 2-site dimer are allowed
    for lx, ly in ((2, 1), (1, 2)):
        nmc.nmc_destroy(nmc.nmc_create(**{**good, "Lx": lx, "Ly": ly}))
    # honeycomb: 2 sites per cell, any cell counts (bipartite by construction)
    for lx, ly, n in ((3, 3, 18), (6, 6, 72), (1, 1, 2)):
        ctx = nmc.nmc_create(**{**good, "Lx": lx, "Ly": ly, "lattice": nmc.NMC_HONEYCOMB})
        assert nmc.nmc_get_dims(ctx)[0] == n
        nmc.nmc_destroy(ctx)
    for b in (dict(lattice=2), dict(lattice=-1), dict(lattice=nmc.NMC_HONEYCOMB, Lx=32, Ly=17)):
        with pytest.raises(nmc.NmcError) as e:
            nmc.nmc_create(**{**good, **b})
        assert e.value.status == nmc.NMC_EINVAL, b


def test_state_errors_without_gpu_work(nmc):
    ctx = nmc.nmc_create(4, 4, 1.0, 4.0, 2.0, 0.1, 10, 0)
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_sweep(ctx, 1)
    assert e.value.status == nmc.NMC_ESTATE
    s = np.ones((1, 20, 16), dtype=np.int8)
    s[0, 3, 5] = 0
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_set_fields(ctx, s)
    assert e.value.status == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_set_fields(ctx, np.ones((1, 20, 15), dtype=np.int8))
    assert e.value.status == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_generate(ctx, mode=1)
    assert e.value.status == nmc.NMC_EINVAL
    bad = nmc.nmc_default_options()
    bad.n_chains = 0
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_configure(ctx, bad)
    assert e.value.status == nmc.NMC_EINVAL
    # FP32-pair stabilization products exist for the compensated precisions only
    for prec in (nmc.NMC_FP64, nmc.NMC_FP32):
        bad = nmc.nmc_default_options()
        bad.precision, bad.stab_pairs = prec, 1
        with pytest.raises(nmc.NmcError) as e:
            nmc.nmc_configure(ctx, bad)
        assert e.value.status == nmc.NMC_EINVAL
    bad = nmc.nmc_default_options()
    bad.precision, bad.stab_pairs = nmc.NMC_SPLIT_BF16, 2
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_configure(ctx, bad)
    assert e.value.status == nmc.NMC_EINVAL
    nmc.nmc_destroy(ctx)


def test_host_philox_equals_oracle(nmc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        w = [int(x) for x in rng.integers(0, 2 ** 32, size=6, dtype=np.uint64)]
        mine = nmc.nmc_philox(*w)
        ref = [int(x) for x in philox4x32_10(*w)]
        assert mine == ref


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (2, 1), (2, 2), (6, 4), (8, 8), (1, 2)])
def test_host_expk_equals_oracle(nmc, Lx, Ly):
    for c in (-0.1, 0.1, -0.05, 0.025):
        mine = nmc.nmc_expk(Lx, Ly, 1.0, c)
        ref = dqmc.expm_sym(dqmc.hopping_matrix(Lx, Ly, 1.0), c)
        # two eigensolvers: agreement to a few N * eps
        assert np.max(np.abs(mine - ref)) < 1e-13


@pytest.mark.parametrize("Lx,Ly", [(3, 3), (6, 6), (2, 1), (4, 2)])
def test_host_honeycomb_expk_equals_oracle(nmc, Lx, Ly):
    model = dqmc.Model(Lx, Ly, 1.0, 0.0, 1.0, 0.1, 10, lattice="honeycomb")
    K = dqmc.lattice_hopping(model)
    for c in (-0.1, 0.05):
        mine = nmc.nmc_expk(Lx, Ly, 1.0, c, lattice="honeycomb")
        assert np.max(np.abs(mine - dqmc.expm_sym(K, c))) < 1e-13


def test_expk_plane_wave_closed_form(nmc):
    """e^{cK}_{ij} = (1/N) sum_k cos(k.(r_i - r_j)) e^{c eps_k} on the periodic lattice."""
    L, c, t = 6, -0.1, 1.0
    mine = nmc.nmc_expk(L, L, t, c)
    ks = 2 * np.pi * np.arange(L) / L
    xs = np.array([i % L for i in range(L * L)])
    ys = np.array([i // L for i in range(L * L)])
    ref = np.zeros((L * L, L * L))
    for kx in ks:
        for ky in ks:
            eps = -2 * t * (np.cos(kx) + np.cos(ky))
            ph = kx * (xs[:, None] - xs[None, :]) + ky * (ys[:, None] - ys[None, :])
            ref += np.cos(ph) * np.exp(c * eps)
    ref /= L * L
    assert np.max(np.abs(mine - ref)) < 1e-14
