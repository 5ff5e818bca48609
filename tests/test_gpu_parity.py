"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bar: bit-exact for integer work (Philox words, initial fields, every flip decision, seen
as the field after each sweep); G to 1e-10 relative in the FP64 path; observables to
1e-9. Reduced-precision paths are compared on the oracle's own trajectory (replay).
"""
import numpy as np
import pytest

from oracle import dqmc
from oracle.dqmc import Chain, Model, initial_fields
from oracle.philox import init_fields, philox4x32_10
from paper_2106_00712_gb300.workloads import random_fields

pytestmark = pytest.mark.gpu

G_REL = 1e-10
OBS_ABS = 1e-9


@pytest.fixture(scope="module")
def nmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc as m
    m.load()
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _ctx(nmc, model, **kw):
    return nmc.Context(model.Lx, model.Ly, model.t, model.U, model.beta, model.dtau,
                       model.n_wrap, seed=model.seed, lattice=model.lattice, **kw)


def _compare_run(nmc, model, chains, n_sweeps, measure_from=0, delay_k=16, fields=None,
                 check_chains=None, chain_offset=0, precision=0, g_rel=G_REL, ph=0,
                 after=None, **opts):
    """Run n_sweeps on the GPU and on the oracle for the checked chains; compare the
    field after every sweep (bit-exact), G at the end and the accumulated observables.
    `after(c)`, if given, runs on the context before it closes."""
    check = list(range(chains)) if check_chains is None else check_chains
    with _ctx(nmc, model, n_chains=chains, delay_k=delay_k, chain_offset=chain_offset,
              drift_tol=1e-3, precision=precision, ph_symmetric=ph, **opts) as c:
        if fields is None:
            c.generate()
            refs = {ch: Chain(model, initial_fields(model, ch + chain_offset), ch + chain_offset)
                    for ch in check}
        else:
            c.set_fields(fields)
            refs = {ch: Chain(model, fields[ch], ch + chain_offset) for ch in check}
        f = c.fields()
        for ch in check:
            assert np.array_equal(f[ch], refs[ch].s)
        for sw in range(n_sweeps):
            meas = sw >= measure_from
            c.sweep(1, measure=int(meas))
            for r in refs.values():
                r.sweep(meas)
            f = c.fields()
            for ch in check:
                assert np.array_equal(f[ch], refs[ch].s), f"decisions differ: sweep {sw} chain {ch}"
        for ch in check:
            for spin in (0, 1):
                assert _rel(c.green(ch, spin), refs[ch].G[spin]) < g_rel
        if n_sweeps > measure_from:
            _, per = c.measure(per_chain=True)
            for ch in check:
                want = refs[ch].means()
                got = per[ch]
                for k in ("energy", "ekin", "double_occ", "s_pipi", "density"):
                    assert abs(getattr(got, k).mean - want[k]) < OBS_ABS, (k, ch)
                assert abs(got.accept - want["accept"]) < 1e-15
                # same arithmetic class as the oracle: drift of the same order
                assert got.max_drift < max(1e-8, 100 * refs[ch].max_drift), (
                    got.max_drift, refs[ch].max_drift)
        if after is not None:
            after(c)
        return c.measure()


def test_device_philox_equals_oracle(nmc):
    import torch
    n = 4096
    rng = np.random.default_rng(3)
    c0 = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    d_c0 = torch.from_numpy(c0.view(np.int32).copy()).cuda()
    d_out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    for (c1, c2, c3, k0, k1) in ((0, 0, 0, 0, 0), (7, 255, 1, 0xDEADBEEF, 0x12345678),
                                 (2 ** 32 - 1, 3, 0, 1, 2 ** 32 - 1)):
        nmc.nmc_philox_device(d_c0.data_ptr(), n, c1, c2, c3, k0, k1, d_out.data_ptr())
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32).reshape(n, 4)
        ref = np.stack([w.astype(np.uint32) for w in
                        philox4x32_10(c0.astype(np.uint64), c1, c2, c3, k0, k1)], axis=1)
        np.testing.assert_array_equal(got, ref)


def test_generated_fields_equal_oracle(nmc):
    model = Model(6, 4, 1.0, 4.0, 1.5, 0.1, 5, seed=0xABCDEF0123)
    with _ctx(nmc, model, n_chains=5, chain_offset=1000) as c:
        c.generate()
        f = c.fields()
    for ch in range(5):
        np.testing.assert_array_equal(f[ch], init_fields(model.seed, model.L_tau, model.N,
                                                         1000 + ch))


@pytest.mark.parametrize("Lx,Ly,n_wrap", [(4, 4, 10), (2, 1, 2), (6, 6, 5), (10, 10, 4)])
def test_initial_green_equals_oracle(nmc, Lx, Ly, n_wrap):
    model = Model(Lx, Ly, 1.0, 4.0, 2.0, 0.1, n_wrap, seed=5)
    fields = random_fields(3, model.L_tau, model.N, seed=11)
    with _ctx(nmc, model, n_chains=3) as c:
        c.set_fields(fields)
        for ch in range(3):
            ref = Chain(model, fields[ch], ch)
            for spin in (0, 1):
                assert _rel(c.green(ch, spin), ref.G[spin]) < G_REL


def test_config_4x4_full_run_matches_oracle(nmc):
    """4x4, U=4, beta=2, dtau=0.1, n_wrap=10, seed 0, Philox init, 200 sweeps (measure
    from sweep 51): every decision identical, G and observables equal."""
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=0)
    pooled = _compare_run(nmc, model, chains=1, n_sweeps=200, measure_from=50)
    assert pooled.n_meas == 150 * 2
    assert abs(pooled.sign.mean - 1.0) < 1e-15
    assert abs(pooled.density.mean - 1.0) < 1e-12


@pytest.mark.parametrize("Lx,Ly,U,beta,dtau,n_wrap,k,chains", [
    (2, 1, 4.0, 1.0, 0.25, 2, 16, 3),     # dimer, N=2
    (1, 2, 3.0, 1.0, 0.1, 10, 4, 2),      # one bond along y
    (2, 2, 6.0, 1.2, 0.1, 1, 2, 2),       # n_wrap = 1
    (6, 6, 4.0, 2.0, 0.1, 20, 5, 3),      # N=36 ragged tiles, n_wrap = L_tau, odd k
    (6, 4, 8.0, 1.0, 0.1, 5, 16, 2),      # rectangular, U=8
    (10, 10, 4.0, 1.0, 0.1, 5, 16, 2),    # N=100: G in global memory in the flip kernel
    (12, 12, 2.0, 0.6, 0.1, 3, 8, 1),     # N=144 > 111: stabilization in global workspace
])
def test_ragged_and_edge_sizes(nmc, Lx, Ly, U, beta, dtau, n_wrap, k, chains):
    model = Model(Lx, Ly, 1.0, U, beta, dtau, n_wrap, seed=17)
    _compare_run(nmc, model, chains=chains, n_sweeps=4, measure_from=1, delay_k=k)


def test_u_zero_all_accepted_closed_form(nmc):
    model = Model(4, 4, 1.0, 0.0, 2.0, 0.1, 10, seed=1)
    with _ctx(nmc, model, n_chains=2) as c:
        c.generate()
        c.sweep(3, measure=1)
        obs = c.measure()
        assert obs.accept == 1.0
        K = dqmc.hopping_matrix(4, 4, 1.0)
        w, V = np.linalg.eigh(K)
        G_exact = V @ np.diag(1 / (1 + np.exp(-2.0 * w))) @ V.T
        assert _rel(c.green(1, 0), G_exact) < 1e-11
        assert abs(obs.double_occ.mean - 0.25) < 1e-12


def test_config_8x8_256_chains_sampled(nmc):
    """8x8, U=4, beta=4, L_tau=40, n_wrap=10, k=16, 256 chains (the benchmark launch
    configuration); oracle on sampled chains for two sweeps (one each direction)."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=256, n_sweeps=2, measure_from=0, delay_k=16,
                 check_chains=[0, 1, 137, 255])


def test_checkpoint_resume_is_exact(nmc):
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 5, seed=9)
    with _ctx(nmc, model, n_chains=3) as a:
        a.generate()
        a.sweep(5, measure=1)
        blob = a.checkpoint()
        a.sweep(4, measure=1)
        want_f, want_o = a.fields(), a.measure()
    with _ctx(nmc, model, n_chains=3) as b:
        b.restore(blob)
        b.sweep(4, measure=1)
        np.testing.assert_array_equal(b.fields(), want_f)
        got = b.measure()
        assert abs(got.energy.mean - want_o.energy.mean) < 1e-10
        assert got.n_meas == want_o.n_meas


def test_chain_sharding_is_partition_independent(nmc):
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=4)
    with _ctx(nmc, model, n_chains=6) as full:
        full.generate()
        full.sweep(3, measure=0)
        f_all = full.fields()
    parts = []
    for off, n in ((0, 2), (2, 4)):
        with _ctx(nmc, model, n_chains=n, chain_offset=off) as c:
            c.generate()
            c.sweep(3, measure=0)
            parts.append(c.fields())
    np.testing.assert_array_equal(np.concatenate(parts), f_all)


def test_fp32_replay_follows_oracle_trajectory(nmc):
    """Plain FP32 propagation on the oracle's trajectory (replay). Wrap errors grow about
    2-3x per slice here (cond(B) ~ 6.5), so FP32 cannot hold 1e-5 over n_wrap = 10 (the
    recorded drift against the FP64 recompute is O(0.1)). The fields follow the oracle
    exactly, and the observables, measured on the FP64-recomputed G of identical fields,
    equal the oracle's."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)
    chains = 2
    refs = [Chain(model, initial_fields(model, ch), ch) for ch in range(chains)]
    with _ctx(nmc, model, n_chains=chains, precision=nmc.NMC_FP32, drift_tol=1.0) as c:
        c.generate()
        for sw in range(4):
            before = np.stack([r.s.copy() for r in refs])
            for r in refs:
                r.sweep(True)
            accept = (np.stack([r.s for r in refs]) != before).astype(np.uint8)
            c.sweep_replay(accept, measure=1)
            np.testing.assert_array_equal(c.fields(), np.stack([r.s for r in refs]))
        obs, per = c.measure(per_chain=True)
        attempts = 4 * chains * model.N * model.L_tau
        assert obs.max_drift < 1.0, obs.max_drift
        assert obs.n_disagree <= 0.05 * attempts
        for ch in range(chains):
            want = refs[ch].means()
            for k in ("energy", "double_occ", "s_pipi", "density"):
                assert abs(getattr(per[ch], k).mean - want[k]) < OBS_ABS, k


# compensated FP32-pair propagation: ~2^-44 per operation, so G tracks FP64 to ~1e-10
G_REL_X2 = 1e-8


def test_fp32x2_replay_meets_accuracy_bar(nmc):
    """FP32X2 on the oracle's trajectory: max|G - G_fp64| <= 1e-5 before every
    stabilization (recorded drift against the FP64 recompute), G at the end within 1e-8
    of the oracle's, no decision of its own differs, observables equal the oracle's."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)
    chains = 2
    refs = [Chain(model, initial_fields(model, ch), ch) for ch in range(chains)]
    with _ctx(nmc, model, n_chains=chains, precision=nmc.NMC_SPLIT_BF16) as c:
        c.generate()
        for sw in range(4):
            before = np.stack([r.s.copy() for r in refs])
            for r in refs:
                r.sweep(True)
            accept = (np.stack([r.s for r in refs]) != before).astype(np.uint8)
            c.sweep_replay(accept, measure=1)
            np.testing.assert_array_equal(c.fields(), np.stack([r.s for r in refs]))
        obs, per = c.measure(per_chain=True)
        assert obs.max_drift <= 1e-5, obs.max_drift
        assert obs.n_disagree == 0
        for ch in range(chains):
            for spin in (0, 1):
                assert _rel(c.green(ch, spin), refs[ch].G[spin]) < G_REL_X2
            want = refs[ch].means()
            for k in ("energy", "double_occ", "s_pipi", "density"):
                assert abs(getattr(per[ch], k).mean - want[k]) < OBS_ABS, k


def test_fp32x2_free_running_decisions_equal_oracle(nmc):
    """Free-running FP32X2 chains make the oracle's decisions (4x4, 60 sweeps)."""
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=1, n_sweeps=60, measure_from=10,
                 precision=nmc.NMC_SPLIT_BF16, g_rel=G_REL_X2)


@pytest.mark.parametrize("prec", [2, 4])    # NMC_SPLIT_BF16, NMC_FP32X2
@pytest.mark.parametrize("Lx,Ly,n_wrap,k,chains", [
    (2, 1, 2, 16, 2), (6, 6, 5, 5, 2), (10, 10, 5, 16, 2), (12, 12, 5, 8, 1)])
def test_fp32x2_ragged_sizes(nmc, Lx, Ly, n_wrap, k, chains, prec):
    model = Model(Lx, Ly, 1.0, 4.0, 1.0, 0.1, n_wrap, seed=23)
    _compare_run(nmc, model, chains=chains, n_sweeps=3, measure_from=1, delay_k=k,
                 precision=prec, g_rel=G_REL_X2)


def test_fp32x2_8x8_256_chains_sampled(nmc):
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=256, n_sweeps=2, measure_from=0, delay_k=16,
                 check_chains=[3, 200], precision=nmc.NMC_SPLIT_BF16, g_rel=G_REL_X2)


def test_bench_config_graph_replayed_tensor_core_sampled(nmc):
    """The benchmark configuration as bench.py times it: 8x8, U=4, beta=4, L_tau=40,
    n_wrap=10, k=16, 256 chains, NMC_SPLIT_BF16 (products on the tensor cores), sweeps
    replayed from recorded CUDA graphs. Eight measuring sweeps: the first two launch
    directly (the graphs are recorded after them), the other six replay the recorded graph
    of their direction. Oracle on four sampled chains: fields after every sweep bit-exact,
    G at the end to 1e-8 relative, per-chain observables to 1e-9."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)

    def replayed(c):
        rec, rep = c.graph_stats()
        assert rec == 2 and rep == 6, (rec, rep)
        st = c.kernel_stats()
        assert st["gemm_tc"][0] > 0 and st["gemm_df"][0] == 0

    _compare_run(nmc, model, chains=256, n_sweeps=8, measure_from=0, delay_k=16,
                 check_chains=[0, 77, 190, 255], precision=nmc.NMC_SPLIT_BF16,
                 g_rel=G_REL_X2, after=replayed)


def test_fp32x2_tensor_core_slicing_equals_simt(nmc):
    """The exact-slicing BF16 tensor-core products and the SIMT double-float products give
    the same chain and the same G to FP64-class accuracy (8x8, beta=4, 3 sweeps)."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=3)
    gs = {}
    for impl, prec in ((0, nmc.NMC_SPLIT_BF16), (1, nmc.NMC_FP32X2)):
        with _ctx(nmc, model, n_chains=8, precision=prec) as c:
            c.generate()
            c.sweep(3, measure=1)
            st = c.kernel_stats()
            assert st["gemm_tc" if impl == 0 else "gemm_df"][0] > 0
            assert st["gemm_df" if impl == 0 else "gemm_tc"][0] == 0
            gs[impl] = (c.fields(), [c.green(ch, sp) for ch in range(8) for sp in (0, 1)],
                        c.measure().max_drift)
    np.testing.assert_array_equal(gs[0][0], gs[1][0])
    for a, b in zip(gs[0][1], gs[1][1]):
        assert np.max(np.abs(a - b)) < 1e-9
    assert gs[0][2] <= 1e-5


# particle-hole single-spin mode: spin down derived from spin up, same chain

@pytest.mark.parametrize("prec", [0, 2])
def test_ph_single_spin_4x4_matches_oracle(nmc, prec):
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=2, n_sweeps=40, measure_from=5, precision=prec,
                 g_rel=G_REL if prec == 0 else G_REL_X2, ph=1)


@pytest.mark.parametrize("Lx,Ly,n_wrap,k,prec", [
    (2, 1, 2, 16, 0), (6, 6, 5, 5, 0), (10, 10, 5, 16, 2), (12, 12, 5, 8, 0)])
def test_ph_single_spin_ragged_sizes(nmc, Lx, Ly, n_wrap, k, prec):
    model = Model(Lx, Ly, 1.0, 4.0, 1.0, 0.1, n_wrap, seed=29)
    _compare_run(nmc, model, chains=2, n_sweeps=3, measure_from=1, delay_k=k, precision=prec,
                 g_rel=G_REL if prec == 0 else G_REL_X2, ph=1)


def test_ph_single_spin_8x8_256_chains_sampled(nmc):
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=256, n_sweeps=2, measure_from=0, delay_k=16,
                 check_chains=[0, 255], precision=nmc.NMC_SPLIT_BF16, g_rel=G_REL_X2, ph=1)


# honeycomb lattice of the paper's Hubbard runs (2 L^2 sites; U = 3.83, beta = 6, dtau = 0.1
# at L = 6); decisions bit-exact in every mode, spin-down G derived by the sublattice signs
@pytest.mark.parametrize("prec,ph", [(0, 0), (2, 0), (0, 1), (2, 1)])
def test_honeycomb_matches_oracle(nmc, prec, ph):
    model = Model(3, 3, 1.0, 3.83, 2.0, 0.1, 10, seed=5, lattice="honeycomb")
    _compare_run(nmc, model, chains=3, n_sweeps=8, measure_from=2, delay_k=5, precision=prec,
                 g_rel=G_REL if prec == 0 else G_REL_X2, ph=ph)


@pytest.mark.parametrize("prec,ph", [(0, 0), (2, 1)])
def test_honeycomb_6x6_paper_point_sampled(nmc, prec, ph):
    model = Model(6, 6, 1.0, 3.83, 6.0, 0.1, 10, seed=0x6C, lattice="honeycomb")
    _compare_run(nmc, model, chains=64, n_sweeps=3, measure_from=1, delay_k=16,
                 check_chains=[1, 62], precision=prec,
                 g_rel=G_REL if prec == 0 else G_REL_X2, ph=ph)


def test_state_errors_on_device(nmc):
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10)
    with _ctx(nmc, model, n_chains=2) as c:
        with pytest.raises(nmc.NmcError):
            c.sweep(1)
        c.generate()
        with pytest.raises(nmc.NmcError):
            c.sweep_replay(np.zeros((2, 20, 15), np.uint8))
        with pytest.raises(nmc.NmcError):
            nmc.nmc_configure(c.ctx, nmc.nmc_default_options())
        with pytest.raises(nmc.NmcError):
            c.green(2, 0)


@pytest.mark.parametrize("prec,ph", [(0, 0), (2, 0), (2, 1)])
def test_sweep_graphs_equal_direct_launches(nmc, prec, ph):
    """Sweeps replayed from recorded CUDA graphs give the same fields, G, observables and
    drift history as direct launches, across warm-up and measuring sweeps, a checkpoint and a
    restore (which re-arranges the stack buffers)."""
    model = Model(6, 4, 1.0, 4.0, 2.0, 0.1, 5, seed=21)
    out = []
    for graphs in (1, 0):
        with _ctx(nmc, model, n_chains=3, precision=prec, ph_symmetric=ph, drift_tol=1e-3,
                  sweep_graphs=graphs) as c:
            c.generate()
            c.sweep(5, measure=0)
            c.sweep(4, measure=1)
            blob = c.checkpoint()
            c.sweep(3, measure=1)
            c.restore(blob)
            c.sweep(5, measure=1)
            o = c.measure()
            out.append((c.fields(), c.green(1, 0), o.energy.mean, o.s_pipi.mean,
                        c.drift_history(), c.series()))
    a, b = out
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]
    np.testing.assert_array_equal(a[4], b[4])
    np.testing.assert_array_equal(a[5], b[5])
