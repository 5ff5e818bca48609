"""The stabilization's products accumulated in FP32 pairs (nmc_options.stab_pairs): the T
updates of the UDT stacks and the three products of the recompute take FP64 operands and
give FP64 results but sum in FP32 pairs. Held to the FP64 bar against the oracle: G of the
initial stacks to 1e-10 relative, every decision of free-running chains bit-exact (the
benchmark configuration, graph-replayed), G at the end and observables as for the
compensated paths."""
import numpy as np
import pytest

from oracle.dqmc import Chain, Model
from paper_2106_00712_gb300.workloads import random_fields

from test_gpu_parity import G_REL, G_REL_X2, _compare_run, _ctx, _rel, nmc  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [2, 4])    # NMC_SPLIT_BF16, NMC_FP32X2
@pytest.mark.parametrize("Lx,Ly,n_wrap", [(4, 4, 10), (2, 1, 2), (6, 6, 5), (10, 10, 4)])
def test_stab_pairs_initial_green_equals_oracle(nmc, Lx, Ly, n_wrap, prec):
    model = Model(Lx, Ly, 1.0, 4.0, 2.0, 0.1, n_wrap, seed=5)
    fields = random_fields(3, model.L_tau, model.N, seed=11)
    with _ctx(nmc, model, n_chains=3, precision=prec, stab_pairs=1) as c:
        c.set_fields(fields)
        for ch in range(3):
            ref = Chain(model, fields[ch], ch)
            for spin in (0, 1):
                assert _rel(c.green(ch, spin), ref.G[spin]) < G_REL


def test_stab_pairs_low_temperature_green_equals_oracle(nmc):
    """beta = 10 at U = 8 (the D of a stack spans many decades): the D-split keeps the
    pair-accumulated operands in the FP32 range, and G of the stacks is as close to the
    oracle's as with FP64 products (1e-10 relative, or 10x the FP64 products' distance)."""
    model = Model(4, 4, 1.0, 8.0, 10.0, 0.1, 10, seed=9)
    fields = random_fields(2, model.L_tau, model.N, seed=4)
    refs = [Chain(model, fields[ch], ch) for ch in range(2)]
    err = {}
    for sp in (0, 1):
        with _ctx(nmc, model, n_chains=2, precision=nmc.NMC_SPLIT_BF16, stab_pairs=sp) as c:
            c.set_fields(fields)
            err[sp] = max(_rel(c.green(ch, s), refs[ch].G[s]) for ch in range(2) for s in (0, 1))
    assert err[1] < max(G_REL, 10 * err[0]), err


def test_stab_pairs_free_running_4x4_matches_oracle(nmc):
    model = Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=0)
    _compare_run(nmc, model, chains=1, n_sweeps=60, measure_from=10,
                 precision=nmc.NMC_SPLIT_BF16, g_rel=G_REL_X2, stab_pairs=1)


@pytest.mark.parametrize("prec", [2, 4])
def test_stab_pairs_ragged_sizes(nmc, prec):
    model = Model(6, 4, 1.0, 4.0, 1.2, 0.1, 4, seed=2)
    _compare_run(nmc, model, chains=3, n_sweeps=4, measure_from=1, delay_k=5,
                 precision=prec, g_rel=G_REL_X2, stab_pairs=1)


def test_stab_pairs_bench_config_graph_replayed_sampled(nmc):
    """The benchmark configuration (8x8, U=4, beta=4, 256 chains, NMC_SPLIT_BF16) with the
    stabilization products in FP32 pairs, eight sweeps of which six replay recorded graphs:
    decisions bit-exact on four sampled chains, no FP64 product launched."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=0)

    def check(c):
        rec, rep = c.graph_stats()
        assert rec == 2 and rep == 6, (rec, rep)
        st = c.kernel_stats()
        assert st["gemm_pair"][0] > 0 and st["gemm"][0] == 0, st

    _compare_run(nmc, model, chains=256, n_sweeps=8, measure_from=0, delay_k=16,
                 check_chains=[0, 77, 190, 255], precision=nmc.NMC_SPLIT_BF16,
                 g_rel=G_REL_X2, after=check, stab_pairs=1)


def test_stab_pairs_recompute_equals_fp64_recompute(nmc):
    """Same fields, both settings: the stacks' G agree to 1e-11 relative, and after three
    sweeps the fields are identical."""
    model = Model(8, 8, 1.0, 4.0, 4.0, 0.1, 10, seed=1)
    out = {}
    for sp in (0, 1):
        with _ctx(nmc, model, n_chains=4, precision=nmc.NMC_SPLIT_BF16, stab_pairs=sp) as c:
            c.generate()
            g0 = np.stack([c.green(ch, s) for ch in range(4) for s in (0, 1)])
            c.sweep(3, measure=1)
            out[sp] = (g0, c.fields())
    assert _rel(out[1][0], out[0][0]) < 1e-11
    np.testing.assert_array_equal(out[1][1], out[0][1])
