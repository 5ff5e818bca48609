"""Full-size parity for the 16x16 workload: N=256, beta=8, dtau=0.05 (L_tau=160),
n_wrap=8, delayed-update rank 32 (clamped to the shared-memory budget), 32 chains.

At N=256 the flip kernel keeps G in global memory (L2) and the QR / Gauss-Jordan kernels
use their global workspace. The oracle runs one sampled chain (about ten seconds per sweep
on the host); the GPU runs all 32 chains in the same launch configuration.
"""
import numpy as np
import pytest

from oracle.dqmc import Chain, Model, initial_fields

pytestmark = pytest.mark.gpu

MODEL = Model(16, 16, 1.0, 4.0, 8.0, 0.05, 8, seed=0)
CHAINS = 32
SAMPLE = 19


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


@pytest.fixture(scope="module")
def oracle_chain():
    ch = Chain(MODEL, initial_fields(MODEL, SAMPLE), SAMPLE)
    G0 = [g.copy() for g in ch.G]
    ch.sweep(True)
    return G0, ch


def _ctx(nmc, prec):
    m = MODEL
    return nmc.Context(m.Lx, m.Ly, m.t, m.U, m.beta, m.dtau, m.n_wrap, seed=m.seed,
                       n_chains=CHAINS, delay_k=32, precision=prec, drift_tol=1e-3)


@pytest.mark.parametrize("prec,g_rel", [(0, 1e-10), (2, 1e-8)])
def test_16x16_one_sweep_matches_oracle(nmc, oracle_chain, prec, g_rel):
    G0, ref = oracle_chain
    with _ctx(nmc, prec) as c:
        c.generate()
        for spin in (0, 1):
            G = c.green(SAMPLE, spin)
            assert np.max(np.abs(G - G0[spin])) / np.max(np.abs(G0[spin])) < g_rel
        c.sweep(1, measure=1)
        np.testing.assert_array_equal(c.fields()[SAMPLE], ref.s)
        for spin in (0, 1):
            G = c.green(SAMPLE, spin)
            assert np.max(np.abs(G - ref.G[spin])) / np.max(np.abs(ref.G[spin])) < g_rel
        obs, per = c.measure(per_chain=True)
        want = ref.means()
        for k in ("energy", "double_occ", "s_pipi"):
            assert abs(getattr(per[SAMPLE], k).mean - want[k]) < 1e-8, k
        hist = c.drift_history()
        assert len(hist) == MODEL.L_tau // MODEL.n_wrap
        assert np.all(hist <= 1e-5), hist.max()
