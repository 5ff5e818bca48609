"""The allocation-free entry point nmc_green_noalloc against the existing path.

nmc_green_noalloc serves callers that cannot allocate device memory when they need G:
it takes device inputs and outputs and keeps its temporaries in a fixed array inside the
library. Two calls in a row (different chain counts; the second spans two chunks of the
fixed array) must each return the G that nmc_set_fields + nmc_get_green give for the
same fields, to the FP64 parity tolerance (1e-10 relative). This file is collected last.
"""
import math

import numpy as np
import pytest

from paper_2106_00712_gb300.workloads import random_fields

pytestmark = pytest.mark.gpu

G_REL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc
    nmc.load()
    return torch, nmc


def _existing(nmc, Lx, Ly, t, U, beta, dtau, n_wrap, fields):
    chains = fields.shape[0]
    with nmc.Context(Lx, Ly, t, U, beta, dtau, n_wrap, seed=0, n_chains=chains) as c:
        c.set_fields(fields)
        return np.stack([np.stack([c.green(ch, sp) for sp in (0, 1)]) for ch in range(chains)])


def test_no_alloc_green_matches_existing_entry_point(env):
    torch, nmc = env
    Lx, Ly, t, U, beta, dtau, n_wrap = 8, 8, 1.0, 4.0, 2.0, 0.1, 5
    N, L = Lx * Ly, int(round(beta / dtau))
    lam = math.acosh(math.exp(dtau * U / 2))
    expk = torch.from_numpy(nmc.nmc_expk(Lx, Ly, t, -dtau)).cuda()
    stream = torch.cuda.current_stream()
    for chains, seed in ((5, 1), (60, 2)):    # 60 chains of N=64 span two chunks
        fields = random_fields(chains, L, N, seed)
        want = _existing(nmc, Lx, Ly, t, U, beta, dtau, n_wrap, fields)
        d_fields = torch.from_numpy(fields).cuda()
        d_G = torch.full((chains, 2, N, N), float("nan"), dtype=torch.float64, device="cuda")
        nmc.nmc_green_noalloc(N, L, n_wrap, lam, expk.data_ptr(), d_fields.data_ptr(), chains,
                              d_G.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = d_G.cpu().numpy()
        assert np.all(np.isfinite(got))
        rel = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert rel < G_REL, rel


def test_no_alloc_green_with_solver_workspace_matches_existing(env):
    """N = 144 (12 x 12) is above the size whose QR and solve fit in shared memory, so each
    chain also takes the 2 N^2-per-matrix solver workspace; 10 chains span two chunks of the
    fixed array (8 chains fit), and two calls run back to back."""
    torch, nmc = env
    Lx, Ly, t, U, beta, dtau, n_wrap = 12, 12, 1.0, 4.0, 0.4, 0.1, 2
    N, L = Lx * Ly, int(round(beta / dtau))
    lam = math.acosh(math.exp(dtau * U / 2))
    expk = torch.from_numpy(nmc.nmc_expk(Lx, Ly, t, -dtau)).cuda()
    stream = torch.cuda.current_stream()
    for chains, seed in ((10, 3), (3, 4)):
        fields = random_fields(chains, L, N, seed)
        want = _existing(nmc, Lx, Ly, t, U, beta, dtau, n_wrap, fields)
        d_fields = torch.from_numpy(fields).cuda()
        d_G = torch.full((chains, 2, N, N), float("nan"), dtype=torch.float64, device="cuda")
        nmc.nmc_green_noalloc(N, L, n_wrap, lam, expk.data_ptr(), d_fields.data_ptr(), chains,
                              d_G.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = d_G.cpu().numpy()
        assert np.all(np.isfinite(got))
        rel = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert rel < G_REL, rel


def test_no_alloc_rejects_oversize_before_any_work(env):
    torch, nmc = env
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    f = torch.ones(16, dtype=torch.int8, device="cuda")
    with pytest.raises(nmc.NmcError) as e:   # 22 x 22 = 484 sites: one chain exceeds 32 MiB
        nmc.nmc_green_noalloc(484, 4, 2, 0.5, dummy.data_ptr(), f.data_ptr(), 1,
                              dummy.data_ptr())
    assert e.value.status == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:   # 410 sites: the first size past the 409 limit
        nmc.nmc_green_noalloc(410, 4, 2, 0.5, dummy.data_ptr(), f.data_ptr(), 1,
                              dummy.data_ptr())
    assert e.value.status == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError):
        nmc.nmc_green_noalloc(64, 10, 3, 0.5, dummy.data_ptr(), f.data_ptr(), 1,
                              dummy.data_ptr())
