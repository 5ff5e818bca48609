"""Failure handling on the device path, without faulting anything.

* NMC_ENUMERIC: a drift tolerance far below any achievable drift makes the host-side check
  after a sweep fail; the sweep itself ran, so the state (fields, G) must equal that of the
  same run with the default tolerance, and the context stays usable.
* NMC_ENOMEM: the allocation-failure hook makes one device allocation of nmc_configure
  fail as if the device were out of memory; the context reports NMC_ENOMEM with a reason,
  is destroyed cleanly, and the next context works. No real memory pressure is created.
"""
import numpy as np
import pytest

from oracle.dqmc import Model

pytestmark = pytest.mark.gpu


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


MODEL = Model(6, 6, 1.0, 4.0, 2.0, 0.1, 5, seed=31)


def _ctx(nmc, **kw):
    m = MODEL
    return nmc.Context(m.Lx, m.Ly, m.t, m.U, m.beta, m.dtau, m.n_wrap, seed=m.seed,
                       n_chains=3, **kw)


@pytest.mark.parametrize("prec", [0, 2])
def test_drift_above_tolerance_returns_enumeric_and_keeps_state(nmc, prec):
    with _ctx(nmc, precision=prec) as ref, _ctx(nmc, precision=prec, drift_tol=1e-300) as c:
        ref.generate()
        c.generate()
        ref.sweep(2, measure=1)
        with pytest.raises(nmc.NmcError) as e:
            c.sweep(2, measure=1)
        assert e.value.status == nmc.NMC_ENUMERIC
        assert "drift" in str(e.value)
        np.testing.assert_array_equal(c.fields(), ref.fields())
        for ch in range(3):
            np.testing.assert_array_equal(c.green(ch, 0), ref.green(ch, 0))
        assert c.measure().max_drift == ref.measure().max_drift > 0
        # still usable: the next sweep runs (and fails the same check again)
        with pytest.raises(nmc.NmcError) as e:
            c.sweep(1, measure=0)
        assert e.value.status == nmc.NMC_ENUMERIC
        ref.sweep(1, measure=0)
        np.testing.assert_array_equal(c.fields(), ref.fields())


def test_injected_allocation_failure_returns_enomem_and_destroys_cleanly(nmc):
    m = MODEL
    for n in (1, 7, 25):   # the first allocation, one in the middle, one late
        nmc.nmc_debug_fail_alloc(n)
        try:
            with pytest.raises(nmc.NmcError) as e:
                _ctx(nmc, precision=2)
            assert e.value.status == nmc.NMC_ENOMEM
            assert "injected" in str(e.value)
        finally:
            nmc.nmc_debug_fail_alloc(0)
    with _ctx(nmc, precision=2) as c:    # the next context allocates and runs
        c.generate()
        c.sweep(1, measure=1)
        assert c.measure().density.mean == pytest.approx(1.0, abs=1e-12)
    # the raw entry points: nmc_configure fails, nmc_destroy releases the partial allocation
    ctx = nmc.nmc_create(m.Lx, m.Ly, m.t, m.U, m.beta, m.dtau, m.n_wrap, m.seed)
    o = nmc.nmc_default_options()
    o.n_chains = 2
    nmc.nmc_debug_fail_alloc(3)
    try:
        with pytest.raises(nmc.NmcError) as e:
            nmc.nmc_configure(ctx, o)
        assert e.value.status == nmc.NMC_ENOMEM
    finally:
        nmc.nmc_debug_fail_alloc(0)
    nmc.nmc_configure(ctx, o)             # a second configure on the same context works
    nmc.nmc_destroy(ctx)
