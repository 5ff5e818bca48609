"""The bounds-checked build (libnmc_debug.so, compiled with NMC_DEBUG) on the small parity
cases: every key index of the kernels is checked (a failed check skips the access and makes
the call return NMC_ECUDA), the results still equal the oracle's, and no check fails.

It runs in a child process that loads the debug library (NMC_LIB_PATH): the test process
may already hold the regular one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2106_00712_gb300 import nmc
from oracle.dqmc import Chain, Model, initial_fields
lib = nmc.load()
assert lib.nmc_debug_build() == 1, "not the bounds-checked build"

def run(model, chains, sweeps, precision, g_rel, ph=0, delay_k=16):
    refs = [Chain(model, initial_fields(model, c), c) for c in range(chains)]
    with nmc.Context(model.Lx, model.Ly, model.t, model.U, model.beta, model.dtau,
                     model.n_wrap, seed=model.seed, n_chains=chains, delay_k=delay_k,
                     precision=precision, drift_tol=1e-3, ph_symmetric=ph) as c:
        c.generate()
        for sw in range(sweeps):
            c.sweep(1, measure=1)
            for r in refs:
                r.sweep(True)
            f = c.fields()
            for ch in range(chains):
                assert np.array_equal(f[ch], refs[ch].s), (model.Lx, sw, ch)
        for ch in range(chains):
            for spin in (0, 1):
                G, want = c.green(ch, spin), refs[ch].G[spin]
                assert np.max(np.abs(G - want)) <= g_rel * np.max(np.abs(want)), (model.Lx, ch)
        if chains >= 2:   # the serving pools' restart path
            c.restart_chains([1], [chains + 5])
            c.sweep(2, measure=1)

run(Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10, seed=0), 1, 6, nmc.NMC_FP64, 1e-10)
run(Model(6, 4, 1.0, 4.0, 1.2, 0.1, 4, seed=2), 3, 4, nmc.NMC_SPLIT_BF16, 1e-8, delay_k=5)
run(Model(6, 4, 1.0, 4.0, 1.2, 0.1, 4, seed=2), 2, 4, nmc.NMC_FP32X2, 1e-8, ph=1)
run(Model(10, 10, 1.0, 4.0, 1.0, 0.1, 5, seed=4), 2, 2, nmc.NMC_SPLIT_BF16, 1e-8)
assert lib.nmc_debug_checks() == 0, lib.nmc_debug_checks()
print("bounds-checked build: parity held, no check failed")
'''


def test_bounds_checked_build_runs_the_parity_cases_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00712_gb300 import build_lib
    lib = build_lib.build(debug=True)
    env = dict(os.environ, NMC_LIB_PATH=lib)
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no check failed" in r.stdout
