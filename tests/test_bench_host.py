"""Host-side logic of the measurement scripts: the roofline arithmetic of bench.py and the
convergence criterion of the network-initialization driver (no GPU)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2106_00712_gb300 import nimc_run  # noqa: E402


def test_class_rooflines_use_the_stated_algorithmic_work():
    N, C = bench.WL.N, bench.WL.n_chains
    # one timed launch of 1 ms per class, both spins
    st = {k: (1, 1, 1.0) for k in ("gemm_tc", "gemm", "flip", "qrp", "solve")}
    rl = bench.class_rooflines(st, "fp32x2", 0, 2, acc=0.5)
    batch = 2 * C
    assert rl["gemm_tc"]["achieved"] == pytest.approx(bench.OZ_PRODUCTS * 2 * N ** 3 * batch / 1e-3 / 1e12)
    assert rl["gemm"]["achieved"] == pytest.approx(2 * N ** 3 * batch / 1e-3 / 1e12)
    k = bench.WL.delay_k
    assert rl["flip"]["achieved"] == pytest.approx(0.5 * N * C * 2 * (2 * N * N + 2 * N * k) / 1e-3 / 1e12)
    assert rl["qrp"]["achieved"] == pytest.approx(8 / 3 * N ** 3 * batch / 1e-3 / 1e12)
    assert rl["solve"]["achieved"] == pytest.approx(3 * N ** 3 * batch / 1e-3 / 1e12)
    for v in rl.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
    # the FP64 path's products and flips are measured against the FP64 pipe
    rl64 = bench.class_rooflines({"gemm": (1, 1, 1.0), "flip": (1, 1, 1.0)}, "fp64", 0, 2, 0.5)
    assert rl64["gemm"]["peak"] == bench.PEAK_TFLOPS["fp64"]
    assert rl64["flip"]["peak"] == bench.PEAK_TFLOPS["fp64"]


def test_traffic_is_reported_only_for_the_captured_source():
    for src, (h, b) in bench.TRAFFIC.items():
        assert b > 0
        assert bench.traffic_of(src) in (b, None)
        assert (bench.traffic_of(src) is not None) == (h == bench.src_hash(src))
    assert bench.traffic_of("no_such_kernel.cu") is None


def test_convergence_criterion():
    ref = (1.0, 0.0)
    def curve(vals, err=0.01):
        return {"x": [[v, err] for v in vals]}
    # within 1 error at sweep 3 and within 3 afterwards
    assert nimc_run._converged_at(curve([1.5, 1.1, 1.005, 0.98, 1.02]), "x", ref) == 3
    # a later excursion beyond 3 errors moves the answer past it
    assert nimc_run._converged_at(curve([1.0, 1.0, 1.05, 1.0, 1.0]), "x", ref) == 4
    assert nimc_run._converged_at(curve([1.5, 1.4]), "x", ref) is None
    # the reference's own error widens the band
    assert nimc_run._converged_at(curve([1.019], err=0.0), "x", (1.0, 0.02)) == 1


def test_table2_golden_fixture():
    """The printed Table 2 values the honeycomb GPU test compares against (tests/golden)."""
    path = os.path.join(ROOT, "tests", "golden", "table2_honeycomb_L6.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        q, *v = line.split()
        rows[q] = [float(x) for x in v]
    assert rows["E_k"] == [-1.360, 0.004, -1.357, 0.003, -1.358, 0.001]
    assert rows["S_Gamma"] == [3.11, 0.10, 2.99, 0.10, 3.00, 0.04]
