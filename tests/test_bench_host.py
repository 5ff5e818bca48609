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


PEAKS = {"fp64": 1.2, "fp32": 75.0, "bf16": 1900.0}


def test_class_rooflines_use_the_stated_algorithmic_work():
    N, C = bench.WL.N, bench.WL.n_chains
    # one timed launch of 1 ms per class, both spins
    st = {k: (1, 1, 1.0) for k in ("gemm_tc", "gemm", "flip", "qrp", "solve")}
    rl = bench.class_rooflines(st, "fp32x2", 2, 0.5, PEAKS, True)
    batch = 2 * C
    assert rl["gemm_tc"]["achieved"] == pytest.approx(bench.OZ_PRODUCTS * 2 * N ** 3 * batch / 1e-3 / 1e12)
    assert rl["gemm"]["achieved"] == pytest.approx(2 * N ** 3 * batch / 1e-3 / 1e12)
    k = bench.WL.delay_k
    assert rl["flip"]["achieved"] == pytest.approx(0.5 * N * C * 2 * (2 * N * N + 2 * N * k) / 1e-3 / 1e12)
    assert rl["qrp"]["achieved"] == pytest.approx(8 / 3 * N ** 3 * batch / 1e-3 / 1e12)
    assert rl["solve"]["achieved"] == pytest.approx(3 * N ** 3 * batch / 1e-3 / 1e12)
    for v in rl.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
    # each class against the pipe it runs on: the tensor class against BF16, the pair
    # kernels against the FP32 SIMT pipe (with the emulation ceiling as a second figure),
    # the FP64 stabilization against the FP64 pipe
    assert rl["gemm_tc"]["peak"] == PEAKS["bf16"]
    assert rl["flip"]["peak"] == PEAKS["fp32"]
    assert rl["flip"]["frac_of_pair_ceiling"] == pytest.approx(
        rl["flip"]["achieved"] / (PEAKS["fp32"] / bench.PAIR_INSTR_PER_FMA))
    assert rl["gemm"]["peak"] == rl["qrp"]["peak"] == rl["solve"]["peak"] == PEAKS["fp64"]
    rl64 = bench.class_rooflines({"gemm": (1, 1, 1.0), "flip": (1, 1, 1.0)}, "fp64", 2, 0.5,
                                 PEAKS, False)
    assert rl64["gemm"]["peak"] == PEAKS["fp64"]
    assert rl64["flip"]["peak"] == PEAKS["fp64"]


def test_whole_step_flop_count():
    """step_flop against the step-by-step count written out for the 8x8 workload."""
    N, L, nb, C = 64, 40, 4, 256
    p = 2.0 * N ** 3
    wraps, stack = 2 * p * L, p * L
    stab = nb * (3 * p + 3 * N ** 3 + 8 / 3 * N ** 3 + p)
    meas = nb * 2 * p
    flips = 0.6 * N * L * 2 * N * N
    want = (wraps + stack + stab + meas + flips) * 2 * C
    assert bench.step_flop(N, L, nb, C, 2, 0.6) == pytest.approx(want)
    # the per-attempt figure sits near the 21 N^2 estimate at this acceptance
    per = bench.step_flop(N, L, nb, C, 2, 0.6) / (C * N * L)
    assert 0.8 * 21 * N * N < per < 1.5 * 21 * N * N


def test_gpus_flag_launches_one_rank_per_gpu_with_disjoint_chains():
    """`bench.py --gpus 2` re-launches itself under torch.distributed.run with two ranks;
    each rank takes its own GPU and a disjoint chain range (no GPU work in --plan-only)."""
    import json
    import subprocess
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                          "--plan-only"], capture_output=True, text=True, timeout=240, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    plans = sorted((json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")),
                   key=lambda d: d["rank"])
    assert [p["rank"] for p in plans] == [0, 1]
    assert all(p["world"] == 2 for p in plans)
    assert [p["device"] for p in plans] == [0, 1]
    (a0, a1), (b0, b1) = plans[0]["chain_range"], plans[1]["chain_range"]
    assert a1 <= b0 and a1 - a0 == b1 - b0 == bench.WL.n_chains


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
