"""Multi-process chain sharding on CPU (gloo, world size 2).

Each rank runs its own range of global chain indices through the FP64 oracle (the
chains the GPU library would run on that rank) and the per-chain results are gathered on
the host. The pooled estimate must equal a single process running all chains, and every
chain's trajectory must be independent of the partition (the Philox counter carries the
global chain index).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.dqmc import Model, run_chain
from paper_2106_00712_gb300 import sharding

MODEL = Model(2, 2, 1.0, 4.0, 1.0, 0.1, 5, seed=12)
TOTAL = 5
SWEEPS = 4


def _chain_results(indices):
    out = {"energy": [], "double_occ": [], "s_pipi": []}
    fields = []
    for c in indices:
        ch = run_chain(MODEL, chain_index=c, n_warm=1, n_meas=SWEEPS)
        m = ch.means()
        for k in out:
            out[k].append(m[k])
        fields.append(ch.s.copy())
    return out, fields


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = sharding.chain_range(rank, world, TOTAL)
        local, fields = _chain_results(range(off, off + cnt))
        merged = sharding.gather_per_chain(local, off, dist)
        pooled = sharding.pool(merged)
        slowest = sharding.max_over_ranks(float(rank + 1), dist)
        all_fields = [None] * world
        dist.all_gather_object(all_fields, (off, fields))
        if rank == 0:
            all_fields.sort(key=lambda t: t[0])
            q.put((pooled, slowest, [f for _, fs in all_fields for f in fs]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_chain_range_partitions_exactly():
    for world in (1, 2, 3, 7):
        got = []
        for r in range(world):
            off, cnt = sharding.chain_range(r, world, 10)
            got.extend(range(off, off + cnt))
        assert got == list(range(10))
    assert sharding.weak_offset(3, 256) == 768
    with pytest.raises(ValueError):
        sharding.chain_range(2, 2, 4)


def test_two_rank_gloo_pooling_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    pooled, slowest, fields = q.get()
    single, single_fields = _chain_results(range(TOTAL))
    ref = sharding.pool(single)
    for k in ref:
        assert pooled[k] == ref[k], k
    assert slowest == 2.0
    assert len(fields) == TOTAL
    for a, b in zip(fields, single_fields):
        np.testing.assert_array_equal(a, b)
