"""Two-rank sharding of an ensemble on the CPU (gloo backend).

Each rank runs its contiguous chain-id range (the FP64 oracle stands in for
the device library here); the FP64 correlator and stress-log sums, summed over
ranks, equal those of one unsharded run of all chains, because the random
numbers are keyed by global chain id.  This covers the N > 1 path: range
arithmetic, chain offsets and the final sum over shards.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import Params
from paper_1106_2899_gb300 import shard

M_TOTAL, STEPS, LEVELS = 96, 300, 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(offset, count):
    p = Params(N=12, N0=3.0)
    e = oracle.Ensemble(p, seed=5, M=count, chain_offset=offset, groups=1, levels=LEVELS, log_every=50,
                        max_logs=STEPS // 50)
    e.init()
    e.run(STEPS, nthreads=1)
    acc, n = e.corr_sums()
    t, L = e.logs()
    return acc.sum(axis=0), L.sum(axis=1), e.get_state()["Z"]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard.shard_range(M_TOTAL, world, rank)
    acc, logs, Z = _run(off, cnt)
    acc_all = shard.allreduce_sum(acc)
    logs_all = shard.allreduce_sum(logs)
    out[rank] = (acc_all, logs_all, Z, off)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_exactly():
    for total, world in [(10, 3), (65536, 8), (7, 7)]:
        ranges = [shard.shard_range(total, world, r) for r in range(world)]
        assert ranges[0][0] == 0
        for (o1, c1), (o2, _) in zip(ranges, ranges[1:]):
            assert o1 + c1 == o2
        assert sum(c for _, c in ranges) == total
    with pytest.raises(ValueError):
        shard.shard_range(3, 4, 0)


def test_two_rank_gloo_sums_equal_unsharded():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    acc_ref, logs_ref, Z_ref = _run(0, M_TOTAL)
    for r in range(world):
        acc_all, logs_all, Z, off = res[r]
        assert np.allclose(acc_all, acc_ref, rtol=1e-12, atol=1e-9)
        assert np.allclose(logs_all, logs_ref, rtol=1e-12, atol=1e-9)
        assert np.array_equal(Z, Z_ref[off:off + len(Z)])
