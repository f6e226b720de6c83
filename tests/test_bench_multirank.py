"""bench.py's multi-rank bookkeeping (the N > 1 path) on two gloo ranks on
the CPU: the job time is the slowest rank's, and the weak-scaling rate counts
every rank's cells; the split of the kv-sweep's fronts across ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + 5.0 * rank, 2.0 - rank]        # ms of the timed steps, e2e seconds
    ms, e2e = bench.max_over_ranks(local, dist)
    out[rank] = (ms, e2e, bench.weak_scaling_rate(1000, 20, world, ms * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, e2e, rate = res[rank]
        assert ms == 15.0 and e2e == 2.0
        assert rate == pytest.approx(1000 * 20 * 2 / 15e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]


def test_instance_shares_cover_and_balance():
    """The N > 1 kv-sweep split: contiguous shares that cover every instance
    once, none empty, each within one instance's length of an equal share of
    the cells."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    lengths = np.random.default_rng(4).integers(512, 8193, size=256)
    for parts in (1, 2, 3, 4, 8, 256):
        shares = bench.instance_shares(lengths, parts)
        assert len(shares) == parts
        assert shares[0][0] == 0 and sum(c for _, c in shares) == len(lengths)
        for (f0, c0), (f1, _) in zip(shares, shares[1:]):
            assert f0 + c0 == f1
        assert all(c >= 1 for _, c in shares)
        cells = [int(lengths[f:f + c].sum()) for f, c in shares]
        if parts < 256:
            assert max(abs(x - lengths.sum() / parts) for x in cells) <= lengths.max()
    # a few long instances first: still one instance per rank at least
    skew = np.array([100000, 100000, 10, 10, 10])
    shares = bench.instance_shares(skew, 4)
    assert [c for _, c in shares] and all(c >= 1 for _, c in shares) and sum(c for _, c in shares) == 5
    with pytest.raises(ValueError):
        bench.instance_shares(skew, 6)


def _kv_rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import argparse
    import numpy as np
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = []

    def fake_run_batch(pr, lengths, vs, phi, cs, cl, *, max_steps, launches_per_graph, dt, steps_per_launch, tol):
        n = np.asarray(lengths)
        assert len(phi) == len(cs) == len(cl) == int(n.sum()) and len(vs) == len(n) == len(dt)
        calls.append((len(n), int(n.sum()), max_steps))
        return {"gpu_ms": 1e-6 * float(n.sum()) * max_steps * (1.0 + rank)}   # rank 1 slower

    try:
        line = bench.kv_sweep_shard(argparse.Namespace(steps=400), dist, world, rank, fake_run_batch, "cpu")
        out[rank] = (calls, line)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_kv_sweep_shards_the_fronts_across_ranks():
    """bench.py --workload kv-sweep under torchrun, its bookkeeping on two gloo
    ranks with a stand-in for the batched run: each rank steps its own share
    (a warm-up, then the timed K steps), the shares cover the 256 fronts, and
    rank 0 reports all instance-steps over the slowest rank's time."""
    sys.path.insert(0, ROOT)
    import bench
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_kv_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    lengths = bench.kv_sweep_inputs()[0]
    shares = bench.instance_shares(lengths, 2)
    for rank in (0, 1):
        calls, _ = res[rank]
        first, count = shares[rank]
        cells = int(lengths[first:first + count].sum())
        assert calls == [(count, cells, 100), (count, cells, 400)]
    assert res[1][1] is None
    line = res[0][1]
    slowest = max(1e-9 * int(lengths[f:f + c].sum()) * 400 * (1 + r) for r, (f, c) in enumerate(shares))
    assert line["n_gpus"] == 2 and line["scaling"] == "strong"
    assert line["value"] == pytest.approx(256 * 400 / slowest)
    assert line["batch_gpu_s"] == pytest.approx(slowest)
