"""Multi-GPU host logic on CPU: world_size-2 gloo ranks.

The path does not exchange data between GPUs (replicas of the dam break,
disjoint shares of a batch's tanks), so what runs across ranks is the
measurement: every rank's units summed over the slowest rank's time, and the
deterministic deal of tanks to ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    el = 1.0 + rank                  # rank 1 is the slowest
    units = 100.0 * (rank + 1)       # 100 and 200 particle-steps
    value, el_max = bench.replica_value(el, units, dist, "cpu")
    shard = bench.shard_tanks(bench_sizes(), world)[rank]
    q.put((rank, value, el_max, shard))
    dist.barrier()
    dist.destroy_process_group()


def bench_sizes():
    from paper_2603_11868_gb300 import cases
    return cases.batched_tank_sizes(256, seed=4)


def test_replica_value_and_tank_shards_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, el_max, _ in res:
        assert el_max == 2.0
        assert value == pytest.approx(300.0 / 2.0)
    shards = [r[3] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(256))
    assert shards == bench.shard_tanks(bench_sizes(), 2)


def test_shard_balance_and_single_rank():
    sizes = bench_sizes()
    assert bench.shard_tanks(sizes, 1) == [list(range(len(sizes)))]
    for ranks in (2, 4, 8):
        sh = bench.shard_tanks(sizes, ranks)
        assert sorted(t for s in sh for t in s) == list(range(len(sizes)))
        loads = np.array([sum(sizes[t] for t in s) for s in sh])
        # largest-first greedy: the spread is at most the largest tank
        assert loads.max() - loads.min() <= max(sizes)


def test_replica_value_without_process_group():
    assert bench.replica_value(2.0, 10.0, None, "cpu") == (5.0, 2.0)
