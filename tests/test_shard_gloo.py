"""Multi-process host logic on CPU: size-balanced sharding of independent graphs over ranks and the
timing reductions, checked with two gloo ranks (the GPU runs use one process per GPU over NCCL
with the same code)."""
import os
import socket

import numpy as np
import pytest

from paper_1610_08128_gb300 import shard, synth

torch = pytest.importorskip("torch")


def test_shard_by_size_is_a_balanced_partition():
    sizes, _ = synth.mix_sizes(1000, 100, 50000, 11)
    for world in (1, 2, 3, 8):
        shards = shard.shard_by_size(sizes, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [int(sum(sizes[i] for i in s)) for s in shards]
        # greedy largest-first: no rank exceeds the mean by more than the largest graph
        assert max(loads) - sum(loads) / world <= int(max(sizes))
        assert all(s == sorted(s) for s in shards)


def test_shard_edge_cases():
    assert shard.shard_by_size([], 3) == [[], [], []]
    assert shard.shard_by_size([5], 2) == [[0], []]
    assert shard.shard_by_size([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.shard_by_size([1], 0)
    assert shard.max_over_ranks(2.5) == 2.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.shard_by_size(sizes, world)[rank]
        work = float(sum(sizes[i] for i in mine))
        slowest = shard.max_over_ranks(1.0 + rank, dist)
        total = shard.sum_over_ranks(work, dist)
        out.put((rank, mine, slowest, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    sizes = [int(x) for x in synth.mix_sizes(200, 100, 50000, 12)[0]]
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mine0, mine1 = res[0][1], res[1][1]
    assert sorted(mine0 + mine1) == list(range(len(sizes)))
    assert not set(mine0) & set(mine1)
    assert res[0][2] == res[1][2] == 2.0              # max over ranks of (1 + rank)
    assert res[0][3] == res[1][3] == float(np.sum(sizes))


def _batch_worker(rank, world, port, G, out):
    """One rank: its size-balanced share of a batch, ordered on the host by the oracle (the GPU
    runs order it with rcm_order_batch), results gathered for reassembly."""
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = synth.c4_specs(G, 20, 400)
        mine = shard.shard_by_size([n for _, n, _ in specs], world)[rank]
        b = synth.c4_batch(G, 20, 400, indices=mine)
        perms = oracle.rcm_batch(b.goff, b.rowptr, b.colidx, threads=2)
        part = {gi: perms[k].tolist() for k, gi in enumerate(mine)}
        parts = [None] * world
        dist.all_gather_object(parts, part)
        out.put((rank, mine, parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_order_one_batch_split_by_size():
    """One batch partitioned by size over two ranks, each ordering only its own graphs; the
    gathered per-graph results reassemble into the whole batch, every graph once and in the
    original order, equal to ordering the unsplit batch."""
    import multiprocessing as mp

    import oracle

    G = 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, G, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][2] == res[1][2]                      # both ranks gathered the same parts
    assert sorted(res[0][1] + res[1][1]) == list(range(G)) and res[0][1] and res[1][1]
    whole = shard.assemble(res[0][2], G)
    full = synth.c4_batch(G, 20, 400)
    ref = oracle.rcm_batch(full.goff, full.rowptr, full.colidx, threads=2)
    for gi in range(G):
        assert whole[gi] == ref[gi].tolist(), gi
    with pytest.raises(ValueError):
        shard.assemble([{0: 1}, {0: 1}], 1)              # a graph from two ranks
    with pytest.raises(ValueError):
        shard.assemble([{0: 1}], 2)                      # a graph from none
