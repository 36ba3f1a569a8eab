"""The N > 1 host logic on CPU ranks (gloo on 127.0.0.1).

* The benchmark: under torchrun every rank factors its own independent
  problems (no data is exchanged), the step time is the maximum over ranks,
  and the reference arm runs on rank 0 alone: distinct per-rank inputs of
  the same shape, max-over-ranks timing, the barrier, and rank 1 of the
  reference arm exiting without work.
* The row-partitioned form's two sums (the sketch and the Gram, Sec. 2.1):
  ordered_scan must leave every rank with the sum of the ranks' block sums
  in ascending global block order, bit for bit, on 2 and 3 ranks.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    w_world, w_rank, _ = bench.dist_setup()
    assert (w_world, w_rank) == (world, rank)
    out = {}
    # independent inputs of the same shape on every rank
    w = bench.rank_workload(W.single_large(m=8192), rank)
    out["single"] = (w.m, w.n, w.seed, w.sketch_seed)
    b = bench.rank_batch(6, rank)
    out["batch_shapes"] = [(x.m, x.n) for x in b]
    out["batch_seeds"] = [x.seed for x in b]
    # the slowest rank sets the step time
    out["max"] = bench.max_over_ranks(10.0 + rank, world)
    bench.barrier(world)
    # reference arm: rank 0 alone runs (a tiny row sample), the others return
    class Args:
        rows, steps, warmup, gpus = 2048, 1, 0, world
    if rank != 0:
        bench.run_reference(Args, world, rank)
        out["ref"] = "returned"
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.timeout(300)
def test_two_cpu_ranks_factor_independent_problems():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0, r1 = res[0], res[1]
    assert r0["single"][:2] == r1["single"][:2]            # same shape
    assert r0["single"][2:] != r1["single"][2:]            # other seeds
    assert r0["single"][2] == 2311083160 + 1               # rank 0: published seed
    assert set(r0["batch_seeds"]).isdisjoint(r1["batch_seeds"])
    assert r0["max"] == r1["max"] == 11.0
    assert r1["ref"] == "returned"


def _blocks(seed, count, size):
    g = torch.Generator()
    g.manual_seed(seed)
    # magnitudes spread over 12 decades: additions in another order round
    # differently
    return [torch.randn(size, generator=g, dtype=torch.float64)
            * torch.pow(10.0, 12 * torch.rand(size, generator=g, dtype=torch.float64) - 6)
            for _ in range(count)]


def _scan_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import paper_2311_08316_gb300 as C
    dist.init_process_group("gloo")
    per = 3
    mine = _blocks(100, per * world, 257)[rank * per:(rank + 1) * per]

    def add_mine(buf):
        for b in mine:                      # this rank's blocks, ascending
            buf.add_(b)

    buf = torch.zeros(257, dtype=torch.float64)
    C.ordered_scan(buf, add_mine)
    # the running sum of the ranks' parts arrived in rank order
    q.put((rank, buf.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 3])
def test_ordered_scan_over_cpu_ranks_is_the_sequential_sum(world):
    # the bookkeeping of the row-partitioned form's two sums: with synthetic
    # block sums, every rank must end with the sum in ascending global block
    # order starting from +0.0, bit for bit, which another order does not give
    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_scan_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks = _blocks(100, 3 * world, 257)
    seq = torch.zeros(257, dtype=torch.float64)
    for b in blocks:
        seq.add_(b)
    rev = torch.zeros(257, dtype=torch.float64)
    for b in reversed(blocks):
        rev.add_(b)
    for r in range(world):
        assert np.array_equal(res[r].view(np.uint64), seq.numpy().view(np.uint64))
    assert not np.array_equal(rev.numpy().view(np.uint64), seq.numpy().view(np.uint64))
