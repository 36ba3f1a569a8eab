"""The row-partitioned form (Sec. 2.1) across processes: two ranks (gloo over
127.0.0.1, both on GPU 0), each holding a range of rows of M, run the
cqrrpt_shard_* phases; the sketch and the Gram are summed over the ranks by
ordered_scan (host copies on gloo).  Each rank's rows of Q, and R, J and k,
must equal the oracle's CQRRPT of the whole M bit for bit (and cqrrpt_d's).
The kernels of the two processes never wait on one another: the only
exchange is the host-side send / receive of the two sums.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix(m, n, rank_planted, seed):
    sv = np.zeros(n)
    if rank_planted:
        sv[:rank_planted] = W.logspaced(rank_planted, -6.0).numpy()
        return np.asfortranarray(W.planted(m, n, sv, seed, noise=1e-15).numpy())
    return np.asfortranarray(W.planted(m, n, W.logspaced(n, -8.0), seed).numpy())


def _worker(rank, world, port, case, bounds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import paper_2311_08316_gb300 as C
    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    m, n, rk, seed, tol, sseed = case
    A = _matrix(m, n, rk, seed)
    r0, r1 = bounds[rank], bounds[rank + 1]
    A_loc = torch.from_numpy(np.ascontiguousarray(A[r0:r1].T)).cuda().t()
    res = C.cqrrpt_sharded(A_loc, m, r0, 1.25, 4, tol, sseed)
    torch.cuda.synchronize()
    q.put((rank, res.status, res.k, res.J.cpu().numpy(),
           np.asfortranarray(res.Qbuf[:, :res.k].cpu().numpy()),
           np.asfortranarray(res.Rbuf[:res.k].cpu().numpy())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def C():
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    import paper_2311_08316_gb300 as lib
    lib.lib()
    return lib


@pytest.mark.timeout(600)
@pytest.mark.parametrize("case,bounds", [
    # m = 3 blocks + a ragged tail, planted rank 40 of 60 (tol 1e-9)
    ((3 * 4096 + 123, 60, 40, 5, 1e-9, 77), [0, 2 * 4096, 3 * 4096 + 123]),
    # n = 300 (a QRCP on several CTAs), full rank, rank 1 holds one block only
    ((5 * 4096 + 77, 300, 0, 6, 1e-12, 78), [0, 4 * 4096, 5 * 4096 + 77]),
])
def test_two_ranks_row_partitioned_bitexact(C, case, bounds):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, bounds, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, st, k, J, Q, R = q.get(timeout=500)
        got[rank] = (st, k, J, Q, R)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, n, rk, seed, tol, sseed = case
    A = _matrix(m, n, rk, seed)
    ref = oracle.cqrrpt(A, 1.25, 4, tol, sseed)
    assert ref.status == 0 and ref.k == (rk or n)
    for rank in range(world):
        st, k, J, Q, R = got[rank]
        assert st == 0 and k == ref.k
        assert np.array_equal(J, ref.J)
        assert np.array_equal(R.view(np.uint64), ref.R.view(np.uint64))
        r0, r1 = bounds[rank], bounds[rank + 1]
        assert np.array_equal(Q.view(np.uint64),
                              np.asfortranarray(ref.Q[r0:r1]).view(np.uint64))
    # and the whole-matrix call on one device gives the same bits
    one = C.cqrrpt(torch.from_numpy(A.T.copy()).cuda().t(), 1.25, 4, tol, sseed)
    assert one.k == ref.k
    assert np.array_equal(np.asfortranarray(one.R.cpu().numpy()).view(np.uint64),
                          ref.R.view(np.uint64))


def test_shard_phases_out_of_order_and_bad_rows(C):
    L = C.lib()
    h = C.Handle()
    A = torch.zeros((64, 5000), dtype=torch.float64, device="cuda").t()
    s = C._stream(None)
    buf = torch.zeros(1000, dtype=torch.float64, device="cuda")
    # accumulate before the sketch: out of order
    assert L.cqrrpt_shard_sketch_accumulate_d(h.h, buf.data_ptr(), s) == -1
    # row0 not a multiple of 4096
    assert L.cqrrpt_shard_sketch_d(h.h, 9000, 5000, 100, 64, A.data_ptr(), 5000, 1.25, 4, 1,
                                   s) == -4
    # rows past m
    assert L.cqrrpt_shard_sketch_d(h.h, 9000, 5000, 8192, 64, A.data_ptr(), 5000, 1.25, 4, 1,
                                   s) == -4
    h.close()
