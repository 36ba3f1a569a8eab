"""The continuous-batching server (cqrrpt_server_*).

Requests submitted while others are on the GPU join later waves; every
result must be the same as a standalone factorisation of the same request
(bit for bit: the batched kernels run the single-problem arithmetic), the
HBM budget must bound admission (requests wait, none is lost), and a request
that can never fit is refused at submission.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    import paper_2311_08316_gb300 as lib
    lib.lib()
    return lib


def pinned_colmajor(a):
    a = np.asfortranarray(a, dtype=np.float64)
    t = torch.from_numpy(a.T.copy()).pin_memory()
    return t.t()


def requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(4, 70))
        m = int(rng.integers(max(2 * n, 100), 12000))
        r = int(rng.integers(max(1, n // 2), n + 1))
        sv = np.zeros(n)
        sv[:r] = W.logspaced(r, -float(rng.uniform(2, 10))).numpy()
        A = W.planted(m, n, sv, seed * 100 + i, noise=(1e-15 if r < n else 0.0)).numpy()
        out.append((np.asfortranarray(A), 1e-9 if r < n else 1e-12, 4000 + i))
    return out


def test_server_results_equal_standalone(C):
    reqs = requests(24, 1)
    srv = C.Server(hbm_budget_bytes=2 << 30, max_inflight=16)
    tickets = []
    for i, (A, tol, seed) in enumerate(reqs):
        tickets.append(srv.submit(pinned_colmajor(A), tol, seed))
        if i % 5 == 0:
            time.sleep(0.002)   # arrivals spread over the first waves
    srv.drain(timeout_us=120_000_000)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    assert stats["waves"] >= 2
    for t, (A, tol, seed) in zip(tickets, reqs):
        got = srv.poll(t)
        assert got is not None
        fac, res = got
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.status == ref.status and res.k == ref.k
        assert res.latency_us > 0 and res.queue_us >= 0
        assert np.array_equal(fac.J.numpy(), ref.J)
        Q = np.asfortranarray(fac.Q.numpy())
        R = np.asfortranarray(fac.R.numpy())
        assert np.array_equal(Q.view(np.uint64), ref.Q.view(np.uint64))
        assert np.array_equal(R.view(np.uint64), ref.R.view(np.uint64))
    srv.close()


def test_server_budget_admission_and_refusal(C):
    reqs = requests(10, 2)
    # budget for about two of these requests at a time
    srv = C.Server(hbm_budget_bytes=48 << 20, max_inflight=8)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed) for A, tol, seed in reqs]
    srv.drain(timeout_us=120_000_000)
    assert srv.stats()["completed"] == len(reqs)
    for t, (A, tol, seed) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        one = C.cqrrpt(torch.from_numpy(A.T.copy()).cuda().t(), 1.25, 4, tol, seed)
        assert res.k == one.k
        assert np.array_equal(fac.R.numpy(), one.R.cpu().numpy())
    big = np.ones((200000, 64), order="F")
    with pytest.raises(C.CqrrptError):
        srv.submit(pinned_colmajor(big), -1.0, 1)      # footprint > whole budget
    srv.close()


def test_server_mixed_precision_requests(C):
    reqs = requests(6, 3)
    srv = C.Server(hbm_budget_bytes=1 << 30, max_inflight=8)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed, precision=(2 if i % 2 else 0))
               for i, (A, tol, seed) in enumerate(reqs)]
    srv.drain(timeout_us=120_000_000)
    for i, (t, (A, tol, seed)) in enumerate(zip(tickets, reqs)):
        fac, res = srv.poll(t)
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.k == ref.k and np.array_equal(fac.J.numpy(), ref.J)
        Q = fac.Q.numpy()
        R = fac.R.numpy()
        AJ = A[:, ref.J]
        assert np.linalg.norm(AJ - Q @ R) / np.linalg.norm(A) <= 1e-12
        assert np.linalg.norm(Q.T @ Q - np.eye(res.k), 2) <= 1e-12
    srv.close()


def test_server_wide_fp64_requests_take_single_path(C):
    # n > 256 runs alone through the multi-CTA path; narrow ones are batched.
    # Either way the result is bit-identical to the oracle, and arrival order
    # decides which unit of work starts next.
    rng = np.random.default_rng(4)
    reqs = []
    for i, n in enumerate([300, 40, 280, 64, 260, 17]):
        m = int(rng.integers(2 * n, 5000))
        A = W.planted(m, n, W.logspaced(n, -6.0), 9000 + i).numpy()
        reqs.append((np.asfortranarray(A), 1e-12, 7000 + i))
    srv = C.Server(hbm_budget_bytes=1 << 30, max_inflight=8)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed) for A, tol, seed in reqs]
    srv.drain(timeout_us=120_000_000)
    assert srv.stats()["completed"] == len(reqs)
    for t, (A, tol, seed) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.status == ref.status and res.k == ref.k
        assert np.array_equal(fac.J.numpy(), ref.J)
        Q = np.asfortranarray(fac.Q.numpy())
        R = np.asfortranarray(fac.R.numpy())
        assert np.array_equal(Q.view(np.uint64), ref.Q.view(np.uint64))
        assert np.array_equal(R.view(np.uint64), ref.R.view(np.uint64))
    srv.close()


@pytest.mark.slow
def test_server_large_requests_both_precisions(C):
    # requests up to m = 2^17 and n = 512 (the serving mix reaches m = 2^20,
    # n = 512), wide ones on the single-problem route, narrow ones batched,
    # FP64 and split-BF16 interleaved
    import split_bounds
    shapes = [(1 << 17, 512, 0, 0), (1 << 16, 300, 2, 0), (100000, 256, 0, 180),
              (70000, 200, 2, 0), (1 << 17, 64, 0, 0), (50000, 128, 2, 90), (30000, 33, 0, 0),
              (9000, 17, 2, 0)]
    reqs = []
    for i, (m, n, prec, r) in enumerate(shapes):
        sv = np.zeros(n)
        if r:
            sv[:r] = W.logspaced(r, -6.0).numpy()
        else:
            sv = W.logspaced(n, -9.0).numpy()
        A = np.asfortranarray(W.planted(m, n, sv, 5100 + i, noise=(1e-15 if r else 0.0)).numpy())
        reqs.append((A, 1e-9 if r else 1e-12, 8100 + i, prec))
    srv = C.Server(hbm_budget_bytes=8 << 30, max_inflight=16)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed, precision=prec)
               for A, tol, seed, prec in reqs]
    srv.drain(timeout_us=600_000_000)
    assert srv.stats()["completed"] == len(reqs)
    for t, (A, tol, seed, prec) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.status == ref.status == 0 and res.k == ref.k, (A.shape, res.status, res.k)
        assert np.array_equal(fac.J.numpy(), ref.J)
        Q = np.asfortranarray(fac.Q.numpy())
        R = np.asfortranarray(fac.R.numpy())
        if prec == 0:
            assert np.array_equal(Q.view(np.uint64), ref.Q.view(np.uint64)), A.shape
            assert np.array_equal(R.view(np.uint64), ref.R.view(np.uint64)), A.shape
        else:
            rq, rr = split_bounds.ratios(Q, R, ref.Q, ref.R, ref.Rsk, A.shape[0])
            assert rq <= 4.0 and rr <= 4.0, (A.shape, rq, rr)
    srv.close()


def test_server_units_overlap_and_stay_bit_identical(C):
    # a wide request (single-problem route) is in flight while small requests
    # arrive: their batched waves run on the other lanes beside it, so at
    # least two units are in flight at once.  Every result equals a
    # standalone call of its precision (FP64: also the oracle) bit for bit.
    big_n, big_m = 400, 1 << 17
    big = np.asfortranarray(W.planted(big_m, big_n, W.logspaced(big_n, -7.0), 6100).numpy())
    reqs = [(big, 1e-12, 6200, 0)] + [(A, tol, seed, (2 if i % 3 == 2 else 0))
                                      for i, (A, tol, seed) in enumerate(requests(12, 9))]
    srv = C.Server(hbm_budget_bytes=4 << 30, max_inflight=32, lanes=3)
    tickets = [srv.submit(pinned_colmajor(reqs[0][0]), reqs[0][1], reqs[0][2])]
    time.sleep(0.01)
    for A, tol, seed, prec in reqs[1:]:
        tickets.append(srv.submit(pinned_colmajor(A), tol, seed, precision=prec))
        time.sleep(0.001)
    srv.drain(timeout_us=300_000_000)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["lanes"] == 3 and st["single_units"] == 1
    assert st["max_busy_lanes"] >= 2, st
    for t, (A, tol, seed, prec) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        assert res.status == 0
        one = C.cqrrpt(torch.from_numpy(A.T.copy()).cuda().t(), 1.25, 4, tol, seed,
                       precision=prec)
        assert res.k == one.k
        assert np.array_equal(fac.J.numpy(), one.J.cpu().numpy())
        assert np.array_equal(np.asfortranarray(fac.Q.numpy()).view(np.uint64),
                              np.asfortranarray(one.Q.cpu().numpy()).view(np.uint64))
        assert np.array_equal(np.asfortranarray(fac.R.numpy()).view(np.uint64),
                              np.asfortranarray(one.R.cpu().numpy()).view(np.uint64))
        if prec == 0 and A.shape[1] <= 64:
            ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
            assert np.array_equal(np.asfortranarray(fac.Q.numpy()).view(np.uint64),
                                  ref.Q.view(np.uint64))
    srv.close()


def test_server_one_lane_still_serves_everything(C):
    # with a single lane the server degenerates to one unit at a time
    reqs = requests(6, 10)
    srv = C.Server(hbm_budget_bytes=1 << 30, max_inflight=8, lanes=1)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed) for A, tol, seed in reqs]
    srv.drain(timeout_us=120_000_000)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["lanes"] == 1 and st["max_busy_lanes"] == 1
    for t, (A, tol, seed) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.k == ref.k
        assert np.array_equal(np.asfortranarray(fac.R.numpy()).view(np.uint64),
                              ref.R.view(np.uint64))
    srv.close()


def test_server_wide_requests_side_by_side(C):
    # several wide requests: up to lanes - 1 single-route units at once, their
    # cooperative QRCP grids one after another on the GPU; results equal the
    # oracle bit for bit
    rng = np.random.default_rng(12)
    reqs = []
    for i, n in enumerate([300, 320, 290, 270, 40, 50]):
        m = int(rng.integers(20000, 40000))
        A = W.planted(m, n, W.logspaced(n, -6.0), 9100 + i).numpy()
        reqs.append((np.asfortranarray(A), 1e-12, 7100 + i))
    srv = C.Server(hbm_budget_bytes=2 << 30, max_inflight=8, lanes=3)
    tickets = [srv.submit(pinned_colmajor(A), tol, seed) for A, tol, seed in reqs]
    srv.drain(timeout_us=300_000_000)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["single_units"] == 4
    assert st["max_busy_lanes"] >= 2
    for t, (A, tol, seed) in zip(tickets, reqs):
        fac, res = srv.poll(t)
        ref = oracle.cqrrpt(A, 1.25, 4, tol, seed)
        assert res.status == ref.status and res.k == ref.k
        assert np.array_equal(fac.J.numpy(), ref.J)
        assert np.array_equal(np.asfortranarray(fac.Q.numpy()).view(np.uint64),
                              ref.Q.view(np.uint64))
        assert np.array_equal(np.asfortranarray(fac.R.numpy()).view(np.uint64),
                              ref.R.view(np.uint64))
    srv.close()
