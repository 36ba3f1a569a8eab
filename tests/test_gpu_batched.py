"""Batched CQRRPT (cqrrpt_batched_d): uneven problems in one batched pass.

Every problem of the batch must give the same J, k, Q and R, bit for bit, as
the oracle and as a standalone cqrrpt_d call; the result of a problem must
not depend on what else shares the batch (checked by reordering the batch
and replaying the cached CUDA graph).  Statuses are per problem.
"""
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


def gpu(a):
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(a.T.copy()).cuda().t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def bits_equal(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.dtype == np.float64:
        return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))
    return np.array_equal(a, b)


def make_batch(count, seed):
    rng = np.random.default_rng(seed)
    mats, tols = [], []
    for i in range(count):
        n = int(rng.integers(3, 90))
        m = int(rng.integers(max(2 * n, 64), 9000))
        r = int(rng.integers(max(1, n // 2), n + 1))
        sv = np.zeros(n)
        sv[:r] = W.logspaced(r, -8.0).numpy()
        A = W.planted(m, n, sv, seed * 1000 + i, noise=(1e-15 if r < n else 0.0)).numpy()
        mats.append(np.asfortranarray(A))
        tols.append(1e-9 if r < n else (1e-12 if i % 3 else -1.0))
    return mats, tols


def test_batched_matches_oracle_and_single(C):
    mats, tols = make_batch(14, 3)
    seeds = [5000 + i for i in range(len(mats))]
    As = [gpu(A) for A in mats]
    res, kd, sd = C.cqrrpt_batched(As, 1.25, 4, tols, seeds)
    for i, (A, r) in enumerate(zip(mats, res)):
        ref = oracle.cqrrpt(A, 1.25, 4, tols[i], seeds[i])
        assert r.status == ref.status and r.k == ref.k, (i, r.status, ref.status, r.k, ref.k)
        assert bits_equal(host(r.J), ref.J), i
        assert bits_equal(host(r.Q), ref.Q), i
        assert bits_equal(host(r.R), ref.R), i
        one = C.cqrrpt(As[i], 1.25, 4, tols[i], seeds[i])
        assert one.k == r.k and torch.equal(one.J, r.J)
        assert torch.equal(one.Q, r.Q) and torch.equal(one.R, r.R)


def test_batched_independent_of_batch_composition_and_graph_replay(C):
    mats, tols = make_batch(9, 4)
    seeds = [77 + i for i in range(len(mats))]
    As = [gpu(A) for A in mats]
    r1, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds)
    r2, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds)          # graph replay
    order = list(reversed(range(len(mats))))
    r3, _, _ = C.cqrrpt_batched([As[i] for i in order], 1.25, 4, [tols[i] for i in order],
                                [seeds[i] for i in order])
    C.set_batch_graphs(False)
    r4, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds)          # direct launches
    C.set_batch_graphs(True)
    for i in range(len(mats)):
        j = order.index(i)
        for other in (r2[i], r3[j], r4[i]):
            assert other.k == r1[i].k
            assert torch.equal(other.J, r1[i].J)
            assert torch.equal(other.Q, r1[i].Q) and torch.equal(other.R, r1[i].R)


def test_batched_per_problem_status(C):
    rng = np.random.default_rng(8)
    good = np.asfortranarray(rng.standard_normal((700, 12)))
    zero = np.zeros((500, 7), order="F")
    bad = np.asfortranarray(rng.standard_normal((400, 9)))
    bad[3, 3] = np.inf
    As = [gpu(good), gpu(zero), gpu(bad), gpu(good)]
    res, kd, sd = C.cqrrpt_batched(As, 1.25, 3, [-1.0] * 4, [1, 2, 3, 1])
    assert [r.status for r in res] == [0, 1, 2, 0]
    assert [r.k for r in res] == [12, 0, 0, 12]
    assert torch.equal(res[0].Q, res[3].Q)
    ref = oracle.cqrrpt(good, 1.25, 3, -1.0, 1)
    assert bits_equal(host(res[0].R), ref.R)


def test_batched_tile_shapes_do_not_change_results(C):
    # every TRSM column block (16 / 32, with the 16-8-4-2-1 remainder) and
    # Gram tile (8 / 16 / 32) gives the oracle's bits; widths cover several
    # buckets and k mod 32 of every residue class a few times
    mats, tols = make_batch(12, 6)
    mats += [np.asfortranarray(W.planted(700, n, W.logspaced(n, -5.0), 60 + n).numpy())
             for n in (31, 33, 47, 64, 65, 97, 130)]
    tols += [1e-12] * 7
    seeds = [900 + i for i in range(len(mats))]
    As = [gpu(A) for A in mats]
    refs = [oracle.cqrrpt(A, 1.25, 4, t, s) for A, t, s in zip(mats, tols, seeds)]
    h = C.Handle()
    for jb, gt in [(16, 16), (32, 32), (16, 32), (32, 16), (32, 8)]:
        C.set_batch_tuning([jb] * 16, [gt] * 16, handle=h)
        res, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, handle=h)
        for i, (r, ref) in enumerate(zip(res, refs)):
            assert r.k == ref.k and bits_equal(host(r.J), ref.J), (jb, gt, i)
            assert bits_equal(host(r.Q), ref.Q) and bits_equal(host(r.R), ref.R), (jb, gt, i)
    with pytest.raises(C.CqrrptError):
        C.set_batch_tuning([24] * 16, None, handle=h)


def test_batched_autotune_picks_shapes_and_keeps_results(C):
    mats, tols = make_batch(16, 7)
    seeds = [300 + i for i in range(len(mats))]
    As = [gpu(A) for A in mats]
    h = C.Handle()
    res, _, _, times = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, handle=h, autotune=True)
    buckets = {min((A.shape[1] - 1) // 32, 15) for A in mats}
    assert set(times) == buckets
    jb, gt = C.get_batch_tuning(handle=h)
    for b, t in times.items():
        assert all(x > 0 for x in t["trsm_us"] + t["gram_us"])
        assert jb[b] == (16 if t["trsm_us"][0] < t["trsm_us"][1] else 32)
        # 8 x 8 Gram tiles are timed too (not reported): 8 or the faster of 16 / 32
        assert gt[b] == 8 or gt[b] == (16 if t["gram_us"][0] < t["gram_us"][1] else 32)
    again, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, handle=h)
    for i, (A, r, r2) in enumerate(zip(mats, res, again)):
        ref = oracle.cqrrpt(A, 1.25, 4, tols[i], seeds[i])
        assert r.k == ref.k and r2.k == ref.k
        for x in (r, r2):
            assert bits_equal(host(x.J), ref.J)
            assert bits_equal(host(x.Q), ref.Q) and bits_equal(host(x.R), ref.R)


def test_batched_split_bf16_matches_single_split_and_oracle(C):
    # lines 4, 5, 7 as batched split products: every problem bit-identical to
    # cqrrpt_d in CQRRPT_SPLITBF16 (same jobs), J and k equal to the oracle's,
    # residuals at FP64 level
    mats, tols = make_batch(10, 8)
    mats.append(np.asfortranarray(W.planted(3000, 140, W.logspaced(140, -9.0), 77).numpy()))
    tols.append(1e-12)
    seeds = [600 + i for i in range(len(mats))]
    As = [gpu(A) for A in mats]
    res, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, precision=C.SPLITBF16)
    for i, (A, r) in enumerate(zip(mats, res)):
        ref = oracle.cqrrpt(A, 1.25, 4, tols[i], seeds[i])
        assert r.status == ref.status and r.k == ref.k, (i, r.status, r.k, ref.k)
        assert bits_equal(host(r.J), ref.J), i
        one = C.cqrrpt(As[i], 1.25, 4, tols[i], seeds[i], precision=C.SPLITBF16)
        assert one.k == r.k
        assert torch.equal(one.Q[:, :r.k], r.Q[:, :r.k]) and torch.equal(one.R[:r.k], r.R[:r.k]), i
        if r.k:
            Q, R = host(r.Q)[:, :r.k], host(r.R)[:r.k]
            AJ = A[:, ref.J]
            # planted rank: the dropped 1e-15 noise tail bounds the residual
            m, n = A.shape
            bound = 1e-12 if r.k == n else max(1e-12, 10e-15 * np.sqrt(m * n) / np.linalg.norm(A))
            assert np.linalg.norm(AJ - Q @ R) / np.linalg.norm(A) <= bound, i
            assert np.linalg.norm(Q.T @ Q - np.eye(r.k), 2) <= 1e-12, i


def pick_uneven(count=16):
    """Problems of the batched workload itself (workloads.batch_uneven: m in
    [4096, 65536], n in [32, 256], planted rank in [n/2, n]): the four with the
    largest sketches n^2 d (their batched QRCP keeps columns in global
    memory), the tallest one, then every 47th of the list."""
    ws = W.batch_uneven(count=512)
    by_size = sorted(range(len(ws)), key=lambda i: -(ws[i].n ** 2 * ws[i].d))
    pick = []
    for i in by_size[:4] + [max(range(len(ws)), key=lambda i: ws[i].m)] + list(range(0, 512, 47)):
        if i not in pick:
            pick.append(i)
    return [ws[i] for i in pick[:count]]


@pytest.mark.slow
def test_batched_uneven_workload_sizes(C):
    import split_bounds
    ws = pick_uneven(16)
    assert len(ws) == 16
    assert any(w.n >= 200 and w.m >= 32768 for w in ws)
    # the largest sketches do not fit one CTA's shared memory
    assert max(w.d * w.n * 8 for w in ws) > 227 * 1024
    As = [w.matrix("cuda") for w in ws]
    tols = [w.tol for w in ws]
    seeds = [w.sketch_seed for w in ws]
    refs = [oracle.cqrrpt(np.asfortranarray(A.cpu().numpy()), w.gamma, w.nnz, w.tol,
                          w.sketch_seed) for A, w in zip(As, ws)]
    h = C.Handle()
    res, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, handle=h)
    res_t, _, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, handle=h, autotune=True)
    for i, (r, rt, ref) in enumerate(zip(res, res_t, refs)):
        assert r.status == ref.status == 0 and r.k == ref.k, (i, r.status, r.k, ref.k)
        for x in (r, rt):
            assert bits_equal(host(x.J), ref.J), i
            assert bits_equal(host(x.Q), ref.Q) and bits_equal(host(x.R), ref.R), i
    sp, _, _ = C.cqrrpt_batched(As, 1.25, 4, tols, seeds, precision=C.SPLITBF16, handle=h)
    for i, (r, ref, w) in enumerate(zip(sp, refs, ws)):
        assert r.status == 0 and r.k == ref.k, (i, r.status, r.k, ref.k)
        assert bits_equal(host(r.J), ref.J), i
        rq, rr = split_bounds.ratios(r.Q, r.R, ref.Q, ref.R, ref.Rsk, w.m)
        assert rq <= 4.0 and rr <= 4.0, (i, w.m, w.n, rq, rr)
    h.close()
