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
