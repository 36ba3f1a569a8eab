"""The bounded device-side waits and their timeout path.

Two kernels wait on other threads of the GPU: the multi-CTA QRCP of the
sketch (Alg. 2 line 2) crosses a grid barrier once per pivot step, and the
split-BF16 tensor-core engine (lines 4, 5, 7) waits on mbarriers for its
copies, products and drains.  Every such wait is bounded; when a bound runs
out the kernel records CQRRPT_TIMEOUT (status 5) and leaves cleanly.  These
tests lower the bounds with cqrrpt_set_wait_limits so that the waits run out
(no fault, trap or endless loop is involved: a wait simply gives up), check
that the call reports status 5, and that the next call on the same handle,
with the default bounds back, gives the oracle's result again.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TIMEOUT = 5


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


def bits(t):
    return np.asfortranarray(t.detach().cpu().numpy()).view(np.uint64)


def test_grid_barrier_timeout_then_clean_call(C):
    # n = 200: the QRCP runs on 25 CTAs with a grid barrier per pivot step
    m, n = 20000, 200
    A_h = np.asfortranarray(W.planted(m, n, W.logspaced(n, -8.0), 31).numpy())
    A = gpu(A_h)
    h = C.Handle()
    C.set_wait_limits(grid_spins=1)
    try:
        C.cqrrpt(A, 1.25, 4, 1e-12, 17, handle=h, sync=False)
        st, k = h.last_status()
    finally:
        C.set_wait_limits(0, 0)
    assert st == TIMEOUT and k == 0
    res = C.cqrrpt(A, 1.25, 4, 1e-12, 17, handle=h)
    ref = oracle.cqrrpt(A_h, 1.25, 4, 1e-12, 17)
    assert res.status == 0 and res.k == ref.k == n
    assert np.array_equal(res.J.cpu().numpy(), ref.J)
    assert np.array_equal(bits(res.Q), ref.Q.view(np.uint64))
    assert np.array_equal(bits(res.R), ref.R.view(np.uint64))
    h.close()


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_engine_wait_timeout_then_clean_call(C, precision):
    # the split-BF16 products of lines 4, 5 and 7 give up on their first
    # mbarrier wait that is not already complete; tensor memory is released
    # (a later call allocates all of it again on every SM)
    m, n = 20000, 96
    A_h = np.asfortranarray(W.planted(m, n, W.logspaced(n, -10.0), 77).numpy())
    A = gpu(A_h)
    h = C.Handle()
    before = C.cqrrpt(A, 1.25, 4, 1e-12, 99, precision=precision, handle=h)
    assert before.status == 0
    C.set_wait_limits(grid_spins=0, tensor_wait_ns=1)
    try:
        C.cqrrpt(A, 1.25, 4, 1e-12, 99, precision=precision, handle=h, sync=False)
        torch.cuda.synchronize()
        st, k = h.last_status()
    finally:
        C.set_wait_limits(0, 0)
    assert st == TIMEOUT and k == 0
    after = C.cqrrpt(A, 1.25, 4, 1e-12, 99, precision=precision, handle=h)
    ref = oracle.cqrrpt(A_h, 1.25, 4, 1e-12, 99)
    assert after.status == 0 and after.k == before.k == ref.k
    assert np.array_equal(after.J.cpu().numpy(), ref.J)
    assert torch.equal(after.Q, before.Q) and torch.equal(after.R, before.R)
    h.close()


def test_wait_limits_reject_negative(C):
    L = C.lib()
    assert L.cqrrpt_set_wait_limits(-1, 0) == -1
    assert L.cqrrpt_set_wait_limits(0, -1) == -2
