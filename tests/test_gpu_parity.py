"""GPU <-> oracle parity, step by step and end to end, through the C ABI.

The library and the oracle implement the same readings of the paper (the
SASO generator, the blocked/ascending summation orders, dot32 inside the
QRCP, the pivot tie-break, the sign convention), so every floating-point
output is compared BIT FOR BIT, and J and k exactly.  Sizes span several
4096-row blocks, several tiles of every kernel, and ragged tails.
"""
import math

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
    t = torch.from_numpy(a.T.copy()).cuda()   # (n, m) contiguous == column-major (m, n)
    return t.t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def assert_bits(got, ref, what):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    same = (got.view(np.uint64) == ref.view(np.uint64)) if got.dtype == np.float64 else (got == ref)
    if not same.all():
        idx = np.argwhere(~same)
        i = tuple(idx[0])
        diff = np.abs(got.astype(np.float64) - ref.astype(np.float64))
        raise AssertionError("%s: %d of %d differ; first at %s got %r ref %r; max abs diff %g"
                             % (what, len(idx), same.size, i, got[i], ref[i], diff.max()))


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- line 1
@pytest.mark.parametrize("m,n,d,s,seed", [
    (4096, 64, 128, 4, 7),
    (3 * 4096 + 123, 13, 40, 8, 11),
    (4097, 5, 16, 1, 3),
    (10000, 33, 42, 32, 2**40 + 9),
    (300, 7, 300, 4, 5),
    # the largest sketch dimension the library takes (28000): the lists
    # kernel's counts then leave shared memory for 8 sorting warps only
    (2 * 4096 + 31, 3, 28000, 8, 13),
])
def test_sketch_bitexact(C, m, n, d, s, seed):
    A = _rng(seed % 1000).standard_normal((m, n))
    ref, st = oracle.sketch(A, d, s, seed)
    got = C.sketch(gpu(A), d, s, seed)
    torch.cuda.synchronize()
    assert st == 0
    assert_bits(host(got), ref, "sketch")


# ---------------------------------------------------------------- line 2
@pytest.mark.parametrize("path", ["auto", "cluster"])
@pytest.mark.parametrize("d,n,seed", [(128, 64, 1), (37, 29, 2), (200, 150, 3), (640, 512, 4),
                                      (9, 9, 5), (1, 1, 6), (80, 57, 7)])
def test_qrcp_bitexact(C, d, n, seed, path, monkeypatch):
    # CQRRPT_QRCP_CLUSTER=1 runs n <= 64 on one thread-block cluster instead
    # of the cooperative grid; both forms give the oracle's bits
    if path == "cluster":
        monkeypatch.setenv("CQRRPT_QRCP_CLUSTER", "1")
    rng = _rng(seed)
    X = rng.standard_normal((d, n)) * np.logspace(0, -8, n)[rng.permutation(n)]
    R_ref, J_ref, *_ = oracle.qrcp(X)
    Xg = gpu(X)
    Rsk, J = C.qrcp(Xg)
    torch.cuda.synchronize()
    assert_bits(host(J), J_ref, "J")
    assert_bits(host(Rsk), R_ref, "R^sk")


@pytest.mark.parametrize("path", ["auto", "cluster"])
@pytest.mark.parametrize("n", [80, 64])
def test_qrcp_rank_deficient_and_ties(C, n, path, monkeypatch):
    if path == "cluster":
        monkeypatch.setenv("CQRRPT_QRCP_CLUSTER", "1")
    rng = _rng(9)
    d = 96
    X = rng.standard_normal((d, 40)) @ rng.standard_normal((40, n))
    X[:, 5] = X[:, 3]           # exact duplicate columns: exact norm ties
    X[:, n - 10] = 0.0          # zero column
    R_ref, J_ref, *_ = oracle.qrcp(X)
    Rsk, J = C.qrcp(gpu(X))
    torch.cuda.synchronize()
    assert_bits(host(J), J_ref, "J")
    assert_bits(host(Rsk), R_ref, "R^sk")


# ---------------------------------------------------------------- line 3
def test_rank_rules(C):
    rng = _rng(10)
    X = rng.standard_normal((60, 50)) * np.logspace(0, -14, 50)
    R_ref, *_ = oracle.qrcp(X)
    Rg = gpu(R_ref)
    for tol in (1e-3, 1e-9, 1e-12, 1e-16):
        k = C.rank(Rg, tol)
        torch.cuda.synchronize()
        assert int(k.item()) == oracle.rank_tol(R_ref, tol)
    k = C.rank(Rg, -1.0)
    assert int(k.item()) == oracle.rank_stage1(R_ref)


# ---------------------------------------------------------------- lines 4, 7
@pytest.mark.parametrize("m,n,k", [(1000, 40, 37), (4096 + 17, 70, 70), (33, 20, 1), (500, 300, 290)])
def test_trsm_bitexact(C, m, n, k):
    rng = _rng(m + k)
    B = rng.standard_normal((m, n))
    T = np.triu(rng.standard_normal((k, k))) + 3 * np.eye(k)
    cols = rng.permutation(n)[:k].astype(np.int64)
    ref = oracle.trsm_rut(B, T, cols)
    got = C.trsm(gpu(B), gpu(T), torch.from_numpy(cols).cuda())
    torch.cuda.synchronize()
    assert_bits(host(got), ref, "trsm gather")
    # in place, identity columns
    ref2 = oracle.trsm_rut(ref, T)
    Xg = gpu(ref)
    C.trsm(Xg, gpu(T), None, out=Xg)
    torch.cuda.synchronize()
    assert_bits(host(Xg), ref2, "trsm in place")


# ---------------------------------------------------------------- line 5
@pytest.mark.parametrize("m,k", [(4096, 64), (3 * 4096 + 77, 45), (100, 1), (9000, 130),
                                 (10 * 4096, 200), (32 * 4096 + 5, 100)])
def test_gram_bitexact(C, m, k):
    # the launch picks 8 x 8 tiles for the small cases, 16 x 16 for
    # (10 * 4096, 200) and 32 x 32 for (32 * 4096 + 5, 100): same bits
    X = _rng(m).standard_normal((m, k))
    ref = oracle.gram(X)
    got = C.gram(gpu(X))
    torch.cuda.synchronize()
    assert_bits(host(got), ref, "gram")


# ---------------------------------------------------------------- line 6
@pytest.mark.parametrize("k", [1, 31, 32, 33, 100, 257])
def test_potrf_bitexact(C, k):
    B = _rng(k).standard_normal((2 * k + 3, k))
    G = B.T @ B
    ref, fail = oracle.potrf_upper(G)
    R, f = C.potrf(gpu(G))
    torch.cuda.synchronize()
    assert fail == -1 and int(f.item()) == -1
    assert_bits(np.triu(host(R)), ref, "potrf")


def test_potrf_failure_column(C):
    rng = _rng(77)
    k = 70
    B = rng.standard_normal((200, k))
    B[:, 45] = B[:, :45] @ rng.standard_normal(45)
    G = B.T @ B
    G[45, 45] -= 1e-3 * G[45, 45]
    ref, fail = oracle.potrf_upper(G)
    R, f = C.potrf(gpu(G))
    torch.cuda.synchronize()
    assert fail == 45 and int(f.item()) == 45
    assert_bits(np.triu(host(R))[:45, :45], ref[:45, :45], "potrf leading block")


# ---------------------------------------------------------------- line 8
@pytest.mark.parametrize("k,n", [(7, 11), (64, 64), (100, 130), (1, 5)])
def test_trmm_bitexact(C, k, n):
    rng = _rng(k * n)
    Rp = np.triu(rng.standard_normal((k, k)))
    Rs = np.triu(rng.standard_normal((k, n)))
    ref = oracle.trmm_upper(Rp, Rs)
    got = C.trmm(gpu(Rp), gpu(Rs))
    torch.cuda.synchronize()
    assert_bits(host(got), ref, "trmm")


# ---------------------------------------------------------------- end to end
def _compare_full(C, A, gamma, nnz, tol, seed):
    ref = oracle.cqrrpt(A, gamma, nnz, tol, seed)
    res = C.cqrrpt(gpu(A), gamma, nnz, tol, seed)
    assert res.status == ref.status
    assert res.k == ref.k
    assert_bits(host(res.J), ref.J, "J")
    if ref.k:
        assert_bits(host(res.Q), ref.Q, "Q")
        assert_bits(host(res.R), ref.R, "R")
    return ref, res


def test_cqrrpt_full_rank_cond1e8(C):
    """m = 4096, n = 64, cond 1e8, d = 2n, 4 nnz/col, tol 1e-12."""
    w = W.single_small()
    A = np.asfortranarray(w.matrix().numpy())
    ref, res = _compare_full(C, A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    assert res.k == 64


@pytest.mark.parametrize("m,n,rank,gamma,nnz,tol", [
    (16384, 128, 100, 1.25, 8, 1e-9),
    (5000, 37, 37, 1.25, 4, -1.0),
    (9000, 70, 35, 1.5, 3, -1.0),
    (4096 * 2 + 1, 50, 50, 1.0, 1, 1e-12),
])
def test_cqrrpt_bitexact_shapes(C, m, n, rank, gamma, nnz, tol):
    sv = np.zeros(n)
    sv[:rank] = W.logspaced(rank, -7.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, m + n, noise=(1e-15 if rank < n else 0.0)).numpy())
    ref, res = _compare_full(C, A, gamma, nnz, tol, 1000 + m)
    if tol > 0 and rank < n:
        assert res.k == rank


def test_cqrrpt_degenerate(C):
    # k = 0: zero matrix
    res = C.cqrrpt(gpu(np.zeros((300, 6))), 1.25, 2, -1.0, 1)
    assert res.status == 1 and res.k == 0
    # n = 1
    A = _rng(4).standard_normal((77, 1))
    _compare_full(C, A, 1.0, 1, -1.0, 3)
    # d == m
    A = _rng(5).standard_normal((20, 16))
    _compare_full(C, A, 1.25, 3, -1.0, 4)
    # non-finite
    A = _rng(6).standard_normal((500, 9))
    A[13, 4] = np.nan
    res = C.cqrrpt(gpu(A), 1.25, 4, -1.0, 4)
    assert res.status == 2 and res.k == 0
    # the handle is usable afterwards
    A = _rng(7).standard_normal((500, 9))
    _compare_full(C, A, 1.25, 4, -1.0, 8)


def test_cqrrpt_invalid_arguments(C):
    import ctypes
    A = gpu(_rng(1).standard_normal((50, 10)))
    with pytest.raises(C.CqrrptError):
        C.cqrrpt(A, 6.0, 4, -1.0, 1)          # d = 60 > m
    with pytest.raises(C.CqrrptError):
        C.cqrrpt(A, 1.25, 40, -1.0, 1)        # nnz > 32
    with pytest.raises(C.CqrrptError):
        C.cqrrpt(A, 0.5, 4, -1.0, 1)          # gamma < 1
    L = C.lib()
    h = C.default_handle()
    assert L.cqrrpt_d(h.h, 50, 10, None, 50, 1.25, 4, -1.0, 1, 0, None, 50, None, 10, None, None,
                      None, None) == -4


def test_cqrrpt_repeatable_across_calls_and_streams(C):
    w = W.single_large(m=8192 + 300, n=96, rank=70)
    A = gpu(np.asfortranarray(w.matrix().numpy()))
    r1 = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r2 = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, stream=s)
    torch.cuda.synchronize()
    assert r1.k == r2.k == 70
    assert torch.equal(r1.J, r2.J)
    assert torch.equal(r1.Q, r2.Q) and torch.equal(r1.R, r2.R)


def test_cqrrpt_async_status(C):
    A = gpu(_rng(3).standard_normal((800, 12)))
    h = C.Handle()
    res = C.cqrrpt(A, 1.25, 4, 1e-12, 5, handle=h, sync=False)
    st, k = h.last_status()
    assert st == 0 and k == 12
    h.close()


def _host_colmajor(A, ld=None, pinned=True):
    """Column-major host tensor holding A (leading dimension ld >= m)."""
    m, n = A.shape
    ld = ld or m
    t = torch.zeros((n, ld), dtype=torch.float64, pin_memory=pinned)
    t[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    return t.t()[:m, :]


def test_host_pipeline_matches_oracle(C):
    """cqrrpt_host_pipeline_d: five host matrices (full rank, planted rank,
    zero, ragged m, padded lda) through the copy/compute pipeline, each
    result bit-identical to the oracle; then the same inputs with two
    alternating output buffers (results copied out in order)."""
    m, n = 4096 + 777, 40
    mats = []
    for i in range(5):
        sv = np.zeros(n)
        rank = [40, 25, 0, 40, 33][i]
        if rank:
            sv[:rank] = W.logspaced(rank, -6.0).numpy()
            mats.append(np.asfortranarray(W.planted(m, n, sv, 50 + i,
                                                    noise=(1e-15 if rank < n else 0.0)).numpy()))
        else:
            mats.append(np.zeros((m, n), order="F"))
    seeds = [11, 12, 13, 14, 2**40 + 15]
    A_h = [_host_colmajor(A, ld=m + 3) for A in mats]
    res = C.cqrrpt_host_pipeline(A_h, 1.25, 4, 1e-9, seeds)
    for i, A in enumerate(mats):
        ref = oracle.cqrrpt(A, 1.25, 4, 1e-9, seeds[i])
        assert res[i].status == ref.status and res[i].k == ref.k, i
        assert_bits(res[i].J.numpy(), ref.J, "J[%d]" % i)
        if ref.k:
            assert_bits(np.asfortranarray(res[i].Q.numpy()), ref.Q, "Q[%d]" % i)
            assert_bits(np.asfortranarray(res[i].R.numpy()), ref.R, "R[%d]" % i)
    assert res[2].status == 1 and res[2].k == 0
    # two output buffers, reused in turn: the last two results are the
    # pipeline's, and equal the first run's
    outs = [(torch.empty((n, m), dtype=torch.float64, pin_memory=True).t(),
             torch.empty((n, n), dtype=torch.float64, pin_memory=True).t(),
             torch.empty(n, dtype=torch.int64, pin_memory=True)) for _ in range(2)]
    res2 = C.cqrrpt_host_pipeline(A_h, 1.25, 4, 1e-9, seeds, outs_host=[outs[i % 2] for i in range(5)])
    assert [r.k for r in res2] == [r.k for r in res]
    for i in (3, 4):
        assert torch.equal(res2[i].J, res[i].J)
        assert torch.equal(res2[i].Q, res[i].Q) and torch.equal(res2[i].R, res[i].R)


def test_host_pipeline_splitbf16_matches_single_calls(C):
    """The split-BF16 precision through the pipeline equals the one-matrix
    call bit for bit (same kernels, same inputs)."""
    w = W.single_large(m=8192 + 300, n=96, rank=70)
    A = np.asfortranarray(w.matrix().numpy())
    A_h = [_host_colmajor(A), _host_colmajor(A)]
    res = C.cqrrpt_host_pipeline(A_h, w.gamma, w.nnz, w.tol, [w.sketch_seed] * 2,
                                 precision=C.SPLITBF16)
    one = C.cqrrpt(gpu(A), w.gamma, w.nnz, w.tol, w.sketch_seed, precision=C.SPLITBF16)
    for r in res:
        assert r.status == 0 and r.k == one.k == 70
        assert torch.equal(r.J, one.J.cpu())
        assert torch.equal(r.Q, one.Q.cpu()) and torch.equal(r.R, one.R.cpu())


# ---------------------------------------------------------------- implicit Q
@pytest.mark.parametrize("m,n,rank,gamma,nnz,tol", [
    (4096 * 2 + 77, 60, 60, 1.25, 4, -1.0),
    (16384 + 5, 96, 70, 1.25, 8, 1e-9),
])
def test_implicit_matches_oracle(C, m, n, rank, gamma, nnz, tol):
    """cqrrpt_implicit_d: M^pre, R^pre, R, J and k bit-identical to the
    oracle's lines 1-6 and 8 (line 7 not formed)."""
    sv = np.zeros(n)
    sv[:rank] = W.logspaced(rank, -7.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, 77 + m, noise=(1e-15 if rank < n else 0.0)).numpy())
    ref = oracle.cqrrpt_implicit(A, gamma, nnz, tol, 5 + n)
    res = C.cqrrpt_implicit(gpu(A), gamma, nnz, tol, 5 + n)
    assert res.status == ref.status and res.k == ref.k
    if tol > 0:
        assert res.k == rank
    assert_bits(host(res.J), ref.J, "J")
    assert_bits(host(res.Apre), ref.Apre, "Apre")
    assert_bits(np.triu(host(res.Rpre)), np.triu(ref.Rpre), "Rpre")
    assert_bits(host(res.R), ref.R, "R")


@pytest.mark.parametrize("r", [1, 5, 17, 40])
def test_apply_q_matches_oracle(C, r):
    """Q X and Q^T Y through cqrrpt_apply_q_d, bit for bit against the
    oracle's apply_q on the oracle's own M^pre and R^pre (ragged row blocks,
    right-hand-side counts across the kernels' 16- and 32-column tiles)."""
    w = W.single_large(m=3 * 4096 + 501, n=72, rank=50)
    A = np.asfortranarray(w.matrix().numpy())
    ref = oracle.cqrrpt_implicit(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    k = ref.k
    assert k == 50
    rng = _rng(100 + r)
    X = np.asfortranarray(rng.standard_normal((k, r)))
    Y = np.asfortranarray(rng.standard_normal((A.shape[0], r)))
    Ap, Rp = gpu(ref.Apre), gpu(ref.Rpre)
    got_q = C.apply_q(Ap, Rp, k, gpu(X))
    got_qt = C.apply_q(Ap, Rp, k, gpu(Y), trans=True)
    assert_bits(host(got_q), oracle.apply_q(ref.Apre, ref.Rpre, X), "QX")
    assert_bits(host(got_qt), oracle.apply_q(ref.Apre, ref.Rpre, Y, trans=True), "QtY")


def test_apply_q_through_the_factorisation_and_k_zero(C):
    """The implicit factorisation's own apply_q equals the explicit Q of
    cqrrpt_d applied with torch to a few u; k = 0 gives Q X = 0."""
    w = W.single_small()
    A = gpu(np.asfortranarray(w.matrix().numpy()))
    imp = C.cqrrpt_implicit(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    exp = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    assert imp.k == exp.k == 64
    assert torch.equal(imp.R, exp.R) and torch.equal(imp.J, exp.J)
    X = torch.randn(64, 3, dtype=torch.float64, device="cuda")
    assert (imp.apply_q(X) - exp.Q @ X).abs().max().item() <= 1e-12 * X.abs().max().item()
    Y = torch.randn(A.shape[0], 3, dtype=torch.float64, device="cuda")
    assert (imp.apply_qt(Y) - exp.Q.t() @ Y).abs().max().item() <= 1e-12 * Y.norm(dim=0).max().item()
    zero = C.cqrrpt_implicit(gpu(np.zeros((300, 6))), 1.25, 2, -1.0, 1)
    assert zero.k == 0 and zero.status == 1
    out = C.apply_q(zero.Abuf, zero.Rprebuf, 0, torch.zeros(0, 2, dtype=torch.float64, device="cuda"))
    assert out.shape == (300, 2) and torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("cap", ["0", "1", "3"])
def test_qrcp_mixed_storage(C, cap, monkeypatch):
    """Sketches too large for the SMs' shared memory keep some owned columns
    in global memory; forcing that on a small sketch (at most `cap` columns
    per CTA in shared memory) leaves J and R^sk bit-identical to the
    oracle, including exact ties and a zero column."""
    monkeypatch.setenv("CQRRPT_QRCP_CACHED_COLUMNS", cap)
    rng = _rng(90 + int(cap))
    d, n = 700, 600
    X = rng.standard_normal((d, 300)) @ rng.standard_normal((300, n))
    X[:, 7] = X[:, 2]
    X[:, 500] = 0.0
    R_ref, J_ref, *_ = oracle.qrcp(X)
    Rsk, J = C.qrcp(gpu(X))
    torch.cuda.synchronize()
    assert_bits(host(J), J_ref, "J")
    assert_bits(host(Rsk), R_ref, "R^sk")
    w = W.single_large(m=8192 + 300, n=96, rank=70)
    A = np.asfortranarray(w.matrix().numpy())
    _compare_full(C, A, w.gamma, w.nnz, w.tol, w.sketch_seed)


# ---------------------------------------------------------- Sec. 1.3 rCholQR
@pytest.mark.parametrize("m,n,seed", [(4096 + 33, 64, 1), (3 * 4096 + 5, 150, 2), (5000, 8, 3),
                                      (9000, 300, 4)])
def test_rcholqr_matches_oracle(C, m, n, seed):
    """The unpivoted randomized CholeskyQR through cqrrpt_rcholqr_d: Q and R
    bit-identical to the oracle's, J the identity, k = n (one CTA and
    several CTAs in the QR of the sketch)."""
    M = np.asfortranarray(W.planted(m, n, W.logspaced(n, -6.0), 300 + seed).numpy())
    ref = oracle.rcholqr(M, 1.25, 4, 40 + seed)
    res = C.rcholqr(gpu(M), 1.25, 4, 40 + seed)
    assert res.status == ref.status == 0 and res.k == ref.k == n
    assert np.array_equal(host(res.J), np.arange(n))
    assert_bits(host(res.Q), ref.Q, "Q")
    assert_bits(host(res.R), ref.R, "R")


# ------------------------------------------- dense (Gaussian) sketching operator
@pytest.mark.parametrize("m,n,d,seed", [
    (2 * 4096 + 77, 20, 40, 1),     # two blocks + ragged tail; d, n not multiples of 32
    (1000, 8, 10, 2),               # less than one row block
    (3 * 4096, 64, 96, 3),          # whole tiles, whole blocks
])
def test_sketch_dense_matches_oracle(C, m, n, d, seed):
    """Line 1 with a Gaussian operator (Sec. 2.3.1): bit-identical to the
    oracle's blocked ascending-fma product."""
    S = np.asfortranarray(W.gaussian_operator(d, m, 500 + seed).numpy())
    M = np.asfortranarray(_rng(seed).standard_normal((m, n)))
    ref, st = oracle.sketch_dense(S, M)
    assert st == 0
    got = C.sketch_dense(gpu(M), gpu(S))
    torch.cuda.synchronize()
    assert_bits(host(got), ref, "S M")


@pytest.mark.parametrize("case", ["planted", "full", "identity"])
def test_cqrrpt_dense_matches_oracle(C, case):
    """Alg. 2 with a dense operator through cqrrpt_dense_d: Q, R, J and k
    bit-identical to the oracle (planted rank with noise; full rank; S = I
    with d = m, where the method is QRCP of M itself)."""
    if case == "planted":
        m, n, rank, tol = 3 * 4096 + 5, 48, 30, 1e-9
        sv = np.zeros(n)
        sv[:rank] = W.logspaced(rank, -6.0).numpy()
        A = np.asfortranarray(W.planted(m, n, sv, 601, noise=1e-15).numpy())
        S = np.asfortranarray(W.gaussian_operator(60, m, 602).numpy())
    elif case == "full":
        m, n, rank, tol = 5000, 64, 64, 1e-12
        A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -8.0), 603).numpy())
        S = np.asfortranarray(W.gaussian_operator(80, m, 604).numpy())
    else:
        m, n, rank, tol = 200, 17, 17, 1e-14
        A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -3.0), 605).numpy())
        S = np.asfortranarray(np.eye(m))
    ref = oracle.cqrrpt_dense(A, S, tol)
    res = C.cqrrpt_dense(gpu(A), gpu(S), tol)
    assert res.status == ref.status == 0 and res.k == ref.k == rank
    assert np.array_equal(host(res.J), ref.J)
    assert_bits(host(res.Q), ref.Q, "Q")
    assert_bits(host(res.R), ref.R, "R")


def test_cqrrpt_dense_one_nonzero_saso_equals_cqrrpt(C):
    """s = 1 gives a SASO with entries +-1 and scale exactly 1: the dense
    path on that operator reproduces cqrrpt_d's outputs bit for bit."""
    m, n, gamma, seed = 2 * 4096 + 300, 40, 1.25, 71
    A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -6.0), 606).numpy())
    d = oracle.sketch_dim(n, gamma)
    S = oracle.saso_dense(seed, d, m, 1)
    a = C.cqrrpt(gpu(A), gamma, 1, 1e-12, seed)
    b = C.cqrrpt_dense(gpu(A), gpu(S), 1e-12)
    assert a.status == b.status == 0 and a.k == b.k == n
    assert torch.equal(a.J, b.J)
    assert_bits(host(b.Q), host(a.Q), "Q")
    assert_bits(host(b.R), host(a.R), "R")


@pytest.mark.parametrize("precision", [2, 3])
def test_cqrrpt_dense_split_modes(C, precision):
    """Dense operator with lines 4, 5, 7 in split-BF16 (with and without the
    second CholeskyQR pass): the FP64 sketch and QRCP give the oracle's J and
    k; residuals at the FP64 level."""
    m, n = 2 * 4096 + 11, 64
    A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -8.0), 607).numpy())
    S = np.asfortranarray(W.gaussian_operator(80, m, 608).numpy())
    ref = oracle.cqrrpt_dense(A, S, 1e-12)
    res = C.cqrrpt_dense(gpu(A), gpu(S), 1e-12, precision=precision)
    assert res.status == ref.status == 0 and res.k == ref.k == n
    assert np.array_equal(host(res.J), ref.J)
    Q, R = host(res.Q), host(res.R)
    assert np.linalg.norm(A[:, ref.J] - Q @ R) / np.linalg.norm(A) <= 1e-13
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13


def test_cqrrpt_dense_nonfinite_and_arguments(C):
    m, n = 300, 10
    A = np.asfortranarray(_rng(9).standard_normal((m, n)))
    A[17, 3] = np.nan
    S = np.asfortranarray(W.gaussian_operator(13, m, 609).numpy())
    res = C.cqrrpt_dense(gpu(A), gpu(S), 1e-12)
    assert res.status == 2 and res.k == 0
    with pytest.raises(Exception):
        C.cqrrpt_dense(gpu(A), gpu(S[:8, :]), 1e-12)          # d < n


# ------------------------------------------- row panels of a host-resident matrix
@pytest.mark.parametrize("panel_rows,tol,case", [
    (4096, 1e-9, "planted"),     # six panels, ragged last one
    (8192, 1e-9, "planted"),
    (65536, 1e-9, "planted"),    # one panel larger than m
    (8192, -1.0, "graded"),      # default rank rule (stage 2 after the Cholesky)
])
def test_panels_host_matches_oracle(C, panel_rows, tol, case):
    """Alg. 2 over row panels streamed from host memory
    (cqrrpt_panels_host_d): the panels' block sums continue the sketch's and
    the Gram's ascending sums, so Q, R, J and k equal the oracle's bit for
    bit whatever the panel height."""
    m, n = 5 * 4096 + 123, 40
    if case == "planted":
        sv = np.zeros(n)
        sv[:30] = W.logspaced(30, -6.0).numpy()
        A = np.asfortranarray(W.planted(m, n, sv, 701, noise=1e-15).numpy())
    else:
        A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -13.0), 702).numpy())
    ref = oracle.cqrrpt(A, 1.25, 4, tol, 77)
    Ah = _host_colmajor(A, ld=m + 3, pinned=panel_rows != 8192)   # padded lda; pageable once
    Q, R, J, k, st = C.cqrrpt_panels(Ah, 1.25, 4, tol, 77, panel_rows=panel_rows)
    assert st == ref.status == 0 and k == ref.k > 0
    assert np.array_equal(J.numpy(), ref.J)
    assert_bits(np.asfortranarray(Q.numpy()), ref.Q, "Q")
    assert_bits(np.asfortranarray(R.numpy()), ref.R, "R")


def test_panels_host_degenerate_cases(C):
    m, n = 2 * 4096 + 5, 12
    Z = _host_colmajor(np.zeros((m, n)))
    _, _, J, k, st = C.cqrrpt_panels(Z, 1.25, 4, 1e-12, 3, panel_rows=4096)
    ref = oracle.cqrrpt(np.zeros((m, n), order="F"), 1.25, 4, 1e-12, 3)
    assert k == 0 and st == ref.status == 1
    assert np.array_equal(J.numpy(), ref.J)
    A = _rng(5).standard_normal((m, n))
    A[4100, 2] = np.inf
    _, _, _, k, st = C.cqrrpt_panels(_host_colmajor(A), 1.25, 4, 1e-12, 3, panel_rows=4096)
    assert k == 0 and st == 2
    with pytest.raises(Exception):
        C.cqrrpt_panels(_host_colmajor(A), 1.25, 4, 1e-12, 3, panel_rows=5000)


# ------------------------------------------- Sec. 2.2 strong rank-revealing QR
@pytest.mark.parametrize("m,n,rank,tol,f", [
    (5000, 48, 30, 1e-9, 1.05),       # planted rank: exchanges
    (5000, 48, 30, 1e-9, 2.0),        # none at f = 2
    (5000, 48, 0, 1e-8, 1.2),         # graded full rank, k < n by the tolerance
    (20000, 400, 300, 1e-9, 1.05),    # k > 256: several blocks per column of A^-1 B
])
def test_srrqr_matches_oracle(C, m, n, rank, tol, f):
    """cqrrpt_srrqr_d: every rho_ij and decision is the oracle's (same sums,
    same tie rule), the refactoring is the unpivoted QRCP, so the number of
    exchanges, J, k, Q and R equal the oracle's bit for bit."""
    if rank:
        sv = np.zeros(n)
        sv[:rank] = W.logspaced(rank, -6.0).numpy()
        A = np.asfortranarray(W.planted(m, n, sv, 701 + n, noise=1e-15).numpy())
    else:
        A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -12.0), 703).numpy())
    ref = oracle.cqrrpt_srrqr(A, 1.25, 4, tol, 77, f)
    res, sw = C.cqrrpt_srrqr(gpu(A), 1.25, 4, tol, 77, f)
    assert res.status == ref.status == 0 and res.k == ref.k
    assert sw == ref.swaps
    assert np.array_equal(host(res.J), ref.J)
    assert_bits(host(res.Q), ref.Q, "Q")
    assert_bits(host(res.R), ref.R, "R")


def test_srrqr_arguments(C):
    A = gpu(_rng(3).standard_normal((300, 10)))
    with pytest.raises(Exception):
        C.cqrrpt_srrqr(A, 1.25, 4, 1e-12, 1, f=1.0)
    res, sw = C.cqrrpt_srrqr(gpu(np.zeros((300, 10))), 1.25, 4, 1e-12, 1, f=2.0)
    assert res.k == 0 and res.status == 1 and sw == 0


# ------------------------------------------- dense operator on the tensor cores
@pytest.mark.parametrize("m,n,d", [(2 * 4096 + 77, 20, 40), (5000, 130, 129), (40000, 64, 300)])
def test_sketch_dense_split_exact_on_integers(C, m, n, d):
    """Split-BF16 dense sketch on integer operands (|S| <= 3, |M| <= 1000):
    every digit, product and 1024-term FP32 sum is exact, so S M equals the
    exact integer product bit for bit (several tiles, slices, ragged tails)."""
    rng = _rng(m + n + d)
    S = rng.integers(-3, 4, size=(d, m)).astype(np.float64)
    M = rng.integers(-1000, 1001, size=(m, n)).astype(np.float64)
    got = host(C.sketch_dense(gpu(M), gpu(S), split=True))
    assert np.array_equal(got, (S.astype(np.int64) @ M.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("m,n,d", [(9000, 130, 150), (3 * 4096 + 5, 64, 80)])
def test_sketch_dense_split_within_the_fp64_bound(C, m, n, d):
    """Gaussian S, graded columns of M: the tensor-core sketch lies within
    the FP64 dot-product bound of the oracle's FP64 sketch."""
    S = np.asfortranarray(W.gaussian_operator(d, m, 611).numpy())
    M = np.asfortranarray(_rng(612).standard_normal((m, n)) * np.logspace(0, -6, n))
    ref, st = oracle.sketch_dense(S, M)
    got = host(C.sketch_dense(gpu(M), gpu(S), split=True))
    bound = 8 * (m / 1024 + 4096 + 16) * 2.0 ** -53 * (np.abs(S) @ np.abs(M))
    assert (np.abs(got - ref) <= bound).all()


def test_cqrrpt_dense_split_sketch_nonfinite(C):
    m, n = 3000, 10
    A = _rng(14).standard_normal((m, n))
    S = np.asfortranarray(W.gaussian_operator(13, m, 613).numpy())
    S[5, 77] = np.inf
    res = C.cqrrpt_dense(gpu(A), gpu(S), 1e-12, precision=2)
    assert res.status == 2 and res.k == 0


# ------------------------------------------- edge cases of the newer entry points
def test_dense_operator_with_padded_leading_dimension(C):
    """S as a view with lds = d + 5 (and A with lda = m + 3): the FP64 dense
    sketch is bit-identical to the oracle's, the tensor-core one equals its
    own contiguous-input result bit for bit."""
    m, n, d = 4096 + 900, 12, 16
    S = np.asfortranarray(W.gaussian_operator(d, m, 620).numpy())
    A = np.asfortranarray(_rng(621).standard_normal((m, n)))
    Sbig = torch.zeros((m, d + 5), dtype=torch.float64, device="cuda")
    Sbig[:, :d] = torch.from_numpy(np.ascontiguousarray(S.T)).cuda()
    Sv = Sbig.t()[:d, :]                      # d x m, stride(1) = d + 5
    Abig = torch.zeros((n, m + 3), dtype=torch.float64, device="cuda")
    Abig[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Av = Abig.t()[:m, :]                      # m x n, stride(1) = m + 3
    assert Sv.stride(1) == d + 5 and Av.stride(1) == m + 3
    ref, _ = oracle.sketch_dense(S, A)
    assert_bits(host(C.sketch_dense(Av, Sv)), ref, "S A (padded)")
    assert_bits(host(C.sketch_dense(Av, Sv, split=True)),
                host(C.sketch_dense(gpu(A), gpu(S), split=True)), "split S A (padded)")
    res = C.cqrrpt_dense(Av, Sv, 1e-12)
    ref2 = oracle.cqrrpt_dense(A, S, 1e-12)
    assert res.k == ref2.k and np.array_equal(host(res.J), ref2.J)
    assert_bits(host(res.Q), ref2.Q, "Q")


def test_single_column_through_panels_and_srrqr(C):
    """n = 1 (d = 2): the row-panel driver and the strong-RRQR entry point
    give the oracle's bits; no exchange is possible."""
    m = 5000
    A = _rng(622).standard_normal((m, 1))
    ref = oracle.cqrrpt(np.asfortranarray(A), 1.25, 2, 1e-12, 9)
    Q, R, J, k, st = C.cqrrpt_panels(_host_colmajor(A), 1.25, 2, 1e-12, 9, panel_rows=4096)
    assert st == ref.status == 0 and k == ref.k == 1
    assert_bits(np.asfortranarray(Q.numpy()), ref.Q, "Q")
    assert_bits(np.asfortranarray(R.numpy()), ref.R, "R")
    res, sw = C.cqrrpt_srrqr(gpu(A), 1.25, 2, 1e-12, 9, f=2.0)
    assert sw == 0 and res.k == 1
    assert_bits(host(res.Q), ref.Q, "Q")


def test_two_handles_on_two_streams_at_once(C):
    # two factorisations queued on two streams without a wait in between,
    # each with its own handle: their multi-CTA QRCP grids must not compete
    # for the SMs (the library runs cooperative grids of a device one after
    # another), and each result is the oracle's bit for bit
    mats = [np.asfortranarray(W.planted(30000, n, W.logspaced(n, -7.0), 4400 + n).numpy())
            for n in (300, 280)]
    refs = [oracle.cqrrpt(A, 1.25, 4, 1e-12, 21) for A in mats]
    hs = [C.Handle(), C.Handle()]
    ss = [torch.cuda.Stream(), torch.cuda.Stream()]
    As = [gpu(A) for A in mats]
    torch.cuda.synchronize()
    outs = []
    for rep in range(3):
        for A, h, s in zip(As, hs, ss):
            outs.append(C.cqrrpt(A, 1.25, 4, 1e-12, 21, handle=h, stream=s, sync=False))
    torch.cuda.synchronize()
    for i, r in enumerate(outs):
        ref = refs[i % 2]
        st, k = hs[i % 2].last_status(ss[i % 2])
        assert st == 0 and k == ref.k
        assert np.array_equal(host(r.J), ref.J)
        assert np.array_equal(host(r.Qbuf[:, :k]).view(np.uint64), ref.Q.view(np.uint64))
        assert np.array_equal(host(r.Rbuf[:k]).view(np.uint64), ref.R.view(np.uint64))
    for h in hs:
        h.close()
