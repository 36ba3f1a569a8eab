"""The split-BF16 precision modes (FP64-accurate tensor-core products by
error-free digit splitting) against the oracle.

* On integer inputs every digit, product and partial sum is exact, so the
  split-BF16 Gram must equal the exact integer Gram bit for bit.
* On general inputs the split-BF16 Gram must agree with the FP64 oracle to
  a few units of u times |X|^T |X| (both are FP64-accurate; the split one has
  exact 1024-term partial sums, the oracle 4096-term sequential ones).
* The split-BF16 TRSM is backward stable: ||X T - B|| <= c u |X| |T|.
* The full method keeps the FP64 sketch, QRCP and rank rule, so J and k are
  bit-identical to the oracle; Q and R satisfy the paper's accuracy
  invariants (Sec. 3) and differ from the oracle entry by entry within the
  graded bound of split_bounds.py (two backward-stable QRs of the same
  matrix: u times the grading of R^sk_11 for the solve of line 4, plus the
  oracle's own Gram summation error).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import split_bounds
import workloads as W

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


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


@pytest.mark.parametrize("m,k", [(5000, 70), (1024, 1), (3000, 129)])
def test_split_gram_exact_on_integers(C, m, k):
    rng = np.random.default_rng(m + k)
    X = rng.integers(-1000, 1001, size=(m, k)).astype(np.float64)
    G = host(C.gram_split(gpu(X)))
    Xi = X.astype(np.int64)
    assert np.array_equal(G, (Xi.T @ Xi).astype(np.float64))


@pytest.mark.parametrize("m,k", [(9000, 130), (70000, 64), (300, 257)])
def test_split_gram_matches_fp64(C, m, k):
    rng = np.random.default_rng(k)
    X = rng.standard_normal((m, k)) * np.logspace(0, -6, k)
    G = host(C.gram_split(gpu(X)))
    ref = oracle.gram(X)
    bound = 8 * (m / 1024 + 4096 + 16) * U * (np.abs(X).T @ np.abs(X))
    assert (np.abs(G - ref) <= bound).all()
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("m,k,grade", [(2000, 64, 0.0), (4096 + 7, 100, -8.0), (500, 33, -3.0)])
def test_split_trsm_backward_stable(C, m, k, grade):
    rng = np.random.default_rng(k)
    n = k + 5
    B = rng.standard_normal((m, n))
    T = np.triu(rng.standard_normal((k, k)) * 0.1) + np.diag(np.logspace(0, grade, k))
    cols = rng.permutation(n)[:k].astype(np.int64)
    X = host(C.trsm_split(gpu(B), gpu(T), torch.from_numpy(cols).cuda()))
    resid = np.abs(X @ T - B[:, cols])
    scale = np.abs(X) @ np.abs(T)
    assert (resid <= 64 * k * U * scale + 1e-300).all()
    # in place, identity columns
    Xg = gpu(B[:, :k])
    C.trsm_split(Xg, gpu(T), None, out=Xg)
    X2 = host(Xg)
    assert (np.abs(X2 @ T - B[:, :k]) <= 64 * k * U * (np.abs(X2) @ np.abs(T)) + 1e-300).all()


# largest |difference| / bound allowed (the bound's constant C, see
# split_bounds.py for the error model the bound comes from)
C_ENTRY = 4.0


def _check_split(C, A, gamma, nnz, tol, seed, precision):
    ref = oracle.cqrrpt(A, gamma, nnz, tol, seed)
    res = C.cqrrpt(gpu(A), gamma, nnz, tol, seed, precision=precision)
    assert res.status == ref.status == 0
    assert res.k == ref.k
    assert np.array_equal(host(res.J), ref.J)
    Q, R = host(res.Q), host(res.R)
    AJ = A[:, ref.J]
    recon = np.linalg.norm(AJ - Q @ R) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(res.k), 2)
    rq, rr = split_bounds.ratios(Q, R, ref.Q, ref.R, ref.Rsk, A.shape[0],
                                 second_pass=(precision == 3))
    print("split precision %d: recon %.2e orth %.2e entry ratios Q %.3g R %.3g"
          % (precision, recon, orth, rq, rr))
    assert rq <= C_ENTRY and rr <= C_ENTRY, (rq, rr)
    return recon, orth


@pytest.mark.parametrize("precision", [2, 3])
def test_split_cqrrpt_full_rank_cond1e8(C, precision):
    w = W.single_small()
    A = np.asfortranarray(w.matrix().numpy())
    recon, orth = _check_split(C, A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision)
    assert recon <= 1e-13 and orth <= 1e-13


@pytest.mark.parametrize("precision", [2, 3])
def test_split_cqrrpt_cond1e10_and_planted_rank(C, precision):
    m, n = 20000, 96
    A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -10.0), 77).numpy())
    recon, orth = _check_split(C, A, 1.25, 4, 1e-12, 99, precision)
    assert recon <= 1e-13 and orth <= 1e-13
    sv = np.zeros(n)
    sv[:60] = W.logspaced(60, -6.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, 78, noise=1e-15).numpy())
    recon, orth = _check_split(C, A, 1.25, 8, 1e-9, 100, precision)
    assert orth <= 1e-13
    assert recon <= max(1e-13, 10 * 1e-15 * math.sqrt(m * n) / np.linalg.norm(A))


def test_split_deterministic(C):
    A = gpu(np.asfortranarray(W.planted(9000, 80, W.logspaced(80, -9.0), 5).numpy()))
    r1 = C.cqrrpt(A, 1.25, 4, 1e-12, 3, precision=2)
    r2 = C.cqrrpt(A, 1.25, 4, 1e-12, 3, precision=2)
    assert torch.equal(r1.Q, r2.Q) and torch.equal(r1.R, r2.R) and torch.equal(r1.J, r2.J)
