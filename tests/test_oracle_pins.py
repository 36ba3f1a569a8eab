"""Pins of the FP64 CPU oracle against facts that do not come from the oracle
itself: published known-answer vectors, exact integer arithmetic, LAPACK
(scipy GEQP3, numpy QR/Cholesky/triangular solves) on special cases that
reduce to them, closed forms from the paper's theorems, and invariants.

Each test names the passage it pins (Alg. = algorithm, Sec. = section).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# S: Philox4x32-10 and the SASO sampling rule (Sec. 2.3.1)
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Salmon et al. SC'11 Philox4x32-10, published known-answer vectors."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert oracle.philox4x32_10(w[:4], w[4:6]) == w[6:]
        n += 1
    assert n == 3


@pytest.mark.parametrize("d,s", [(16, 4), (128, 4), (1280, 8), (5, 5), (7, 1)])
def test_saso_columns_have_s_distinct_rows(d, s):
    """Sec. 2.3.1: each column of S has exactly s nonzeros at distinct rows."""
    for r in range(200):
        rows, neg = oracle.saso_column(12345, r, d, s)
        assert len(set(rows.tolist())) == s
        assert rows.min() >= 0 and rows.max() < d
        assert set(neg.tolist()) <= {0, 1}


def test_saso_subsets_uniform():
    """Sec. 2.3.1: the s locations are uniform over all s-subsets of [0, d):
    chi-square over the C(6,2) = 15 subsets (Floyd's algorithm)."""
    d, s, cols = 6, 2, 30000
    counts = {}
    for r in range(cols):
        rows, _ = oracle.saso_column(777, r, d, s)
        key = tuple(sorted(rows.tolist()))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 15
    exp = cols / 15
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 45.0  # 14 dof: p < 1e-4 for a correct sampler


def test_saso_signs_balanced_and_row_marginals_uniform():
    """Sec. 2.3.1: signs +-1 equally likely; each row equally likely."""
    d, s, cols = 40, 4, 20000
    hist = np.zeros(d)
    negs = 0
    for r in range(cols):
        rows, neg = oracle.saso_column(99, r, d, s)
        hist[rows] += 1
        negs += int(neg.sum())
    tot = cols * s
    assert abs(negs / tot - 0.5) < 0.01
    exp = tot / d
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 90.0  # 39 dof


def test_saso_seed_changes_operator():
    a = oracle.saso_dense(1, 16, 64, 4)
    b = oracle.saso_dense(2, 16, 64, 4)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, oracle.saso_dense(1, 16, 64, 4))
    assert oracle.saso_scale(4) == 0.5


# --------------------------------------------------------------------------
# Alg. 2 line 1: the sketch
# --------------------------------------------------------------------------
def test_sketch_exact_on_integer_matrix():
    """On integer M with |M| <= 2^20 every partial sum is exact, so the sketch
    must equal the exact product S M (Python integers) bit for bit; m spans
    several 4096-row blocks and a ragged tail."""
    rng = _rng(1)
    m, n, d, s = 3 * 4096 + 123, 5, 16, 4
    M = np.asfortranarray(rng.integers(-(2 ** 20), 2 ** 20, size=(m, n)).astype(np.float64))
    Msk, st = oracle.sketch(M, d, s, seed=42)
    assert st == 0
    S2 = (oracle.saso_dense(42, d, m, s) * 2).astype(np.int64)   # entries +-1
    exact = S2 @ M.astype(np.int64)                              # int64, exact
    assert np.array_equal(Msk, exact.astype(np.float64) * 0.5)


def test_sketch_matches_dense_product_general():
    rng = _rng(2)
    m, n, d, s = 5000, 7, 24, 8
    M = np.asfortranarray(rng.standard_normal((m, n)))
    Msk, st = oracle.sketch(M, d, s, seed=7)
    S = oracle.saso_dense(7, d, m, s)
    ref = S @ M
    # sequential-sum error bound: (terms per row) * u * sum |S_ir M_rc|
    bound = (m * s / d + 2) * U * (np.abs(S) @ np.abs(M))
    assert (np.abs(Msk - ref) <= bound).all()


def test_sketch_nonfinite_status():
    M = np.asfortranarray(np.ones((100, 3)))
    M[17, 1] = np.nan
    _, st = oracle.sketch(M, 8, 2, seed=1)
    assert st == 2


# --------------------------------------------------------------------------
# dot32 (the summation reading used inside the QRCP)
# --------------------------------------------------------------------------
def test_dot32_exact_on_integers_and_within_error_bound():
    rng = _rng(3)
    x = rng.integers(-1000, 1000, 333).astype(np.float64)
    y = rng.integers(-1000, 1000, 333).astype(np.float64)
    assert oracle.dot32(x, y) == float(int(x.astype(np.int64) @ y.astype(np.int64)))
    x = rng.standard_normal(1001)
    y = rng.standard_normal(1001)
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x.tolist(), y.tolist()))
    bound = (1001 / 32 + 6) * U * float(np.abs(x) @ np.abs(y))
    assert abs(Fraction(oracle.dot32(x, y)) - exact) <= Fraction(bound)


# --------------------------------------------------------------------------
# Alg. 2 line 2: QRCP (GEQP3 semantics)
# --------------------------------------------------------------------------
def _graded(d, n, seed):
    rng = _rng(seed)
    X = rng.standard_normal((d, n)) * np.logspace(0, -3, n)[rng.permutation(n)]
    return np.asfortranarray(X)


@pytest.mark.parametrize("d,n,seed", [(40, 13, 1), (128, 64, 2), (200, 150, 3), (9, 9, 4)])
def test_qrcp_matches_lapack_geqp3(d, n, seed):
    X = _graded(d, n, seed)
    R, J, tau, piv, sec, _ = oracle.qrcp(X)
    _, Rl, Jl = sl.qr(X, mode="economic", pivoting=True)
    gap = (piv - np.maximum(sec, 0)) / piv
    first_tie = int(np.argmax(gap < 1e-10)) if (gap < 1e-10).any() else n
    assert first_tie >= n - 1
    assert np.array_equal(J, Jl)
    scale = np.abs(Rl).max()
    assert np.abs(np.abs(R) - np.abs(Rl[:n, :])).max() <= 1e-12 * scale
    # R^T R = X_J^T X_J (R^sk is the R factor of the pivoted sketch)
    XJ = X[:, J]
    assert np.abs(R.T @ R - XJ.T @ XJ).max() <= 1e-13 * np.abs(XJ.T @ XJ).max()
    assert (np.diag(R) >= 0).all()
    assert np.array_equal(np.triu(R), R)
    # |R_jj| non-increasing under max-norm pivoting
    dR = np.diag(R)
    assert (dR[1:] <= dR[:-1] * (1 + 1e-12)).all()


def test_qrcp_lowest_index_on_exact_ties():
    """Businger-Golub pivoting with the BLAS idamax convention: the first of
    equal maxima.  Columns 1..3 are signed permutations of one vector of
    powers of two (exactly equal norms), column 0 is smaller."""
    base = np.array([4.0, 2.0, 1.0, 0.5, 0.25, 8.0])
    X = np.zeros((6, 4))
    X[:, 0] = base / 4
    X[:, 1] = base[[1, 0, 2, 3, 4, 5]]
    X[:, 2] = -base[[5, 4, 3, 2, 1, 0]]
    X[:, 3] = base
    R, J, *_ = oracle.qrcp(np.asfortranarray(X))
    assert J[0] == 1


# --------------------------------------------------------------------------
# Alg. 2 line 3: rank (Sec. 3.3)
# --------------------------------------------------------------------------
def test_rank_tol_counts_leading_diagonal():
    R = np.diag([2.0, 1.0, 1e-3, 1e-10, 1e-9, 1e-15])
    assert oracle.rank_tol(R, 1e-9) == 3       # 1e-10/2 < 1e-9 stops the count
    assert oracle.rank_tol(R, 1e-12) == 5
    assert oracle.rank_tol(R, 0.6) == 1
    assert oracle.rank_tol(np.zeros((3, 3)), 1e-9) == 0


def test_rank_stage1_closed_form():
    """eq. initial_numerical_rank: k_o = min{l : ||C_l||_F <= u max|R|}."""
    n = 6
    R = np.triu(np.ones((n, n))) * 0.0
    diag = [1.0, 0.5, 0.25, 1e-17, 1e-18, 0.0]
    R[np.arange(n), np.arange(n)] = diag
    # ||C_3||_F = sqrt(1e-34 + 1e-36) <= u * 1 ; ||C_2|| = 0.25 > u
    assert oracle.rank_stage1(R) == 3
    R[2, 5] = 1e-3   # in row 2 -> C_2 only
    assert oracle.rank_stage1(R) == 3
    R[3, 4] = 1e-10  # C_3 now above u
    assert oracle.rank_stage1(R) == 4


def test_rank_stage2_cond_diag():
    """eq. updated_numerical_rank with cond(diag): largest l with
    max/min of the first l diagonal entries of R^pre <= 10."""
    Rp = np.diag([1.0, 1.2, 0.9, 0.2, 0.09, 5.0])
    assert oracle.rank_stage2(6, Rp) == 4      # 1.2/0.09 > 10 at l = 5
    assert oracle.rank_stage2(3, Rp) == 3
    assert oracle.rank_stage2(6, np.diag([1.0, 0.1, 0.0999, 1, 1, 1])) == 2


# --------------------------------------------------------------------------
# Alg. 2 lines 4-8 kernels against LAPACK
# --------------------------------------------------------------------------
def test_trsm_matches_triangular_solve():
    rng = _rng(5)
    m, n, k = 300, 20, 12
    B = np.asfortranarray(rng.standard_normal((m, n)))
    T = np.triu(rng.standard_normal((k, k))) + 4 * np.eye(k)
    cols = rng.permutation(n)[:k]
    X = oracle.trsm_rut(B, T, cols)
    ref = sl.solve_triangular(T, B[:, cols].T, trans="T", lower=False).T
    assert np.abs(X - ref).max() <= 1e-13 * np.abs(ref).max()


def test_gram_matches_product_several_blocks():
    rng = _rng(6)
    m, k = 3 * 4096 + 77, 9
    X = np.asfortranarray(rng.standard_normal((m, k)))
    G = oracle.gram(X)
    assert np.array_equal(G, G.T)
    assert np.abs(G - X.T @ X).max() <= 1e-13 * m
    Xi = np.asfortranarray(rng.integers(-50, 50, (m, k)).astype(np.float64))
    assert np.array_equal(oracle.gram(Xi), (Xi.astype(np.int64).T @ Xi.astype(np.int64)).astype(float))


def test_gram_sums_256_row_sub_blocks_in_ascending_order():
    """The Gram's summation reading, on inputs where the order shows in the
    result (values derived by hand; u = 2^-53, half an ulp of 1.0).
    Column 0 is all ones, so G[0, 1] is the sum of column 1.
    (a) rows 0..255: 1, then 255 times u; rows 256..511: 255 times u, then -1.
    Sub-block 0 sums to 1 (each 1 + u is a tie and rounds to 1), sub-block 1
    to u*255 - 1 exactly; their sum is 255 u.  One sequential chain over the
    512 rows would give 0 instead (the u's all vanish against 1 or are added
    before the -1).
    (b) rows 0, 256 and 512 hold 1, u and u (the rest 0): the sub-block sums
    1, u, u added in ascending order from +0.0 give 1 (two ties); a tree
    1 + (u + u) would give 1 + 2u."""
    u = 2.0 ** -53
    y = np.zeros(512)
    y[0] = 1.0
    y[1:256] = u
    y[256:511] = u
    y[511] = -1.0
    X = np.asfortranarray(np.stack([np.ones(512), y], axis=1))
    G = oracle.gram(X)
    assert G[0, 1] == 255 * u and G[1, 0] == 255 * u
    y = np.zeros(768)
    y[0], y[256], y[512] = 1.0, u, u
    X = np.asfortranarray(np.stack([np.ones(768), y], axis=1))
    assert oracle.gram(X)[0, 1] == 1.0
    # the same sums in a second 4096-row block start again from +0.0 and the
    # two block sums are added in ascending order
    y2 = np.zeros(4096 + 512)
    y2[4096 + 0] = 1.0
    y2[4096 + 1:4096 + 256] = u
    y2[4096 + 256:4096 + 511] = u
    y2[4096 + 511] = -1.0
    # block 0 sums to 1, block 1 to 255 u; 1 + 255 u lies halfway between
    # 1 + 254 u and 1 + 256 u (the ulp of 1 is 2u) and rounds to the even one
    y2[0] = 1.0
    X = np.asfortranarray(np.stack([np.ones(4096 + 512), y2], axis=1))
    assert oracle.gram(X)[0, 1] == 1.0 + 256 * u


def test_potrf_matches_cholesky_and_reports_failure():
    rng = _rng(7)
    k = 15
    Bm = rng.standard_normal((40, k))
    G = Bm.T @ Bm
    R, fail = oracle.potrf_upper(G)
    assert fail == -1
    assert np.abs(R - np.linalg.cholesky(G).T).max() <= 1e-13 * np.abs(R).max()
    # Remark 4: column 9 depends on columns 0..8 -> failure at 9, leading block valid
    Bm[:, 9] = Bm[:, :9] @ rng.standard_normal(9)
    G = Bm.T @ Bm
    G[9, 9] -= 1e-6 * G[9, 9]
    R, fail = oracle.potrf_upper(G)
    assert fail == 9
    L = R[:9, :9]
    assert np.abs(L.T @ L - G[:9, :9]).max() <= 1e-12 * np.abs(G).max()


def test_trmm_matches_product():
    rng = _rng(8)
    k, n = 7, 11
    Rp = np.triu(rng.standard_normal((k, k)))
    Rs = np.triu(rng.standard_normal((k, n)))
    R = oracle.trmm_upper(Rp, Rs)
    assert np.abs(R - Rp @ Rs).max() <= 1e-14 * 10
    assert np.array_equal(np.triu(R), R)


# --------------------------------------------------------------------------
# The whole method
# --------------------------------------------------------------------------
def test_identity_sketch_reduces_to_geqp3():
    """With S = I (d = m is allowed, Alg. 2 input n <= d <= m) CQRRPT is QRCP
    of M itself: J equals LAPACK GEQP3's pivots and |R| equals |R_geqp3|."""
    X = _graded(90, 17, 11)
    res = oracle.cqrrpt_core_sketched(X, X, tol=1e-14)
    _, Rl, Jl = sl.qr(X, mode="economic", pivoting=True)
    assert res.k == 17
    assert np.array_equal(res.J, Jl)
    assert np.abs(res.R - np.abs(Rl) * np.sign(res.R)).max() <= 1e-12 * np.abs(Rl).max()
    assert np.abs(np.abs(res.R) - np.abs(Rl)).max() <= 1e-12 * np.abs(Rl).max()


def test_full_rank_is_unique_positive_qr_of_pivoted_matrix():
    """Full rank: (Q, R) with diag(R) > 0 is the unique QR of M[:, J]."""
    m, n = 3000, 24
    A = W.planted(m, n, W.logspaced(n, -3.0), 5).numpy()
    A = np.asfortranarray(A)
    res = oracle.cqrrpt(A, 1.25, 4, 1e-12, 17)
    assert res.status == 0 and res.k == n
    Qn, Rn = np.linalg.qr(A[:, res.J])
    sg = np.sign(np.diag(Rn))
    Qn = Qn * sg
    Rn = (Rn.T * sg).T
    assert np.abs(res.R - Rn).max() <= 1e-12 * np.abs(Rn).max()
    assert np.abs(res.Q - Qn).max() <= 1e-11


def test_theorem1_sketch_of_residual_vanishes():
    """Thm. 2: S (M_n - Q_k R_k) = 0 when rank(SM) = rank(M)."""
    m, n, gamma, s, seed = 2048, 16, 1.5, 3, 5
    A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -4.0), 9).numpy())
    res = oracle.cqrrpt(A, gamma, s, 1e-12, seed)
    d = oracle.sketch_dim(n, gamma)
    S = oracle.saso_dense(seed, d, m, s)
    D = A[:, res.J] - res.Q @ res.R
    assert np.linalg.norm(S @ D) <= 1e-14 * np.linalg.norm(S @ A) * 10


def test_theorem2_spectrum_of_preconditioned_matrix():
    """Thm. 3: sigma_i(M^pre) = 1 / sigma_{k-i+1}(S U), U an orthonormal basis
    of range(M)."""
    m, n, gamma, s, seed = 4096, 20, 1.25, 4, 3
    U_ = W.haar(m, n, 21).numpy()
    V_ = W.haar(n, n, 22).numpy()
    A = np.asfortranarray((U_ * W.logspaced(n, -4.0).numpy()) @ V_.T)
    res = oracle.cqrrpt(A, gamma, s, 1e-12, seed)
    assert res.k == n
    Mpre = oracle.trsm_rut(A, res.Rsk[:n, :n], res.J[:n])
    d = oracle.sketch_dim(n, gamma)
    S = oracle.saso_dense(seed, d, m, s)
    sv_pre = np.linalg.svd(Mpre, compute_uv=False)
    sv_su = np.linalg.svd(S @ U_, compute_uv=False)
    assert np.abs(sv_pre - 1.0 / sv_su[::-1]).max() <= 1e-9 * sv_pre.max()


def test_invariants_full_rank_cond_1e8():
    """Full-rank m = 4096, n = 64, cond 1e8, d = 2n, 4 nnz/col, tol 1e-12:
    k = n, R upper-trapezoidal with positive diagonal,
    ||M[:,J] - QR||_F/||M||_F <= 1e-13 and ||Q^T Q - I||_2 <= 1e-13."""
    w = W.single_small()
    A = np.asfortranarray(w.matrix().numpy())
    res = oracle.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    assert res.status == 0 and res.k == 64
    assert np.array_equal(np.triu(res.R), res.R) and (np.diag(res.R) > 0).all()
    assert np.linalg.norm(A[:, res.J] - res.Q @ res.R) / np.linalg.norm(A) <= 1e-13
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(64), 2) <= 1e-13
    assert sorted(res.J.tolist()) == list(range(64))


@pytest.mark.parametrize("m,n,rank,gamma,s", [(8192, 96, 60, 1.25, 8), (4100, 33, 20, 1.25, 4)])
def test_planted_rank_recovered(m, n, rank, gamma, s):
    sv = np.zeros(n)
    sv[:rank] = W.logspaced(rank, -6.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, 31, noise=1e-15).numpy())
    res = oracle.cqrrpt(A, gamma, s, 1e-9, 77)
    assert res.k == rank
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(rank), 2) <= 1e-13
    noise = 1e-15 * math.sqrt(m * n)
    assert np.linalg.norm(A[:, res.J] - res.Q @ res.R) / np.linalg.norm(A) <= \
        max(1e-13, 10 * noise / np.linalg.norm(A))


def test_default_rank_rule_and_degenerate_cases():
    rng = _rng(12)
    # zero matrix -> k = 0, status 1
    res = oracle.cqrrpt(np.zeros((64, 4), order="F"), 1.25, 2, -1.0, 1)
    assert res.status == 1 and res.k == 0
    # n = 1
    A = np.asfortranarray(rng.standard_normal((50, 1)))
    res = oracle.cqrrpt(A, 1.0, 1, -1.0, 3)
    assert res.k == 1 and abs(res.R[0, 0] - np.linalg.norm(A)) <= 1e-14 * np.linalg.norm(A)
    # d == m (gamma n = m)
    A = np.asfortranarray(rng.standard_normal((20, 16)))
    res = oracle.cqrrpt(A, 1.25, 3, -1.0, 4)
    assert res.k == 16
    assert np.linalg.norm(A[:, res.J] - res.Q @ res.R) <= 1e-13 * np.linalg.norm(A)
    # invalid arguments
    assert oracle.cqrrpt(A, 2.0, 3, -1.0, 4).status == -5      # d > m
    assert oracle.cqrrpt(A, 0.9, 3, -1.0, 4).status == -5      # gamma < 1
    assert oracle.cqrrpt(A, 1.0, 17, -1.0, 4).status == -6     # nnz > d
    # non-finite input
    A[3, 2] = np.inf
    assert oracle.cqrrpt(A, 1.0, 2, -1.0, 4).status == 2


# --------------------------------------------------------------------------
# Implicit Q (Sec. 2.1: Q_k = M^pre (R^pre)^{-1}): apply Q and Q^T
# --------------------------------------------------------------------------
def test_apply_q_exact_on_integer_factors():
    """With an integer M^pre and an upper R^pre whose diagonal holds powers
    of two and whose solves stay integral, every step is exact: Q X and
    Q^T Y equal exact rational arithmetic (pins the substitution direction,
    the transposes and the indexing)."""
    rng = _rng(41)
    m, k, r = 2 * 4096 + 19, 5, 3
    Apre = np.asfortranarray(rng.integers(-8, 9, (m, k)).astype(np.float64))
    Rpre = np.triu(rng.integers(-3, 4, (k, k)).astype(np.float64), 1) + np.diag([1.0, 2.0, 1.0, 4.0, 1.0])
    # X such that W = Rpre^{-1} X is integral: X = Rpre @ Wi
    Wi = rng.integers(-5, 6, (k, r)).astype(np.float64)
    X = Rpre @ Wi
    Y = oracle.apply_q(Apre, Rpre, X)
    assert np.array_equal(Y, Apre @ Wi)
    # Q^T Y0: Z = Apre^T Y0 in exact integers, then the forward substitution
    # with R^T in exact rationals (the divisors are powers of two)
    Y0 = np.asfortranarray(rng.integers(-4, 5, (m, r)).astype(np.float64))
    Z = [[sum(Fraction(int(a)) * Fraction(int(b)) for a, b in zip(Apre[:, t], Y0[:, c]))
          for c in range(r)] for t in range(k)]
    # exact forward substitution with R^T
    Vx = [[None] * r for _ in range(k)]
    for c in range(r):
        for j in range(k):
            s = Z[j][c] - sum(Fraction(Rpre[t, j]) * Vx[t][c] for t in range(j))
            Vx[j][c] = s / Fraction(Rpre[j, j])
    V = oracle.apply_q(Apre, Rpre, Y0, trans=True)
    for j in range(k):
        for c in range(r):
            assert V[j, c] == float(Vx[j][c]), (j, c)


def test_apply_q_matches_explicit_q_and_adjoint():
    """On a cond-1e8 factorisation: the implicit Q X and Q^T Y match the
    explicit Q of Alg. 2 line 7 to a few u, <Qx, y> = <x, Q^T y>, and
    Q^T Q x = x (orthonormal columns, Theorem 3)."""
    w = W.single_small()
    M = np.asfortranarray(w.matrix().numpy())
    res = oracle.cqrrpt_implicit(M, w.gamma, w.nnz, w.tol, w.sketch_seed)
    k = res.k
    assert k == 64 and res.Apre.shape == (M.shape[0], k)
    rng = _rng(42)
    X = rng.standard_normal((k, 4))
    Yq = oracle.apply_q(res.Apre, res.Rpre, X)
    assert np.abs(Yq - res.Q @ X).max() <= 1e-12 * np.abs(X).max()
    Y = rng.standard_normal((M.shape[0], 4))
    Z = oracle.apply_q(res.Apre, res.Rpre, Y, trans=True)
    assert np.abs(Z - res.Q.T @ Y).max() <= 1e-12 * np.linalg.norm(Y, axis=0).max()
    lhs = np.sum(Yq * Y, axis=0)
    rhs = np.sum(X * Z, axis=0)
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(lhs).max()
    back = oracle.apply_q(res.Apre, res.Rpre, Yq, trans=True)
    assert np.abs(back - X).max() <= 1e-12 * np.abs(X).max()
    # the implicit pieces are the explicit run's intermediates
    assert np.array_equal(oracle.trsm_rut(res.Apre, res.Rpre), res.Q)


# --------------------------------------------------------------------------
# Sec. 1.3: randomized CholeskyQR (unpivoted)
# --------------------------------------------------------------------------
def test_qr_nopivot_matches_lapack_qr():
    """The unpivoted Householder QR (same reflectors, diagonal made
    non-negative) equals LAPACK's R up to row signs."""
    rng = _rng(51)
    X = rng.standard_normal((60, 40)) * np.logspace(0, -4, 40)
    R = oracle.qr_nopivot(X)
    Rl = np.linalg.qr(X, mode="r")
    Rl = Rl * np.where(np.diag(Rl) < 0, -1.0, 1.0)[:, None]
    assert (np.diag(R) >= 0).all()
    assert np.abs(R - Rl).max() <= 1e-13 * np.abs(Rl).max()


def test_rcholqr_factorises_a_full_rank_matrix():
    """Sec. 1.3 on a cond-1e6 matrix: J is the identity, k = n, M = Q R,
    Q^T Q = I, and R equals LAPACK's R of M (unique with a positive
    diagonal) to the conditioning."""
    m, n = 3000, 30
    M = np.asfortranarray(W.planted(m, n, W.logspaced(n, -6.0), 52).numpy())
    res = oracle.rcholqr(M, 1.25, 4, 17)
    assert res.status == 0 and res.k == n
    assert np.array_equal(res.J, np.arange(n))
    assert np.linalg.norm(M - res.Q @ res.R) / np.linalg.norm(M) <= 1e-14
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(n), 2) <= 1e-13
    Rl = np.linalg.qr(M, mode="r")
    Rl = Rl * np.where(np.diag(Rl) < 0, -1.0, 1.0)[:, None]
    assert np.abs(res.R - Rl).max() <= 1e-9 * np.abs(Rl).max()


def test_rcholqr_equals_cqrrpt_when_the_pivots_are_the_identity():
    """Columns whose norms fall by 10x each: the QRCP of the sketch picks
    them in order, so CQRRPT (with the same near-zero rank tolerance) and
    the unpivoted method run the same arithmetic: identical bits."""
    m, n = 2500, 12
    rng = _rng(53)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    M = np.asfortranarray(U * np.logspace(0, -11, n))
    a = oracle.rcholqr(M, 1.25, 4, 9)
    b = oracle.cqrrpt(M, 1.25, 4, 1e-300, 9)
    assert np.array_equal(b.J, np.arange(n)) and a.k == b.k == n
    assert np.array_equal(a.Q.view(np.uint64), b.Q.view(np.uint64))
    assert np.array_equal(a.R.view(np.uint64), b.R.view(np.uint64))


# --------------------------------------------------------------------------
# Dense sketching operators (Sec. 2.3.1's Gaussian family)
# --------------------------------------------------------------------------
def test_sketch_dense_exact_on_integer_operands():
    """Integer S (|S| <= 3) and M (|M| <= 2^20): every product and partial
    sum is exact, so the dense sketch equals the exact product S M (int64)
    bit for bit; m spans two 4096-row blocks and a ragged tail."""
    rng = _rng(41)
    m, n, d = 2 * 4096 + 77, 5, 24
    S = np.asfortranarray(rng.integers(-3, 4, size=(d, m)).astype(np.float64))
    M = np.asfortranarray(rng.integers(-(2 ** 20), 2 ** 20, size=(m, n)).astype(np.float64))
    Msk, st = oracle.sketch_dense(S, M)
    assert st == 0
    exact = S.astype(np.int64) @ M.astype(np.int64)
    assert np.array_equal(Msk, exact.astype(np.float64))


def test_sketch_dense_of_the_saso_pattern_is_the_saso_sketch():
    """With S = the SASO's +-1 pattern, fma(+-1, a, p) rounds exactly like
    p +- a, zero entries change nothing, and the blocks are summed in the same
    order, so scale * (S_pattern M) equals the SASO sketch bit for bit."""
    rng = _rng(42)
    m, n, d, s = 3 * 4096 + 123, 6, 40, 4
    M = np.asfortranarray(rng.standard_normal((m, n)))
    scale = oracle.saso_scale(s)
    pattern = np.asfortranarray(oracle.saso_dense(9, d, m, s) / scale)
    assert set(np.unique(pattern).tolist()) <= {-1.0, 0.0, 1.0}
    Md, st = oracle.sketch_dense(pattern, M)
    assert st == 0
    Ms, st2 = oracle.sketch(M, d, s, seed=9)
    assert st2 == 0
    assert np.array_equal(Md * scale, Ms)


def test_sketch_dense_within_the_dot_product_bound():
    """Gaussian S: against the exact sum of the exact products (rationals),
    every entry lies within (4096 + blocks) u sum |S_ir M_rc|."""
    rng = _rng(43)
    m, n, d = 4096 + 50, 2, 3
    S = np.asfortranarray(W.gaussian_operator(d, m, 5).numpy())
    M = np.asfortranarray(rng.standard_normal((m, n)))
    Msk, st = oracle.sketch_dense(S, M)
    assert st == 0
    absprod = np.abs(S) @ np.abs(M)
    for i in range(d):
        for c in range(n):
            exact = sum((Fraction(float(S[i, r])) * Fraction(float(M[r, c])) for r in range(m)),
                        Fraction(0))
            err = abs(Fraction(float(Msk[i, c])) - exact)
            assert err <= Fraction((4096 + 2) * U * absprod[i, c])


def test_sketch_dense_nonfinite_status():
    S = np.asfortranarray(np.ones((4, 10)))
    M = np.asfortranarray(np.ones((10, 2)))
    M[3, 1] = np.inf
    _, st = oracle.sketch_dense(S, M)
    assert st == 2
    assert oracle.cqrrpt_dense(M, S, 1e-12).status == 2


def test_cqrrpt_dense_identity_operator_is_geqp3():
    """S = I_m (d = m): the sketch is M exactly, and CQRRPT is QRCP of M:
    J equals LAPACK GEQP3's pivots and |R| its |R|."""
    X = np.asfortranarray(_graded(90, 17, 13))
    I = np.asfortranarray(np.eye(90))
    Msk, st = oracle.sketch_dense(I, X)
    assert st == 0 and np.array_equal(Msk, X)
    res = oracle.cqrrpt_dense(X, I, 1e-14)
    _, Rl, Jl = sl.qr(X, mode="economic", pivoting=True)
    assert res.k == 17
    assert np.array_equal(res.J, Jl)
    assert np.abs(np.abs(res.R) - np.abs(Rl)).max() <= 1e-12 * np.abs(Rl).max()


def test_cqrrpt_dense_with_one_nonzero_saso_equals_cqrrpt():
    """s = 1: the SASO's entries are +-1 and its scale is exactly 1, so CQRRPT
    with that dense S is CQRRPT with the SASO, bit for bit."""
    m, n, gamma, seed = 5000, 24, 1.25, 31
    A = np.asfortranarray(W.planted(m, n, W.logspaced(n, -5.0), 8).numpy())
    d = oracle.sketch_dim(n, gamma)
    S = oracle.saso_dense(seed, d, m, 1)
    ref = oracle.cqrrpt(A, gamma, 1, 1e-12, seed)
    res = oracle.cqrrpt_dense(A, S, 1e-12)
    assert ref.status == 0 and res.status == 0 and res.k == ref.k == n
    assert np.array_equal(res.J, ref.J)
    assert np.array_equal(res.Q, ref.Q) and np.array_equal(res.R, ref.R)


def test_cqrrpt_dense_gaussian_theorem2_and_invariants():
    """Gaussian S (Sec. 2.3.1): sigma_i(M^pre) = 1 / sigma_{k-i+1}(S U)
    (Thm. 3, with M^pre = Q R^pre), and the factorisation invariants."""
    m, n = 4096 + 300, 20
    d = oracle.sketch_dim(n, 1.25)
    U_ = W.haar(m, n, 51).numpy()
    V_ = W.haar(n, n, 52).numpy()
    A = np.asfortranarray((U_ * W.logspaced(n, -4.0).numpy()) @ V_.T)
    S = np.asfortranarray(W.gaussian_operator(d, m, 53).numpy())
    res = oracle.cqrrpt_dense(A, S, 1e-12)
    assert res.status == 0 and res.k == n
    Mpre = res.Q @ res.Rpre
    sv_pre = np.linalg.svd(Mpre, compute_uv=False)
    sv_su = np.linalg.svd(S @ U_, compute_uv=False)
    assert np.abs(sv_pre - 1.0 / sv_su[::-1]).max() <= 1e-9 * sv_pre.max()
    assert np.array_equal(np.triu(res.R), res.R) and (np.diag(res.R) > 0).all()
    assert np.linalg.norm(A[:, res.J] - res.Q @ res.R) / np.linalg.norm(A) <= 1e-13
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(n), 2) <= 1e-13


def test_cqrrpt_dense_planted_rank_and_argument_errors():
    sv = np.zeros(40)
    sv[:25] = W.logspaced(25, -6.0).numpy()
    m = 6000
    A = np.asfortranarray(W.planted(m, 40, sv, 61, noise=1e-15).numpy())
    S = np.asfortranarray(W.gaussian_operator(50, m, 62).numpy())
    res = oracle.cqrrpt_dense(A, S, 1e-9)
    assert res.k == 25
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(25), 2) <= 1e-13
    Sbad = np.asfortranarray(W.gaussian_operator(30, m, 63).numpy())   # d < n
    assert oracle.cqrrpt_dense(A, Sbad, 1e-9).status == -5


# --------------------------------------------------------------------------
# Sec. 2.2: strong rank-revealing QR of the sketch (Gu-Eisenstat exchanges)
# --------------------------------------------------------------------------
def _kahan(n, c=0.285):
    s = math.sqrt(1.0 - c * c)
    K = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    K = np.diag(s ** np.arange(n)) @ K
    return np.asfortranarray(K @ np.diag(1.0 - 1e-7 * np.arange(n)))  # QRCP keeps the order


def _qrcp_R(X):
    X = np.asfortranarray(X, dtype=np.float64)
    d, n = X.shape
    W = X.copy(order="F")
    J = np.zeros(n, dtype=np.int64)
    oracle.lib().oracle_qrcp(d, n, oracle._ptr(W), d, oracle._ptr(J), None, None, None)
    return np.asfortranarray(np.triu(W[:n, :])), J


def _strong_bounds(R, k):
    A, B, Cm = R[:k, :k], R[:k, k:], R[k:, k:]
    AB = sl.solve_triangular(A, B)
    Ainv = sl.solve_triangular(A, np.eye(k))
    ratio = np.linalg.norm(Cm, axis=0)[None, :] * np.linalg.norm(Ainv, axis=1)[:, None]
    return np.abs(AB).max(), ratio.max()


def test_srrqr_repairs_the_kahan_matrix():
    """Kahan's matrix defeats max-norm pivoting (no exchange, R[n-1,n-1] far
    above sigma_min).  The strong RRQR exchanges at k = n - 1 give
    |(A^-1 B)_ij| <= f, ||C_j|| / omega_i <= f (checked with LAPACK solves),
    sigma_min <= R[n-1,n-1] <= sigma_min sqrt(1 + f^2 k (n-k)) (Gu-Eisenstat),
    and R is the R factor of K[:, J] (numpy QR, up to row signs)."""
    n, f = 30, 2.0
    K = _kahan(n)
    R0, J0 = _qrcp_R(K)
    assert np.array_equal(J0, np.arange(n))
    smin = np.linalg.svd(K, compute_uv=False)[-1]
    assert R0[-1, -1] > 100 * smin
    R, J, sw = oracle.srrqr(R0, n - 1, f, J0)
    assert sw >= 1 and sorted(J.tolist()) == list(range(n))
    ab, ratio = _strong_bounds(R, n - 1)
    assert ab <= f and ratio <= f
    assert smin * (1 - 1e-10) <= R[-1, -1] <= smin * math.sqrt(1 + f * f * (n - 1))
    Rn = np.linalg.qr(K[:, J], mode="r")
    assert np.abs(np.abs(R) - np.abs(Rn)).max() <= 1e-13 * np.abs(Rn).max()
    assert (np.diag(R) >= 0).all() and np.array_equal(np.triu(R), R)


def _vol(X, cols):
    return math.sqrt(abs(np.linalg.det(X[:, cols].T @ X[:, cols])))


def _volume_case(seed):
    """seed 0: greedy max-norm pivoting picks (a, b) with volume 70 while
    (b, c) has 98; seeds > 0: random columns with one near-dependence."""
    rng = _rng(900 + seed)
    if seed == 0:
        X = 0.01 * rng.standard_normal((12, 8))
        X[:3, 0] = [10.0, 0.0, 0.0]
        X[:3, 1] = [7.0, 7.0, 0.0]
        X[:3, 2] = [7.0, -7.0, 0.0]
        return X, 2
    X = rng.standard_normal((12, 8)) * (1.0 + 3.0 * rng.random(8))
    X[:, 5] = X[:, 0] + 0.3 * X[:, 6]
    return X, 4


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5, 6])
def test_srrqr_no_exchange_grows_the_volume_beyond_f(seed):
    """Brute force on small matrices: exchanging column i < k with column
    j >= k multiplies |det A| (the volume of the k selected columns of X)
    by sqrt(rho_ij) (Gu-Eisenstat's Lemma 3.1).  After the exchanges no single
    exchange grows the volume by more than f, and the volume did not
    shrink."""
    X, k = _volume_case(seed)
    n, f = X.shape[1], 1.02
    R0, J0 = _qrcp_R(X)
    R, J, sw = oracle.srrqr(R0, k, f, J0)
    v = _vol(X, J[:k])
    assert v >= _vol(X, J0[:k]) * (1 - 1e-12)
    for i in range(k):
        for j in range(k, n):
            cols = J.copy()
            cols[i], cols[j] = cols[j], cols[i]
            assert _vol(X, cols[:k]) <= f * v * (1 + 1e-10)


def test_srrqr_exchange_on_the_greedy_counterexample():
    """Max-norm pivoting keeps (a, b), volume 70; one exchange reaches
    (b, c), volume 98 (rho = (98/70)^2 = 1.96 > f^2)."""
    X, k = _volume_case(0)
    R0, J0 = _qrcp_R(X)
    assert sorted(J0[:2].tolist()) == [0, 1]
    R, J, sw = oracle.srrqr(R0, k, 1.2, J0)
    assert sw == 1 and sorted(J[:2].tolist()) == [1, 2]
    assert abs(_vol(X, J[:2]) / _vol(X, J0[:2]) - 1.4) < 1e-3


def test_srrqr_leaves_a_strong_factorisation_alone():
    X = _rng(77).standard_normal((200, 40))
    R0, J0 = _qrcp_R(X)
    R, J, sw = oracle.srrqr(R0, 20, 2.0, J0)
    assert sw == 0 and np.array_equal(J, J0) and np.array_equal(R, R0)


def test_cqrrpt_srrqr_planted_rank():
    """The method with the exchanges: with f = 1.05 the planted-rank matrix
    needs exchanges, and the result keeps k, the factorisation invariants
    and the strong bounds on R^sk; with f = 2 no exchange happens and the
    result is CQRRPT's, bit for bit."""
    m, n = 5000, 48
    sv = np.zeros(n)
    sv[:30] = W.logspaced(30, -6.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, 701, noise=1e-15).numpy())
    res = oracle.cqrrpt_srrqr(A, 1.25, 4, 1e-9, 77, 1.05)
    assert res.status == 0 and res.k == 30 and res.swaps > 0
    assert sorted(res.J.tolist()) == list(range(n))
    ab, ratio = _strong_bounds(res.Rsk, 30)
    assert ab <= 1.05 and ratio <= 1.05
    assert np.linalg.norm(A[:, res.J] - res.Q @ res.R) / np.linalg.norm(A) <= 1e-11
    assert np.linalg.norm(res.Q.T @ res.Q - np.eye(30), 2) <= 1e-13
    r2 = oracle.cqrrpt_srrqr(A, 1.25, 4, 1e-9, 77, 2.0)
    ref = oracle.cqrrpt(A, 1.25, 4, 1e-9, 77)
    assert r2.swaps == 0 and np.array_equal(r2.J, ref.J)
    assert np.array_equal(r2.Q, ref.Q) and np.array_equal(r2.R, ref.R)
    assert oracle.cqrrpt_srrqr(A, 1.25, 4, 1e-9, 77, 1.0).status == -10


def test_gaussian_operator_moments():
    """The input generator's Gaussian operator has iid entries of mean 0 and
    variance 1/d (Sec. 2.3.1): sample moments within a few standard errors,
    and E[S^T S] = I_m shows in the column norms (mean 1)."""
    d, m = 64, 20000
    S = W.gaussian_operator(d, m, 99).numpy()
    assert S.shape == (d, m)
    n = S.size
    assert abs(S.mean()) <= 5 / math.sqrt(n * d)
    assert abs(S.var() * d - 1.0) <= 5 * math.sqrt(2.0 / n)
    col = (S * S).sum(axis=0)
    assert abs(col.mean() - 1.0) <= 5 * math.sqrt(2.0 / d / m)


def test_cqrrpt_dense_theorem2_sketch_of_residual_vanishes():
    """Thm. 2 with a Gaussian S: S (M_n - Q_k R_k) = 0 when rank(SM) =
    rank(M), here on a planted rank-12 matrix."""
    m, n = 3000, 20
    sv = np.zeros(n)
    sv[:12] = W.logspaced(12, -4.0).numpy()
    A = np.asfortranarray(W.planted(m, n, sv, 71).numpy())
    S = np.asfortranarray(W.gaussian_operator(25, m, 72).numpy())
    res = oracle.cqrrpt_dense(A, S, 1e-10)
    assert res.k == 12
    D = A[:, res.J] - res.Q @ res.R
    assert np.linalg.norm(S @ D) <= 1e-13 * np.linalg.norm(S @ A)
