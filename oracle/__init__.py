"""Python access to the CQRRPT oracle (plain FP64 C, see ``cqrrpt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports this package.

All matrices are numpy float64 arrays in Fortran (column-major) order, the
LAPACK layout (the paper's implementation is built on LAPACK, Sec. 5).
Indices are 0-based.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_philox4x32_10.argtypes = [_p, _p, _p]
        L.oracle_saso_column.argtypes = [_u64, _i64, _i64, ctypes.c_int, _p, _p]
        L.oracle_saso_dense.argtypes = [_u64, _i64, _i64, ctypes.c_int, _d, _p]
        L.oracle_sketch.argtypes = [_i64, _i64, _p, _i64, _i64, ctypes.c_int, _u64, _d, _p, _i64]
        L.oracle_sketch.restype = ctypes.c_int
        L.oracle_dot32.argtypes = [_p, _p, _i64]
        L.oracle_dot32.restype = _d
        L.oracle_qrcp.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p]
        L.oracle_rank_tol.argtypes = [_i64, _p, _i64, _d]
        L.oracle_rank_tol.restype = _i64
        L.oracle_rank_stage1.argtypes = [_i64, _p, _i64]
        L.oracle_rank_stage1.restype = _i64
        L.oracle_rank_stage2.argtypes = [_i64, _p, _i64]
        L.oracle_rank_stage2.restype = _i64
        L.oracle_trsm_rut.argtypes = [_i64, _i64, _p, _i64, _p, _p, _i64, _p, _i64]
        L.oracle_gram.argtypes = [_i64, _i64, _p, _i64, _p, _i64]
        L.oracle_potrf_upper.argtypes = [_i64, _p, _i64, _p, _i64]
        L.oracle_potrf_upper.restype = _i64
        L.oracle_trmm_upper.argtypes = [_i64, _i64, _p, _i64, _p, _i64, _p, _i64]
        L.oracle_qr_nopivot.argtypes = [_i64, _i64, _p, _i64, _p, _p]
        L.oracle_rcholqr.argtypes = [_i64, _i64, _p, _i64, _d, ctypes.c_int, _u64, _p, _i64, _p,
                                     _i64, _p, _p, _p, _p]
        L.oracle_rcholqr.restype = ctypes.c_int
        L.oracle_apply_q.argtypes = [ctypes.c_int, _i64, _i64, _p, _i64, _p, _i64, _i64, _p,
                                     _i64, _p, _i64]
        L.oracle_sketch_dim.argtypes = [_i64, _d]
        L.oracle_sketch_dim.restype = _i64
        L.oracle_cqrrpt.argtypes = [_i64, _i64, _p, _i64, _d, ctypes.c_int, _d, _u64,
                                    _p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]
        L.oracle_cqrrpt.restype = ctypes.c_int
        L.oracle_cqrrpt_core_sketched.argtypes = [_i64, _i64, _p, _i64, _p, _i64, _d,
                                                  _p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]
        L.oracle_cqrrpt_core_sketched.restype = ctypes.c_int
        L.oracle_srrqr.argtypes = [_i64, _i64, _d, _p, _i64, _p, _i64]
        L.oracle_srrqr.restype = _i64
        L.oracle_cqrrpt_srrqr.argtypes = [_i64, _i64, _p, _i64, _d, ctypes.c_int, _d, _u64, _d,
                                          _p, _i64, _p, _i64, _p, _p, _p, _p]
        L.oracle_cqrrpt_srrqr.restype = ctypes.c_int
        L.oracle_sketch_dense.argtypes = [_i64, _i64, _i64, _p, _i64, _p, _i64, _p, _i64]
        L.oracle_sketch_dense.restype = ctypes.c_int
        L.oracle_cqrrpt_dense.argtypes = [_i64, _i64, _p, _i64, _i64, _p, _i64, _d,
                                          _p, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]
        L.oracle_cqrrpt_dense.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _fortran(a, dtype=np.float64):
    return np.asfortranarray(a, dtype=dtype)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words and 2 key words -> 4 words."""
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def saso_column(seed, r, d, s):
    """Rows (draw order) and negative-sign flags of column r of S."""
    rows = np.zeros(s, dtype=np.int32)
    neg = np.zeros(s, dtype=np.uint8)
    lib().oracle_saso_column(seed, r, d, s, _ptr(rows), _ptr(neg))
    return rows, neg


def saso_scale(s):
    """1/sqrt(s) as one IEEE division (the value both sides use)."""
    return 1.0 / math.sqrt(float(s))


def saso_dense(seed, d, m, s):
    S = np.zeros((d, m), dtype=np.float64, order="F")
    lib().oracle_saso_dense(seed, d, m, s, saso_scale(s), _ptr(S))
    return S


def sketch_dim(n, gamma):
    return int(lib().oracle_sketch_dim(n, gamma))


def sketch(M, d, s, seed):
    """M^sk = S M (Alg. 2 line 1).  Returns (Msk, status)."""
    M = _fortran(M)
    m, n = M.shape
    Msk = np.zeros((d, n), dtype=np.float64, order="F")
    st = lib().oracle_sketch(m, n, _ptr(M), m, d, s, seed, saso_scale(s), _ptr(Msk), d)
    return Msk, st


def sketch_dense(S, M):
    """M^sk = S M for a dense operator S (d x m), the blocked order of every
    tall sum, no final scaling.  Returns (Msk, status)."""
    S = _fortran(S)
    M = _fortran(M)
    d, m = S.shape
    n = M.shape[1]
    assert M.shape[0] == m
    Msk = np.zeros((d, n), dtype=np.float64, order="F")
    st = lib().oracle_sketch_dense(m, n, d, _ptr(S), d, _ptr(M), m, _ptr(Msk), d)
    return Msk, st


def dot32(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().oracle_dot32(_ptr(x), _ptr(y), x.size)


def qrcp(X):
    """QRCP of X (d x n) -> (R n x n upper, J, tau, pivot norms, runner-up norms, work)."""
    W = _fortran(X).copy(order="F")
    d, n = W.shape
    J = np.zeros(n, dtype=np.int64)
    tau = np.zeros(n)
    piv = np.zeros(n)
    sec = np.zeros(n)
    lib().oracle_qrcp(d, n, _ptr(W), d, _ptr(J), _ptr(tau), _ptr(piv), _ptr(sec))
    R = np.triu(W[:n, :]).copy(order="F")
    return R, J, tau, piv, sec, W


def rank_tol(R, tol):
    R = _fortran(R)
    return int(lib().oracle_rank_tol(R.shape[1], _ptr(R), R.shape[0], tol))


def rank_stage1(R):
    R = _fortran(R)
    return int(lib().oracle_rank_stage1(R.shape[1], _ptr(R), R.shape[0]))


def rank_stage2(ko, Rpre):
    Rpre = _fortran(Rpre)
    return int(lib().oracle_rank_stage2(ko, _ptr(Rpre), Rpre.shape[0]))


def trsm_rut(B, T, cols=None):
    """X = B[:, cols] T^{-1} (T upper triangular k x k), row-wise substitution."""
    B = _fortran(B)
    T = _fortran(T)
    m = B.shape[0]
    k = T.shape[0]
    X = np.zeros((m, k), dtype=np.float64, order="F")
    c = None if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    lib().oracle_trsm_rut(m, k, _ptr(B), m, _ptr(c), _ptr(T), k, _ptr(X), m)
    return X


def gram(X):
    X = _fortran(X)
    m, k = X.shape
    G = np.zeros((k, k), dtype=np.float64, order="F")
    lib().oracle_gram(m, k, _ptr(X), m, _ptr(G), k)
    return G


def potrf_upper(G):
    """Upper Cholesky; returns (R, fail) with fail = -1 or the failing column."""
    G = _fortran(G)
    k = G.shape[0]
    R = np.zeros((k, k), dtype=np.float64, order="F")
    fail = lib().oracle_potrf_upper(k, _ptr(G), k, _ptr(R), k)
    return R, int(fail)


def trmm_upper(Rpre, Rsk_k):
    """R = Rpre (k x k upper) @ Rsk_k (k x n upper trapezoidal)."""
    Rpre = _fortran(Rpre)
    Rsk_k = _fortran(Rsk_k)
    k, n = Rsk_k.shape
    R = np.zeros((k, n), dtype=np.float64, order="F")
    lib().oracle_trmm_upper(k, n, _ptr(Rpre), k, _ptr(Rsk_k), k, _ptr(R), k)
    return R


def apply_q(Apre, Rpre, X, trans=False):
    """Q X (trans False; X k x r) or Q^T X (trans True; X m x r) for the
    implicit Q = Apre Rpre^{-1} (Apre m x k, Rpre k x k upper)."""
    Apre = _fortran(Apre)
    Rpre = _fortran(Rpre)
    X = _fortran(X if X.ndim == 2 else X.reshape(-1, 1))
    m, k = Apre.shape
    r = X.shape[1]
    Y = np.zeros((k if trans else m, r), dtype=np.float64, order="F")
    lib().oracle_apply_q(1 if trans else 0, m, k, _ptr(Apre), m, _ptr(Rpre), k, r, _ptr(X),
                         X.shape[0], _ptr(Y), Y.shape[0])
    return Y


def qr_nopivot(X):
    """Householder QR of X (d x n) without pivoting, with the QRCP's
    reflectors and sign convention: returns (R n x n upper, positive
    diagonal)."""
    X = _fortran(X).copy(order="F")
    d, n = X.shape
    J = np.zeros(n, dtype=np.int64)
    tau = np.zeros(n)
    lib().oracle_qr_nopivot(d, n, _ptr(X), d, _ptr(J), _ptr(tau))
    return np.triu(X[:n, :]).copy(order="F")


def rcholqr(M, gamma=1.25, nnz=4, seed=0):
    """Sec. 1.3's randomized CholeskyQR (no pivoting; M of full column
    rank): Result with Q, R, J (identity), k, status, Rsk, Rpre."""
    M = _fortran(M)
    m, n = M.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    J = np.zeros(n, dtype=np.int64)
    k = np.zeros(1, dtype=np.int64)
    Rsk = np.zeros((n, n), dtype=np.float64, order="F")
    Rpre = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().oracle_rcholqr(m, n, _ptr(M), m, gamma, nnz, seed, _ptr(Q), m, _ptr(R), n,
                              _ptr(J), _ptr(k), _ptr(Rsk), _ptr(Rpre))
    kk = int(k[0])
    return Result(Q=Q[:, :kk], R=R[:kk, :], J=J, k=kk, status=int(st), Rsk=Rsk,
                  Rpre=Rpre[:kk, :kk], Qfull=Q, Rfull=R)


def cqrrpt_implicit(M, gamma=1.25, nnz=4, tol=-1.0, seed=0):
    """Alg. 1 without line 7: J, k, R as cqrrpt, plus M^pre[:, :k] (the
    preconditioned matrix, line 4) and R^pre[:k, :k] (line 6), which
    represent Q_k = M^pre (R^pre)^{-1}."""
    res = cqrrpt(M, gamma, nnz, tol, seed)
    k = res.k
    if k:
        res.Apre = trsm_rut(_fortran(M), res.Rsk[:k, :k], res.J[:k])
    else:
        res.Apre = np.zeros((_fortran(M).shape[0], 0), order="F")
    return res


class Result:
    """Output of the oracle's CQRRPT: Q (m x k), R (k x n), J (n), k, status,
    plus diagnostics R^sk, R^pre, pivot norms and runner-up norms per step."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def cqrrpt(M, gamma=1.25, nnz=4, tol=-1.0, seed=0):
    """Alg. 1: sample S from seed, d = ceil(gamma n), run Alg. 2."""
    M = _fortran(M)
    m, n = M.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    J = np.zeros(n, dtype=np.int64)
    k = np.zeros(1, dtype=np.int64)
    Rsk = np.zeros((n, n), dtype=np.float64, order="F")
    Rpre = np.zeros((n, n), dtype=np.float64, order="F")
    piv = np.zeros(n)
    sec = np.zeros(n)
    st = lib().oracle_cqrrpt(m, n, _ptr(M), m, gamma, nnz, tol, seed, _ptr(Q), m, _ptr(R), n,
                             _ptr(J), _ptr(k), _ptr(Rsk), _ptr(Rpre), _ptr(piv), _ptr(sec))
    kk = int(k[0])
    return Result(Q=Q[:, :kk], R=R[:kk, :], J=J, k=kk, status=int(st), Rsk=Rsk,
                  Rpre=Rpre[:kk, :kk], pivnorm=piv, second=sec, Qfull=Q, Rfull=R)


def cqrrpt_core_sketched(M, Msk, tol=-1.0):
    """Alg. 2 lines 2-8 for a given sketch Msk (any S), e.g. S = I."""
    M = _fortran(M)
    W = _fortran(Msk).copy(order="F")
    m, n = M.shape
    d = W.shape[0]
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    J = np.zeros(n, dtype=np.int64)
    k = np.zeros(1, dtype=np.int64)
    Rsk = np.zeros((n, n), dtype=np.float64, order="F")
    Rpre = np.zeros((n, n), dtype=np.float64, order="F")
    piv = np.zeros(n)
    sec = np.zeros(n)
    st = lib().oracle_cqrrpt_core_sketched(m, n, _ptr(M), m, _ptr(W), d, tol, _ptr(Q), m,
                                           _ptr(R), n, _ptr(J), _ptr(k), _ptr(Rsk), _ptr(Rpre),
                                           _ptr(piv), _ptr(sec))
    kk = int(k[0])
    return Result(Q=Q[:, :kk], R=R[:kk, :], J=J, k=kk, status=int(st), Rsk=Rsk,
                  Rpre=Rpre[:kk, :kk], pivnorm=piv, second=sec, Qfull=Q, Rfull=R)


def cqrrpt_dense(M, S, tol=-1.0):
    """Alg. 2 with the dense sketching operator S (d x m) given, e.g. a
    Gaussian operator (Sec. 2.3.1)."""
    M = _fortran(M)
    S = _fortran(S)
    m, n = M.shape
    d = S.shape[0]
    assert S.shape[1] == m
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    J = np.zeros(n, dtype=np.int64)
    k = np.zeros(1, dtype=np.int64)
    Rsk = np.zeros((n, n), dtype=np.float64, order="F")
    Rpre = np.zeros((n, n), dtype=np.float64, order="F")
    piv = np.zeros(n)
    sec = np.zeros(n)
    st = lib().oracle_cqrrpt_dense(m, n, _ptr(M), m, d, _ptr(S), d, tol, _ptr(Q), m, _ptr(R), n,
                                   _ptr(J), _ptr(k), _ptr(Rsk), _ptr(Rpre), _ptr(piv), _ptr(sec))
    kk = int(k[0])
    return Result(Q=Q[:, :kk], R=R[:kk, :], J=J, k=kk, status=int(st), Rsk=Rsk,
                  Rpre=Rpre[:kk, :kk], pivnorm=piv, second=sec, Qfull=Q, Rfull=R)


def srrqr(R, k, f=2.0, J=None, max_swaps=None):
    """Sec. 2.2's strong RRQR exchanges (Gu-Eisenstat, tuning parameter f) at
    rank k on an n x n upper-triangular R with J.  Returns (R, J, swaps)."""
    R = _fortran(R).copy(order="F")
    n = R.shape[0]
    J = np.arange(n, dtype=np.int64) if J is None else np.array(J, dtype=np.int64)
    sw = lib().oracle_srrqr(n, k, f, _ptr(R), n, _ptr(J), 64 * n if max_swaps is None else max_swaps)
    return R, J, int(sw)


def cqrrpt_srrqr(M, gamma=1.25, nnz=4, tol=-1.0, seed=0, f=2.0):
    """Alg. 1 with the strong RRQR exchanges after the rank rule (Sec. 2.2)."""
    M = _fortran(M)
    m, n = M.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    J = np.zeros(n, dtype=np.int64)
    k = np.zeros(1, dtype=np.int64)
    Rsk = np.zeros((n, n), dtype=np.float64, order="F")
    sw = np.zeros(1, dtype=np.int64)
    st = lib().oracle_cqrrpt_srrqr(m, n, _ptr(M), m, gamma, nnz, tol, seed, f, _ptr(Q), m,
                                   _ptr(R), n, _ptr(J), _ptr(k), _ptr(Rsk), _ptr(sw))
    kk = int(k[0])
    return Result(Q=Q[:, :kk], R=R[:kk, :], J=J, k=kk, status=int(st), Rsk=Rsk,
                  swaps=int(sw[0]), Qfull=Q, Rfull=R)
