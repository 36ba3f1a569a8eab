/*
 * CQRRPT oracle: a plain, slow, FP64 CPU implementation of CholeskyQR with
 * randomization and pivoting (Melnichenko et al., arXiv 2311.08316).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * path (the CUDA library) shares no code with it and never calls it.
 *
 * Every routine follows one passage of the paper, step by step, in the
 * paper's notation:
 *   Alg. 1 (cqrrpt)        -> oracle_cqrrpt          d = ceil(gamma n)
 *   Alg. 2 line 1 (sketch) -> oracle_sketch          M^sk = S M
 *                             oracle_sketch_dense    the same for a dense S
 *                             (Sec. 2.3.1's Gaussian operators), with
 *                             oracle_cqrrpt_dense for the whole method
 *   Alg. 2 line 2 (qrcp)   -> oracle_qrcp            GEQP3-style QRCP
 *   Alg. 2 line 3 (rank)   -> oracle_rank_tol / oracle_rank_stage1 / _stage2
 *                             (Sec. 3.3, eqs. initial_numerical_rank and
 *                              updated_numerical_rank)
 *   Alg. 2 line 4          -> oracle_trsm_rut        M^pre = M_k (A^sk_k)^-1
 *   Alg. 2 line 5          -> oracle_gram            G = (M^pre)^T M^pre
 *   Alg. 2 line 6          -> oracle_potrf_upper     R^pre = chol(G), Remark 4
 *   Alg. 2 line 7          -> oracle_trsm_rut        Q_k = M^pre (R^pre)^-1
 *   Alg. 2 line 8          -> oracle_trmm_upper      R_k = R^pre R^sk_k
 *   Q_k = M^pre (R^pre)^-1 -> oracle_apply_q         Q X and Q^T Y without forming Q
 *   Sec. 1.3 (rCholQR)     -> oracle_rcholqr         unpivoted randomized CholeskyQR
 *   Sec. 2.2 (strong RRQR) -> oracle_srrqr           Gu-Eisenstat exchanges at rank k,
 *                             oracle_cqrrpt_srrqr    the method with them
 *   (implicit Q: Sec. 2.1 notes that M^pre and R^pre represent Q_k)
 * The SASO operator is the one of Sec. 2.3.1 (each column of S has exactly s
 * nonzeros at uniformly random rows with values +-1/sqrt(s)).
 *
 * Where the paper is silent (random number generator, sampling rule,
 * summation order, pivot tie-break, sign convention) this file takes the
 * following readings; the CUDA library implements the same readings in code
 * of its own:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) drives S.  Column r
 *     of S uses key (seed lo, seed hi); row draws read the word stream
 *     Philox((r lo, r hi, t, 0)) t = 0,1,..; sign draws read
 *     Philox((r lo, r hi, t, 1)).  Rows are drawn by Floyd's algorithm for
 *     s distinct values of [0, d), each uniform draw by Lemire's
 *     multiply-shift with rejection (at most 64 rejections, then the last
 *     draw is kept).  Nonzero j is negative iff bit (j mod 32) of sign word
 *     j/32 is set.  The scale 1/sqrt(s) is a single IEEE division.
 *   - Every sum over the tall dimension m is blocked: rows are split into
 *     blocks of ROW_BLOCK = 4096; inside a block terms are added in
 *     ascending row order starting from +0.0; block sums are added in
 *     ascending block order starting from +0.0.  The Gram (line 5) blocks
 *     once more: its sum over a block is the ascending sum, from +0.0, of
 *     the block's GRAM_SUB_BLOCK = 256-row sub-block sums, each of which
 *     adds its terms in ascending row order from +0.0.
 *   - Dot products inside the QRCP of the d x n sketch ("dot32"): element i
 *     of a vector goes to lane i mod 32; each lane accumulates its elements
 *     in ascending order with fma from +0.0; lanes are combined by the fixed
 *     tree (l += l+16, l += l+8, l += l+4, l += l+2, l += l+1).
 *   - All other sums (substitution, Cholesky, triangular product) run in
 *     ascending index order, one fma per term.
 *   - QRCP pivots on the largest partial column norm, lowest position on
 *     exact ties; reflectors as LAPACK's dlarfg: beta = -sign(alpha) ||x||,
 *     tau = (beta - alpha) / beta, v = x * (1 / (alpha - beta)) (one
 *     division, then a scaling); the LAPACK dlaqp2 downdate with the
 *     Drmac-Bujanovic recompute safeguard (threshold sqrt(u)); after the
 *     n steps every row
 *     of R^sk with a negative diagonal is negated, so diag(R^sk) >= 0 and
 *     the returned R has a positive diagonal.
 *   - Plain a*b+c is never contracted: build with -ffp-contract=off; every
 *     fused multiply-add is written as fma().
 *
 * Layout: all matrices column-major (LAPACK), 0-based indices.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors, brute-force
 * rational sketch on integer inputs, scipy GEQP3 pivots on the sketch, the
 * S = I special case (CQRRPT reduces to GEQP3 on M), the unique
 * positive-diagonal QR of M[:, J] from numpy, Theorem 2 (S (M_n - Q_k R_k)
 * = 0), Theorem 3 (singular values of M^pre are the inverses of those of
 * S U), and planted-rank recovery.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ROW_BLOCK 4096
#define GRAM_SUB_BLOCK 256

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2).                           */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word stream: word w of stream `tag` for column r. */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;
} word_stream;

static void ws_init(word_stream* ws, uint64_t seed, int64_t r, uint32_t tag) {
    ws->key[0] = (uint32_t)seed;
    ws->key[1] = (uint32_t)(seed >> 32);
    ws->ctr[0] = (uint32_t)(uint64_t)r;
    ws->ctr[1] = (uint32_t)((uint64_t)r >> 32);
    ws->ctr[2] = 0;
    ws->ctr[3] = tag;
    ws->pos = 4;
}

static uint32_t ws_next(word_stream* ws) {
    if (ws->pos == 4) {
        oracle_philox4x32_10(ws->ctr, ws->key, ws->buf);
        ws->ctr[2] += 1;
        ws->pos = 0;
    }
    return ws->buf[ws->pos++];
}

/* Uniform integer in [0, range) (Lemire 2019, multiply-shift with rejection). */
static uint32_t uniform_below(word_stream* ws, uint32_t range) {
    uint64_t prod = (uint64_t)ws_next(ws) * range;
    uint32_t low = (uint32_t)prod;
    if (low < range) {
        uint32_t thresh = (uint32_t)(-range) % range;
        int tries = 0;
        while (low < thresh && tries < 64) {
            prod = (uint64_t)ws_next(ws) * range;
            low = (uint32_t)prod;
            ++tries;
        }
    }
    return (uint32_t)(prod >> 32);
}

/* Column r of the SASO S (Sec. 2.3.1): s distinct rows of [0, d) in draw
 * order and their signs (1 = negative). */
void oracle_saso_column(uint64_t seed, int64_t r, int64_t d, int s, int32_t* rows, uint8_t* neg) {
    word_stream rs, ss;
    ws_init(&rs, seed, r, 0u);
    ws_init(&ss, seed, r, 1u);
    /* Floyd's algorithm: for j = d-s .. d-1 draw t in [0, j]; take j if t was
     * already taken, else t. */
    for (int q = 0; q < s; ++q) {
        uint32_t jj = (uint32_t)(d - s + q);
        uint32_t t = uniform_below(&rs, jj + 1u);
        int taken = 0;
        for (int p = 0; p < q; ++p)
            if ((uint32_t)rows[p] == t) taken = 1;
        rows[q] = (int32_t)(taken ? jj : t);
    }
    uint32_t word = 0;
    for (int q = 0; q < s; ++q) {
        if (q % 32 == 0) word = ws_next(&ss);
        neg[q] = (uint8_t)((word >> (q % 32)) & 1u);
    }
}

/* Dense S (d x m, column-major) for tests on tiny sizes. */
void oracle_saso_dense(uint64_t seed, int64_t d, int64_t m, int s, double scale, double* S) {
    int32_t rows[4096];
    uint8_t neg[4096];
    memset(S, 0, sizeof(double) * (size_t)(d * m));
    for (int64_t r = 0; r < m; ++r) {
        oracle_saso_column(seed, r, d, s, rows, neg);
        for (int q = 0; q < s; ++q) S[rows[q] + r * d] = neg[q] ? -scale : scale;
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 line 1: sketch M^sk = S M (d x n).                                 */
/* ------------------------------------------------------------------------ */
/* Returns 0, or 2 if the sketch holds a non-finite value. */
int oracle_sketch(int64_t m, int64_t n, const double* M, int64_t ldm, int64_t d, int s,
                  uint64_t seed, double scale, double* Msk, int64_t ldsk) {
    int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m * s));
    uint8_t* neg = (uint8_t*)malloc((size_t)(m * s));
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) oracle_saso_column(seed, r, d, s, rows + r * s, neg + r * s);

    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int64_t c = 0; c < n; ++c) {
        double* total = (double*)malloc(sizeof(double) * (size_t)d);
        double* part = (double*)malloc(sizeof(double) * (size_t)d);
        for (int64_t i = 0; i < d; ++i) total[i] = 0.0;
        for (int64_t r0 = 0; r0 < m; r0 += ROW_BLOCK) {
            int64_t r1 = r0 + ROW_BLOCK < m ? r0 + ROW_BLOCK : m;
            for (int64_t i = 0; i < d; ++i) part[i] = 0.0;
            for (int64_t r = r0; r < r1; ++r) {
                double a = M[r + c * ldm];
                for (int q = 0; q < s; ++q) {
                    int64_t i = rows[r * s + q];
                    part[i] = neg[r * s + q] ? part[i] - a : part[i] + a;
                }
            }
            for (int64_t i = 0; i < d; ++i) total[i] = total[i] + part[i];
        }
        for (int64_t i = 0; i < d; ++i) {
            double v = total[i] * scale;
            Msk[i + c * ldsk] = v;
            if (!isfinite(v)) bad = 1;
        }
        free(total);
        free(part);
    }
    free(rows);
    free(neg);
    return bad ? 2 : 0;
}

/* Alg. 2 line 1 with a dense operator S (d x m, column-major, ld lds) that
 * the caller drew, e.g. from the Gaussian family of Sec. 2.3.1 (iid entries
 * of mean 0 and variance 1/d).  M^sk[i, c] = sum_r S[i, r] M[r, c], blocked
 * over the rows like every tall sum: one fma per term in ascending r from
 * +0.0 inside a block, block sums added in ascending block order from +0.0.
 * There is no final scaling: S carries its own.  Returns 0, or 2 if the
 * sketch holds a non-finite value. */
int oracle_sketch_dense(int64_t m, int64_t n, int64_t d, const double* S, int64_t lds,
                        const double* M, int64_t ldm, double* Msk, int64_t ldsk) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int64_t c = 0; c < n; ++c) {
        double* total = (double*)malloc(sizeof(double) * (size_t)d);
        double* part = (double*)malloc(sizeof(double) * (size_t)d);
        for (int64_t i = 0; i < d; ++i) total[i] = 0.0;
        for (int64_t r0 = 0; r0 < m; r0 += ROW_BLOCK) {
            int64_t r1 = r0 + ROW_BLOCK < m ? r0 + ROW_BLOCK : m;
            for (int64_t i = 0; i < d; ++i) part[i] = 0.0;
            for (int64_t r = r0; r < r1; ++r) {
                double a = M[r + c * ldm];
                const double* Sr = S + r * lds;
                for (int64_t i = 0; i < d; ++i) part[i] = fma(Sr[i], a, part[i]);
            }
            for (int64_t i = 0; i < d; ++i) total[i] = total[i] + part[i];
        }
        for (int64_t i = 0; i < d; ++i) {
            Msk[i + c * ldsk] = total[i];
            if (!isfinite(total[i])) bad = 1;
        }
        free(total);
        free(part);
    }
    return bad ? 2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 line 2: QRCP of the sketch (Businger-Golub max-norm pivoting as in  */
/* LAPACK GEQP3, Sec. 1 and Sec. 2.1 flop count).                          */
/* ------------------------------------------------------------------------ */
/* dot32 of x[0..len) and y[0..len) (the reading stated in the header). */
double oracle_dot32(const double* x, const double* y, int64_t len) {
    double lane[32];
    for (int l = 0; l < 32; ++l) lane[l] = 0.0;
    for (int64_t i = 0; i < len; ++i) lane[i % 32] = fma(x[i], y[i], lane[i % 32]);
    for (int off = 16; off >= 1; off /= 2)
        for (int l = 0; l < off; ++l) lane[l] = lane[l] + lane[l + off];
    return lane[0];
}

/* X: d x n column-major (in: sketch; out: R^sk in rows 0..n-1, upper part,
 * rows with negative diagonal negated; below the diagonal: Householder data).
 * J: n pivots (position -> original column).  vn_out (optional): vn1 at the
 * moment each column was chosen (the pivot norm), for near-tie analysis. */
/* pivoting == 0: plain Householder QR (the column at position j is step j's
 * pivot; Sec. 1.3's randomized CholeskyQR), same reflectors and updates. */
static void qrcp_ex(int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J, double* tau_out,
                    double* pivnorm_out, double* second_out, int pivoting);

void oracle_qrcp(int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J, double* tau_out,
                 double* pivnorm_out, double* second_out) {
    qrcp_ex(d, n, X, ldx, J, tau_out, pivnorm_out, second_out, 1);
}

void oracle_qr_nopivot(int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J,
                       double* tau_out) {
    qrcp_ex(d, n, X, ldx, J, tau_out, NULL, NULL, 0);
}

static void qrcp_ex(int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J, double* tau_out,
                    double* pivnorm_out, double* second_out, int pivoting) {
    const double u = ldexp(1.0, -53);
    const double tol3z = sqrt(u);
    double* vn1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* vn2 = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t c = 0; c < n; ++c) {
        const double* col = X + c * ldx;
        vn1[c] = sqrt(oracle_dot32(col, col, d));
        vn2[c] = vn1[c];
        J[c] = c;
    }
    for (int64_t j = 0; j < n; ++j) {
        /* pivot: largest vn1 over positions j..n-1, lowest position on ties */
        int64_t p = j;
        if (pivoting)
            for (int64_t c = j + 1; c < n; ++c)
                if (vn1[c] > vn1[p]) p = c;
        if (pivnorm_out) pivnorm_out[j] = vn1[p];
        if (second_out) {
            double sec = -1.0;
            for (int64_t c = j; c < n; ++c)
                if (c != p && vn1[c] > sec) sec = vn1[c];
            second_out[j] = sec;
        }
        if (p != j) {
            for (int64_t r = 0; r < d; ++r) {
                double t = X[r + p * ldx];
                X[r + p * ldx] = X[r + j * ldx];
                X[r + j * ldx] = t;
            }
            int64_t tj = J[p]; J[p] = J[j]; J[j] = tj;
            vn1[p] = vn1[j];
            vn2[p] = vn2[j];
        }
        /* Householder reflector H = I - tau v v^T with v[0] = 1 on X[j:, j] */
        double* colj = X + j * ldx;
        double alpha = colj[j];
        double sumsq = (j + 1 < d) ? oracle_dot32(colj + j + 1, colj + j + 1, d - j - 1) : 0.0;
        double tau;
        if (sumsq == 0.0) {
            tau = 0.0;
        } else {
            double nrm = sqrt(fma(alpha, alpha, sumsq));
            double beta = (alpha >= 0.0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            /* v = x (1 / (alpha - beta)): one division, then a scaling, as
             * LAPACK's reflector generator (dlarfg) does in GEQP3 */
            double rden = 1.0 / (alpha - beta);
            for (int64_t r = j + 1; r < d; ++r) colj[r] = colj[r] * rden;
            colj[j] = beta;
        }
        if (tau_out) tau_out[j] = tau;
        /* apply H to the trailing columns, then downdate their norms */
        double* v = (double*)malloc(sizeof(double) * (size_t)(d - j));
        v[0] = 1.0;
        for (int64_t r = j + 1; r < d; ++r) v[r - j] = colj[r];
        for (int64_t c = j + 1; c < n; ++c) {
            double* colc = X + c * ldx;
            double w = oracle_dot32(v, colc + j, d - j);
            double t = -tau * w;
            for (int64_t r = j; r < d; ++r) colc[r] = fma(v[r - j], t, colc[r]);
            if (vn1[c] != 0.0) {
                double temp = fabs(colc[j]) / vn1[c];
                temp = 1.0 - temp * temp;
                temp = temp > 0.0 ? temp : 0.0;
                double ratio = vn1[c] / vn2[c];
                double temp2 = temp * (ratio * ratio);
                if (temp2 <= tol3z) {
                    if (j + 1 < d) {
                        vn1[c] = sqrt(oracle_dot32(colc + j + 1, colc + j + 1, d - j - 1));
                    } else {
                        vn1[c] = 0.0;
                    }
                    vn2[c] = vn1[c];
                } else {
                    vn1[c] = vn1[c] * sqrt(temp);
                }
            }
        }
        free(v);
    }
    /* sign convention: diag(R^sk) >= 0 (absorbed into the discarded Q^sk) */
    for (int64_t j = 0; j < n; ++j) {
        if (X[j + j * ldx] < 0.0)
            for (int64_t c = j; c < n; ++c) X[j + c * ldx] = -X[j + c * ldx];
    }
    free(vn1);
    free(vn2);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 line 3: rank.                                                      */
/* ------------------------------------------------------------------------ */
/* tol > 0: number of leading j with R[j,j] > tol * R[0,0]. */
int64_t oracle_rank_tol(int64_t n, const double* R, int64_t ldr, double tol) {
    double thresh = tol * R[0];
    int64_t k = 0;
    while (k < n && R[k + k * ldr] > thresh) ++k;
    return k;
}

/* Stage 1 (eq. initial_numerical_rank): k_o = min{l : ||C^sk_l||_F <= u s},
 * s = max |R^sk|, C^sk_l = R^sk[l:, l:].  ||C_l||^2 = ||R[l, l:]||^2 +
 * ||C_{l+1}||^2, each row sum in ascending column order. */
int64_t oracle_rank_stage1(int64_t n, const double* R, int64_t ldr) {
    const double u = ldexp(1.0, -53);
    double smax = 0.0;
    for (int64_t c = 0; c < n; ++c)
        for (int64_t i = 0; i <= c; ++i) {
            double a = fabs(R[i + c * ldr]);
            if (a > smax) smax = a;
        }
    double* f2 = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    f2[n] = 0.0;
    for (int64_t l = n - 1; l >= 0; --l) {
        double rs = 0.0;
        for (int64_t c = l; c < n; ++c) rs = fma(R[l + c * ldr], R[l + c * ldr], rs);
        f2[l] = f2[l + 1] + rs;
    }
    double thresh = u * smax;
    int64_t ko = n;
    for (int64_t l = 0; l <= n; ++l)
        if (sqrt(f2[l]) <= thresh) { ko = l; break; }
    free(f2);
    return ko;
}

/* Stage 2 (eq. updated_numerical_rank with cond = cond(diag)):
 * largest l <= ko with max_{i<l} Rpre_ii / min_{i<l} Rpre_ii <= 10
 * (10 = sqrt(eps_tol / u) with eps_tol = 100 u). */
int64_t oracle_rank_stage2(int64_t ko, const double* Rpre, int64_t ldr) {
    int64_t k = 0;
    double mx = 0.0, mn = 0.0;
    for (int64_t l = 1; l <= ko; ++l) {
        double dl = Rpre[(l - 1) + (l - 1) * ldr];
        if (l == 1) { mx = dl; mn = dl; }
        else { if (dl > mx) mx = dl; if (dl < mn) mn = dl; }
        if (mx / mn <= 10.0) k = l; else break;
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 lines 4 and 7: X = B(:, cols) * T^{-1}, T upper triangular k x k,  */
/* by row-wise substitution in ascending order.  cols == NULL: identity.     */
/* ------------------------------------------------------------------------ */
void oracle_trsm_rut(int64_t m, int64_t k, const double* B, int64_t ldb, const int64_t* cols,
                     const double* T, int64_t ldt, double* X, int64_t ldx) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < k; ++j) {
            int64_t bc = cols ? cols[j] : j;
            double s = B[i + bc * ldb];
            for (int64_t t = 0; t < j; ++t) s = fma(-X[i + t * ldx], T[t + j * ldt], s);
            X[i + j * ldx] = s / T[j + j * ldt];
        }
    }
}

/* Alg. 2 line 5: G = X^T X (k x k, both triangles), blocked sum over rows:
 * 256-row sub-blocks inside 4096-row blocks (the reading above). */
void oracle_gram(int64_t m, int64_t k, const double* X, int64_t ldx, double* G, int64_t ldg) {
#pragma omp parallel for schedule(dynamic)
    for (int64_t b = 0; b < k; ++b) {
        for (int64_t a = 0; a <= b; ++a) {
            const double* xa = X + a * ldx;
            const double* xb = X + b * ldx;
            double total = 0.0;
            for (int64_t r0 = 0; r0 < m; r0 += ROW_BLOCK) {
                int64_t r1 = r0 + ROW_BLOCK < m ? r0 + ROW_BLOCK : m;
                double part = 0.0;
                for (int64_t s0 = r0; s0 < r1; s0 += GRAM_SUB_BLOCK) {
                    int64_t s1 = s0 + GRAM_SUB_BLOCK < r1 ? s0 + GRAM_SUB_BLOCK : r1;
                    double sub = 0.0;
                    for (int64_t r = s0; r < s1; ++r) sub = fma(xa[r], xb[r], sub);
                    part = part + sub;
                }
                total = total + part;
            }
            G[a + b * ldg] = total;
            G[b + a * ldg] = total;
        }
    }
}

/* Alg. 2 line 6: upper Cholesky G = R^T R (unblocked, ascending sums).
 * Returns -1 on success or the first column j whose pivot is not positive
 * (Remark 4: the leading j x j block of R is then valid). */
int64_t oracle_potrf_upper(int64_t k, const double* G, int64_t ldg, double* R, int64_t ldr) {
    for (int64_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < k; ++i) R[i + c * ldr] = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        double s = G[j + j * ldg];
        for (int64_t t = 0; t < j; ++t) s = fma(-R[t + j * ldr], R[t + j * ldr], s);
        if (!(s > 0.0)) return j;
        double rjj = sqrt(s);
        R[j + j * ldr] = rjj;
        for (int64_t c = j + 1; c < k; ++c) {
            double sc = G[j + c * ldg];
            for (int64_t t = 0; t < j; ++t) sc = fma(-R[t + j * ldr], R[t + c * ldr], sc);
            R[j + c * ldr] = sc / rjj;
        }
    }
    return -1;
}

/* Alg. 2 line 8: R_k = R^pre (k x k upper) * R^sk[0:k, :] (k x n upper
 * trapezoidal); entries below the diagonal are set to zero. */
void oracle_trmm_upper(int64_t k, int64_t n, const double* Rpre, int64_t ldp, const double* Rsk,
                       int64_t ldsk, double* R, int64_t ldr) {
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t i = 0; i < k; ++i) {
            if (c < i) { R[i + c * ldr] = 0.0; continue; }
            int64_t tend = c < k - 1 ? c : k - 1;
            double s = 0.0;
            for (int64_t t = i; t <= tend; ++t) s = fma(Rpre[i + t * ldp], Rsk[t + c * ldsk], s);
            R[i + c * ldr] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: strong rank-revealing QR of the sketch at rank k (Gu and        */
/* Eisenstat 1996, with tuning parameter f > 1; the paper names f = 2).      */
/* ------------------------------------------------------------------------ */
/* R = [A B; 0 C] (n x n upper triangular, diag >= 0, ld ldr) with A the
 * leading k x k block.  While some pair (i < k <= j) has
 *     rho_ij = (A^{-1} B)_{i, j-k}^2 + ||C[:, j-k]||^2 ||row i of A^{-1}||^2
 * above f^2, the pair with the largest rho_ij (lowest i, then lowest j, on
 * ties) has its columns exchanged (in R and in J) and R is refactored by
 * an unpivoted Householder QR (the QRCP's reflectors and sign convention,
 * Q discarded).  Each exchange multiplies |det A| by sqrt(rho_ij) > f, so
 * the loop ends; max_swaps bounds it all the same.  Sums run in ascending
 * index order with one fma per term:
 *     W = A^{-1} by columns, column-oriented back substitution (column c:
 *         x = e_c; for t = c down to 0: x_t = x_t / A[t,t], then
 *         x_i = fma(-A[i,t], x_t, x_i) for every i < t);
 *     (A^{-1}B)[i,j] = sum_{t=i..k-1} W[i,t] R[t,k+j];
 *     w2_i = sum_{t=i..k-1} W[i,t]^2;  g2_j = sum_{t=k..k+j} R[t,k+j]^2;
 *     rho_ij = fma(ab, ab, g2_j * w2_i).
 * Returns the number of exchanges. */
int64_t oracle_srrqr(int64_t n, int64_t k, double f, double* R, int64_t ldr, int64_t* J,
                     int64_t max_swaps) {
    if (k <= 0 || k >= n) return 0;
    const int64_t nk = n - k;
    double* W = (double*)calloc((size_t)(k * k), sizeof(double));
    double* w2 = (double*)malloc(sizeof(double) * (size_t)k);
    double* g2 = (double*)malloc(sizeof(double) * (size_t)nk);
    double* X = (double*)malloc(sizeof(double) * (size_t)(n * n));
    int64_t* Jt = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    double* tau = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t swaps = 0;
    while (swaps < max_swaps) {
        for (int64_t c = 0; c < k; ++c) {
            double* x = W + c * k;
            for (int64_t i = 0; i < k; ++i) x[i] = i == c ? 1.0 : 0.0;
            for (int64_t t = c; t >= 0; --t) {
                x[t] = x[t] / R[t + t * ldr];
                for (int64_t i = 0; i < t; ++i) x[i] = fma(-R[i + t * ldr], x[t], x[i]);
            }
        }
        for (int64_t i = 0; i < k; ++i) {
            double s = 0.0;
            for (int64_t t = i; t < k; ++t) s = fma(W[i + t * k], W[i + t * k], s);
            w2[i] = s;
        }
        for (int64_t j = 0; j < nk; ++j) {
            double s = 0.0;
            for (int64_t t = k; t <= k + j; ++t) s = fma(R[t + (k + j) * ldr], R[t + (k + j) * ldr], s);
            g2[j] = s;
        }
        double best = -1.0;
        int64_t bi = -1, bj = -1;
        for (int64_t i = 0; i < k; ++i)
            for (int64_t j = 0; j < nk; ++j) {
                double ab = 0.0;
                for (int64_t t = i; t < k; ++t) ab = fma(W[i + t * k], R[t + (k + j) * ldr], ab);
                double rho = fma(ab, ab, g2[j] * w2[i]);
                if (rho > best) { best = rho; bi = i; bj = j; }
            }
        if (!(best > f * f)) break;
        /* exchange columns bi and k + bj, then refactor */
        const int64_t jc = k + bj;
        for (int64_t c = 0; c < n; ++c) {
            const int64_t src = c == bi ? jc : (c == jc ? bi : c);
            for (int64_t r = 0; r < n; ++r) X[r + c * n] = R[r + src * ldr];
        }
        int64_t tj = J[bi]; J[bi] = J[jc]; J[jc] = tj;
        qrcp_ex(n, n, X, n, Jt, tau, NULL, NULL, 0);
        for (int64_t c = 0; c < n; ++c)
            for (int64_t r = 0; r < n; ++r) R[r + c * ldr] = r <= c ? X[r + c * n] : 0.0;
        ++swaps;
    }
    free(W); free(w2); free(g2); free(X); free(Jt); free(tau);
    return swaps;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 + Alg. 2: the full method.                                         */
/* ------------------------------------------------------------------------ */
int64_t oracle_sketch_dim(int64_t n, double gamma) { return (int64_t)ceil(gamma * (double)n); }

/* Alg. 2 lines 2-8 given the sketch Msk (d x n, ld d, overwritten).
 * Returns 0, or 1 when k == 0.  Q: m x n capacity (first k columns
 * written); R: n x n capacity (first k rows written); J: n pivots; *k_out:
 * rank.  Optional diagnostics (may be NULL): Rsk_out (n x n, ld n) R^sk;
 * Rpre_out (n x n, ld n) R^pre; pivnorm/second (n). */
static int core_ex(int64_t m, int64_t n, const double* M, int64_t ldm, double* Msk, int64_t d,
                   double tol, double* Q, int64_t ldq, double* R, int64_t ldr, int64_t* J,
                   int64_t* k_out, double* Rsk_out, double* Rpre_out, double* pivnorm,
                   double* second, int pivoting, double srrqr_f, int64_t* swaps_out);

int oracle_cqrrpt_core_sketched(int64_t m, int64_t n, const double* M, int64_t ldm, double* Msk,
                                int64_t d, double tol, double* Q, int64_t ldq, double* R,
                                int64_t ldr, int64_t* J, int64_t* k_out, double* Rsk_out,
                                double* Rpre_out, double* pivnorm, double* second) {
    return core_ex(m, n, M, ldm, Msk, d, tol, Q, ldq, R, ldr, J, k_out, Rsk_out, Rpre_out,
                   pivnorm, second, 1, 0.0, NULL);
}

static int core_ex(int64_t m, int64_t n, const double* M, int64_t ldm, double* Msk, int64_t d,
                   double tol, double* Q, int64_t ldq, double* R, int64_t ldr, int64_t* J,
                   int64_t* k_out, double* Rsk_out, double* Rpre_out, double* pivnorm,
                   double* second, int pivoting, double srrqr_f, int64_t* swaps_out) {
    *k_out = 0;
    double* tau = (double*)malloc(sizeof(double) * (size_t)n);
    qrcp_ex(d, n, Msk, d, J, tau, pivnorm, second, pivoting);
    /* R^sk: upper n x n */
    double* Rsk = (double*)calloc((size_t)(n * n), sizeof(double));
    for (int64_t c = 0; c < n; ++c)
        for (int64_t i = 0; i <= c; ++i) Rsk[i + c * n] = Msk[i + c * d];
    if (Rsk_out) memcpy(Rsk_out, Rsk, sizeof(double) * (size_t)(n * n));
    if (Rpre_out) memset(Rpre_out, 0, sizeof(double) * (size_t)(n * n));

    int stage2 = !(tol > 0.0);
    int64_t k = stage2 ? oracle_rank_stage1(n, Rsk, n) : oracle_rank_tol(n, Rsk, n, tol);
    if (srrqr_f > 0.0) {
        int64_t sw = oracle_srrqr(n, k, srrqr_f, Rsk, n, J, 64 * n);
        if (swaps_out) *swaps_out = sw;
        if (Rsk_out) memcpy(Rsk_out, Rsk, sizeof(double) * (size_t)(n * n));
    }
    if (k > 0) {
        /* M^pre into Q's storage */
        oracle_trsm_rut(m, k, M, ldm, J, Rsk, n, Q, ldq);
        double* G = (double*)malloc(sizeof(double) * (size_t)(k * k));
        oracle_gram(m, k, Q, ldq, G, k);
        double* Rpre = (double*)malloc(sizeof(double) * (size_t)(k * k));
        int64_t fail = oracle_potrf_upper(k, G, k, Rpre, k);
        int64_t kc = fail >= 0 ? fail : k; /* Remark 4 */
        if (stage2 && kc > 0) kc = oracle_rank_stage2(kc, Rpre, k);
        k = kc;
        if (k > 0) {
            /* Q_k = M^pre (R^pre)^{-1}, in place, row by row */
            oracle_trsm_rut(m, k, Q, ldq, NULL, Rpre, k, Q, ldq);
            oracle_trmm_upper(k, n, Rpre, k, Rsk, n, R, ldr);
            if (Rpre_out)
                for (int64_t c = 0; c < k; ++c)
                    for (int64_t i = 0; i <= c; ++i) Rpre_out[i + c * n] = Rpre[i + c * k];
        }
        free(G);
        free(Rpre);
    }
    *k_out = k;
    free(Rsk);
    free(tau);
    return k == 0 ? 1 : 0;
}

/* Alg. 1: d = ceil(gamma n), sample the SASO S from seed, then Alg. 2.
 * Returns 0 on success, -i for invalid argument i, 1 when k == 0, 2 for a
 * non-finite sketch (then J, Q, R are not written and k = 0). */
int oracle_cqrrpt(int64_t m, int64_t n, const double* M, int64_t ldm, double gamma, int nnz,
                  double tol, uint64_t seed, double* Q, int64_t ldq, double* R, int64_t ldr,
                  int64_t* J, int64_t* k_out, double* Rsk_out, double* Rpre_out, double* pivnorm,
                  double* second) {
    *k_out = 0;
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (ldm < m) return -4;
    if (!(gamma >= 1.0)) return -5;
    int64_t d = oracle_sketch_dim(n, gamma);
    if (d > m) return -5;
    if (nnz < 1 || nnz > d) return -6;
    if (ldq < m) return -10;
    if (ldr < n) return -12;
    double scale = 1.0 / sqrt((double)nnz);
    double* Msk = (double*)malloc(sizeof(double) * (size_t)(d * n));
    int st = oracle_sketch(m, n, M, ldm, d, nnz, seed, scale, Msk, d);
    if (st == 0)
        st = oracle_cqrrpt_core_sketched(m, n, M, ldm, Msk, d, tol, Q, ldq, R, ldr, J, k_out,
                                         Rsk_out, Rpre_out, pivnorm, second);
    free(Msk);
    return st;
}

/* Alg. 1 with the strong rank-revealing QR of Sec. 2.2 in line 2: the QRCP
 * of the sketch, the rank k of line 3, then oracle_srrqr at that k (J and
 * R^sk exchanged and refactored), then lines 4-8 as oracle_cqrrpt.
 * *swaps_out receives the number of exchanges.  Returns as oracle_cqrrpt
 * (-10 for f <= 1). */
int oracle_cqrrpt_srrqr(int64_t m, int64_t n, const double* M, int64_t ldm, double gamma, int nnz,
                        double tol, uint64_t seed, double f, double* Q, int64_t ldq, double* R,
                        int64_t ldr, int64_t* J, int64_t* k_out, double* Rsk_out,
                        int64_t* swaps_out) {
    *k_out = 0;
    if (swaps_out) *swaps_out = 0;
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (ldm < m) return -4;
    if (!(gamma >= 1.0)) return -5;
    int64_t d = oracle_sketch_dim(n, gamma);
    if (d > m) return -5;
    if (nnz < 1 || nnz > d) return -6;
    if (!(f > 1.0)) return -10;
    if (ldq < m) return -11;
    if (ldr < n) return -13;
    double scale = 1.0 / sqrt((double)nnz);
    double* Msk = (double*)malloc(sizeof(double) * (size_t)(d * n));
    int st = oracle_sketch(m, n, M, ldm, d, nnz, seed, scale, Msk, d);
    if (st == 0)
        st = core_ex(m, n, M, ldm, Msk, d, tol, Q, ldq, R, ldr, J, k_out, Rsk_out, NULL, NULL,
                     NULL, 1, f, swaps_out);
    free(Msk);
    return st;
}

/* Alg. 2 with a dense sketching operator S (d x m, ld lds) given by the
 * caller (Sec. 2.3.1's Gaussian family, or any operator of the family F that
 * Alg. 1 takes as a parameter): line 1 by oracle_sketch_dense, then lines 2-8
 * as oracle_cqrrpt.  Returns 0, -i for invalid argument i, 1 when k == 0, 2
 * for a non-finite sketch. */
int oracle_cqrrpt_dense(int64_t m, int64_t n, const double* M, int64_t ldm, int64_t d,
                        const double* S, int64_t lds, double tol, double* Q, int64_t ldq,
                        double* R, int64_t ldr, int64_t* J, int64_t* k_out, double* Rsk_out,
                        double* Rpre_out, double* pivnorm, double* second) {
    *k_out = 0;
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (ldm < m) return -4;
    if (d < n || d > m) return -5;
    if (lds < d) return -7;
    if (ldq < m) return -10;
    if (ldr < n) return -12;
    double* Msk = (double*)malloc(sizeof(double) * (size_t)(d * n));
    int st = oracle_sketch_dense(m, n, d, S, lds, M, ldm, Msk, d);
    if (st == 0)
        st = oracle_cqrrpt_core_sketched(m, n, M, ldm, Msk, d, tol, Q, ldq, R, ldr, J, k_out,
                                         Rsk_out, Rpre_out, pivnorm, second);
    free(Msk);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Implicit Q (Sec. 2.1: Q_k = M^pre (R^pre)^{-1}, Alg. 2 line 7 not formed): */
/* trans == 0: Y (m x r) = Q X with X k x r:                                  */
/*     W = (R^pre)^{-1} X by back substitution (row j: terms t = k-1 down to  */
/*     j+1, one fma each, then one division), Y = M^pre W in ascending t     */
/*     from +0.0, one fma per term;                                           */
/* trans == 1: Y (k x r) = Q^T X with X m x r:                                */
/*     Z = (M^pre)^T X as a blocked sum over the rows (ROW_BLOCK blocks,     */
/*     ascending rows inside from +0.0, blocks added in ascending order from */
/*     +0.0), then Y = (R^pre)^{-T} Z by forward substitution (row j: terms   */
/*     t = 0 up to j-1, one fma each, then one division).                     */
/* ------------------------------------------------------------------------ */
void oracle_apply_q(int trans, int64_t m, int64_t k, const double* Apre, int64_t lda,
                    const double* Rpre, int64_t ldr, int64_t nrhs, const double* X, int64_t ldx,
                    double* Y, int64_t ldy) {
    double* W = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t c = 0; c < nrhs; ++c) {
        const double* x = X + c * ldx;
        double* y = Y + c * ldy;
        if (trans == 0) {
            for (int64_t j = k - 1; j >= 0; --j) {
                double s = x[j];
                for (int64_t t = k - 1; t > j; --t) s = fma(-Rpre[j + t * ldr], W[t], s);
                W[j] = s / Rpre[j + j * ldr];
            }
            for (int64_t i = 0; i < m; ++i) {
                double s = 0.0;
                for (int64_t t = 0; t < k; ++t) s = fma(Apre[i + t * lda], W[t], s);
                y[i] = s;
            }
        } else {
            for (int64_t t = 0; t < k; ++t) {
                const double* a = Apre + t * lda;
                double total = 0.0;
                for (int64_t r0 = 0; r0 < m; r0 += ROW_BLOCK) {
                    int64_t r1 = r0 + ROW_BLOCK < m ? r0 + ROW_BLOCK : m;
                    double part = 0.0;
                    for (int64_t r = r0; r < r1; ++r) part = fma(a[r], x[r], part);
                    total = total + part;
                }
                W[t] = total;
            }
            for (int64_t j = 0; j < k; ++j) {
                double s = W[j];
                for (int64_t t = 0; t < j; ++t) s = fma(-Rpre[t + j * ldr], y[t], s);
                y[j] = s / Rpre[j + j * ldr];
            }
        }
    }
    free(W);
}

/* ------------------------------------------------------------------------ */
/* Sec. 1.3: randomized CholeskyQR (the method CQRRPT extends) -- sketch,    */
/* unpivoted QR of the sketch, M^pre = M (R^sk)^{-1}, G, R^pre = chol(G),   */
/* Q = M^pre (R^pre)^{-1}, R = R^pre R^sk.  M must have full column rank:  */
/* k = n, except that an exactly zero diagonal of R^sk (below DBL_MIN times */
/* R^sk[0,0]) ends k there and a Cholesky breakdown lowers k (Remark 4).    */
/* J is the identity.  Returns as oracle_cqrrpt.                            */
/* ------------------------------------------------------------------------ */
int oracle_rcholqr(int64_t m, int64_t n, const double* M, int64_t ldm, double gamma, int nnz,
                   uint64_t seed, double* Q, int64_t ldq, double* R, int64_t ldr, int64_t* J,
                   int64_t* k_out, double* Rsk_out, double* Rpre_out) {
    *k_out = 0;
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (ldm < m) return -4;
    if (!(gamma >= 1.0)) return -5;
    int64_t d = oracle_sketch_dim(n, gamma);
    if (d > m) return -5;
    if (nnz < 1 || nnz > d) return -6;
    if (ldq < m) return -10;
    if (ldr < n) return -12;
    double scale = 1.0 / sqrt((double)nnz);
    double* Msk = (double*)malloc(sizeof(double) * (size_t)(d * n));
    int st = oracle_sketch(m, n, M, ldm, d, nnz, seed, scale, Msk, d);
    if (st == 0)
        st = core_ex(m, n, M, ldm, Msk, d, DBL_MIN, Q, ldq, R, ldr, J, k_out, Rsk_out, Rpre_out,
                     NULL, NULL, 0, 0.0, NULL);
    free(Msk);
    return st;
}
