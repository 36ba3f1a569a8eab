/*
 * cqrrpt.h -- C ABI of the GB300 (sm_103a) CQRRPT library.
 *
 * CQRRPT ("CholeskyQR with Randomization and Pivoting for Tall matrices",
 * Melnichenko, Balabanov, Murray, Demmel, Mahoney, Luszczek; arXiv
 * 2311.08316) computes a column-pivoted QR decomposition M[:, J] = Q_k R_k
 * of a tall m x n matrix M (Def. 1 of the paper, Sec. 1.6.2):
 *   Alg. 1: d = ceil(gamma n), sample a d x m sketching operator S;
 *   Alg. 2: M^sk = S M; [Q^sk, R^sk, J] = qrcp(M^sk); k = rank(R^sk);
 *           M^pre = M[:, J[:k]] (R^sk[:k,:k])^{-1}; G = M^pre^T M^pre;
 *           R^pre = chol(G); Q_k = M^pre (R^pre)^{-1}; R_k = R^pre R^sk[:k,:].
 *
 * Conventions for every entry point:
 *   - matrices are FP64, column-major (LAPACK layout), with a leading
 *     dimension argument; indices are 0-based (the paper's are 1-based);
 *   - every matrix/vector pointer is a DEVICE pointer unless the argument
 *     name ends in _host; the caller owns every buffer it passes; the
 *     library only reads A and writes the outputs it is given;
 *   - calls are enqueued on `stream` and return without waiting, unless a
 *     _host output pointer is given, in which case the call waits for the
 *     stream and returns the final status;
 *   - a handle owns the library's device workspace and device status words;
 *     it is not thread safe: use one handle per concurrently used stream;
 *   - argument errors are returned immediately as -i (argument i, counting
 *     the handle as argument 1), nothing is enqueued;
 *   - results do not depend on the launch configuration: the arithmetic
 *     order of every sum is fixed (see the library's design notes), so the
 *     same inputs give bit-identical outputs on every call.
 *
 * The sketching operator is the SASO of Sec. 2.3.1: each of the m columns of
 * S has exactly nnz_per_col nonzeros at distinct uniformly random rows, each
 * +-1/sqrt(nnz_per_col); S is generated on the fly from `seed` by the
 * counter-based Philox4x32-10 generator and never stored.
 */
#ifndef CQRRPT_H
#define CQRRPT_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (>= 0); negative values -i flag argument i. */
#define CQRRPT_OK 0
#define CQRRPT_RANK_ZERO 1   /* k == 0: M is numerically zero; J is valid  */
#define CQRRPT_NONFINITE 2   /* the sketch of M holds Inf/NaN; k = 0       */
#define CQRRPT_CUDA_ERROR 3  /* a CUDA call or launch failed              */
#define CQRRPT_NO_MEMORY 4   /* workspace allocation failed               */
#define CQRRPT_TIMEOUT 5     /* a bounded device-side wait expired        */
#define CQRRPT_TOO_LARGE 6   /* problem exceeds the fixed scratch of
                                cqrrpt_sketch_noalloc_d                  */

/* Precision of the O(m n^2) steps (Alg. 2 lines 4, 5 and 7).  In every
 * mode the sketch, the QRCP of the sketch, the rank rule, the Cholesky and
 * R = R^pre R^sk run in FP64, so J and k are the same in all modes.
 *   CQRRPT_FP64       FP64 FMA, fixed summation order: bit-identical to the
 *                     library's documented arithmetic on every call.
 *   CQRRPT_SPLITBF16  lines 4, 5, 7 on the BF16 tensor cores through an
 *                     error-free split of every operand into eight 7-bit
 *                     digits (56 bits), exact FP32 accumulation of chunks of
 *                     1024 terms, exact 64-bit integer combination of the
 *                     digit levels, two FP64 roundings per entry: FP64-level
 *                     accuracy, not bit-identical to CQRRPT_FP64.
 *   CQRRPT_SPLITBF16_CHOLQR2  as CQRRPT_SPLITBF16, followed by a second
 *                     Cholesky-QR pass on Q (G2 = Q^T Q, R2 = chol(G2),
 *                     Q := Q R2^{-1}, R := R2 R) in the same arithmetic. */
#define CQRRPT_FP64 0
#define CQRRPT_SPLITBF16 2
#define CQRRPT_SPLITBF16_CHOLQR2 3

typedef struct cqrrpt_ctx* cqrrpt_handle;

/* Create a handle bound to CUDA device `device` (made current for the
 * call).  Returns 0 or CQRRPT_CUDA_ERROR. */
int cqrrpt_create(cqrrpt_handle* h, int device);

/* Release the handle and its workspace (waits for the device). */
int cqrrpt_destroy(cqrrpt_handle h);

/* Workspace bytes cqrrpt_d needs for an m x n problem. */
int cqrrpt_workspace_size(int64_t m, int64_t n, double gamma, int nnz_per_col, int precision,
                          size_t* bytes_host);

/* Grow the handle's workspace to at least `bytes` now (a later call that
 * fits allocates nothing).  Returns 0 or CQRRPT_NO_MEMORY. */
int cqrrpt_reserve(cqrrpt_handle h, size_t bytes);

/* Full CQRRPT, Alg. 1 + Alg. 2 (the paper's cqrrpt(M, gamma, F) with F the
 * SASO family; defaults gamma = 1.25, nnz_per_col = 4, Sec. 5.1).
 *   m, n          M is m x n, n <= ceil(gamma n) = d <= m, n <= 16384.
 *   A, lda        M (read only), lda >= m.
 *   gamma         sampling factor >= 1 (Alg. 1).
 *   nnz_per_col   nonzeros per column of S, 1 <= nnz_per_col <= min(d, 32).
 *   tol           rank rule (Alg. 2 line 3, Sec. 3.3): tol > 0 keeps the
 *                 leading columns with R^sk[j,j] > tol R^sk[0,0];
 *                 tol <= 0 runs the paper's two-stage estimate (stage 1:
 *                 smallest l with ||R^sk[l:,l:]||_F <= u max|R^sk|; stage 2
 *                 after the Cholesky: largest l with
 *                 cond(diag(R^pre[:l,:l])) <= sqrt(100u/u) = 10).  In both
 *                 cases a Cholesky breakdown at column j sets k = j
 *                 (Remark 4).
 *   seed          seed of S.
 *   precision     CQRRPT_FP64, CQRRPT_SPLITBF16 or CQRRPT_SPLITBF16_CHOLQR2.
 *   Q, ldq        m x n capacity, ldq >= m; columns 0..k-1 receive Q_k
 *                 (column j of M^pre is formed there first).
 *   R, ldr        n x n capacity, ldr >= n; rows 0..k-1 receive R_k, upper
 *                 trapezoidal with a positive diagonal.
 *   J             n int64 entries: the full pivot vector, column j of
 *                 M[:, J] is column J[j] of M.
 *   k_dev         device int64 or NULL: receives k.
 *   k_host        host int64 or NULL: if given, the call waits for the
 *                 stream, stores k and returns the final status.
 * Without k_host the return value covers argument and launch errors only;
 * device-detected conditions (CQRRPT_RANK_ZERO, CQRRPT_NONFINITE,
 * CQRRPT_TIMEOUT) are then read with cqrrpt_last_status. */
int cqrrpt_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda, double gamma,
             int nnz_per_col, double tol, uint64_t seed, int precision, double* Q, int64_t ldq,
             double* R, int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host,
             cudaStream_t stream);

/* ---- randomized CholeskyQR (Sec. 1.3) ------------------------------------ */

/* The method CQRRPT extends, in FP64: M^sk = S M (the same SASO S),
 * [Q^sk, R^sk] = qr(M^sk) WITHOUT pivoting (the QRCP's reflectors, every
 * pivot the next column), M^pre = M (R^sk)^{-1}, G = M^pre^T M^pre,
 * R^pre = chol(G), Q = M^pre (R^pre)^{-1}, R = R^pre R^sk.  M must have full
 * column rank: k = n, except that an exactly zero diagonal of R^sk ends k
 * there and a Cholesky breakdown lowers k (Remark 4).  J receives the
 * identity.  Arguments and errors as cqrrpt_d (no tol, no precision). */
int cqrrpt_rcholqr_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                     double gamma, int nnz_per_col, uint64_t seed, double* Q, int64_t ldq,
                     double* R, int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host,
                     cudaStream_t stream);

/* ---- strong rank-revealing pivots ----------------------------------------- */

/* Alg. 1 in FP64 with a strong rank-revealing QR of the sketch (Sec. 2.2:
 * Gu and Eisenstat's algorithm, tuning parameter f; the paper names f = 2).
 * Lines 1-3 as cqrrpt_d; then, with A = R^sk[:k, :k], B = R^sk[:k, k:],
 * C = R^sk[k:, k:], while some i < k <= j has
 *     rho_ij = (A^{-1} B)_{i, j-k}^2 + ||C[:, j-k]||^2 ||row i of A^{-1}||^2 > f^2,
 * the pair with the largest rho_ij (lowest i, then j, on ties) is
 * exchanged in J and R^sk, and R^sk is refactored by an unpivoted
 * Householder QR (at most 64 n exchanges); then lines 4-8 at the same k.
 * Afterwards |(A^{-1} B)_{ij}| <= f and ||C[:, j]|| / omega_i(A) <= f.
 * The host waits for k after line 3 and once per exchange step.
 *   f           tuning parameter, f > 1 (argument 10).
 *   swaps_host  host int64 or NULL: the number of exchanges (argument 18).
 * Other arguments, outputs and errors as cqrrpt_d (FP64; argument numbers
 * from Q on shift by one: Q is 11). */
int cqrrpt_srrqr_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                   double gamma, int nnz_per_col, double tol, uint64_t seed, double f, double* Q,
                   int64_t ldq, double* R, int64_t ldr, int64_t* J, int64_t* k_dev,
                   int64_t* k_host, int64_t* swaps_host, cudaStream_t stream);

/* ---- row panels of a host-resident matrix --------------------------------- */

/* The row-partitioned form of Alg. 2 (Sec. 2.1 notes that the sketch and the
 * Gram matrix are sums over row blocks, so rows can be split among
 * processors with one reduction each) run on one GPU over row panels of a
 * host-resident M that need not fit in device memory.  Panels of
 * panel_rows rows are streamed through two device slots (copy-in, compute
 * and copy-out on three streams):
 *   pass 1: line 1 per panel; each panel's 4096-row block sums continue the
 *           sketch's ascending block sum (the reduction); then lines 2-3;
 *   pass 2: lines 4-5 per panel; M^pre is parked in Q_host's first k
 *           columns and its Gram blocks continue G's ascending block sum;
 *           then line 6;
 *   pass 3: line 7 per panel, in place on the parked M^pre; then line 8.
 * Because panel_rows is a multiple of 4096, every sum keeps cqrrpt_d's
 * order: Q, R, J and k equal cqrrpt_d's (FP64) bit for bit.  Device memory:
 * 4 panel_rows n 8 bytes plus one panel_rows-row workspace.  Host traffic:
 * M read twice, M^pre written and read once, Q written once.  The host
 * waits for k after line 3 and after line 6.  Pin A_host and Q_host
 * (cudaHostRegister) for copies that overlap the kernels.
 *   A_host, lda   m x n host matrix (lda >= m), read only (arguments 4, 5).
 *   panel_rows    a positive multiple of 4096 (else -10).
 *   Q_host, ldq   m x n host capacity, ldq >= m; first k columns receive Q
 *                 (the first columns hold M^pre in between) (11, 12).
 *   R_host, ldr   n x n host capacity, ldr >= n; first k rows receive R (13, 14).
 *   J_host        n host int64 pivots (15); k_host: host int64 rank (16).
 * Other arguments as cqrrpt_d (FP64 only).  Returns 0 or a status of
 * cqrrpt_d (the call completes before returning). */
int cqrrpt_panels_host_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A_host,
                         int64_t lda, double gamma, int nnz_per_col, double tol, uint64_t seed,
                         int64_t panel_rows, double* Q_host, int64_t ldq, double* R_host,
                         int64_t ldr, int64_t* J_host, int64_t* k_host, cudaStream_t stream);

/* ---- dense sketching operators -------------------------------------------- */

/* Alg. 2 with a dense sketching operator S that the caller drew: the
 * Gaussian family of Sec. 2.3.1 (iid entries of mean 0 and variance 1/d), or
 * any other d x m operator (Alg. 1 takes the distribution F as a parameter).
 * With CQRRPT_FP64, line 1 is M^sk = S M in FP64: for each 4096-row block
 * one fma per term in ascending row order from +0.0, the blocks then added
 * in ascending order, no scaling (S carries its own); 2 d m n flops against
 * the m n s additions of a SASO.  In the split-BF16 precisions line 1 is the
 * tensor-core product of cqrrpt_sketch_dense_split_d (FP64-accurate).
 * Lines 2-8 are those of cqrrpt_d in the chosen precision.
 *   d          sketch rows, n <= d <= m and d <= 28000 (else -6).
 *   S, lds     d x m column-major device matrix, lds >= d; read only,
 *              owned by the caller (arguments 7, 8).
 *   tol        rank rule as cqrrpt_d (argument 9).
 *   precision  as cqrrpt_d (argument 10).
 *   Q ... k_host as cqrrpt_d (arguments 11-17).
 * Errors and statuses as cqrrpt_d. */
int cqrrpt_dense_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda, int64_t d,
                   const double* S, int64_t lds, double tol, int precision, double* Q,
                   int64_t ldq, double* R, int64_t ldr, int64_t* J, int64_t* k_dev,
                   int64_t* k_host, cudaStream_t stream);

/* Line 1 alone with a dense operator: Ask (d x n, ldsk >= d) = S A in the
 * sum order of cqrrpt_dense_d; S d x m (lds >= d), 1 <= d <= 65536.  A non-finite result
 * sets the handle's status (CQRRPT_NONFINITE, read by cqrrpt_last_status).
 * Uses the handle's workspace ((m/4096 + 1) n d 8 bytes); no host wait. */
int cqrrpt_sketch_dense_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                          int64_t d, const double* S, int64_t lds, double* Ask, int64_t ldsk,
                          cudaStream_t stream);

/* Line 1 with a dense operator on the BF16 tensor cores: Ask = S A as the
 * split-BF16 product (S transposed, both operands split into eight 7-bit
 * digit planes along m, 36 digit-pair products with exact FP32 sums of 1024
 * terms, exact integer combination, one rounding per K slice, the slices
 * added in ascending order).  FP64-accurate, not bit-identical to
 * cqrrpt_sketch_dense_d.  A non-finite entry of S or A sets CQRRPT_NONFINITE.
 * Arguments as cqrrpt_sketch_dense_d (n, d <= 65536).  Workspace: S^T and the
 * digit planes, about (8 + 16 (d + n)) m bytes. */
int cqrrpt_sketch_dense_split_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A,
                                int64_t lda, int64_t d, const double* S, int64_t lds, double* Ask,
                                int64_t ldsk, cudaStream_t stream);

/* ---- implicit Q --------------------------------------------------------- */

/* Alg. 1 in FP64 stopped before Alg. 2 line 7: M^pre = M[:, J[:k]]
 * (R^sk_11)^{-1} (line 4) and R^pre = chol(M^pre^T M^pre) (line 6) are
 * returned instead of Q_k; together they represent Q_k = M^pre (R^pre)^{-1}
 * (Sec. 2.1), which cqrrpt_apply_q_d applies.  A client that only applies Q
 * skips the line-7 solve, one of the two O(m k^2) triangular solves.
 * J, k and R (= R^pre R^sk_k, line 8) are those of cqrrpt_d, bit for bit;
 * Apre holds column j of cqrrpt_d's M^pre.  Arguments as cqrrpt_d, plus:
 *   Apre, ldp     m x n capacity, ldp >= m; columns 0..k-1 receive M^pre.
 *   Rpre, ldrp    n x n capacity, ldrp >= n; the leading k x k upper
 *                 triangle receives R^pre. */
int cqrrpt_implicit_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                      double gamma, int nnz_per_col, double tol, uint64_t seed, double* Apre,
                      int64_t ldp, double* Rpre, int64_t ldrp, double* R, int64_t ldr, int64_t* J,
                      int64_t* k_dev, int64_t* k_host, cudaStream_t stream);

/* Y = Q X (trans 0) or Y = Q^T X (trans 1) for Q = Apre Rpre^{-1} (m x k,
 * from cqrrpt_implicit_d; k is the host value it returned):
 *   trans 0: X k x nrhs (ldx >= k), Y m x nrhs (ldy >= m):
 *            W = Rpre^{-1} X by back substitution, then Y = Apre W;
 *   trans 1: X m x nrhs (ldx >= m), Y k x nrhs (ldy >= k):
 *            Z = Apre^T X as a sum over 4096-row blocks in ascending order,
 *            then Y = Rpre^{-T} Z by forward substitution.
 * Every sum has a fixed order (documented in applyq.cu), so results repeat
 * bit for bit.  k = 0 gives Y = 0 (trans 0) or nothing (trans 1).  Device
 * pointers; uses the handle's workspace; no host wait. */
int cqrrpt_apply_q_d(cqrrpt_handle h, int trans, int64_t m, int64_t k, const double* Apre,
                     int64_t ldp, const double* Rpre, int64_t ldrp, int64_t nrhs, const double* X,
                     int64_t ldx, double* Y, int64_t ldy, cudaStream_t stream);

/* ---- many factorisations from host memory -------------------------------- */

/* `count` factorisations of m x n host-resident matrices (the same
 * `[Q,R,J] = cqrrpt(M, gamma, F)` as cqrrpt_d, one per matrix) in a
 * copy/compute pipeline: while matrix i is factored on `stream`, matrix i+1
 * is copied in on a second stream and the result of matrix i-1 is copied
 * out on a third (double-buffered device copies of A, Q, R and J owned by
 * the handle).  The call returns when every result is in host memory.
 *   count             number of matrices >= 1.
 *   A_host[i], lda    host pointers (column-major, lda >= m); pinned host
 *                     memory lets the copies run as asynchronous DMA.  The
 *                     same pointer may appear more than once.
 *   seeds[i]          host array: seed of S for matrix i.
 *   Q_host[i], ldq    host, m x n capacity; columns 0..k_i-1 receive Q.
 *   R_host[i], ldr    host, n x n capacity; rows 0..k_i-1 receive R.
 *   J_host[i]         host, n int64 entries.
 *   k_host, status_host  host arrays of count entries: k and the final
 *                     status of each factorisation (as cqrrpt_last_status).
 * Output buffers of different i may alias (results are copied out in
 * order).  gamma, nnz_per_col, tol and precision as in cqrrpt_d.  Returns
 * the first argument or launch error (negative or CQRRPT_CUDA_ERROR /
 * CQRRPT_NO_MEMORY); per-matrix device conditions are in status_host. */
int cqrrpt_host_pipeline_d(cqrrpt_handle h, int count, int64_t m, int64_t n,
                           const double* const* A_host, int64_t lda, double gamma,
                           int nnz_per_col, double tol, const uint64_t* seeds, int precision,
                           double* const* Q_host, int64_t ldq, double* const* R_host, int64_t ldr,
                           int64_t* const* J_host, int64_t* k_host, int* status_host,
                           cudaStream_t stream);

/* ---- batched CQRRPT ------------------------------------------------------ */

/* Workspace bytes cqrrpt_batched_d needs for `batch` problems (m, n: host
 * arrays of batch entries). */
int cqrrpt_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, double gamma,
                                  int nnz_per_col, size_t* bytes_host);

/* Many independent problems of uneven sizes in one batched pass: one launch
 * per phase of Alg. 2 covers every problem (the QRCP and the Cholesky give
 * one CTA to each problem), and the whole sequence is captured once into a
 * CUDA graph and replayed while the batch's launch shapes repeat.
 *   batch                       number of problems >= 1.
 *   m, n, lda, tol, seed, ldq, ldr      HOST arrays of `batch` entries.
 *   A, Q, R, J                  HOST arrays of `batch` DEVICE pointers with
 *                               the meaning and sizes of cqrrpt_d.
 *   gamma, nnz_per_col, precision      shared by all problems; precision
 *                               CQRRPT_FP64 or CQRRPT_SPLITBF16.  In
 *                               CQRRPT_SPLITBF16 the sketch, QRCP, rank rule,
 *                               Cholesky and TRMM run as batched FP64
 *                               kernels and lines 4, 5 and 7 as batched
 *                               split-BF16 products; the call then waits for
 *                               the stream twice (the products are sized by
 *                               each problem's k) and grows a second,
 *                               handle-owned workspace for the digit planes
 *                               (about 16 m k bytes per problem).
 *   k_dev, status_dev           DEVICE arrays of `batch` entries (or NULL):
 *                               each problem's k and final status.
 * Every problem's J, k, Q and R are bit-identical to cqrrpt_d on the same
 * inputs in the same precision.  In CQRRPT_FP64 the call returns after
 * enqueueing (argument errors: -i for argument i, counting the handle as
 * 1). */
int cqrrpt_batched_d(cqrrpt_handle h, int batch, const int64_t* m, const int64_t* n,
                     const double* const* A, const int64_t* lda, double gamma, int nnz_per_col,
                     const double* tol, const uint64_t* seed, int precision, double* const* Q,
                     const int64_t* ldq, double* const* R, const int64_t* ldr, int64_t* const* J,
                     int64_t* k_dev, int* status_dev, cudaStream_t stream);

/* enable = 0: cqrrpt_batched_d launches its kernels directly instead of
 * through its cached CUDA graph. */
int cqrrpt_set_batch_graphs(cqrrpt_handle h, int enable);

/* Autotuner of the batched path.  The two O(m n^2) batched kernels have
 * tile shapes chosen per problem width bucket b = min((n - 1) / 32, 15):
 * the widest register block of the substitution of Alg. 2 lines 4 and 7
 * (16 or 32 columns) and the output tile of the Gram partial sums of line 5
 * (8 x 8, 16 x 16 or 32 x 32).  This call factors the batch once with the
 * handle's current shapes, then, for every bucket present, times every shape
 * of both kernels on that bucket's problems (best of 3 launches, CUDA events),
 * stores the faster shape per bucket and kernel in the handle (every later
 * cqrrpt_batched_d and server wave on the handle uses it), and factors the
 * batch again with the chosen shapes: on return the outputs are those of
 * cqrrpt_batched_d.  The shapes change the blocking only, never the order
 * of any sum, so outputs are bit-identical whatever is chosen.  Waits for
 * the stream.
 *   arguments 1-18      as cqrrpt_batched_d (precision CQRRPT_FP64 only:
 *                       the tuned shapes are those of the FP64 kernels).
 *   times_us_host       HOST array of 64 doubles or NULL: for bucket b,
 *                       [4b + 0, 4b + 1] = TRSM time with 16 / 32 columns,
 *                       [4b + 2, 4b + 3] = Gram time with 16 / 32 tiles
 *                       (microseconds; 0 for buckets absent from the batch;
 *                       the 8 x 8 Gram time is compared but not reported).
 * Returns 0, an argument error, CQRRPT_NO_MEMORY or CQRRPT_CUDA_ERROR. */
int cqrrpt_batched_autotune(cqrrpt_handle h, int batch, const int64_t* m, const int64_t* n,
                            const double* const* A, const int64_t* lda, double gamma,
                            int nnz_per_col, const double* tol, const uint64_t* seed,
                            int precision, double* const* Q, const int64_t* ldq,
                            double* const* R, const int64_t* ldr, int64_t* const* J,
                            int64_t* k_dev, int* status_dev, double* times_us_host,
                            cudaStream_t stream);

/* The handle's batched tile shapes: HOST arrays of 16 entries (either may be
 * NULL), TRSM column block (16 or 32) and Gram tile edge (8, 16 or 32) per
 * width bucket.  set_tuning returns -2 for a TRSM block other than 16 or 32
 * and -3 for a Gram edge other than 8, 16 or 32, and then changes nothing.
 * A new handle starts with 32-column blocks, 8 x 8 Gram tiles for
 * n <= 256 and 32 x 32 above. */
int cqrrpt_batched_get_tuning(cqrrpt_handle h, int* trsm_jb_host, int* gram_tile_host);
int cqrrpt_batched_set_tuning(cqrrpt_handle h, const int* trsm_jb_host, const int* gram_tile_host);

/* ---- row-partitioned CQRRPT over ranks (Sec. 2.1, communication cost) ---- */

/* The paper's distributed form: the rows of M are split among ranks (each a
 * process with its own device and handle), each rank sketches its rows, the
 * d x n sketch is summed over the ranks, every rank factors the sketch
 * (lines 2-3, the same J and k everywhere), each rank forms M^pre and its
 * Gram contribution on its rows, the k x k Gram is summed over the ranks,
 * and every rank finishes (lines 6-8) with Q on its own rows.  The two sums
 * are the only communication: d n + k^2 words, plus their broadcast.
 *
 * Rank r holds rows [row0, row0 + rows) of M, with row0 a multiple of 4096;
 * the ranks' ranges, in rank order, tile 0 .. m-1.  Each sum is an ordered
 * scan: rank 0 starts from +0.0, rank r adds its 4096-row block sums in
 * ascending block order to the running sum it receives from rank r-1 and
 * passes it on; the last rank's sum is broadcast.  Every sum then runs in
 * exactly the order of cqrrpt_d on the whole M (blocks ascending), so J, k,
 * R and each rank's rows of Q are bit-identical to cqrrpt_d's.  The library
 * does the arithmetic; the caller moves the two buffers between ranks (any
 * transport: they are plain device arrays).
 *
 * Per rank, all calls on one handle and one stream, in this order:
 *   cqrrpt_shard_sketch_d            block sums of S M on this rank's rows
 *   cqrrpt_shard_sketch_accumulate_d acc += them (after receiving acc)
 *   cqrrpt_shard_qrcp_d              lines 1-3 on the summed sketch
 *   cqrrpt_shard_gram_d              line 4 on this rank's rows, and the
 *                                    block sums of line 5
 *   cqrrpt_shard_gram_accumulate_d   G += them (after receiving G)
 *   cqrrpt_shard_finish_d            lines 6-8
 * A phase called out of order returns -1.  The handle keeps the rank's state
 * (and A's pointer: A must stay valid until cqrrpt_shard_gram_d). */

/* Phase 1: m = rows of the whole M; rows, row0: this rank's rows; A: this
 * rank's rows x n block (column-major, lda >= rows); gamma, nnz, seed as
 * cqrrpt_d (the same on every rank).  Errors: -i for argument i (row0 not a
 * multiple of 4096 or past m: -4; d > m: -8), CQRRPT_NO_MEMORY,
 * CQRRPT_CUDA_ERROR. */
int cqrrpt_shard_sketch_d(cqrrpt_handle h, int64_t m, int64_t rows, int64_t row0, int64_t n,
                          const double* A, int64_t lda, double gamma, int nnz, uint64_t seed,
                          cudaStream_t stream);

/* Phase 2: acc (d x n, ld d, device) += this rank's block sums in ascending
 * block order.  acc must hold +0.0 everywhere on rank 0, else the running
 * sum received from the previous rank. */
int cqrrpt_shard_sketch_accumulate_d(cqrrpt_handle h, double* acc, cudaStream_t stream);

/* Phase 3: M^sk = acc / sqrt(nnz) (the complete sum, every rank the same),
 * the QRCP (line 2) and the rank rule (line 3, tol as cqrrpt_d).  J: n
 * device int64 pivots, which must stay valid until cqrrpt_shard_gram_d. */
int cqrrpt_shard_qrcp_d(cqrrpt_handle h, const double* acc, double tol, int64_t* J,
                        cudaStream_t stream);

/* Phase 4: Q[:, :k] = A[:, J[:k]] (R^sk_11)^-1 on this rank's rows (M^pre,
 * Q: rows x n capacity, ldq >= rows), then its 4096-row Gram block sums. */
int cqrrpt_shard_gram_d(cqrrpt_handle h, double* Q, int64_t ldq, cudaStream_t stream);

/* Phase 5: G (n x n, ld n, device; both triangles of the leading k x k
 * written) += this rank's Gram block sums in ascending block order.  G must
 * hold +0.0 on rank 0, else the running sum received from the previous
 * rank. */
int cqrrpt_shard_gram_accumulate_d(cqrrpt_handle h, double* G, cudaStream_t stream);

/* Phase 6: with the complete G (overwritten as working storage): R^pre =
 * chol(G) with Remark 4 and the second rank stage, Q[:, :k] = M^pre
 * (R^pre)^-1 in place on this rank's rows, R = R^pre R^sk_k (n x n
 * capacity, ldr >= n; every rank the same).  k_dev / k_host as cqrrpt_d. */
int cqrrpt_shard_finish_d(cqrrpt_handle h, double* G, double* Q, int64_t ldq, double* R,
                          int64_t ldr, int64_t* k_dev, int64_t* k_host, cudaStream_t stream);

/* ---- serving: continuous batching ---------------------------------------- */

/* One request: a host matrix and host output buffers (pinned host memory
 * makes the copies asynchronous).  All pointers are HOST pointers. */
typedef struct {
  int64_t m, n;         /* n <= ceil(gamma n) <= m                          */
  const double* A_host; /* m x n, column-major, lda >= m                     */
  int64_t lda;
  double tol;           /* rank rule as in cqrrpt_d                          */
  uint64_t seed;        /* seed of S                                         */
  int precision;        /* CQRRPT_FP64 or a CQRRPT_SPLITBF16 mode            */
  double* Q_host;       /* m x n capacity, ldq >= m (first k columns valid)  */
  int64_t ldq;
  double* R_host;       /* n x n capacity, ldr >= n (first k rows valid)     */
  int64_t ldr;
  int64_t* J_host;      /* n pivots                                          */
} cqrrpt_request;

typedef struct {
  int64_t k;
  int status;           /* as cqrrpt_d                                        */
  double latency_us;    /* submit -> results in the host buffers              */
  double queue_us;      /* submit -> admitted (device memory reserved)        */
} cqrrpt_result;

typedef struct cqrrpt_server_s* cqrrpt_server;

/* A server that factors submitted requests with continuous batching, its
 * units of work overlapping on the GPU (the paper has no serving layer; the
 * arithmetic of every unit is Alg. 1 + Alg. 2 as in cqrrpt_d).  A scheduler
 * thread admits requests in arrival order while their device footprint (A,
 * Q, R, J and, for requests of a batched route, the batched workspace) fits
 * hbm_budget_bytes (one allocation made here) and at most max_inflight are
 * in flight, and copies their inputs in while other work runs.  Work runs on
 * `lanes` lanes (1..8), each a handle, a stream and a worker thread, so that
 * up to `lanes` units are in flight at once, the oldest arrived request
 * deciding the next unit:
 *   - a request with n > 256 or in CQRRPT_SPLITBF16_CHOLQR2 runs alone
 *     through cqrrpt_d (multi-CTA QRCP) on its lane, at most lanes - 1 such
 *     units at a time (their cooperative QRCP grids run one after another on
 *     the GPU, everything else side by side);
 *   - other requests run as batched waves: one batched pass over the arrived
 *     requests of the oldest one's precision (CQRRPT_FP64 or
 *     CQRRPT_SPLITBF16).  A wave starts at once when the GPU is idle;
 *     while any unit is in flight, arrivals gather until 4 are waiting or
 *     the oldest has waited 8 ms.
 * Results are bit-identical to standalone calls of the same precision.  The
 * server owns `h` (lane 0) until cqrrpt_server_destroy; lanes 1.. get
 * handles of their own (with h's batched tile shapes).  Single-route runs
 * and the split-BF16 digit planes use the lanes' handle workspaces, outside
 * the budget.  The current device is used.  Returns 0, -i for argument i,
 * CQRRPT_NO_MEMORY or CQRRPT_CUDA_ERROR. */
int cqrrpt_server_create_lanes(cqrrpt_handle h, size_t hbm_budget_bytes, int max_inflight,
                               double gamma, int nnz_per_col, int lanes, cqrrpt_server* server);

/* cqrrpt_server_create_lanes with 3 lanes. */
int cqrrpt_server_create(cqrrpt_handle h, size_t hbm_budget_bytes, int max_inflight, double gamma,
                         int nnz_per_col, cqrrpt_server* server);

/* Non-blocking: queues the request and returns its ticket.  The request's
 * buffers must stay valid until its completion is polled.  A request whose
 * footprint exceeds the whole budget returns CQRRPT_NO_MEMORY. */
int cqrrpt_server_submit(cqrrpt_server s, const cqrrpt_request* req, uint64_t* ticket);

/* *done = 1 once the request's results are in its host buffers; then *out
 * (if not NULL) receives k, status and latencies and the ticket is retired. */
int cqrrpt_server_poll(cqrrpt_server s, uint64_t ticket, int* done, cqrrpt_result* out);

/* Waits until no request is queued or in flight (timeout_us < 0: no limit).
 * Returns CQRRPT_TIMEOUT when the limit passes first. */
int cqrrpt_server_drain(cqrrpt_server s, int64_t timeout_us);

/* Counters: units of work launched (batched waves and single-route runs),
 * requests completed, in flight, queued. */
int cqrrpt_server_stats(cqrrpt_server s, int64_t* waves, int64_t* completed, int64_t* inflight,
                        int64_t* queued);

/* The first `count` (at most 10) of: units launched, requests completed, in
 * flight, queued, lanes, the largest number of units in flight at the same
 * time so far, single-route units, batched waves, requests in batched
 * waves, units in flight now.  out: host array.  Returns 0, -1 or -2. */
int cqrrpt_server_stats_ex(cqrrpt_server s, int64_t* out, int count);

/* Finishes every queued and in-flight request, stops the scheduler and frees
 * the server's memory. */
int cqrrpt_server_destroy(cqrrpt_server s);

/* Wait for `stream` and return the device-detected status of the handle's
 * last cqrrpt_d call (0, 1, 2 or 5) in *status_host, and its k in *k_host
 * (either pointer may be NULL). */
int cqrrpt_last_status(cqrrpt_handle h, cudaStream_t stream, int* status_host, int64_t* k_host);

const char* cqrrpt_status_string(int status);

/* ---- tracing ------------------------------------------------------------ */

/* enable != 0: cqrrpt_d records a CUDA event between its phases (the
 * per-subroutine runtime breakdown of the paper's Sec. 5.2 profiling). */
int cqrrpt_set_profiling(cqrrpt_handle h, int enable);

/* Waits for the last profiled cqrrpt_d and writes the device time in ms of
 * its first `nphases` (<= 8) phases to ms_host, in this order: sketch,
 * qrcp, rank, M^pre TRSM (line 4), Gram (line 5), Cholesky + rank stage 2
 * (line 6), Q TRSM (line 7), TRMM (line 8). */
int cqrrpt_phase_times(cqrrpt_handle h, float* ms_host, int nphases);

/* Number of kernels this library has launched in this process. */
long long cqrrpt_kernel_launches(void);

/* Bounds of the device-side waits on the current device, for tests of the
 * timeout path (the paper has no counterpart).  grid_spins: polls of the
 * QRCP's grid barrier (Alg. 2 line 2, multi-CTA) before a CTA gives up;
 * tensor_wait_ns: nanoseconds an mbarrier wait of the tensor-core engine
 * (CQRRPT_SPLITBF16*) waits before it gives up.  0 restores each default
 * (2^25 polls; 2 s).  A wait that gives up records CQRRPT_TIMEOUT in the
 * call's status (read by cqrrpt_last_status or returned through k_host);
 * the kernels then leave cleanly: the engine waits, with the default bound,
 * for its copies and products in flight and releases its tensor memory, and
 * every later kernel of the call sees the status and does nothing.  The
 * next call starts from a clean state.  Process-wide per device, not tied
 * to a handle; do not change it while calls are in flight.  Returns 0, -1 /
 * -2 for a negative argument, or CQRRPT_CUDA_ERROR. */
int cqrrpt_set_wait_limits(int64_t grid_spins, int64_t tensor_wait_ns);

/* Measured FP64 fma rate of CUDA device `device` (GFLOP/s, 2 flop per fma):
 * threads running 8, 16 or 32 independent register fma chains (the same
 * flop count: 8 * iters fma per thread), 4 or 8 CTAs of 256 threads per SM;
 * each shape is launched once to warm up, then timed with CUDA events; the
 * best rate is returned.  The roofline denominator of the FP64 kernels (the
 * paper has no counterpart).  *ms_host (may be NULL) receives the best
 * shape's timed ms.  Returns 0, -2 (iters < 1), -3 (gflops_host NULL) or
 * CQRRPT_CUDA_ERROR. */
int cqrrpt_probe_fp64_gflops(int device, int iters, double* gflops_host, double* ms_host);

/* ---- single steps of Alg. 2 (same kernels as cqrrpt_d) ------------------ */

/* Line 1: M^sk = S M, S the SASO of (seed, d, nnz_per_col).  Ask: d x n,
 * ldsk >= d.  Sum order: per block of 4096 rows ascending, blocks in
 * ascending order, then one multiply by 1/sqrt(nnz_per_col). */
int cqrrpt_sketch_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                    int64_t d, int nnz_per_col, uint64_t seed, double* Ask, int64_t ldsk,
                    cudaStream_t stream);

/* The sketch S A without any allocation (a deployment variant with the same
 * result as cqrrpt_sketch_d; the paper has no counterpart).  For callers
 * that cannot allocate device memory when they sketch -- code inside a
 * pre-sized, locked memory pool, or hosts that may not create a handle
 * because a handle owns a workspace -- this computes exactly what
 * cqrrpt_sketch_d computes (same kernels, same bits) but needs no handle:
 * its scratch is one file-scope device array of 32 MiB that every GPU
 * loading this library holds until the process exits.  It calls no
 * cudaMalloc/cudaFree.  The scratch a problem needs is, with
 * nb = ceil(m / 4096) and a256(x) = x rounded up to a multiple of 256,
 *     a256(nb (d + 1) 4) + a256(nb 4096 nnz_per_col 4) + a256(nb n d 8)
 * bytes; above cqrrpt_sketch_noalloc_max_bytes() the call returns
 * CQRRPT_TOO_LARGE before any work is queued.  The first call in each CUDA
 * context of a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it with the
 * context's id (a context created again after cudaDeviceReset is looked up
 * afresh); make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents; calls whose
 * executions overlap on the GPU race on it and must not be issued.  A
 * non-finite entry of A sets the status word in the array, which
 * cqrrpt_sketch_noalloc_status reads.  Arguments as cqrrpt_sketch_d without
 * the handle (argument numbers shift by one: m is argument 1).  The device
 * is the current one. */
int cqrrpt_sketch_noalloc_d(int64_t m, int64_t n, const double* A, int64_t lda, int64_t d,
                            int nnz_per_col, uint64_t seed, double* Ask, int64_t ldsk,
                            cudaStream_t stream);

/* Largest sketch scratch (bytes) cqrrpt_sketch_noalloc_d accepts. */
size_t cqrrpt_sketch_noalloc_max_bytes(void);

/* Status of the last cqrrpt_sketch_noalloc_d queued on the current device,
 * read in stream order: copies the status word of the fixed scratch array
 * into *status_host (pageable host memory is fine) on `stream` and waits
 * for the stream.  *status_host = 0 (CQRRPT_OK) or CQRRPT_NONFINITE (A held
 * a NaN or an infinity).  Allocates nothing.  Returns 0, -2 (status_host
 * NULL) or CQRRPT_CUDA_ERROR. */
int cqrrpt_sketch_noalloc_status(cudaStream_t stream, int* status_host);

/* Line 2: QRCP of X (d x n, ldx >= d, overwritten with Householder data).
 * J: n int64 pivots; Rsk: n x n (ldr >= n) sign-normalised R^sk (diagonal
 * >= 0, zero below the diagonal). */
int cqrrpt_qrcp_d(cqrrpt_handle h, int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J,
                  double* Rsk, int64_t ldr, cudaStream_t stream);

/* Line 3 (stage 1 only when tol <= 0): rank of R^sk into the device int64
 * *k_dev. */
int cqrrpt_rank_d(cqrrpt_handle h, int64_t n, const double* Rsk, int64_t ldr, double tol,
                  int64_t* k_dev, cudaStream_t stream);

/* Lines 4 and 7: X[:, 0:k] = B[:, cols[0:k]] T^{-1}, T upper triangular
 * k x k; cols: k device int64 or NULL (identity); X may equal B when cols
 * is NULL (in-place). */
int cqrrpt_trsm_d(cqrrpt_handle h, int64_t m, int64_t k, const double* B, int64_t ldb,
                  const int64_t* cols, const double* T, int64_t ldt, double* X, int64_t ldx,
                  cudaStream_t stream);

/* Line 5: G = X^T X (k x k, both triangles), X m x k. */
int cqrrpt_gram_d(cqrrpt_handle h, int64_t m, int64_t k, const double* X, int64_t ldx, double* G,
                  int64_t ldg, cudaStream_t stream);

/* Line 6: upper Cholesky of G (k x k, overwritten as working storage) into
 * R (upper triangle written).  *fail_dev (device int64) receives -1 or the
 * first column whose pivot is not positive (Remark 4). */
int cqrrpt_potrf_d(cqrrpt_handle h, int64_t k, double* G, int64_t ldg, double* R, int64_t ldr,
                   int64_t* fail_dev, cudaStream_t stream);

/* Line 5 in the CQRRPT_SPLITBF16 arithmetic: G = X^T X (k x k) as 36 BF16
 * tensor-core products of 7-bit digit planes: exact FP32 chunk sums of 1024
 * terms, combined exactly in integers (two 64-bit groups of four levels,
 * then one 128-bit sum) and rounded once to FP64.  A bounded device wait that expires is
 * reported as CQRRPT_TIMEOUT by cqrrpt_last_status. */
int cqrrpt_gram_split_d(cqrrpt_handle h, int64_t m, int64_t k, const double* X, int64_t ldx,
                        double* G, int64_t ldg, cudaStream_t stream);

/* Lines 4 and 7 in the CQRRPT_SPLITBF16 arithmetic: X = B[:, cols] T^{-1}
 * (recursive halving; off-diagonal blocks as split-BF16 products, 32-column
 * diagonal blocks by FP64 row-wise substitution): backward stable for any
 * upper triangular T.  X may equal B when cols is NULL.  A bounded device
 * wait that expires is reported as CQRRPT_TIMEOUT by cqrrpt_last_status. */
int cqrrpt_trsm_split_d(cqrrpt_handle h, int64_t m, int64_t k, const double* B, int64_t ldb,
                        const int64_t* cols, const double* T, int64_t ldt, double* X,
                        int64_t ldx, cudaStream_t stream);

/* Line 8: R = Rpre (k x k upper) * Rsk[0:k, 0:n] (upper trapezoidal), zero
 * below the diagonal. */
int cqrrpt_trmm_d(cqrrpt_handle h, int64_t k, int64_t n, const double* Rpre, int64_t ldp,
                  const double* Rsk, int64_t ldsk, double* R, int64_t ldr, cudaStream_t stream);

/* ---- host helpers (no GPU needed) --------------------------------------- */

/* d = ceil(gamma n) (Alg. 1). */
int64_t cqrrpt_sketch_dim(int64_t n, double gamma);

/* One Philox4x32-10 block (Salmon et al., SC'11) as used for S. */
void cqrrpt_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Column r of S: rows[0..nnz) in draw order and neg[q] = 1 when nonzero q
 * is negative (nnz_per_col <= 32). */
void cqrrpt_saso_column(uint64_t seed, int64_t r, int64_t d, int nnz_per_col, int32_t* rows,
                        uint8_t* neg);

#ifdef __cplusplus
}
#endif
#endif /* CQRRPT_H */
