// Internal launch interface between the C-ABI layer (api.cu, batched.cu) and
// the kernel translation units.  Every launcher enqueues on `stream`, never
// synchronises, and returns the launch error (cudaSuccess if none).  Ranks
// and status words live in device memory so that a whole factorisation can
// be enqueued without a host round trip.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "batch.cuh"
#include "common.cuh"

namespace cqrrpt {

constexpr int kSkCols = 2;        // sketch: columns per CTA
constexpr int kSkThreads = 1024;  // sketch: threads per CTA, at most
constexpr int kQrcpThreads = 256;
constexpr int64_t kQrcpSmemCap = 200 * 1024;  // QRCP: dynamic shared memory per CTA, at most
constexpr int kTrsmThreads = 128;
constexpr int kTrsmJB = 32;       // TRSM: columns solved per register block
constexpr int kTrsmTB = 64;       // TRSM: rows of T staged per chunk
constexpr int kGramTile = 32;     // SYRK: output tile edge
constexpr int kGramRows = 32;     // SYRK: rows staged per chunk
constexpr int kCholNB = 32;       // Cholesky panel width
constexpr int kCombineThreads = 256;

inline int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Process-wide count of kernels this library has launched.
void count_launches(int n);
// Raises (never lowers) the dynamic shared-memory limit of kernel `fn` on
// the current device to `bytes`; thread-safe.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);

// ---- Alg. 2 line 1 -------------------------------------------------------
int64_t sketch_workspace_bytes(int64_t m, int64_t n, int d, int s);
// Carves the scratch of one sketch out of `work` into D.
void sketch_carve(SketchDesc& D, void* work);
cudaError_t launch_sketch(int64_t m, int64_t n, const double* M, int64_t ldm, int d, int s,
                          uint64_t seed, double scale, double* Msk, int64_t ldsk, void* work,
                          int* status, cudaStream_t stream);
// Line 1 with a dense operator S (d x m, ld lds): M^sk = S M, one fma per
// term in ascending row order inside each kRowBlock block, blocks added in
// ascending order, no scaling.  work: sketch_dense_workspace_bytes.
int64_t sketch_dense_workspace_bytes(int64_t m, int64_t n, int d);
cudaError_t launch_sketch_dense(int64_t m, int64_t n, const double* S, int64_t lds,
                                const double* M, int64_t ldm, int d, double* Msk, int64_t ldsk,
                                void* work, int* status, cudaStream_t stream);
// Row panels of M (rows [row0, row0 + rows), row0 a multiple of kRowBlock):
// acc (d x n, ld d) += the panel's block sums in ascending block order;
// acc = +0.0 before the first panel; after the last, sketch_finish writes
// M^sk = scale * acc, bit-identical to launch_sketch on the whole M.
cudaError_t launch_sketch_panel(int64_t rows, int64_t n, const double* M, int64_t ldm, int d,
                                int s, uint64_t seed, int64_t row0, double* acc, void* work,
                                cudaStream_t stream);
cudaError_t launch_sketch_finish(int d, int64_t n, const double* acc, double scale, double* Msk,
                                 int64_t ldsk, int* status, cudaStream_t stream);
// The two halves of launch_sketch_panel: the panel's block sums into `work`,
// then acc += those sums in ascending block order (the same work carve).
cudaError_t launch_sketch_panel_partials(int64_t rows, int64_t n, const double* M, int64_t ldm,
                                         int d, int s, uint64_t seed, int64_t row0, void* work,
                                         cudaStream_t stream);
cudaError_t launch_sketch_panel_accumulate(int64_t rows, int64_t n, int d, int s, double* acc,
                                           void* work, cudaStream_t stream);
// The same product on the BF16 tensor cores (split-BF16, FP64-accurate, not
// bit-identical): S transposed, then the Gram's K-sliced product of S^T and M.
// work: sketch_dense_split_workspace_bytes.
int64_t sketch_dense_split_workspace_bytes(int64_t m, int64_t n, int d);
cudaError_t launch_sketch_dense_split(int64_t m, int64_t n, const double* S, int64_t lds,
                                      const double* M, int64_t ldm, int d, double* Msk,
                                      int64_t ldsk, void* work, int* status,
                                      cudaStream_t stream);
int64_t sketch_list_tiles(const SketchDesc& D);
int64_t sketch_partial_tiles(const SketchDesc& D);
int64_t sketch_combine_tiles(const SketchDesc& D);
// phase 0: lists, 1: partial sums, 2: combine
cudaError_t launch_sketch_batched(int phase, const SketchDesc* D, const int64_t* base, int nprob,
                                  int64_t total_tiles, int max_d, cudaStream_t stream);

// ---- Alg. 2 line 2 -------------------------------------------------------
// polls of the QRCP's grid barrier before it records kTimeout, on the
// current device; 0 restores kSpinLimit (test hook of the timeout path)
cudaError_t qrcp_set_spin_limit(unsigned long long spins);
int64_t qrcp_workspace_bytes(int64_t n);
QrcpWork qrcp_carve(void* work, int n);
// X (d x n, ld ldx) is overwritten; J (n, int64) receives the pivots;
// Rsk (n x n, ld ldr) receives the sign-normalised upper triangle.
cudaError_t launch_qrcp(int d, int n, double* X, int64_t ldx, int64_t* J, double* Rsk,
                        int64_t ldr, void* work, DeviceScalars* sc, int num_sms,
                        cudaStream_t stream, bool nopivot = false);
// one CTA per problem (no grid barrier), then the gather
// qrcp_smem_bytes > 0: one CTA per problem in shared memory (sketch columns
// that do not fit stay in global memory); 0: the global-memory kernel.
cudaError_t launch_qrcp_batched(const QrcpDesc* D, int nprob, const int64_t* gather_base,
                                int64_t gather_tiles, int64_t qrcp_smem_bytes,
                                cudaStream_t stream);

// Sec. 2.2: strong RRQR exchanges (Gu-Eisenstat, f > 1) on R^sk (n x n,
// upper triangular) and J at the host rank k, after line 3.  Loops with one
// host wait per step (best_host: 32 pinned bytes); at most max_swaps
// exchanges, counted in *swaps_out.  work: srrqr_workspace_bytes(n);
// qrcp_work: qrcp_workspace_bytes(n).
int64_t srrqr_workspace_bytes(int n);
cudaError_t srrqr_exchange(int n, int k, double f, double* Rsk, int64_t ldr, int64_t* J,
                           void* work, void* qrcp_work, DeviceScalars* sc, int num_sms,
                           double* best_host, int64_t max_swaps, int64_t* swaps_out,
                           cudaStream_t stream);

// ---- Alg. 2 line 3 -------------------------------------------------------
// tol > 0: leading count of R_jj > tol R_00; tol <= 0: stage 1.
// f2: n + 1 doubles of scratch.
cudaError_t launch_rank(int n, const double* Rsk, int64_t ldr, double tol, DeviceScalars* sc,
                        double* f2, cudaStream_t stream);
cudaError_t launch_rank_batched(const RankDesc* D, int nprob, cudaStream_t stream);
// stage 2 on R^pre after the Cholesky (k := min(k, fail) first).
cudaError_t launch_rank_stage2(const double* Rpre, int64_t ldp, bool stage2, DeviceScalars* sc,
                               cudaStream_t stream);
cudaError_t launch_rank_stage2_batched(const Stage2Desc* D, int nprob, cudaStream_t stream);

// ---- Alg. 2 lines 4 and 7 ------------------------------------------------
// X[:, 0:k] = B[:, cols[0:k]] * T^{-1}; cols may be null (identity); X may
// alias B when cols is null.  k read from *k_dev.
int64_t trsm_tiles(int64_t m);
cudaError_t launch_trsm_rut(int64_t m, int kmax, const int64_t* k_dev, const double* B,
                            int64_t ldb, const int64_t* cols, const double* T, int64_t ldt,
                            double* X, int64_t ldx, const int* status, cudaStream_t stream);
cudaError_t launch_trsm_rut_batched(const TrsmDesc* D, const int64_t* base, int nprob,
                                    int64_t total_tiles, cudaStream_t stream);

// ---- Alg. 2 line 5 -------------------------------------------------------
// Workspace of launch_gram (either form); gram_block_workspace_bytes: of
// the block-partial form alone (launch_gram_partials, the batched Gram).
int64_t gram_workspace_bytes(int64_t m, int64_t n);
int64_t gram_block_workspace_bytes(int64_t m, int64_t n);
int64_t gram_partial_tiles(int64_t m, int kmax, int tile);
int64_t gram_combine_tiles(int kmax);
// accumulate: G (both triangles) += this X's blocks, continuing G's sums
// in ascending block order (row panels; G = 0 before the first panel).
// sub_ok: `work` holds gram_workspace_bytes(m, kmax), so a small problem
// may take the sub-block partial form (same bits, shorter chains).
cudaError_t launch_gram(int64_t m, int kmax, const int64_t* k_dev, const double* X, int64_t ldx,
                        double* G, int64_t ldg, void* work, const int* status,
                        cudaStream_t stream, bool accumulate = false, bool sub_ok = false);
// The two halves of launch_gram: the block sums into `work`, then G (both
// triangles) = (accumulate: G +) their ascending sum.
cudaError_t launch_gram_partials(int64_t m, int kmax, const int64_t* k_dev, const double* X,
                                 int64_t ldx, void* work, const int* status,
                                 cudaStream_t stream);
cudaError_t launch_gram_sum(int64_t m, int kmax, const int64_t* k_dev, double* G, int64_t ldg,
                            void* work, const int* status, cudaStream_t stream, bool accumulate);
// phase 0: partial tiles, 1: combine
cudaError_t launch_gram_batched(int phase, const GramDesc* D, const int64_t* base, int nprob,
                                int64_t total_tiles, cudaStream_t stream);

// ---- Alg. 2 line 6 -------------------------------------------------------
// Factors G (overwritten as working storage) into R (upper); on a
// non-positive pivot at column j records sc->fail = j (Remark 4).
// Implicit Q = M^pre (R^pre)^{-1} (applyq.cu): Y = Q X (trans 0, X k x r,
// Y m x r) or Y = Q^T X (trans 1, X m x r, Y k x r); host k and r.
int64_t apply_q_workspace_bytes(int trans, int64_t m, int64_t k, int64_t r);
cudaError_t launch_apply_q(int trans, int64_t m, int k, const double* Apre, int64_t ldp,
                           const double* Rpre, int64_t ldrp, int r, const double* X, int64_t ldx,
                           double* Y, int64_t ldy, void* work, cudaStream_t s);

cudaError_t launch_potrf(int kmax, double* G, int64_t ldg, double* R, int64_t ldr,
                         DeviceScalars* sc, cudaStream_t stream);
// one CTA per problem runs every panel
cudaError_t launch_potrf_batched(const PotrfDesc* D, int nprob, cudaStream_t stream);

// ---- Alg. 2 line 8 -------------------------------------------------------
int64_t trmm_tiles(int n);
cudaError_t launch_trmm(int n, const int64_t* k_dev, const double* Rpre, int64_t ldp,
                        const double* Rsk, int64_t ldsk, double* R, int64_t ldr,
                        const int* status, cudaStream_t stream);
cudaError_t launch_trmm_batched(const TrmmDesc* D, const int64_t* base, int nprob,
                                int64_t total_tiles, cudaStream_t stream);

// ---- small helpers -------------------------------------------------------
cudaError_t launch_init_scalars(DeviceScalars* sc, int64_t k, cudaStream_t stream);
cudaError_t launch_init_scalars_batched(DeviceScalars* sc, int nprob, cudaStream_t stream);
cudaError_t launch_finalize(DeviceScalars* sc, int64_t* k_out, int* status_out,
                            cudaStream_t stream);
cudaError_t launch_finalize_batched(const FinalDesc* D, int nprob, cudaStream_t stream);

}  // namespace cqrrpt
