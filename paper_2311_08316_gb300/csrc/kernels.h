// Internal launch interface between the C-ABI layer (api.cu) and the kernel
// translation units.  Every launcher enqueues on `stream`, never
// synchronises, and returns the launch error (cudaSuccess if none).
// Ranks and status words live in device memory so that a whole
// factorisation can be enqueued without a host round trip.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cqrrpt {

constexpr int kSkCols = 4;        // sketch: columns per CTA
constexpr int kSkThreads = 512;   // sketch: threads per CTA
constexpr int kQrcpThreads = 256;
constexpr int kTrsmThreads = 128;
constexpr int kTrsmJB = 16;       // TRSM: columns solved per register block
constexpr int kTrsmTB = 64;       // TRSM: rows of T staged per chunk
constexpr int kGramTile = 32;     // SYRK: output tile edge
constexpr int kGramRows = 32;     // SYRK: rows staged per chunk
constexpr int kCholNB = 32;       // Cholesky panel width

inline int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Device scalars of one factorisation.
struct DeviceScalars {
  int64_t k;         // current rank (rank rule, then Remark 3, then stage 2)
  int64_t fail;      // Cholesky failure column or -1
  int status;        // kOk / kNonFinite / kTimeout ...
  int pad;
  GridBarrier bar;
};

// ---- Alg. 2 line 1 -------------------------------------------------------
int64_t sketch_workspace_bytes(int64_t m, int64_t n, int d, int s);
cudaError_t launch_sketch(int64_t m, int64_t n, const double* M, int64_t ldm, int d, int s,
                          uint64_t seed, double scale, double* Msk, int64_t ldsk, void* work,
                          int* status, cudaStream_t stream);

// ---- Alg. 2 line 2 -------------------------------------------------------
int64_t qrcp_workspace_bytes(int64_t n);
// X (d x n, ld ldx) is overwritten; J (n, int64) receives the pivots;
// Rsk (n x n, ld ldr) receives the sign-normalised upper triangle.
cudaError_t launch_qrcp(int d, int n, double* X, int64_t ldx, int64_t* J, double* Rsk,
                        int64_t ldr, void* work, DeviceScalars* sc, int num_sms,
                        cudaStream_t stream);

// ---- Alg. 2 line 3 -------------------------------------------------------
// tol > 0: leading count of R_jj > tol R_00; tol <= 0: stage 1.
// f2: n + 1 doubles of scratch.
cudaError_t launch_rank(int n, const double* Rsk, int64_t ldr, double tol, DeviceScalars* sc,
                        double* f2, cudaStream_t stream);
// stage 2 on R^pre after the Cholesky (k := min(k, fail) first).
cudaError_t launch_rank_stage2(const double* Rpre, int64_t ldp, bool stage2, DeviceScalars* sc,
                               cudaStream_t stream);

// ---- Alg. 2 lines 4 and 7 ------------------------------------------------
// X[:, 0:k] = B[:, cols[0:k]] * T^{-1}; cols may be null (identity); X may
// alias B when cols is null.  k read from *k_dev; kmax bounds the grid.
cudaError_t launch_trsm_rut(int64_t m, int kmax, const int64_t* k_dev, const double* B,
                            int64_t ldb, const int64_t* cols, const double* T, int64_t ldt,
                            double* X, int64_t ldx, const int* status, cudaStream_t stream);

// ---- Alg. 2 line 5 -------------------------------------------------------
int64_t gram_workspace_bytes(int64_t m, int64_t n);
cudaError_t launch_gram(int64_t m, int kmax, const int64_t* k_dev, const double* X, int64_t ldx,
                        double* G, int64_t ldg, void* work, const int* status,
                        cudaStream_t stream);

// ---- Alg. 2 line 6 -------------------------------------------------------
// Factors G (overwritten as working storage) into R (upper); on a
// non-positive pivot at column j records sc->fail = j (Remark 3).
cudaError_t launch_potrf(int kmax, double* G, int64_t ldg, double* R, int64_t ldr,
                         DeviceScalars* sc, cudaStream_t stream);

// ---- Alg. 2 line 8 -------------------------------------------------------
cudaError_t launch_trmm(int n, const int64_t* k_dev, const double* Rpre, int64_t ldp,
                        const double* Rsk, int64_t ldsk, double* R, int64_t ldr,
                        const int* status, cudaStream_t stream);

// ---- small helpers -------------------------------------------------------
// Process-wide count of kernels this library has launched.
void count_launches(int n);
cudaError_t launch_init_scalars(DeviceScalars* sc, int64_t k, cudaStream_t stream);
cudaError_t launch_finalize(DeviceScalars* sc, int64_t* k_out, int* status_out,
                            cudaStream_t stream);

}  // namespace cqrrpt
