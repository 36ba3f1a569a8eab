// FP64-accurate products on the BF16 tensor cores by error-free digit
// splitting (see ozaki.cu).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cqrrpt {

constexpr int kOzDigits = 8;     // 7-bit digits per entry (56 bits)
constexpr int kOzLevels = 9;     // keep digit pairs with p + q <= 9
constexpr int kOzPairs = 36;     // number of such pairs
constexpr int kOzChunk = 1024;   // exact FP32 accumulation length (1024 * 127^2 < 2^24)
constexpr int kOzTrsmNB = 32;    // diagonal block size of the split-BF16 TRSM
constexpr int kOzStore = 0, kOzSub = 1;

// C[i, j] (op)= 2^(ea[i] + eb[j]) sum_{p+q<=9} 2^(-7(p+q)) sum_k A_p[i][k] B_q[j][k]
struct OzGemm {
  int64_t M;
  int N;
  int64_t Kpad;       // multiple of 32, digits beyond the true K are zero
  int64_t kslice;     // K range per CTA (multiple of 32); partial results per slice
  const __nv_bfloat16* A;  // planes [8][M][Kpad]
  int64_t a_plane;
  const __nv_bfloat16* B;  // planes [8][N][Kpad]
  int64_t b_plane;
  const int* ea;
  const int* eb;
  double* C;
  int64_t ldc;
  int64_t c_slice;    // offset between the partial results of two K slices
  int mode;           // kOzStore: C = v; kOzSub: C = C - v
  int upper_only;     // skip tiles strictly below the diagonal
  int* err;           // device status word (or null): set to CQRRPT_TIMEOUT
                      // when a bounded wait of the engine expires
};

// tcgen05 engine (ozaki_tc.cu)
cudaError_t oz_gemm_tc_launch(const OzGemm& G, cudaStream_t s);
cudaError_t oz_gemm_launch(const OzGemm& G, cudaStream_t s);
int64_t oz_gram_workspace(int64_t m, int k, int64_t* nslices_out);
cudaError_t oz_gram(int64_t m, int k, const double* X, int64_t ldx, double* G, int64_t ldg,
                    void* work, cudaStream_t s, int* status = nullptr);
int64_t oz_trsm_workspace(int64_t m, int k);
// X := B[:, cols] T^{-1} through the FP64 (row-wise) inverse of T
int64_t oz_trsm_inv_workspace(int64_t m, int k);
cudaError_t oz_trsm_inv(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                        const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                        cudaStream_t s, int* status = nullptr);
cudaError_t oz_trsm(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                    const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                    cudaStream_t s, int* status = nullptr);

}  // namespace cqrrpt
