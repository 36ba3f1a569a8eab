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
  const __nv_bfloat16* A;  // planes [8][Kpad/a_kblk][M][a_kblk] ([8][M][Kpad] unblocked)
  int64_t a_plane;
  const __nv_bfloat16* B;  // planes [8][Kpad/b_kblk][N][b_kblk]
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
  int64_t a_kblk;     // K extent of one plane block of A (0: Kpad, unblocked)
  int64_t b_kblk;     // the same for B
};

// tcgen05 engine (ozaki_tc.cu)
cudaError_t oz_gemm_tc_launch(const OzGemm& G, cudaStream_t s);
// bound (ns) of the tensor-core engine's pipeline waits on the current
// device; 0 restores the default (test hook of the timeout path)
cudaError_t oz_set_wait_ns(unsigned long long ns);
cudaError_t oz_gemm_launch(const OzGemm& G, cudaStream_t s);
// many products in one launch: jobs, their two TMA maps each (A, B; 64-byte
// aligned CUtensorMap objects in device memory) and the CTA prefix table
// (job j owns CTAs [base[j], base[j + 1])).
int64_t oz_gemm_tiles(const OzGemm& G);
bool oz_gemm_valid(const OzGemm& G);
bool oz_gemm_encode_maps(const OzGemm& G, void* maps_host /* 2 CUtensorMap */);
constexpr size_t kOzMapBytes = 128;  // sizeof(CUtensorMap)
cudaError_t oz_gemm_tc_batched_launch(const OzGemm* jobs, const void* maps, const int64_t* base,
                                      int njobs, int64_t total_tiles, cudaStream_t s);

// Operand splits and the small helper steps, as jobs so that one body serves
// a single launch and a batched launch over many problems.
struct OzRowSplit {   // row operand: digit planes of X[r, map[k]], K = cols
  const double* X;
  int64_t ldx;
  const int64_t* map;  // column map or null (identity)
  int64_t rows;
  int cols;
  int64_t kpad;
  int* e;              // rows exponents (written)
  __nv_bfloat16* D;    // planes [8][rows][kpad]
  int64_t plane;
};
struct OzColSplit {   // column operand: digit planes of X[k, c], K = rows
  const double* X;
  int64_t ldx;
  int64_t rows;
  int cols;
  int64_t kpad;
  int* e;              // cols exponents (written)
  __nv_bfloat16* D;    // planes [8][kpad/kblk][cols][kblk]
  int64_t plane;
  int64_t kblk;        // 0 (= kpad: planes [8][cols][kpad]) or kOzChunk
};
struct OzTrinv {      // W = T^{-1}, row by row
  const double* T;
  int64_t ldt;
  int k;
  double* W;
  int64_t ldw;
};
struct OzCombine {    // G = sum of the K-slice partials, mirrored
  const double* P;
  int64_t slice;
  int nslices;
  int n;
  double* G;
  int64_t ldg;
};
int64_t oz_rowexp_tiles(const OzRowSplit& J);
int64_t oz_splitrows_tiles(const OzRowSplit& J);
int64_t oz_colexp_tiles(const OzColSplit& J);
int64_t oz_splitcols_tiles(const OzColSplit& J);
int oz_trinv_warps(int kmax);
// one CTA per row of W (every k of a batch at most kmax): then a job's tiles
// are its k rows (oz_trinv_tiles with warps = 1)
bool oz_trinv_row_mode(int kmax);
int64_t oz_trinv_tiles(const OzTrinv& J, int warps);
int64_t oz_combine_tiles(const OzCombine& J);
cudaError_t oz_rowsplit_batched(const OzRowSplit* jobs, const int64_t* base_exp,
                                int64_t tiles_exp, const int64_t* base_split,
                                int64_t tiles_split, int njobs, cudaStream_t s);
cudaError_t oz_colsplit_batched(const OzColSplit* jobs, const int64_t* base_exp,
                                int64_t tiles_exp, const int64_t* base_split,
                                int64_t tiles_split, int njobs, cudaStream_t s);
cudaError_t oz_trinv_batched(const OzTrinv* jobs, const int64_t* base, int64_t tiles, int njobs,
                             int warps, int kmax, cudaStream_t s);
cudaError_t oz_combine_batched(const OzCombine* jobs, const int64_t* base, int64_t tiles,
                               int njobs, cudaStream_t s);
// number of K slices the Gram of an m x k matrix uses (as oz_gram)
int64_t oz_gram_slices(int64_t m, int k);
int64_t oz_gram_workspace(int64_t m, int k, int64_t* nslices_out);
cudaError_t oz_gram(int64_t m, int k, const double* X, int64_t ldx, double* G, int64_t ldg,
                    void* work, cudaStream_t s, int* status = nullptr);
// C = X^T Y (ka x kb, ld ldc) from X (m x ka) and Y (m x kb), column-major:
// the Gram's K-sliced split-BF16 product with two operands (all tiles).
int64_t oz_gemm_tn_workspace(int64_t m, int ka, int kb, int64_t* nslices_out);
cudaError_t oz_gemm_tn(int64_t m, int ka, int kb, const double* X, int64_t ldx, const double* Y,
                       int64_t ldy, double* C, int64_t ldc, void* work, cudaStream_t s,
                       int* status = nullptr);
int64_t oz_trsm_workspace(int64_t m, int k);
// X := B[:, cols] T^{-1} through the FP64 (row-wise) inverse of T.  side
// (or null): a second stream and two events on which T^{-1} is formed while
// B[:, cols] is split on s (joined before the product).
struct OzSide {
  cudaStream_t stream;
  cudaEvent_t fork, join;
};
int64_t oz_trsm_inv_workspace(int64_t m, int k);
cudaError_t oz_trsm_inv(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                        const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                        cudaStream_t s, int* status = nullptr, const OzSide* side = nullptr);
cudaError_t oz_trsm(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                    const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                    cudaStream_t s, int* status = nullptr);

}  // namespace cqrrpt
