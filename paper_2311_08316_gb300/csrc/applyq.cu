// The implicit Q of a factorisation stopped before Alg. 2 line 7: the
// preconditioned matrix M^pre (m x k, line 4) and R^pre (k x k, line 6)
// represent Q_k = M^pre (R^pre)^{-1} (Sec. 2.1), and Q X or Q^T Y is applied
// without forming Q (a client that only applies Q skips the line-7 TRSM,
// one of the two O(m k^2) solves).
//
//   Q X   (X k x r):  W = (R^pre)^{-1} X by back substitution, then
//                     Y = M^pre W, one thread per row, ascending t, one fma
//                     per term from +0.0;
//   Q^T Y (Y m x r):  Z = (M^pre)^T Y as a blocked sum over the rows (blocks
//                     of kRowBlock rows, ascending rows inside from +0.0,
//                     block partials added in ascending order from +0.0),
//                     then W = (R^pre)^{-T} Z by forward substitution.
//
// The substitutions run one CTA per right-hand side.  Element t of the
// right-hand side belongs to thread t mod blockDim (kept in shared memory),
// so the owner of the next pivot already holds its value: one barrier per
// step.  Element t receives its terms in the order of the steps (descending
// j for the back substitution, ascending j for the forward one), one fma
// each, then one division by the diagonal.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

namespace {

constexpr int kTrsvThreads = 256;
constexpr int kQaRows = 128;    // Q X: rows (threads) per CTA
constexpr int kQaCols = 16;     // Q X: right-hand sides per CTA (register accumulators)
constexpr int kQaChunk = 128;   // Q X: rows of W staged per chunk
constexpr int kQtTile = 32;     // Q^T Y: output tile edge in t
constexpr int kQtRows = 32;     // Q^T Y: rows staged per chunk

// Solve T w = b for every column of B (T upper k x k: back substitution),
// or T^T w = b (forward substitution; Tt = T^T, so that the column of Tt
// read in step j is contiguous).  One CTA per column.
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_cols_kernel(int lower, int k, const double* __restrict__ T, int64_t ldt,
                     const double* __restrict__ B, int64_t ldb, double* __restrict__ W,
                     int64_t ldw) {
  extern __shared__ double s[];  // k entries
  __shared__ double wslot[2];
  const int c = blockIdx.x;
  const double* b = B + (int64_t)c * ldb;
  double* w = W + (int64_t)c * ldw;
  for (int t = threadIdx.x; t < k; t += kTrsvThreads) s[t] = b[t];
  // no barrier needed: every thread only touches its own entries of s until
  // the first wslot exchange
  if (!lower) {
    for (int j = k - 1; j >= 0; --j) {
      if (threadIdx.x == j % kTrsvThreads) {
        const double x = __ddiv_rn(s[j], T[(int64_t)j * ldt + j]);
        wslot[j & 1] = x;
        w[j] = x;
      }
      __syncthreads();
      const double x = wslot[j & 1];
      const double* tc = T + (int64_t)j * ldt;  // column j of T: rows t < j
      for (int t = threadIdx.x; t < j; t += kTrsvThreads) s[t] = __fma_rn(-tc[t], x, s[t]);
    }
  } else {
    for (int j = 0; j < k; ++j) {
      if (threadIdx.x == j % kTrsvThreads) {
        const double x = __ddiv_rn(s[j], T[(int64_t)j * ldt + j]);
        wslot[j & 1] = x;
        w[j] = x;
      }
      __syncthreads();
      const double x = wslot[j & 1];
      const double* tc = T + (int64_t)j * ldt;  // column j of T^T = row j of T
      for (int t = threadIdx.x; t < k; t += kTrsvThreads)
        if (t > j) s[t] = __fma_rn(-tc[t], x, s[t]);
    }
  }
}

// Tt = T^T (k x k) through 32 x 32 shared tiles.
__global__ void transpose_kernel(int k, const double* __restrict__ T, int64_t ldt,
                                 double* __restrict__ Tt) {
  __shared__ double tl[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int j = ty; j < 32; j += 8)
    if (bx + tx < k && by + j < k) tl[j][tx] = T[(int64_t)(by + j) * ldt + bx + tx];
  __syncthreads();
  for (int j = ty; j < 32; j += 8)
    if (by + tx < k && bx + j < k) Tt[(int64_t)(bx + j) * k + by + tx] = tl[tx][j];
}

// Y[:, c0:c0+16] = A W[:, c0:c0+16]: thread = row, W staged kQaChunk rows at
// a time (broadcast reads).
__global__ void __launch_bounds__(kQaRows)
    qx_kernel(int64_t m, int k, int r, const double* __restrict__ A, int64_t lda,
              const double* __restrict__ W, int64_t ldw, double* __restrict__ Y, int64_t ldy) {
  __shared__ double Ws[kQaChunk][kQaCols];
  const int64_t i = (int64_t)blockIdx.x * kQaRows + threadIdx.x;
  const int c0 = blockIdx.y * kQaCols;
  const int nc = min(kQaCols, r - c0);
  double acc[kQaCols];
#pragma unroll
  for (int c = 0; c < kQaCols; ++c) acc[c] = 0.0;
  for (int t0 = 0; t0 < k; t0 += kQaChunk) {
    const int tn = min(kQaChunk, k - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < kQaChunk * kQaCols; e += kQaRows) {
      const int t = e / kQaCols, c = e % kQaCols;
      Ws[t][c] = (t < tn && c < nc) ? W[(int64_t)(c0 + c) * ldw + t0 + t] : 0.0;
    }
    __syncthreads();
    if (i < m) {
      for (int t = 0; t < tn; ++t) {
        const double a = A[(int64_t)(t0 + t) * lda + i];
#pragma unroll
        for (int c = 0; c < kQaCols; ++c) acc[c] = __fma_rn(a, Ws[t][c], acc[c]);
      }
    }
  }
  if (i < m)
#pragma unroll
    for (int c = 0; c < kQaCols; ++c)
      if (c < nc) Y[(int64_t)(c0 + c) * ldy + i] = acc[c];
}

// Partial P_b[t, c] = sum_{rows of block b} A[row, t] X[row, c] (ascending
// rows, one fma per term from +0.0): one CTA per (block, 32 x TC tile), 64
// threads in an 8 x 8 grid with 4 x (TC / 8) register tiles (TC = 16 when
// there are at most 16 right-hand sides).
template <int TC>
__global__ void __launch_bounds__(64)
    qt_partial_kernel(int64_t m, int k, int r, const double* __restrict__ A, int64_t lda,
                      const double* __restrict__ X, int64_t ldx, double* __restrict__ P) {
  __shared__ double As[kQtTile][kQtRows + 1];
  __shared__ double Xs[TC][kQtRows + 1];
  constexpr int RT = kQtTile / 8, RC = TC / 8;
  const int tiles_t = (k + kQtTile - 1) / kQtTile;
  const int tiles_c = (r + TC - 1) / TC;
  const int64_t b = blockIdx.x / ((int64_t)tiles_t * tiles_c);
  const int rem = (int)(blockIdx.x - b * (int64_t)tiles_t * tiles_c);
  const int t0 = (rem / tiles_c) * kQtTile, c0 = (rem % tiles_c) * TC;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, m - r0);
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc[RT][RC];
#pragma unroll
  for (int u = 0; u < RT; ++u)
#pragma unroll
    for (int v = 0; v < RC; ++v) acc[u][v] = 0.0;
  for (int rr0 = 0; rr0 < rows; rr0 += kQtRows) {
    const int nr = min(kQtRows, rows - rr0);
    __syncthreads();
    for (int e = threadIdx.x; e < kQtTile * kQtRows; e += 64) {
      const int col = e / kQtRows, row = e % kQtRows;
      const int64_t rr = r0 + rr0 + row;
      const bool rok = row < nr;
      As[col][row] = (rok && t0 + col < k) ? A[(int64_t)(t0 + col) * lda + rr] : 0.0;
      if (col < TC) Xs[col][row] = (rok && c0 + col < r) ? X[(int64_t)(c0 + col) * ldx + rr] : 0.0;
    }
    __syncthreads();
    for (int row = 0; row < nr; ++row) {
      double va[RT], vx[RC];
#pragma unroll
      for (int u = 0; u < RT; ++u) va[u] = As[ty * RT + u][row];
#pragma unroll
      for (int v = 0; v < RC; ++v) vx[v] = Xs[tx * RC + v][row];
#pragma unroll
      for (int u = 0; u < RT; ++u)
#pragma unroll
        for (int v = 0; v < RC; ++v) acc[u][v] = __fma_rn(va[u], vx[v], acc[u][v]);
    }
  }
  double* Pb = P + b * (int64_t)k * r;
#pragma unroll
  for (int u = 0; u < RT; ++u)
#pragma unroll
    for (int v = 0; v < RC; ++v) {
      const int t = t0 + ty * RT + u, c = c0 + tx * RC + v;
      if (t < k && c < r) Pb[(int64_t)c * k + t] = acc[u][v];
    }
}

// Z[t, c] = ((P_0 + P_1) + P_2) + ... (ascending blocks from +0.0).
__global__ void __launch_bounds__(kCombineThreads)
    qt_combine_kernel(int64_t nblocks, int k, int r, const double* __restrict__ P,
                      double* __restrict__ Z) {
  const int64_t idx = (int64_t)blockIdx.x * kCombineThreads + threadIdx.x;
  if (idx >= (int64_t)k * r) return;
  double s = 0.0;
  for (int64_t b = 0; b < nblocks; ++b) s = __dadd_rn(s, P[b * (int64_t)k * r + idx]);
  Z[idx] = s;
}

cudaError_t trsv_cols(int lower, int k, const double* T, int64_t ldt, const double* B,
                      int64_t ldb, double* W, int64_t ldw, int r, cudaStream_t s) {
  const size_t smem = (size_t)k * sizeof(double);
  cudaError_t e = raise_smem_limit((const void*)trsv_cols_kernel, smem);
  if (e != cudaSuccess) return e;
  trsv_cols_kernel<<<(unsigned)r, kTrsvThreads, smem, s>>>(lower, k, T, ldt, B, ldb, W, ldw);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int64_t apply_q_workspace_bytes(int trans, int64_t m, int64_t k, int64_t r) {
  const int64_t w = align256(k * r * 8);
  if (!trans) return w;
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  return w + align256(k * r * 8) + align256(nb * k * r * 8) + align256(k * k * 8);
}

cudaError_t launch_apply_q(int trans, int64_t m, int k, const double* Apre, int64_t ldp,
                           const double* Rpre, int64_t ldrp, int r, const double* X, int64_t ldx,
                           double* Y, int64_t ldy, void* work, cudaStream_t s) {
  char* w = (char*)work;
  double* W = (double*)w;
  w += align256((int64_t)k * r * 8);
  if (!trans) {
    cudaError_t e = trsv_cols(0, k, Rpre, ldrp, X, ldx, W, k, r, s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((m + kQaRows - 1) / kQaRows), (unsigned)((r + kQaCols - 1) / kQaCols));
    qx_kernel<<<grid, kQaRows, 0, s>>>(m, k, r, Apre, ldp, W, k, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
  }
  double* Z = (double*)w;
  w += align256((int64_t)k * r * 8);
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  double* P = (double*)w;
  w += align256(nb * k * r * 8);
  double* Tt = (double*)w;
  const dim3 tg((unsigned)((k + 31) / 32), (unsigned)((k + 31) / 32));
  transpose_kernel<<<tg, 256, 0, s>>>(k, Rpre, ldrp, Tt);
  const int tc = r <= 16 ? 16 : 32;
  const int64_t tiles = nb * ((k + kQtTile - 1) / kQtTile) * ((r + tc - 1) / tc);
  if (tc == 16)
    qt_partial_kernel<16><<<(unsigned)tiles, 64, 0, s>>>(m, k, r, Apre, ldp, X, ldx, P);
  else
    qt_partial_kernel<32><<<(unsigned)tiles, 64, 0, s>>>(m, k, r, Apre, ldp, X, ldx, P);
  qt_combine_kernel<<<(unsigned)(((int64_t)k * r + kCombineThreads - 1) / kCombineThreads),
                      kCombineThreads, 0, s>>>(nb, k, r, P, Z);
  count_launches(3);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // W = (R^pre)^{-T} Z straight into Y (k x r, ld ldy)
  return trsv_cols(1, k, Tt, k, Z, k, Y, ldy, r, s);
}

}  // namespace cqrrpt
