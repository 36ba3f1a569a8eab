// Alg. 2 lines 4 and 7: X = B[:, cols] T^{-1} with T upper triangular
// (k x k), by row-wise substitution:
//   X[i, j] = (B[i, cols[j]] - sum_{t<j} X[i, t] T[t, j]) / T[j, j],
// the sum in ascending t with one fma per term.  Line 4 uses the pivot
// gather cols = J[0:k] and T = R^sk_11 (M^pre = M_k (A^sk_k)^{-1}); line 7
// runs in place with cols = identity and T = R^pre (Q_k = M^pre (R^pre)^{-1}).
//
// One thread owns one row i.  Columns are solved in register blocks of
// kTrsmJB columns (16 where a batched problem's descriptor asks for it; the
// batched autotuner picks the width per problem size), the last k mod that
// width in blocks of 16, 8, 4, 2, 1.  A block's partial sums are seeded
// with B, then receive the terms t < j0 chunk by chunk (kTrsmTB rows of T
// staged in shared memory, X[i, t] re-read from the thread's own, already
// solved row), then the triangular part of the block in ascending t.  Every
// partial sum therefore receives its terms in ascending t, so the result
// does not depend on the blocking.  The kernel is bound by the FP64 pipe
// (one DFMA per term).
//
// The single-problem kernel and the batched kernel (one launch over many
// independent problems; CTA -> (problem, row tile) through a prefix table)
// share the same body.
#include "batch.cuh"
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

// Columns j0 .. j0 + JB - 1 of the thread's row i (all of them exist);
// THREADS threads per CTA.
template <int JB, int THREADS>
__device__ __forceinline__ void trsm_rut_block(int j0, int64_t i, bool active, double* Ts,
                                               double* Td, const TrsmDesc& D) {
  const double* B = D.B;
  const int64_t* cols = D.cols;
  const double* T = D.T;
  double* X = D.X;
  const int64_t ldb = D.ldb, ldt = D.ldt, ldx = D.ldx;
  double s[JB];
#pragma unroll
  for (int jj = 0; jj < JB; ++jj) {
    s[jj] = 0.0;
    if (active) {
      const int64_t bc = cols ? cols[j0 + jj] : (int64_t)(j0 + jj);
      s[jj] = B[bc * ldb + i];
    }
  }
  // terms t < j0
  for (int t0 = 0; t0 < j0; t0 += kTrsmTB) {
    const int tb = min(kTrsmTB, j0 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < tb * JB; e += THREADS) {
      const int tt = e / JB, jj = e % JB;
      Ts[tt * JB + jj] = T[(int64_t)(j0 + jj) * ldt + (t0 + tt)];
    }
    __syncthreads();
    if (active) {
      for (int tt = 0; tt < tb; ++tt) {
        const double x = -X[(int64_t)(t0 + tt) * ldx + i];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) s[jj] = __fma_rn(x, Ts[tt * JB + jj], s[jj]);
      }
    }
  }
  // triangular block
  __syncthreads();
  for (int e = threadIdx.x; e < JB * JB; e += THREADS) {
    const int tt = e / JB, jj = e % JB;
    Td[tt * JB + jj] = T[(int64_t)(j0 + jj) * ldt + (j0 + tt)];
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      const double x = __ddiv_rn(s[jj], Td[jj * JB + jj]);
      X[(int64_t)(j0 + jj) * ldx + i] = x;
      const double nx = -x;
#pragma unroll
      for (int j2 = jj + 1; j2 < JB; ++j2) s[j2] = __fma_rn(nx, Td[jj * JB + j2], s[j2]);
    }
  }
}

// Blocks of JBMAX columns, then the remainder k mod JBMAX as blocks of
// halving width (16, 8, 4, 2, 1), so no block computes a column that does not
// exist.
// Ts (kTrsmTB x kTrsmJB) and Td (kTrsmJB x kTrsmJB): shared staging.
template <int JBMAX, int THREADS = kTrsmThreads>
__device__ __forceinline__ void trsm_rut_body(int64_t tile, const TrsmDesc& D, double* Ts,
                                              double* Td) {
  static_assert(JBMAX == 16 || JBMAX == 32, "column block of 16 or 32");
  if (*D.status != kOk) return;
  const int k = (int)*D.k_dev;
  const int64_t i = tile * (int64_t)THREADS + threadIdx.x;
  const bool active = i < D.m;
  int j0 = 0;
  for (; j0 + JBMAX <= k; j0 += JBMAX) trsm_rut_block<JBMAX, THREADS>(j0, i, active, Ts, Td, D);
  if (JBMAX > 16 && k - j0 >= 16) {
    trsm_rut_block<16, THREADS>(j0, i, active, Ts, Td, D);
    j0 += 16;
  }
  if (k - j0 >= 8) { trsm_rut_block<8, THREADS>(j0, i, active, Ts, Td, D); j0 += 8; }
  if (k - j0 >= 4) { trsm_rut_block<4, THREADS>(j0, i, active, Ts, Td, D); j0 += 4; }
  if (k - j0 >= 2) { trsm_rut_block<2, THREADS>(j0, i, active, Ts, Td, D); j0 += 2; }
  if (k - j0 >= 1) trsm_rut_block<1, THREADS>(j0, i, active, Ts, Td, D);
}

__global__ void __launch_bounds__(kTrsmThreads) trsm_rut_kernel(TrsmDesc D) {
  __shared__ double Ts[kTrsmTB * kTrsmJB];
  __shared__ double Td[kTrsmJB * kTrsmJB];
  trsm_rut_body<kTrsmJB>(blockIdx.x, D, Ts, Td);
}

// Small m: four lanes per row.  A warp owns 8 rows; lane 4 r + g holds, for
// row r, the partial sums of the block's columns j with j mod 4 = g.  The
// terms t < j0 arrive as in trsm_rut_block (each lane re-reads the row's
// solved X[i, t]); in the triangular part the owner of column j divides and
// passes x_j to the row's other three lanes by a width-4 shuffle, and each
// updates its later columns.  Every partial sum receives the same terms in
// ascending t with one fma each, then the same division: the bits of
// trsm_rut_kernel.  A warp issues a quarter of the fmas per row, and a row's
// work spreads over four lanes of more warps (a single warp issues one FP64
// instruction per 64 cycles on this part).
constexpr int kTrsmSplitThreads = 128;  // 32 rows per CTA
template <int JB>
__device__ __forceinline__ void trsm_split_block(int j0, int64_t i, bool active, int g,
                                                 double* Ts, double* Td, const TrsmDesc& D) {
  constexpr int NJ = (JB + 3) / 4;  // columns per lane (JB >= 4), one for JB < 4
  const double* B = D.B;
  const int64_t* cols = D.cols;
  const double* T = D.T;
  double* X = D.X;
  const int64_t ldb = D.ldb, ldt = D.ldt, ldx = D.ldx;
  double s[NJ];
#pragma unroll
  for (int u = 0; u < NJ; ++u) {
    const int jj = u * 4 + g;
    s[u] = 0.0;
    if (active && jj < JB) {
      const int64_t bc = cols ? cols[j0 + jj] : (int64_t)(j0 + jj);
      s[u] = B[bc * ldb + i];
    }
  }
  for (int t0 = 0; t0 < j0; t0 += kTrsmTB) {
    const int tb = min(kTrsmTB, j0 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < tb * JB; e += kTrsmSplitThreads) {
      const int tt = e / JB, jj = e % JB;
      Ts[tt * JB + jj] = T[(int64_t)(j0 + jj) * ldt + (t0 + tt)];
    }
    __syncthreads();
    if (active) {
      for (int tt = 0; tt < tb; ++tt) {
        const double x = -X[(int64_t)(t0 + tt) * ldx + i];
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
          const int jj = u * 4 + g;
          if (jj < JB) s[u] = __fma_rn(x, Ts[tt * JB + jj], s[u]);
        }
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < JB * JB; e += kTrsmSplitThreads) {
    const int tt = e / JB, jj = e % JB;
    Td[tt * JB + jj] = T[(int64_t)(j0 + jj) * ldt + (j0 + tt)];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int jj = 0; jj < JB; ++jj) {
    const int owner = jj & 3;
    double x = 0.0;
    if (g == owner && active) {
      x = __ddiv_rn(s[jj >> 2], Td[jj * JB + jj]);
      X[(int64_t)(j0 + jj) * ldx + i] = x;
    }
    x = __shfl_sync(0xffffffffu, x, (lane & ~3) | owner);
    const double nx = -x;
#pragma unroll
    for (int u = 0; u < NJ; ++u) {
      const int j2 = u * 4 + g;
      if (j2 > jj && j2 < JB) s[u] = __fma_rn(nx, Td[jj * JB + j2], s[u]);
    }
  }
}

__global__ void __launch_bounds__(kTrsmSplitThreads) trsm_rut_small_kernel(TrsmDesc D) {
  __shared__ double Ts[kTrsmTB * kTrsmJB];
  __shared__ double Td[kTrsmJB * kTrsmJB];
  if (*D.status != kOk) return;
  const int k = (int)*D.k_dev;
  const int g = threadIdx.x & 3;
  const int64_t i = (int64_t)blockIdx.x * (kTrsmSplitThreads / 4) + (threadIdx.x >> 2);
  const bool active = i < D.m;
  int j0 = 0;
  for (; j0 + 32 <= k; j0 += 32) trsm_split_block<32>(j0, i, active, g, Ts, Td, D);
  if (k - j0 >= 16) { trsm_split_block<16>(j0, i, active, g, Ts, Td, D); j0 += 16; }
  if (k - j0 >= 8) { trsm_split_block<8>(j0, i, active, g, Ts, Td, D); j0 += 8; }
  if (k - j0 >= 4) { trsm_split_block<4>(j0, i, active, g, Ts, Td, D); j0 += 4; }
  if (k - j0 >= 2) { trsm_split_block<2>(j0, i, active, g, Ts, Td, D); j0 += 2; }
  if (k - j0 >= 1) trsm_split_block<1>(j0, i, active, g, Ts, Td, D);
}

__global__ void __launch_bounds__(kTrsmThreads) trsm_rut_batched_kernel(const TrsmDesc* D,
                                                                         const int64_t* base,
                                                                         int nprob) {
  int64_t local;
  __shared__ double Ts[kTrsmTB * kTrsmJB];
  __shared__ double Td[kTrsmJB * kTrsmJB];
  const int p = find_problem(base, nprob, blockIdx.x, &local);
  if (D[p].jb == 16)
    trsm_rut_body<16>(local, D[p], Ts, Td);
  else
    trsm_rut_body<32>(local, D[p], Ts, Td);
}

int64_t trsm_tiles(int64_t m) { return (m + kTrsmThreads - 1) / kTrsmThreads; }

cudaError_t launch_trsm_rut(int64_t m, int kmax, const int64_t* k_dev, const double* B,
                            int64_t ldb, const int64_t* cols, const double* T, int64_t ldt,
                            double* X, int64_t ldx, const int* status, cudaStream_t stream) {
  (void)kmax;
  TrsmDesc D{m, k_dev, B, ldb, cols, T, ldt, X, ldx, status, kTrsmJB};
  if (trsm_tiles(m) < 152) {  // less than one CTA per SM at 128 rows per CTA
    const int64_t rows_per_cta = kTrsmSplitThreads / 4;
    trsm_rut_small_kernel<<<(unsigned)((m + rows_per_cta - 1) / rows_per_cta),
                            kTrsmSplitThreads, 0, stream>>>(D);
  } else {
    trsm_rut_kernel<<<(unsigned)trsm_tiles(m), kTrsmThreads, 0, stream>>>(D);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trsm_rut_batched(const TrsmDesc* D_dev, const int64_t* base_dev, int nprob,
                                    int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  trsm_rut_batched_kernel<<<(unsigned)total_tiles, kTrsmThreads, 0, stream>>>(D_dev, base_dev,
                                                                             nprob);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
