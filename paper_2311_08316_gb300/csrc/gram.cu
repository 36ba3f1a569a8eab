// Alg. 2 line 5: the Gram matrix G = (M^pre)^T M^pre (k x k, the SYRK of
// the CholeskyQR step, Sec. 2.1).
//
// The sum over the m rows is blocked: for each row block b of kRowBlock rows
// gram_partial_kernel forms P_b[a, c] = sum_{r in b} X[r, a] X[r, c] in
// ascending r with one fma per term (a <= c); gram_combine_kernel then adds
// the blocks in ascending order, G[a, c] = ((P_0 + P_1) + P_2) + ..., and
// mirrors the upper triangle.  One CTA computes one kGramTile x kGramTile
// output tile of one row block; each of its 64 threads owns a 4 x 4
// register tile, and rows are staged kGramRows at a time in shared memory.
// The kernel is bound by the FP64 pipe.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

int64_t gram_workspace_bytes(int64_t m, int64_t n) {
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  return align256(nb * n * n * 8);
}

__global__ void __launch_bounds__(64) gram_partial_kernel(int64_t m, int n_ld,
                                                          const int64_t* __restrict__ k_dev,
                                                          const double* __restrict__ X, int64_t ldx,
                                                          double* partial,
                                                          const int* __restrict__ status) {
  __shared__ double Xa[kGramTile][kGramRows + 1];  // [col][row]
  __shared__ double Xc[kGramTile][kGramRows + 1];
  if (*status != kOk) return;
  const int k = (int)*k_dev;
  // tile index -> (ta, tc) with ta <= tc
  const int tiles_1d = (k + kGramTile - 1) / kGramTile;
  int t = blockIdx.x, ta = 0;
  while (ta < tiles_1d && t >= tiles_1d - ta) { t -= tiles_1d - ta; ++ta; }
  if (ta >= tiles_1d) return;
  const int tc = ta + t;
  const int64_t b = blockIdx.y;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, m - r0);
  if (rows <= 0) return;
  const int a0 = ta * kGramTile, c0 = tc * kGramTile;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

  for (int rr0 = 0; rr0 < rows; rr0 += kGramRows) {
    const int nr = min(kGramRows, rows - rr0);
    __syncthreads();
    for (int e = threadIdx.x; e < kGramTile * kGramRows; e += 64) {
      const int col = e / kGramRows, row = e % kGramRows;
      const int64_t r = r0 + rr0 + row;
      const bool rok = row < nr;
      Xa[col][row] = (rok && a0 + col < k) ? X[(int64_t)(a0 + col) * ldx + r] : 0.0;
      Xc[col][row] = (rok && c0 + col < k) ? X[(int64_t)(c0 + col) * ldx + r] : 0.0;
    }
    __syncthreads();
    for (int row = 0; row < nr; ++row) {
      double va[4], vc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) va[u] = Xa[ty * 4 + u][row];
#pragma unroll
      for (int v = 0; v < 4; ++v) vc[v] = Xc[tx * 4 + v][row];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = __fma_rn(va[u], vc[v], acc[u][v]);
    }
  }
  double* P = partial + b * (int64_t)n_ld * n_ld;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int a = a0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (a < k && c < k && a <= c) P[(int64_t)c * n_ld + a] = acc[u][v];
    }
}

__global__ void gram_combine_kernel(int64_t nblocks, int n_ld, const int64_t* __restrict__ k_dev,
                                    const double* __restrict__ partial, double* G, int64_t ldg,
                                    const int* __restrict__ status) {
  if (*status != kOk) return;
  const int k = (int)*k_dev;
  const int64_t total = (int64_t)k * k;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / k), a = (int)(idx - (int64_t)c * k);
    if (a > c) continue;
    const int64_t off = (int64_t)c * n_ld + a;
    double tsum = 0.0;
    for (int64_t b = 0; b < nblocks; ++b)
      tsum = __dadd_rn(tsum, partial[b * (int64_t)n_ld * n_ld + off]);
    G[(int64_t)c * ldg + a] = tsum;
    G[(int64_t)a * ldg + c] = tsum;
  }
}

cudaError_t launch_gram(int64_t m, int kmax, const int64_t* k_dev, const double* X, int64_t ldx,
                        double* G, int64_t ldg, void* work, const int* status,
                        cudaStream_t stream) {
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  const int t1 = (kmax + kGramTile - 1) / kGramTile;
  const int tiles = t1 * (t1 + 1) / 2;
  double* partial = (double*)work;
  dim3 grid((unsigned)tiles, (unsigned)nb);
  gram_partial_kernel<<<grid, 64, 0, stream>>>(m, kmax, k_dev, X, ldx, partial, status);
  const int64_t total = (int64_t)kmax * kmax;
  const unsigned cgrid = (unsigned)min64((total + 255) / 256, 152 * 16);
  gram_combine_kernel<<<cgrid, 256, 0, stream>>>(nb, kmax, k_dev, partial, G, ldg, status);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace cqrrpt
