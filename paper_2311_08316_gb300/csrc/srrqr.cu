// Sec. 2.2: strong rank-revealing QR of the sketch at rank k (Gu and
// Eisenstat 1996, tuning parameter f > 1; the paper names f = 2), applied
// after the rank rule of line 3 to R^sk = [A B; 0 C] (A the leading k x k
// block) and J.
//
// One exchange step:
//   srrqr_inv      W = A^{-1}, one warp per column c, column-oriented
//                  back substitution: x = e_c; for t = c down to 0,
//                  x_t = x_t / A[t,t], then x_i = fma(-A[i,t], x_t, x_i), i < t;
//   srrqr_norms    w2_i = sum_{t=i..k-1} W[i,t]^2, g2_j = ||C[:, j]||^2;
//   srrqr_rho      one thread per pair (i < k <= k+j):
//                  ab = sum_{t=i..k-1} W[i,t] R[t,k+j],
//                  rho_ij = fma(ab, ab, g2_j w2_i), and the block's largest;
//   srrqr_reduce   the largest rho_ij (lowest i, then lowest j, on ties);
// every sum in ascending index order with one fma per term, so rho and the
// decision are those of the oracle bit for bit.  The host reads the winner;
// if rho_ij > f^2, srrqr_swap exchanges columns i and k+j of R (into a
// scratch copy) and in J, and the unpivoted QRCP kernels refactor it into
// R^sk (same reflectors and sign convention as line 2).  Each exchange
// multiplies |det A| by sqrt(rho_ij) > f, so the loop ends; a cap bounds it.
// The work is O(k^2 (n-k)) per step on a k x n triangle: small next to
// lines 4-7, and most inputs need no exchange at f = 2 (one step, one host
// wait).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

constexpr int kSrThreads = 256;

// One warp per column c of W (up to kInvWarps columns per CTA, each column
// in shared memory), column-oriented back substitution: x = e_c; for t = c
// down to 0, x_t = x_t / A[t,t], then x_i = fma(-A[i,t], x_t, x_i) for all
// i < t, the lanes splitting the i (column t of A is contiguous).  Each x_i
// takes its terms in descending t, as the oracle does; c steps per column.
constexpr int kInvWarps = 8;
__global__ void __launch_bounds__(kInvWarps * 32) srrqr_inv_kernel(int k, const double* R,
                                                                   int64_t ldr, double* W) {
  extern __shared__ double inv_cols[];  // [warps][k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (int)(blockDim.x >> 5) + warp;
  if (c >= k) return;
  double* x = inv_cols + (int64_t)warp * k;
  for (int i = lane; i <= c; i += 32) x[i] = i == c ? 1.0 : 0.0;
  __syncwarp();
  for (int t = c; t >= 0; --t) {
    const double* col = R + (int64_t)t * ldr;
    if (lane == 0) x[t] = __ddiv_rn(x[t], col[t]);
    __syncwarp();
    const double xt = x[t];
    for (int i = lane; i < t; i += 32) x[i] = __fma_rn(-col[i], xt, x[i]);
    __syncwarp();
  }
  double* out = W + (int64_t)c * k;
  for (int i = lane; i < k; i += 32) out[i] = i <= c ? x[i] : 0.0;
}

__global__ void __launch_bounds__(kSrThreads) srrqr_norms_kernel(int n, int k, const double* W,
                                                                 const double* R, int64_t ldr,
                                                                 double* w2, double* g2) {
  const int x = blockIdx.x * kSrThreads + threadIdx.x;
  if (x < k) {
    double s = 0.0;
    for (int t = x; t < k; ++t) {
      const double v = W[(int64_t)t * k + x];
      s = __fma_rn(v, v, s);
    }
    w2[x] = s;
  } else if (x < n) {
    const int j = x - k;
    const double* col = R + (int64_t)x * ldr;
    double s = 0.0;
    for (int t = k; t <= x; ++t) s = __fma_rn(col[t], col[t], s);
    g2[j] = s;
  }
}

// candidate a beats b: larger rho, then lower i, then lower j (rho never NaN
// here: a NaN rho loses every comparison and is never taken)
__device__ __forceinline__ bool sr_better(double ra, int ia, int ja, double rb, int ib, int jb) {
  return ra > rb || (ra == rb && (ia < ib || (ia == ib && ja < jb)));
}

// grid (ceil(k / kSrThreads), n - k): thread i of column j of (A^{-1} B)
__global__ void __launch_bounds__(kSrThreads) srrqr_rho_kernel(int n, int k, const double* W,
                                                               const double* R, int64_t ldr,
                                                               const double* w2,
                                                               const double* g2,
                                                               double* blk_rho, int* blk_ij) {
  __shared__ double s_rho[kSrThreads];
  __shared__ int s_i[kSrThreads], s_j[kSrThreads];
  const int i = blockIdx.x * kSrThreads + threadIdx.x;
  const int j = blockIdx.y;
  double rho = -1.0;
  int bi = 0x7fffffff, bj = 0x7fffffff;
  if (i < k) {
    const double* col = R + (int64_t)(k + j) * ldr;
    double ab = 0.0;
    for (int t = i; t < k; ++t) ab = __fma_rn(W[(int64_t)t * k + i], col[t], ab);
    const double r = __fma_rn(ab, ab, __dmul_rn(g2[j], w2[i]));
    if (r > rho) { rho = r; bi = i; bj = j; }
  }
  s_rho[threadIdx.x] = rho;
  s_i[threadIdx.x] = bi;
  s_j[threadIdx.x] = bj;
  __syncthreads();
  for (int off = kSrThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const int o = threadIdx.x + off;
      if (sr_better(s_rho[o], s_i[o], s_j[o], s_rho[threadIdx.x], s_i[threadIdx.x],
                    s_j[threadIdx.x])) {
        s_rho[threadIdx.x] = s_rho[o];
        s_i[threadIdx.x] = s_i[o];
        s_j[threadIdx.x] = s_j[o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    blk_rho[b] = s_rho[0];
    blk_ij[2 * b] = s_i[0];
    blk_ij[2 * b + 1] = s_j[0];
  }
}

// one block: the best of nblk block results -> out (rho, then i, j and the
// factorisation's status as doubles, 32 bytes)
__global__ void __launch_bounds__(kSrThreads) srrqr_reduce_kernel(int64_t nblk,
                                                                  const double* blk_rho,
                                                                  const int* blk_ij,
                                                                  const DeviceScalars* sc,
                                                                  double* out) {
  __shared__ double s_rho[kSrThreads];
  __shared__ int s_i[kSrThreads], s_j[kSrThreads];
  double rho = -1.0;
  int bi = 0x7fffffff, bj = 0x7fffffff;
  for (int64_t b = threadIdx.x; b < nblk; b += kSrThreads)
    if (sr_better(blk_rho[b], blk_ij[2 * b], blk_ij[2 * b + 1], rho, bi, bj)) {
      rho = blk_rho[b];
      bi = blk_ij[2 * b];
      bj = blk_ij[2 * b + 1];
    }
  s_rho[threadIdx.x] = rho;
  s_i[threadIdx.x] = bi;
  s_j[threadIdx.x] = bj;
  __syncthreads();
  for (int off = kSrThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const int o = threadIdx.x + off;
      if (sr_better(s_rho[o], s_i[o], s_j[o], s_rho[threadIdx.x], s_i[threadIdx.x],
                    s_j[threadIdx.x])) {
        s_rho[threadIdx.x] = s_rho[o];
        s_i[threadIdx.x] = s_i[o];
        s_j[threadIdx.x] = s_j[o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_rho[0];
    out[1] = (double)s_i[0];
    out[2] = (double)s_j[0];
    out[3] = (double)sc->status;
  }
}

// X = R with columns a and b exchanged (n x n, ld n); J[a] <-> J[b]
__global__ void __launch_bounds__(kSrThreads) srrqr_swap_kernel(int n, const double* R,
                                                                int64_t ldr, int a, int b,
                                                                double* X, int64_t* J) {
  const int64_t idx = (int64_t)blockIdx.x * kSrThreads + threadIdx.x;
  if (idx < (int64_t)n * n) {
    const int c = (int)(idx / n), r = (int)(idx - (int64_t)c * n);
    const int src = c == a ? b : (c == b ? a : c);
    X[idx] = R[(int64_t)src * ldr + r];
  }
  if (idx == 0) {
    const int64_t t = J[a];
    J[a] = J[b];
    J[b] = t;
  }
}

static int64_t rho_blocks(int n, int k) {
  return (int64_t)((k + kSrThreads - 1) / kSrThreads) * (n - k);
}
// at least rho_blocks(n, k) for every 0 < k < n
static int64_t rho_blocks_max(int n) { return (int64_t)n * (n / kSrThreads + 1); }

int64_t srrqr_workspace_bytes(int n) {
  const int64_t nn = (int64_t)n * n;
  return align256(nn * 8) * 2 + align256((int64_t)n * 8) * 2 +
         align256(rho_blocks_max(n) * 8) * 2 + align256((int64_t)n * 8) + 256;
}

cudaError_t srrqr_exchange(int n, int k, double f, double* Rsk, int64_t ldr, int64_t* J,
                           void* work, void* qrcp_work, DeviceScalars* sc, int num_sms,
                           double* best_host, int64_t max_swaps, int64_t* swaps_out,
                           cudaStream_t stream) {
  *swaps_out = 0;
  if (k <= 0 || k >= n) return cudaSuccess;
  const int64_t nn = (int64_t)n * n;
  char* w = (char*)work;
  double* W = (double*)w; w += align256(nn * 8);
  double* X = (double*)w; w += align256(nn * 8);
  double* w2 = (double*)w; w += align256((int64_t)n * 8);
  double* g2 = (double*)w; w += align256((int64_t)n * 8);
  double* blk_rho = (double*)w; w += align256(rho_blocks_max(n) * 8);
  int* blk_ij = (int*)w; w += align256(rho_blocks_max(n) * 8);
  int64_t* Jtmp = (int64_t*)w; w += align256((int64_t)n * 8);
  double* best_dev = (double*)w;
  const unsigned gk = (unsigned)((k + kSrThreads - 1) / kSrThreads);
  // warps per CTA: as many columns as fit in 200 KB of shared memory, 1..8
  const int inv_warps = (int)std::max<int64_t>(1, std::min<int64_t>(kInvWarps,
                                                                     (200 << 10) / (8ll * k)));
  const unsigned ginv = (unsigned)((k + inv_warps - 1) / inv_warps);
  const size_t inv_smem = (size_t)inv_warps * k * 8;
  cudaError_t e = cudaSuccess;
  if (inv_smem > 48 * 1024)
    e = raise_smem_limit((const void*)srrqr_inv_kernel, inv_smem);
  if (e != cudaSuccess) return e;
  const unsigned gn = (unsigned)((n + kSrThreads - 1) / kSrThreads);
  const dim3 grho(gk, (unsigned)(n - k));
  const double f2 = f * f;
  for (int64_t s = 0; s < max_swaps; ++s) {
    srrqr_inv_kernel<<<ginv, inv_warps * 32, inv_smem, stream>>>(k, Rsk, ldr, W);
    srrqr_norms_kernel<<<gn, kSrThreads, 0, stream>>>(n, k, W, Rsk, ldr, w2, g2);
    srrqr_rho_kernel<<<grho, kSrThreads, 0, stream>>>(n, k, W, Rsk, ldr, w2, g2, blk_rho, blk_ij);
    srrqr_reduce_kernel<<<1, kSrThreads, 0, stream>>>(rho_blocks(n, k), blk_rho, blk_ij, sc,
                                                      best_dev);
    count_launches(4);
    e = cudaMemcpyAsync(best_host, best_dev, 32, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (best_host[3] != (double)kOk) break;  // the status stands; later kernels skip
    if (!(best_host[0] > f2)) break;
    const int bi = (int)best_host[1], bj = (int)best_host[2];
    if (bi < 0 || bi >= k || bj < 0 || bj >= n - k) return cudaErrorUnknown;
    srrqr_swap_kernel<<<(unsigned)((nn + kSrThreads - 1) / kSrThreads), kSrThreads, 0, stream>>>(
        n, Rsk, ldr, bi, k + bj, X, J);
    count_launches(1);
    e = launch_qrcp(n, n, X, n, Jtmp, Rsk, ldr, qrcp_work, sc, num_sms, stream, true);
    if (e != cudaSuccess) return e;
    ++*swaps_out;
  }
  return cudaGetLastError();
}

}  // namespace cqrrpt
