// Alg. 2 line 6: R^pre = chol(G), upper (G = R^T R), with the failure rule
// of Remark 4 (Sec. 3.3): if the pivot of column j is not positive the
// factorisation stops, records fail = j, and the leading j x j block of R is
// the valid factor of G[0:j, 0:j].
//
// Every entry follows the unblocked recurrence
//   R[j, c] = (G[j, c] - sum_{t<j} R[t, j] R[t, c]) / R[j, j],
//   R[j, j] = sqrt(G[j, j] - sum_{t<j} R[t, j]^2),
// each sum in ascending t with one fma per term.  It is evaluated
// right-looking in panels of kCholNB columns, which keeps that order: G is
// used as working storage S and receives the terms t of earlier panels in
// ascending order (update step), the terms of the current panel are added
// by the diagonal-block and panel steps, again in ascending t.
//
// Single problem: three launches per panel (diagonal block, panel rows,
// trailing update).  Batch: one CTA per problem runs every panel with block
// barriers between the steps; same bodies, same arithmetic.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

// Diagonal block [jb, jb + nb) by one warp, lane = column.  Returns false
// (and records sc->fail) on a non-positive pivot.
__device__ __forceinline__ bool potrf_diag_body(int jb, const PotrfDesc& D) {
  __shared__ double rdiag;
  __shared__ int failed;
  DeviceScalars* sc = D.sc;
  double* S = D.G;
  double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int lane = threadIdx.x & 31;
  if (lane == 0) failed = 0;
  __syncwarp();
  for (int jj = 0; jj < nb; ++jj) {
    const int j = jb + jj;
    if (lane == 0) {
      double s = S[(int64_t)j * lds + j];
      for (int t = jb; t < j; ++t) {
        const double r = R[(int64_t)j * ldr + t];
        s = __fma_rn(-r, r, s);
      }
      if (!(s > 0.0)) {
        failed = 1;
        sc->fail = j;
      } else {
        rdiag = __dsqrt_rn(s);
        R[(int64_t)j * ldr + j] = rdiag;
      }
    }
    __syncwarp();
    if (failed) return false;
    const int c = jb + lane;
    if (lane > jj && lane < nb) {
      double s = S[(int64_t)c * lds + j];
      for (int t = jb; t < j; ++t) s = __fma_rn(-R[(int64_t)j * ldr + t], R[(int64_t)c * ldr + t], s);
      R[(int64_t)c * ldr + j] = __ddiv_rn(s, rdiag);
    }
    __syncwarp();
  }
  return true;
}

// Panel rows [jb, jb + nb) of column c >= jb + nb.
__device__ __forceinline__ void potrf_panel_col(int jb, int nb, int c, const PotrfDesc& D) {
  const double* S = D.G;
  double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  for (int jj = 0; jj < nb; ++jj) {
    const int j = jb + jj;
    double s = S[(int64_t)c * lds + j];
    for (int t = jb; t < j; ++t) s = __fma_rn(-R[(int64_t)j * ldr + t], R[(int64_t)c * ldr + t], s);
    R[(int64_t)c * ldr + j] = __ddiv_rn(s, R[(int64_t)j * ldr + j]);
  }
}

// Trailing update of S[a, c] (a <= c, both >= jb + nb) by the panel's rows.
__device__ __forceinline__ void potrf_update_elem(int jb, int base, int a, int c,
                                                  const PotrfDesc& D) {
  double* S = D.G;
  const double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  double s = S[(int64_t)c * lds + a];
  for (int t = jb; t < base; ++t) s = __fma_rn(-R[(int64_t)a * ldr + t], R[(int64_t)c * ldr + t], s);
  S[(int64_t)c * lds + a] = s;
}

// ---- single problem: one launch per step ------------------------------------
__global__ void potrf_diag_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  if (jb >= (int)sc->k) return;
  potrf_diag_body(jb, D);
}

__global__ void potrf_panel_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int c = jb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (jb >= k || c >= k) return;
  potrf_panel_col(jb, nb, c, D);
}

__global__ void potrf_update_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int base = jb + nb;
  if (jb >= k || base >= k) return;
  const int a = base + blockIdx.y * 16 + threadIdx.y;
  const int c = base + blockIdx.x * 16 + threadIdx.x;
  if (a >= k || c >= k || a > c) return;
  potrf_update_elem(jb, base, a, c, D);
}

// ---- batch: one CTA per problem -----------------------------------------------
__global__ void __launch_bounds__(256) potrf_batched_kernel(const PotrfDesc* Dv) {
  const PotrfDesc& D = Dv[blockIdx.x];
  DeviceScalars* sc = D.sc;
  __shared__ int go;
  for (int jb = 0; jb < D.kmax; jb += kCholNB) {
    if (threadIdx.x == 0)
      go = (*(volatile int*)&sc->status == kOk && *(volatile int64_t*)&sc->fail < 0 &&
            jb < (int)sc->k);
    __syncthreads();
    if (!go) return;
    const int k = (int)sc->k;
    const int nb = min(kCholNB, k - jb);
    const int base = jb + nb;
    if (threadIdx.x < 32) potrf_diag_body(jb, D);
    __syncthreads();
    if (threadIdx.x == 0) go = (*(volatile int64_t*)&sc->fail < 0);
    __syncthreads();
    if (!go) return;
    for (int c = base + threadIdx.x; c < k; c += blockDim.x) potrf_panel_col(jb, nb, c, D);
    __syncthreads();
    const int w = k - base;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int a = base + e / w, c = base + e % w;
      if (a <= c) potrf_update_elem(jb, base, a, c, D);
    }
    __syncthreads();
  }
}

cudaError_t launch_potrf(int kmax, double* G, int64_t ldg, double* R, int64_t ldr,
                         DeviceScalars* sc, cudaStream_t stream) {
  PotrfDesc D{kmax, G, ldg, R, ldr, sc};
  for (int jb = 0; jb < kmax; jb += kCholNB) {
    potrf_diag_kernel<<<1, 32, 0, stream>>>(jb, D);
    count_launches(1);
    const int rest = kmax - jb - kCholNB;
    if (rest > 0) {
      count_launches(2);
      potrf_panel_kernel<<<(rest + 127) / 128, 128, 0, stream>>>(jb, D);
      dim3 grid((rest + 15) / 16, (rest + 15) / 16);
      potrf_update_kernel<<<grid, dim3(16, 16), 0, stream>>>(jb, D);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_potrf_batched(const PotrfDesc* D, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  potrf_batched_kernel<<<nprob, 256, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
