// Alg. 2 line 6: R^pre = chol(G), upper (G = R^T R), with the failure rule
// of Remark 3 (Sec. 4.3): if the pivot of column j is not positive the
// factorisation stops, records fail = j, and the leading j x j block of R is
// the valid factor of G[0:j, 0:j].
//
// Every entry follows the unblocked recurrence
//   R[j, c] = (G[j, c] - sum_{t<j} R[t, j] R[t, c]) / R[j, j],
//   R[j, j] = sqrt(G[j, j] - sum_{t<j} R[t, j]^2),
// each sum in ascending t with one fma per term.  It is evaluated
// right-looking in panels of kCholNB columns, which keeps that order: G is
// used as working storage S and receives the terms t of earlier panels in
// ascending order (update kernel), the terms of the current panel are added
// by the diagonal-block and panel kernels, again in ascending t.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

// Diagonal block [jb, jb + nb) of the panel: one warp, lane = column.
__global__ void potrf_diag_kernel(int jb, double* S, int64_t lds, double* R, int64_t ldr,
                                  DeviceScalars* sc) {
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  if (jb >= k) return;
  const int nb = min(kCholNB, k - jb);
  const int lane = threadIdx.x;
  __shared__ double rdiag;
  __shared__ int failed;
  if (lane == 0) failed = 0;
  __syncwarp();
  for (int jj = 0; jj < nb; ++jj) {
    const int j = jb + jj;
    // column j of the block's row j: diagonal first (lane 0)
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
    if (failed) return;
    const int c = jb + lane;
    if (lane > jj && lane < nb) {
      double s = S[(int64_t)c * lds + j];
      for (int t = jb; t < j; ++t) s = __fma_rn(-R[(int64_t)j * ldr + t], R[(int64_t)c * ldr + t], s);
      R[(int64_t)c * ldr + j] = __ddiv_rn(s, rdiag);
    }
    __syncwarp();
  }
}

// Panel rows [jb, jb + nb) for columns c >= jb + nb: one thread per column.
__global__ void potrf_panel_kernel(int jb, const double* S, int64_t lds, double* R, int64_t ldr,
                                   DeviceScalars* sc) {
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int c = jb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (jb >= k || c >= k) return;
  for (int jj = 0; jj < nb; ++jj) {
    const int j = jb + jj;
    double s = S[(int64_t)c * lds + j];
    for (int t = jb; t < j; ++t) s = __fma_rn(-R[(int64_t)j * ldr + t], R[(int64_t)c * ldr + t], s);
    R[(int64_t)c * ldr + j] = __ddiv_rn(s, R[(int64_t)j * ldr + j]);
  }
}

// Trailing update: S[a, c] -= sum_{t in panel} R[t, a] R[t, c], a <= c,
// a, c >= jb + nb, in ascending t.
__global__ void potrf_update_kernel(int jb, double* S, int64_t lds, const double* R, int64_t ldr,
                                    DeviceScalars* sc) {
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int base = jb + nb;
  if (jb >= k || base >= k) return;
  const int a = base + blockIdx.y * 16 + threadIdx.y;
  const int c = base + blockIdx.x * 16 + threadIdx.x;
  if (a >= k || c >= k || a > c) return;
  double s = S[(int64_t)c * lds + a];
  for (int t = jb; t < base; ++t) s = __fma_rn(-R[(int64_t)a * ldr + t], R[(int64_t)c * ldr + t], s);
  S[(int64_t)c * lds + a] = s;
}

cudaError_t launch_potrf(int kmax, double* G, int64_t ldg, double* R, int64_t ldr,
                         DeviceScalars* sc, cudaStream_t stream) {
  for (int jb = 0; jb < kmax; jb += kCholNB) {
    potrf_diag_kernel<<<1, 32, 0, stream>>>(jb, G, ldg, R, ldr, sc);
    count_launches(1);
    const int rest = kmax - jb - kCholNB;
    if (rest > 0) {
      count_launches(2);
      potrf_panel_kernel<<<(rest + 127) / 128, 128, 0, stream>>>(jb, G, ldg, R, ldr, sc);
      dim3 grid((rest + 15) / 16, (rest + 15) / 16);
      potrf_update_kernel<<<grid, dim3(16, 16), 0, stream>>>(jb, G, ldg, R, ldr, sc);
    }
  }
  return cudaGetLastError();
}

}  // namespace cqrrpt
