// Alg. 2 line 8: undo the preconditioning, R_k = R^pre R^sk_k, where R^pre is
// k x k upper triangular and R^sk_k = R^sk[0:k, :] is k x n upper
// trapezoidal (a TRMM, Appendix A.1 step 4).  Entry (i, c), i <= c, is
//   sum_{t = i}^{min(c, k-1)} R^pre[i, t] R^sk[t, c]
// in ascending t with one fma per term, starting from +0.0; entries with
// c < i are set to zero so R is upper trapezoidal.  One thread per entry;
// rows >= k are not touched.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

__global__ void trmm_kernel(int n, const int64_t* __restrict__ k_dev, const double* __restrict__ Rp,
                            int64_t ldp, const double* __restrict__ Rs, int64_t lds, double* R,
                            int64_t ldr, const int* __restrict__ status) {
  if (*status != kOk) return;
  const int k = (int)*k_dev;
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k || c >= n) return;
  double s = 0.0;
  if (c >= i) {
    const int tend = min(c, k - 1);
    for (int t = i; t <= tend; ++t) s = __fma_rn(Rp[(int64_t)t * ldp + i], Rs[(int64_t)c * lds + t], s);
  }
  R[(int64_t)c * ldr + i] = s;
}

cudaError_t launch_trmm(int n, const int64_t* k_dev, const double* Rpre, int64_t ldp,
                        const double* Rsk, int64_t ldsk, double* R, int64_t ldr,
                        const int* status, cudaStream_t stream) {
  dim3 grid((unsigned)((n + 127) / 128), (unsigned)n);
  trmm_kernel<<<grid, 128, 0, stream>>>(n, k_dev, Rpre, ldp, Rsk, ldsk, R, ldr, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
