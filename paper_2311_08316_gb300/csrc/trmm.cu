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

constexpr int kTrmmThreads = 128;

int64_t trmm_tiles(int n) { return (int64_t)((n + kTrmmThreads - 1) / kTrmmThreads) * n; }

// tile -> (column c, row chunk)
__device__ __forceinline__ void trmm_body(int64_t tile, const TrmmDesc& D) {
  if (*D.status != kOk) return;
  const int n = D.n;
  const int k = (int)*D.k_dev;
  const int chunks = (n + kTrmmThreads - 1) / kTrmmThreads;
  const int c = (int)(tile / chunks);
  const int i = (int)(tile % chunks) * kTrmmThreads + threadIdx.x;
  if (i >= k || c >= n) return;
  double s = 0.0;
  if (c >= i) {
    const int tend = min(c, k - 1);
    for (int t = i; t <= tend; ++t)
      s = __fma_rn(D.Rp[(int64_t)t * D.ldp + i], D.Rs[(int64_t)c * D.lds + t], s);
  }
  D.R[(int64_t)c * D.ldr + i] = s;
}

__global__ void __launch_bounds__(kTrmmThreads) trmm_kernel(TrmmDesc D) {
  trmm_body(blockIdx.x, D);
}

__global__ void __launch_bounds__(kTrmmThreads) trmm_batched_kernel(const TrmmDesc* D,
                                                                     const int64_t* base, int np) {
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  trmm_body(t, D[p]);
}

cudaError_t launch_trmm(int n, const int64_t* k_dev, const double* Rpre, int64_t ldp,
                        const double* Rsk, int64_t ldsk, double* R, int64_t ldr,
                        const int* status, cudaStream_t stream) {
  TrmmDesc D{n, k_dev, Rpre, ldp, Rsk, ldsk, R, ldr, status};
  trmm_kernel<<<(unsigned)trmm_tiles(n), kTrmmThreads, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trmm_batched(const TrmmDesc* D, const int64_t* base, int nprob,
                                int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  trmm_batched_kernel<<<(unsigned)total_tiles, kTrmmThreads, 0, stream>>>(D, base, nprob);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
