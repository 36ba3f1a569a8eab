// Shared device helpers of the CQRRPT CUDA library (sm_103a).
//
// Arithmetic conventions (the library's readings of what the paper leaves
// open; every kernel follows them so that results do not depend on launch
// shapes):
//   * sums over the tall dimension m run in row blocks of kRowBlock rows,
//     ascending inside a block from +0.0, block sums added in ascending block
//     order from +0.0;
//   * dot products inside the QRCP of the sketch are "dot32": element i goes
//     to lane i mod 32, each lane accumulates with fma from +0.0, lanes are
//     combined by the fixed tree 16, 8, 4, 2, 1;
//   * other sums (substitutions, Cholesky, triangular product) run in
//     ascending index order with one fma per term;
//   * the library is compiled with --fmad=false, so a*b+c is never fused
//     unless written as fma().
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cqrrpt {

constexpr int kRowBlock = 4096;

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Status codes shared by kernels and host (match include/cqrrpt.h).
enum : int {
  kOk = 0,
  kRankZero = 1,
  kNonFinite = 2,
  kCudaError = 3,
  kNoMemory = 4,
  kTimeout = 5,
};

// Upper bound on spin iterations of any device-side wait (with a short
// sleep per iteration this is a few seconds); on expiry the waiting CTA
// records kTimeout and leaves.
constexpr unsigned long long kSpinLimit = 1ull << 25;

__device__ __forceinline__ double warp_tree_sum32(double v) {
  // lanes l < off add lane l + off; the result ends in lane 0 and is then
  // broadcast.  The tree (16, 8, 4, 2, 1) is the dot32 combination order.
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    double o = __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) < off) v = __dadd_rn(v, o);
  }
  return __shfl_sync(0xffffffffu, v, 0);
}

// Grid-wide barrier for cooperative launches: arrival counter plus a
// generation word.  Waits are bounded: after spin_limit polls (kSpinLimit
// unless a test lowered it) the CTA sets *status = kTimeout and returns
// false.
struct GridBarrier {
  unsigned int count;
  unsigned int generation;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, int* status,
                                          unsigned long long spin_limit = kSpinLimit) {
  __shared__ int ok_flag;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (nblocks > 1) {
      volatile unsigned int* genp = &bar->generation;
      unsigned int gen = *genp;
      __threadfence();
      unsigned int arrived = atomicAdd(&bar->count, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(&bar->count, 0u);
        __threadfence();
        atomicAdd(&bar->generation, 1u);
      } else {
        unsigned long long spins = 0;
        while (*genp == gen) {
          if (++spins > spin_limit) {
            atomicExch(status, kTimeout);
            ok = 0;
            break;
          }
          if (spins > 256) __nanosleep(64);  // poll tightly first, then back off
        }
      }
      __threadfence();
    }
    ok_flag = ok;
  }
  __syncthreads();
  return ok_flag != 0;
}

}  // namespace cqrrpt

#define CQ_CHECK(expr)                                  \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return cqrrpt::kCudaError;   \
  } while (0)
