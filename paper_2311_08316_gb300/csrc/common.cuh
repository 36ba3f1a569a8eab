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
constexpr int kGramSub = 256;  // the Gram's sub-blocks inside a row block

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

// Grid-wide barrier for cooperative launches: a counter that only grows.
// Barrier b of a launch is passed once the counter reaches (b + 1) G: each
// CTA adds 1 and waits until the counter reaches the next multiple of G, so
// the last CTA to arrive releases the others by its own addition (no reset,
// no second word on the critical path).  grid_release() at the end of the
// kernel puts the counter back to 0 for the next launch; init_scalars also
// zeroes it.  Waits are bounded: after spin_limit polls (kSpinLimit unless a
// test lowered it) the CTA sets *status = kTimeout and returns false.
struct GridBarrier {
  unsigned int count;
  unsigned int released;  // CTAs past their last barrier (grid_release)
};

// One thread's side of the barrier: arrive for its CTA (after the CTA's
// writes, which a block-level barrier orders before this call) and wait.
__device__ __forceinline__ bool grid_arrive_wait(GridBarrier* bar, unsigned int nblocks,
                                                 int* status, unsigned long long spin_limit) {
  if (nblocks <= 1) return true;
  bool ok = true;
  __threadfence();  // the CTA's writes before its arrival
  const unsigned int arrived = atomicAdd(&bar->count, 1u);
  const unsigned int target = arrived - arrived % nblocks + nblocks;
  if (arrived + 1 != target) {
    volatile unsigned int* cp = &bar->count;
    unsigned long long spins = 0;
    while ((int)(*cp - target) < 0) {
      if (++spins > spin_limit) {
        atomicExch(status, kTimeout);
        ok = false;
        break;
      }
      if (spins > 256) __nanosleep(64);  // poll tightly first, then back off
    }
  }
  __threadfence();
  return ok;
}

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, int* status,
                                          unsigned long long spin_limit = kSpinLimit) {
  __shared__ int ok_flag;
  __syncthreads();
  if (threadIdx.x == 0) ok_flag = grid_arrive_wait(bar, nblocks, status, spin_limit) ? 1 : 0;
  __syncthreads();
  return ok_flag != 0;
}

// After a CTA's last grid_sync of the launch: the last CTA to get here (all
// others are past every barrier and read the counter no more) zeroes it.
__device__ __forceinline__ void grid_release(GridBarrier* bar, unsigned int nblocks) {
  if (nblocks > 1 && threadIdx.x == 0) {
    if (atomicAdd(&bar->released, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      atomicExch(&bar->released, 0u);
    }
  }
}

}  // namespace cqrrpt

#define CQ_CHECK(expr)                                  \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return cqrrpt::kCudaError;   \
  } while (0)
