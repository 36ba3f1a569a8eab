// Measured FP64 FMA rate of the device: the denominator of the roofline of
// the FP64 kernels (every FP64 step of the method is bound by the FP64
// pipe, not by HBM).  Not part of the method.
//
// Each thread runs CHAINS independent fma chains on registers (no memory
// traffic inside the loop).  Shapes of 8, 16 and 32 chains per thread with
// 4 or 8 CTAs of 256 threads per SM are each launched twice (a warm-up,
// then a timed launch, CUDA events on a private stream); the best rate is
// reported.  flop = 2 * CHAINS * iters * threads.
#include <cuda_runtime.h>

#include "../../include/cqrrpt.h"

namespace {

constexpr int kThreads = 256;

__device__ double g_probe_sink;

template <int CHAINS>
__global__ void __launch_bounds__(kThreads) fp64_fma_probe_kernel(int iters, double seed) {
  double a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = seed + (double)(threadIdx.x + c);
  const double x = 0.999999999, y = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = __fma_rn(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  if (s == 12345.678) g_probe_sink = s;  // keeps the chains alive
}

template <int CHAINS>
cudaError_t timed(int blocks, int iters, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                  double* gflops, float* ms_out) {
  const int it = iters * 8 / CHAINS;  // the same flop count for every shape
  fp64_fma_probe_kernel<CHAINS><<<blocks, kThreads, 0, s>>>(it, 1.0);
  cudaEventRecord(e0, s);
  fp64_fma_probe_kernel<CHAINS><<<blocks, kThreads, 0, s>>>(it, 2.0);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess || ms <= 0.f) return e != cudaSuccess ? e : cudaErrorUnknown;
  *gflops = 2.0 * CHAINS * (double)it * (double)blocks * kThreads / (ms * 1e-3) / 1e9;
  *ms_out = ms;
  return cudaSuccess;
}

}  // namespace

extern "C" int cqrrpt_probe_fp64_gflops(int device, int iters, double* gflops_host,
                                        double* ms_host) {
  if (iters < 1) return -2;
  if (!gflops_host) return -3;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return CQRRPT_CUDA_ERROR;
  int sms = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CQRRPT_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = CQRRPT_CUDA_ERROR;
  } else {
    double best = 0.0, g = 0.0;
    float best_ms = 0.f, ms = 0.f;
    for (int per_sm = 4; per_sm <= 8 && rc == CQRRPT_OK; per_sm *= 2) {
      const int blocks = per_sm * sms;
      for (int shape = 0; shape < 3 && rc == CQRRPT_OK; ++shape) {
        cudaError_t e = shape == 0   ? timed<8>(blocks, iters, s, e0, e1, &g, &ms)
                        : shape == 1 ? timed<16>(blocks, iters, s, e0, e1, &g, &ms)
                                     : timed<32>(blocks, iters, s, e0, e1, &g, &ms);
        if (e != cudaSuccess) rc = CQRRPT_CUDA_ERROR;
        else if (g > best) { best = g; best_ms = ms; }
      }
    }
    if (rc == CQRRPT_OK) {
      *gflops_host = best;
      if (ms_host) *ms_host = best_ms;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
