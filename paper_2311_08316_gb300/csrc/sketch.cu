// Alg. 2 line 1: the sketch M^sk = S M with the SASO S of Sec. 3.3.1.
//
// Three kernels:
//   saso_lists_kernel     per row block (kRowBlock rows) of M, the SASO
//                         columns of that block regrouped by target row i:
//                         for each i the rows r of the block with S[i,r] != 0
//                         in ascending r, with their signs (a CSR of the
//                         block of S by target row).
//   sketch_partial_kernel per (row block b, group of kSkCols columns): stages
//                         the block of M in shared memory (coalesced), then
//                         one thread per target row i walks its list and
//                         accumulates +-M[r, c] in ascending r from +0.0,
//                         giving P_b[i, c].
//   sketch_combine_kernel M^sk[i, c] = scale * (P_0 + P_1 + ...) in
//                         ascending block order from +0.0; flags non-finite
//                         results.
// The arithmetic (FP64 additions in that order, one final scale) is fixed by
// the data, not by the launch shape.
#include "common.cuh"
#include "kernels.h"
#include "saso.cuh"

namespace cqrrpt {

// entries: (r_local << 1) | negative
__global__ void saso_lists_kernel(int64_t m, int d, int s, uint64_t seed, int* seg_start,
                                  uint32_t* entries) {
  extern __shared__ int sh_lists[];
  int* count = sh_lists;          // d
  int* start = sh_lists + d;      // d + 1
  const int64_t b = blockIdx.x;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, m - r0);
  int* gstart = seg_start + b * (int64_t)(d + 1);
  uint32_t* gent = entries + b * (int64_t)kRowBlock * s;

  for (int i = threadIdx.x; i < d; i += blockDim.x) count[i] = 0;
  __syncthreads();
  int tr[kMaxNnzInline];
  uint32_t neg;
  for (int rl = threadIdx.x; rl < rows; rl += blockDim.x) {
    saso_column(seed, r0 + rl, d, s, tr, &neg);
    for (int q = 0; q < s; ++q) atomicAdd(&count[tr[q]], 1);
  }
  __syncthreads();
  // exclusive scan of count -> start (single warp, sequential chunks)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < d; base += 32) {
      int v = (base + lane < d) ? count[base + lane] : 0;
      int x = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
      }
      if (base + lane < d) start[base + lane] = carry + x - v;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) start[d] = carry;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= d; i += blockDim.x) gstart[i] = start[i];
  for (int i = threadIdx.x; i < d; i += blockDim.x) count[i] = start[i];  // cursors
  __syncthreads();
  for (int rl = threadIdx.x; rl < rows; rl += blockDim.x) {
    saso_column(seed, r0 + rl, d, s, tr, &neg);
    for (int q = 0; q < s; ++q) {
      const int pos = atomicAdd(&count[tr[q]], 1);
      gent[pos] = ((uint32_t)rl << 1) | ((neg >> q) & 1u);
    }
  }
  __syncthreads();
  // each segment to ascending r (insertion sort; segments are short)
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const int a = start[i], e = start[i + 1];
    for (int x = a + 1; x < e; ++x) {
      const uint32_t key = gent[x];
      int y = x - 1;
      while (y >= a && gent[y] > key) {
        gent[y + 1] = gent[y];
        --y;
      }
      gent[y + 1] = key;
    }
  }
}

__global__ void __launch_bounds__(kSkThreads) sketch_partial_kernel(
    int64_t m, int64_t n, const double* __restrict__ M, int64_t ldm, int d, int s,
    const int* __restrict__ seg_start, const uint32_t* __restrict__ entries, double* partial) {
  extern __shared__ double tile[];  // [kRowBlock][kSkCols], row-major
  const int64_t b = blockIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * kSkCols;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, m - r0);
  const int ncols = (int)min64(kSkCols, n - c0);
  for (int cc = 0; cc < kSkCols; ++cc) {
    if (cc < ncols) {
      const double* col = M + (c0 + cc) * ldm + r0;
      for (int rl = threadIdx.x; rl < rows; rl += blockDim.x) tile[rl * kSkCols + cc] = col[rl];
    }
  }
  __syncthreads();
  const int* st = seg_start + b * (int64_t)(d + 1);
  const uint32_t* ent = entries + b * (int64_t)kRowBlock * s;
  double* P = partial + b * n * (int64_t)d;  // P_b: d x n, ld d
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double acc[kSkCols];
#pragma unroll
    for (int cc = 0; cc < kSkCols; ++cc) acc[cc] = 0.0;
    const int e1 = st[i + 1];
    for (int e = st[i]; e < e1; ++e) {
      const uint32_t w = ent[e];
      const double* row = tile + (w >> 1) * kSkCols;
      if (w & 1u) {
#pragma unroll
        for (int cc = 0; cc < kSkCols; ++cc) acc[cc] = __dsub_rn(acc[cc], row[cc]);
      } else {
#pragma unroll
        for (int cc = 0; cc < kSkCols; ++cc) acc[cc] = __dadd_rn(acc[cc], row[cc]);
      }
    }
    for (int cc = 0; cc < ncols; ++cc) P[(c0 + cc) * d + i] = acc[cc];
  }
}

__global__ void sketch_combine_kernel(int64_t nblocks, int64_t n, int d, double scale,
                                      const double* __restrict__ partial, double* Msk, int64_t ldsk,
                                      int* status) {
  const int64_t total = n * (int64_t)d;
  bool bad = false;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / d, i = idx - c * d;
    double t = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) t = __dadd_rn(t, partial[b * total + idx]);
    const double v = __dmul_rn(t, scale);
    Msk[c * ldsk + i] = v;
    bad |= !isfinite(v);
  }
  if (bad) atomicExch(status, kNonFinite);
}

int64_t sketch_workspace_bytes(int64_t m, int64_t n, int d, int s) {
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  int64_t bytes = 0;
  bytes += align256(nb * (int64_t)(d + 1) * 4);
  bytes += align256(nb * (int64_t)kRowBlock * s * 4);
  bytes += align256(nb * n * (int64_t)d * 8);
  return bytes;
}

cudaError_t launch_sketch(int64_t m, int64_t n, const double* M, int64_t ldm, int d, int s,
                          uint64_t seed, double scale, double* Msk, int64_t ldsk, void* work,
                          int* status, cudaStream_t stream) {
  const int64_t nb = (m + kRowBlock - 1) / kRowBlock;
  char* p = (char*)work;
  int* seg_start = (int*)p;
  p += align256(nb * (int64_t)(d + 1) * 4);
  uint32_t* entries = (uint32_t*)p;
  p += align256(nb * (int64_t)kRowBlock * s * 4);
  double* partial = (double*)p;

  const size_t sh_lists = (size_t)(2 * d + 1) * sizeof(int);
  if (sh_lists > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(saso_lists_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_lists);
    if (e != cudaSuccess) return e;
  }
  saso_lists_kernel<<<(unsigned)nb, 256, sh_lists, stream>>>(m, d, s, seed, seg_start, entries);
  const size_t sh_tile = (size_t)kRowBlock * kSkCols * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(sketch_partial_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_tile);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)nb, (unsigned)((n + kSkCols - 1) / kSkCols));
  sketch_partial_kernel<<<grid, kSkThreads, sh_tile, stream>>>(m, n, M, ldm, d, s, seg_start,
                                                                entries, partial);
  const int64_t total = n * (int64_t)d;
  const unsigned cgrid = (unsigned)min64((total + 255) / 256, 152 * 16);
  sketch_combine_kernel<<<cgrid, 256, 0, stream>>>(nb, n, d, scale, partial, Msk, ldsk, status);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace cqrrpt
