// Alg. 2 line 1: the sketch M^sk = S M with the SASO S of Sec. 2.3.1.
//
// Three kernels:
//   saso_lists     per row block (kRowBlock rows) of M, the SASO columns of
//                  that block regrouped by target row i: for each i the rows
//                  r of the block with S[i,r] != 0 in ascending r, with their
//                  signs (a CSR of the block of S by target row).
//   sketch_partial per (row block b, pair of columns): stages the block of
//                  M in shared memory (coalesced, one double2 per row; 64 KB,
//                  so that three CTAs share an SM and one stages while the
//                  others add), then one thread per target row i walks its
//                  list and accumulates +-M[r, c] in ascending r from +0.0,
//                  giving P_b[i, c].  The kernel is bound by the FP64 add
//                  pipe (m s n additions).
//   sketch_combine M^sk[i, c] = scale * (P_0 + P_1 + ...) in ascending block
//                  order from +0.0; flags non-finite results.
// The arithmetic (FP64 additions in that order, one final scale) is fixed by
// the data, not by the launch shape.  Each kernel exists as a single-problem
// launch and a batched launch (CTA -> (problem, tile)) over the same body.
//
// A dense operator S (d x m, given by the caller: Sec. 2.3.1's Gaussian
// family) replaces the first two kernels by sketch_dense_partial, which forms
// P_b[i, c] = sum_{r in b} S[i, r] M[r, c] with one fma per term in ascending
// r from +0.0; sketch_combine then adds the blocks with scale 1 (exact).
#include "common.cuh"
#include "kernels.h"
#include "ozaki.h"
#include "saso.cuh"

namespace cqrrpt {

constexpr int kListThreads = 1024;  // saso_lists: threads per CTA
constexpr int kListMapWords = kRowBlock / 32;  // one bit per row of a block
constexpr int kListSmemMax = 227 * 1024;       // dynamic shared memory per CTA, at most
// warps that sort segments: one row map and one sign map of kListMapWords
// words each per warp, as many as fit beside the counts and starts (2 d + 1
// ints; d <= 28000 leaves room for 8)
__host__ __device__ inline int lists_sort_warps(int d) {
  const int room = (kListSmemMax - (2 * d + 1) * 4) / (2 * kListMapWords * 4);
  return room < 1 ? 1 : (room > kListThreads / 32 ? kListThreads / 32 : room);
}
// dynamic shared memory of saso_lists
static size_t lists_smem_bytes(int d) {
  return (size_t)(2 * d + 1) * sizeof(int) +
         (size_t)lists_sort_warps(d) * 2 * kListMapWords * sizeof(uint32_t);
}

// seg_start of a block holds, for t < d, start[t] (the offset of target t's
// segment) in its low 17 bits and, in its high 15, the target that thread t
// of sketch_partial takes: the targets in descending order of list length, so
// that a warp's lanes walk lists of about the same length (within one length
// the order is free; every target's sum is the same whichever thread forms
// it).  seg_start[d] is the total.  Only when every start fits 17 bits and
// every target 15 (s < 32, d < 32768); otherwise the plain starts, in target
// order.
__host__ __device__ inline bool seg_packed(int d, int s) { return d < 32768 && s < 32; }
constexpr uint32_t kSegMask = (1u << 17) - 1;
constexpr int kLenBins = 128;  // list lengths of 127 and more share the last bin

// entries: (r_local << 1) | negative
__device__ __forceinline__ void saso_lists_body(int64_t b, const SketchDesc& D, int* sh_lists) {
  const int d = D.d, s = D.s;
  int* count = sh_lists;          // d
  int* start = sh_lists + d;      // d + 1
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, D.m - r0);
  int* gstart = D.seg_start + b * (int64_t)(d + 1);
  uint32_t* gent = D.entries + b * (int64_t)kRowBlock * s;

  for (int i = threadIdx.x; i < d; i += blockDim.x) count[i] = 0;
  __syncthreads();
  int tr[kMaxNnzInline];
  uint32_t neg;
  for (int rl = threadIdx.x; rl < rows; rl += blockDim.x) {
    saso_column(D.seed, D.row0 + r0 + rl, d, s, tr, &neg);
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
    saso_column(D.seed, D.row0 + r0 + rl, d, s, tr, &neg);
    for (int q = 0; q < s; ++q) {
      const int pos = atomicAdd(&count[tr[q]], 1);
      gent[pos] = ((uint32_t)rl << 1) | ((neg >> q) & 1u);
    }
  }
  __syncthreads();
  // each segment to ascending r: one warp per segment marks its rows (and
  // their signs) in two 4096-bit maps in shared memory -- the rows of a
  // segment are distinct, a row having s distinct targets -- then writes
  // them back in bit order, lane l taking map words 4l .. 4l+3 at the offset
  // of a warp prefix sum of the words' popcounts: O(L + 128) per segment of
  // L entries instead of an O(L^2) insertion sort
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = lists_sort_warps(d);
    uint32_t* rowmap = (uint32_t*)(start + d + 1) + warp * 2 * kListMapWords;
    uint32_t* negmap = rowmap + kListMapWords;
    for (int i = warp; warp < nwarps && i < d; i += nwarps) {
      const int a = start[i], e = start[i + 1];
      if (e - a < 2) continue;  // uniform over the warp
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        rowmap[4 * lane + u] = 0u;
        negmap[4 * lane + u] = 0u;
      }
      __syncwarp();
      for (int x = a + lane; x < e; x += 32) {
        const uint32_t w = gent[x];
        const uint32_t r = w >> 1;
        atomicOr(&rowmap[r >> 5], 1u << (r & 31));
        if (w & 1u) atomicOr(&negmap[r >> 5], 1u << (r & 31));
      }
      __syncwarp();
      uint32_t words[4], negs[4];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        words[u] = rowmap[4 * lane + u];
        negs[u] = negmap[4 * lane + u];
        cnt += __popc(words[u]);
      }
      int x = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
      }
      int pos = a + x - cnt;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint32_t bits = words[u];
        while (bits) {
          const int bit = __ffs(bits) - 1;
          bits &= bits - 1u;
          const uint32_t r = (uint32_t)((4 * lane + u) * 32 + bit);
          gent[pos++] = (r << 1) | ((negs[u] >> bit) & 1u);
        }
      }
      __syncwarp();
    }
  }
  if (!seg_packed(d, s)) return;
  // targets by descending list length: a counting sort on the length (the
  // sort warps' maps are free again: their first kLenBins words hold it)
  __syncthreads();
  int* hist = start + d + 1;
  for (int i = threadIdx.x; i < kLenBins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const int len = start[i + 1] - start[i];
    atomicAdd(&hist[kLenBins - 1 - (len < kLenBins - 1 ? len : kLenBins - 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the bins (longest first)
    const int lane = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < kLenBins; base += 32) {
      const int v = hist[base + lane];
      int x = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
      }
      hist[base + lane] = carry + x - v;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const int len = start[i + 1] - start[i];
    const int pos = atomicAdd(&hist[kLenBins - 1 - (len < kLenBins - 1 ? len : kLenBins - 1)], 1);
    gstart[pos] = (int)(((uint32_t)i << 17) | (uint32_t)start[pos]);
  }
}

// tile: the block's rows of the kSkCols (= 2) columns, one double2 per row.
__device__ __forceinline__ void sketch_partial_body(int64_t b, int64_t cg, const SketchDesc& D,
                                                    double2* tile /* [kRowBlock] */) {
  static_assert(kSkCols == 2, "two columns per CTA, staged as double2");
  const int d = D.d;
  const int64_t n = D.n;
  const int64_t c0 = cg * kSkCols;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, D.m - r0);
  const bool two = c0 + 1 < n;
  {
    const double* col0 = D.M + c0 * D.ldm + r0;
    const double* col1 = D.M + (two ? c0 + 1 : c0) * D.ldm + r0;
    for (int rl = threadIdx.x; rl < rows; rl += blockDim.x)
      tile[rl] = make_double2(col0[rl], two ? col1[rl] : 0.0);
  }
  __syncthreads();
  const uint32_t* st = (const uint32_t*)D.seg_start + b * (int64_t)(d + 1);
  const uint32_t* ent = D.entries + b * (int64_t)kRowBlock * D.s;
  double* P = D.partial + b * n * (int64_t)d;  // P_b: d x n, ld d
  const bool packed = seg_packed(d, D.s);
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    // thread t takes target i (longest lists first when packed)
    const int i = packed ? (int)(st[t] >> 17) : t;
    const int e0 = packed ? (int)(st[i] & kSegMask) : (int)st[i];
    const int e1 = i + 1 < d ? (packed ? (int)(st[i + 1] & kSegMask) : (int)st[i + 1]) : (int)st[d];
    double a0 = 0.0, a1 = 0.0;
    for (int e = e0; e < e1; ++e) {
      const uint32_t w = ent[e];
      const double2 v = tile[w >> 1];
      // a - x == a + (-x) exactly; the sign flip runs on the integer pipe
      const unsigned long long neg = (unsigned long long)(w & 1u) << 63;
      a0 = __dadd_rn(a0, __longlong_as_double(__double_as_longlong(v.x) ^ neg));
      a1 = __dadd_rn(a1, __longlong_as_double(__double_as_longlong(v.y) ^ neg));
    }
    P[c0 * d + i] = a0;
    if (two) P[(c0 + 1) * d + i] = a1;
  }
}

__device__ __forceinline__ void sketch_combine_body(int64_t tile, const SketchDesc& D) {
  const int d = D.d;
  const int64_t total = D.n * (int64_t)d;
  const int64_t nblocks = (D.m + kRowBlock - 1) / kRowBlock;
  const int64_t idx = tile * kCombineThreads + threadIdx.x;
  bool bad = false;
  if (idx < total) {
    const int64_t c = idx / d, i = idx - c * d;
    double t = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) t = __dadd_rn(t, D.partial[b * total + idx]);
    const double v = __dmul_rn(t, D.scale);
    D.Msk[c * D.ldsk + i] = v;
    bad = !isfinite(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(D.status, kNonFinite);
}

// Row panels: acc[i, c] continues the ascending block sum of the panels
// before this one (acc = +0.0 before the first panel), so that after the
// last panel acc equals the combine's sum bit for bit when every panel
// starts on a kRowBlock boundary; sketch_finish then scales.
__global__ void __launch_bounds__(kCombineThreads) sketch_accumulate_kernel(SketchDesc D,
                                                                            double* acc) {
  const int64_t total = D.n * (int64_t)D.d;
  const int64_t nblocks = (D.m + kRowBlock - 1) / kRowBlock;
  const int64_t idx = (int64_t)blockIdx.x * kCombineThreads + threadIdx.x;
  if (idx >= total) return;
  double t = acc[idx];
  for (int64_t b = 0; b < nblocks; ++b) t = __dadd_rn(t, D.partial[b * total + idx]);
  acc[idx] = t;
}

__global__ void __launch_bounds__(kCombineThreads) sketch_finish_kernel(const double* acc, int d,
                                                                        int64_t n, double scale,
                                                                        double* Msk, int64_t ldsk,
                                                                        int* status) {
  const int64_t idx = (int64_t)blockIdx.x * kCombineThreads + threadIdx.x;
  bool bad = false;
  if (idx < n * (int64_t)d) {
    const int64_t c = idx / d, i = idx - c * d;
    const double v = __dmul_rn(acc[idx], scale);
    Msk[c * ldsk + i] = v;
    bad = !isfinite(v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(status, kNonFinite);
}

// ---- single-problem kernels -------------------------------------------------
__global__ void __launch_bounds__(kListThreads) saso_lists_kernel(SketchDesc D) {
  extern __shared__ int sh_lists[];
  saso_lists_body(blockIdx.x, D, sh_lists);
}

__global__ void __launch_bounds__(kSkThreads) sketch_partial_kernel(SketchDesc D, int64_t ncg) {
  extern __shared__ double2 tile[];
  sketch_partial_body(blockIdx.x / ncg, blockIdx.x % ncg, D, tile);
}

__global__ void __launch_bounds__(kCombineThreads) sketch_combine_kernel(SketchDesc D) {
  sketch_combine_body(blockIdx.x, D);
}

// ---- batched kernels --------------------------------------------------------
__global__ void __launch_bounds__(kListThreads) saso_lists_batched_kernel(const SketchDesc* D,
                                                                   const int64_t* base, int np) {
  extern __shared__ int sh_lists[];
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  saso_lists_body(t, D[p], sh_lists);
}

__global__ void __launch_bounds__(kSkThreads) sketch_partial_batched_kernel(const SketchDesc* D,
                                                                            const int64_t* base,
                                                                            int np) {
  extern __shared__ double2 tile[];
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  const int64_t ncg = (D[p].n + kSkCols - 1) / kSkCols;
  sketch_partial_body(t / ncg, t % ncg, D[p], tile);
}

__global__ void __launch_bounds__(kCombineThreads) sketch_combine_batched_kernel(
    const SketchDesc* D, const int64_t* base, int np) {
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  sketch_combine_body(t, D[p]);
}

// ---- dense operators --------------------------------------------------------
// One CTA per (row block b, 32 x 32 tile of the d x n output); 64 threads in
// an 8 x 8 grid, each with a 4 x 4 register tile; rows staged kDsRows at a
// time in shared memory (S read along i, M along r: both coalesced).  The
// kernel is bound by the FP64 pipe (2 d m n flops); the CTAs of one row block
// are adjacent in launch order, so its slices of S and M are read from HBM
// about once and reused from L2 by the block's tiles.
constexpr int kDsTile = 32;
constexpr int kDsRows = 32;

struct DenseSketchDesc {
  int64_t m, n;
  int d;
  const double* S;
  int64_t lds;
  const double* M;
  int64_t ldm;
  double* partial;  // nblocks x (n x d), ld d
};

__global__ void __launch_bounds__(64, 14) sketch_dense_partial_kernel(DenseSketchDesc D,
                                                                      int ti_count, int tiles) {
  __shared__ double Ss[kDsTile][kDsRows + 1];  // [i][row]
  __shared__ double Ms[kDsTile][kDsRows + 1];  // [c][row]
  const int64_t b = blockIdx.x / tiles;
  const int t = (int)(blockIdx.x - b * tiles);
  const int i0 = (t % ti_count) * kDsTile, c0 = (t / ti_count) * kDsTile;
  const int64_t r0 = b * kRowBlock;
  const int rows = (int)min64(kRowBlock, D.m - r0);
  const int d = D.d;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

  for (int rr0 = 0; rr0 < rows; rr0 += kDsRows) {
    const int nr = min(kDsRows, rows - rr0);
    __syncthreads();
    for (int e = threadIdx.x; e < kDsTile * kDsRows; e += 64) {
      const int i = e % kDsTile, srow = e / kDsTile;
      Ss[i][srow] = (srow < nr && i0 + i < d)
                        ? D.S[(r0 + rr0 + srow) * D.lds + (i0 + i)] : 0.0;
      const int c = e / kDsRows, mrow = e % kDsRows;
      Ms[c][mrow] = (mrow < nr && c0 + c < D.n)
                        ? D.M[(int64_t)(c0 + c) * D.ldm + (r0 + rr0 + mrow)] : 0.0;
    }
    __syncthreads();
    for (int row = 0; row < nr; ++row) {
      double va[4], vc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) va[u] = Ss[ty * 4 + u][row];
#pragma unroll
      for (int v = 0; v < 4; ++v) vc[v] = Ms[tx * 4 + v][row];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = __fma_rn(va[u], vc[v], acc[u][v]);
    }
  }
  double* P = D.partial + b * D.n * (int64_t)d;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (i < d && c < D.n) P[(int64_t)c * d + i] = acc[u][v];
    }
}

// ---- host side --------------------------------------------------------------
static int64_t nblocks_of(int64_t m) { return (m + kRowBlock - 1) / kRowBlock; }

// Threads of a partial-sum CTA: the d target rows spread evenly over at most
// kSkThreads threads (every thread the same number of rows, up to the last
// warp), a whole number of warps.
static int sketch_threads(int d) {
  const int passes = (d + kSkThreads - 1) / kSkThreads;
  const int per = (d + passes - 1) / passes;
  return (per + 31) / 32 * 32;
}

int64_t sketch_workspace_bytes(int64_t m, int64_t n, int d, int s) {
  const int64_t nb = nblocks_of(m);
  int64_t bytes = 0;
  bytes += align256(nb * (int64_t)(d + 1) * 4);
  bytes += align256(nb * (int64_t)kRowBlock * s * 4);
  bytes += align256(nb * n * (int64_t)d * 8);
  return bytes;
}

void sketch_carve(SketchDesc& D, void* work) {
  const int64_t nb = nblocks_of(D.m);
  char* p = (char*)work;
  D.seg_start = (int*)p;
  p += align256(nb * (int64_t)(D.d + 1) * 4);
  D.entries = (uint32_t*)p;
  p += align256(nb * (int64_t)kRowBlock * D.s * 4);
  D.partial = (double*)p;
}

int64_t sketch_list_tiles(const SketchDesc& D) { return nblocks_of(D.m); }
int64_t sketch_partial_tiles(const SketchDesc& D) {
  return nblocks_of(D.m) * ((D.n + kSkCols - 1) / kSkCols);
}
int64_t sketch_combine_tiles(const SketchDesc& D) {
  return (D.n * (int64_t)D.d + kCombineThreads - 1) / kCombineThreads;
}

static cudaError_t set_smem_attrs(size_t lists_bytes) {
  cudaError_t e = cudaSuccess;
  if (lists_bytes > 48 * 1024) {
    e = raise_smem_limit((const void*)saso_lists_kernel, lists_bytes);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)saso_lists_batched_kernel, lists_bytes);
    if (e != cudaSuccess) return e;
  }
  const int tile_bytes = kRowBlock * (int)sizeof(double2);
  e = raise_smem_limit((const void*)sketch_partial_kernel, (size_t)tile_bytes);
  if (e == cudaSuccess)
    e = raise_smem_limit((const void*)sketch_partial_batched_kernel, (size_t)tile_bytes);
  return e;
}

cudaError_t launch_sketch(int64_t m, int64_t n, const double* M, int64_t ldm, int d, int s,
                          uint64_t seed, double scale, double* Msk, int64_t ldsk, void* work,
                          int* status, cudaStream_t stream) {
  SketchDesc D{};
  D.m = m; D.n = n; D.d = d; D.s = s; D.seed = seed; D.scale = scale;
  D.M = M; D.ldm = ldm; D.Msk = Msk; D.ldsk = ldsk; D.status = status;
  sketch_carve(D, work);
  const size_t sh_lists = lists_smem_bytes(d);
  cudaError_t e = set_smem_attrs(sh_lists);
  if (e != cudaSuccess) return e;
  saso_lists_kernel<<<(unsigned)sketch_list_tiles(D), kListThreads, sh_lists, stream>>>(D);
  const int64_t ncg = (n + kSkCols - 1) / kSkCols;
  sketch_partial_kernel<<<(unsigned)sketch_partial_tiles(D), sketch_threads(d),
                          kRowBlock * sizeof(double2), stream>>>(D, ncg);
  sketch_combine_kernel<<<(unsigned)sketch_combine_tiles(D), kCombineThreads, 0, stream>>>(D);
  count_launches(3);
  return cudaGetLastError();
}

int64_t sketch_dense_workspace_bytes(int64_t m, int64_t n, int d) {
  return align256(nblocks_of(m) * n * (int64_t)d * 8);
}

cudaError_t launch_sketch_dense(int64_t m, int64_t n, const double* S, int64_t lds,
                                const double* M, int64_t ldm, int d, double* Msk, int64_t ldsk,
                                void* work, int* status, cudaStream_t stream) {
  const int ti_count = (d + kDsTile - 1) / kDsTile;
  const int tiles = ti_count * (int)((n + kDsTile - 1) / kDsTile);
  DenseSketchDesc P{m, n, d, S, lds, M, ldm, (double*)work};
  sketch_dense_partial_kernel<<<(unsigned)(nblocks_of(m) * tiles), 64, 0, stream>>>(P, ti_count,
                                                                                 tiles);
  SketchDesc D{};
  D.m = m; D.n = n; D.d = d; D.scale = 1.0;
  D.partial = (double*)work; D.Msk = Msk; D.ldsk = ldsk; D.status = status;
  sketch_combine_kernel<<<(unsigned)sketch_combine_tiles(D), kCombineThreads, 0, stream>>>(D);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_sketch_panel_partials(int64_t rows, int64_t n, const double* M, int64_t ldm,
                                         int d, int s, uint64_t seed, int64_t row0, void* work,
                                         cudaStream_t stream) {
  SketchDesc D{};
  D.m = rows; D.n = n; D.d = d; D.s = s; D.seed = seed; D.row0 = row0; D.scale = 1.0;
  D.M = M; D.ldm = ldm;
  sketch_carve(D, work);
  const size_t sh_lists = lists_smem_bytes(d);
  cudaError_t e = set_smem_attrs(sh_lists);
  if (e != cudaSuccess) return e;
  saso_lists_kernel<<<(unsigned)sketch_list_tiles(D), kListThreads, sh_lists, stream>>>(D);
  const int64_t ncg = (n + kSkCols - 1) / kSkCols;
  sketch_partial_kernel<<<(unsigned)sketch_partial_tiles(D), sketch_threads(d),
                          kRowBlock * sizeof(double2), stream>>>(D, ncg);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_sketch_panel_accumulate(int64_t rows, int64_t n, int d, int s, double* acc,
                                           void* work, cudaStream_t stream) {
  SketchDesc D{};
  D.m = rows; D.n = n; D.d = d; D.s = s;
  sketch_carve(D, work);
  sketch_accumulate_kernel<<<(unsigned)sketch_combine_tiles(D), kCombineThreads, 0, stream>>>(
      D, acc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sketch_panel(int64_t rows, int64_t n, const double* M, int64_t ldm, int d,
                                int s, uint64_t seed, int64_t row0, double* acc, void* work,
                                cudaStream_t stream) {
  cudaError_t e = launch_sketch_panel_partials(rows, n, M, ldm, d, s, seed, row0, work, stream);
  if (e != cudaSuccess) return e;
  return launch_sketch_panel_accumulate(rows, n, d, s, acc, work, stream);
}

cudaError_t launch_sketch_finish(int d, int64_t n, const double* acc, double scale, double* Msk,
                                 int64_t ldsk, int* status, cudaStream_t stream) {
  const unsigned grid = (unsigned)((n * (int64_t)d + kCombineThreads - 1) / kCombineThreads);
  sketch_finish_kernel<<<grid, kCombineThreads, 0, stream>>>(acc, d, n, scale, Msk, ldsk, status);
  count_launches(1);
  return cudaGetLastError();
}

// ---- dense operators on the tensor cores ------------------------------------
// M^sk = S M as the split-BF16 product (S^T)^T M: S is transposed into
// S^T (m x d, column-major, 32 x 32 tiles through shared memory) so that both
// operands are split along their m rows like the Gram's, then oz_gemm_tn.
// Non-finite entries of S (seen by the transpose) or of M set kNonFinite:
// the digit split does not carry them.
__global__ void __launch_bounds__(256) sketch_transpose_kernel(const double* S, int64_t lds,
                                                               int d, int64_t m, double* St,
                                                               int* status) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;  // columns of S (rows of S^T)
  const int i0 = blockIdx.y * 32;               // rows of S
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  bool bad = false;
  for (int j = ty; j < 32; j += 8) {
    const int i = i0 + tx;
    const int64_t r = r0 + j;
    double v = 0.0;
    if (i < d && r < m) {
      v = S[r * lds + i];
      bad |= !isfinite(v);
    }
    tile[j][tx] = v;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + tx;
    const int i = i0 + j;
    if (i < d && r < m) St[(int64_t)i * m + r] = tile[tx][j];
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(status, kNonFinite);
}

__global__ void __launch_bounds__(256) nonfinite_scan_kernel(const double* M, int64_t ldm,
                                                             int64_t rows, int64_t cols,
                                                             int* status) {
  bool bad = false;
  const int64_t total = rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * 256) {
    const int64_t c = idx / rows, r = idx - c * rows;
    bad |= !isfinite(M[c * ldm + r]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(status, kNonFinite);
}

int64_t sketch_dense_split_workspace_bytes(int64_t m, int64_t n, int d) {
  return align256(m * (int64_t)d * 8) + oz_gemm_tn_workspace(m, d, (int)n, nullptr);
}

cudaError_t launch_sketch_dense_split(int64_t m, int64_t n, const double* S, int64_t lds,
                                      const double* M, int64_t ldm, int d, double* Msk,
                                      int64_t ldsk, void* work, int* status,
                                      cudaStream_t stream) {
  double* St = (double*)work;
  void* rest = (char*)work + align256(m * (int64_t)d * 8);
  const dim3 gt((unsigned)((m + 31) / 32), (unsigned)((d + 31) / 32));
  sketch_transpose_kernel<<<gt, 256, 0, stream>>>(S, lds, d, m, St, status);
  nonfinite_scan_kernel<<<4 * 152, 256, 0, stream>>>(M, ldm, m, n, status);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return oz_gemm_tn(m, d, (int)n, St, m, M, ldm, Msk, ldsk, rest, stream, status);
}

cudaError_t sketch_set_attributes(int max_d) { return set_smem_attrs(lists_smem_bytes(max_d)); }

// The shared-memory attributes must have been set by sketch_set_attributes
// (outside any stream capture).
cudaError_t launch_sketch_batched(int phase, const SketchDesc* D, const int64_t* base, int np,
                                  int64_t total_tiles, int max_d, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  const size_t sh_lists = lists_smem_bytes(max_d);
  if (phase == 0)
    saso_lists_batched_kernel<<<(unsigned)total_tiles, kListThreads, sh_lists, stream>>>(D, base,
                                                                                        np);
  else if (phase == 1)
    sketch_partial_batched_kernel<<<(unsigned)total_tiles, sketch_threads(max_d),
                                    kRowBlock * sizeof(double2), stream>>>(D, base, np);
  else
    sketch_combine_batched_kernel<<<(unsigned)total_tiles, kCombineThreads, 0, stream>>>(D, base,
                                                                                        np);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
