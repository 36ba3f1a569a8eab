// Alg. 2 line 5: the Gram matrix G = (M^pre)^T M^pre (k x k, the SYRK of
// the CholeskyQR step, Sec. 1.2).
//
// The sum over the m rows is blocked twice: rows fall into blocks of
// kRowBlock rows and each block into sub-blocks of kGramSub rows.  A
// sub-block sum S[a, c] = sum_{r in s} X[r, a] X[r, c] runs in ascending r
// with one fma per term from +0.0 (a <= c); a block sum is
// P_b = ((0 + S_b0) + S_b1) + ... over its sub-blocks in ascending order,
// and G[a, c] = ((0 + P_0) + P_1) + ... over the blocks; the upper triangle
// is mirrored.  Two forms give these bits:
//   * block partials (every caller): one CTA per output tile and block
//     folds each sub-block sum into the block sum as it goes (in registers
//     for 8- and 16-wide tiles, in the block partial in global memory for
//     32-wide ones), gram_combine adds the blocks;
//   * sub-block partials (launch_gram with sub_ok, a small problem whose
//     sub-block partials fit the workspace): one CTA per output tile and
//     sub-block, so a sum's dependent chain is kGramSub fmas instead of
//     kRowBlock (m = 4096: 256 instead of 4096); gram_combine forms the
//     block sums and their sum.
// One CTA computes one output tile of one row block (or sub-block)
// (kGramTile x kGramTile, or 16 x 16 where a batched problem's descriptor
// asks for it: less padding when k is small; the batched autotuner picks the
// edge per problem size; a small single problem uses 16 x 16 or 8 x 8 tiles
// so that enough CTAs share the work); its 64 threads own 4 x 4 (2 x 2,
// 1 x 1) register tiles, and rows are staged kGramRows at a time in shared
// memory.  Each entry is
// the same ascending-r fma chain whatever the tile, so the tile does not
// change the result.  The kernel is bound by the FP64 pipe.  Single-problem
// and batched launches share the bodies.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

static __host__ __device__ int64_t gram_nblocks(int64_t m) {
  return (m + kRowBlock - 1) / kRowBlock;
}
static __host__ __device__ int64_t gram_nsub(int64_t m) { return (m + kGramSub - 1) / kGramSub; }
// sub-block partials for a small problem: m within 8 blocks and at most
// 64 MiB of partials
static bool gram_sub_mode(int64_t m, int64_t n) {
  return m <= 8 * (int64_t)kRowBlock && gram_nsub(m) * n * n * 8 <= (64ll << 20);
}
static __host__ __device__ int gram_tile_edge(int tile) {
  return tile == 8 ? 8 : tile == 16 ? 16 : kGramTile;
}
static __host__ __device__ int64_t gram_ntri(int kmax, int tile) {
  const int e = gram_tile_edge(tile);
  const int64_t t1 = (kmax + e - 1) / e;
  return t1 * (t1 + 1) / 2;
}

int64_t gram_block_workspace_bytes(int64_t m, int64_t n) {
  return align256(gram_nblocks(m) * n * n * 8);
}
int64_t gram_workspace_bytes(int64_t m, int64_t n) {
  const int64_t a = gram_block_workspace_bytes(m, n);
  const int64_t b = gram_sub_mode(m, n) ? align256(gram_nsub(m) * n * n * 8) : 0;
  return a > b ? a : b;
}
int64_t gram_partial_tiles(int64_t m, int kmax, int tile) {
  return gram_nblocks(m) * gram_ntri(kmax, tile);
}
static int64_t gram_sub_partial_tiles(int64_t m, int kmax, int tile) {
  return gram_nsub(m) * gram_ntri(kmax, tile);
}
int64_t gram_combine_tiles(int kmax) {
  return ((int64_t)kmax * kmax + kCombineThreads - 1) / kCombineThreads;
}

// One TILE x TILE output tile of one row block; 64 threads in an 8 x 8
// grid, each with a (TILE/8) x (TILE/8) register tile.
typedef double GramStage[kGramTile][kGramRows + 1];  // [col][row]

template <int TILE>
__device__ __forceinline__ void gram_partial_tile(int64_t tile, const GramDesc& D, GramStage& Xa,
                                                  GramStage& Xc) {
  constexpr int R = TILE / 8;
  const int k = (int)*D.k_dev;
  const int64_t ntri = gram_ntri(D.n_ld, TILE);
  const int64_t b = tile / ntri;
  int t = (int)(tile - b * ntri);
  // triangular tile index -> (ta, tc) with ta <= tc, for the device k
  const int tiles_1d = (k + TILE - 1) / TILE;
  int ta = 0;
  while (ta < tiles_1d && t >= tiles_1d - ta) { t -= tiles_1d - ta; ++ta; }
  if (ta >= tiles_1d) return;
  const int tc = ta + t;
  // D.sub: b is a sub-block (its sum alone); else a block (sub-block sums
  // folded into the block sum)
  const int64_t r0 = D.sub ? b * kGramSub : b * kRowBlock;
  const int rows = (int)min64(D.sub ? kGramSub : kRowBlock, D.m - r0);
  if (rows <= 0) return;
  const double* X = D.X;
  const int64_t ldx = D.ldx;
  const int a0 = ta * TILE, c0 = tc * TILE;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int n_ld = D.n_ld;
  double* P = D.partial + b * (int64_t)n_ld * n_ld;
  double acc[R][R];  // the current sub-block's sums
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int v = 0; v < R; ++v) acc[u][v] = 0.0;
  // the block sums (registers)
  constexpr bool kBlkRegs = true;
  double blk[kBlkRegs ? R : 1][kBlkRegs ? R : 1];
#pragma unroll
  for (int u = 0; u < (kBlkRegs ? R : 1); ++u)
#pragma unroll
    for (int v = 0; v < (kBlkRegs ? R : 1); ++v) blk[u][v] = 0.0;
  auto fold = [&](bool first) {  // block sum += sub-block sum; sub-block sum = 0
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
      for (int v = 0; v < R; ++v) {
        if constexpr (kBlkRegs) {
          blk[u][v] = __dadd_rn(blk[u][v], acc[u][v]);
        } else {
          const int a = a0 + ty * R + u, c = c0 + tx * R + v;
          if (a < k && c < k && a <= c) {
            double* e = P + (int64_t)c * n_ld + a;
            *e = __dadd_rn(first ? 0.0 : *e, acc[u][v]);
          }
        }
        acc[u][v] = 0.0;
      }
  };

  // small tiles (few CTAs, latency-bound): the next chunk's rows are loaded
  // into registers while the current chunk is summed
  constexpr bool kPrefetch = TILE <= 16;
  constexpr int kPer = kPrefetch ? TILE * kGramRows / 64 : 1;  // staged elements per thread
  double pa[kPer], pc[kPer];
  auto load_chunk = [&](int rr0) {
    const int nr = min(kGramRows, rows - rr0);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x + 64 * q;
      const int col = e / kGramRows, row = e % kGramRows;
      const int64_t r = r0 + rr0 + row;
      const bool rok = row < nr;
      pa[q] = (rok && a0 + col < k) ? X[(int64_t)(a0 + col) * ldx + r] : 0.0;
      pc[q] = (rok && c0 + col < k) ? X[(int64_t)(c0 + col) * ldx + r] : 0.0;
    }
  };
  if constexpr (kPrefetch) load_chunk(0);
  for (int rr0 = 0; rr0 < rows; rr0 += kGramRows) {
    const int nr = min(kGramRows, rows - rr0);
    __syncthreads();
    if constexpr (kPrefetch) {
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e = threadIdx.x + 64 * q;
        Xa[e / kGramRows][e % kGramRows] = pa[q];
        Xc[e / kGramRows][e % kGramRows] = pc[q];
      }
    } else {
      for (int e = threadIdx.x; e < TILE * kGramRows; e += 64) {
        const int col = e / kGramRows, row = e % kGramRows;
        const int64_t r = r0 + rr0 + row;
        const bool rok = row < nr;
        Xa[col][row] = (rok && a0 + col < k) ? X[(int64_t)(a0 + col) * ldx + r] : 0.0;
        Xc[col][row] = (rok && c0 + col < k) ? X[(int64_t)(c0 + col) * ldx + r] : 0.0;
      }
    }
    __syncthreads();
    if constexpr (kPrefetch)
      if (rr0 + kGramRows < rows) load_chunk(rr0 + kGramRows);
    for (int row = 0; row < nr; ++row) {
      double va[R], vc[R];
#pragma unroll
      for (int u = 0; u < R; ++u) va[u] = Xa[ty * R + u][row];
#pragma unroll
      for (int v = 0; v < R; ++v) vc[v] = Xc[tx * R + v][row];
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) acc[u][v] = __fma_rn(va[u], vc[v], acc[u][v]);
    }
    // end of a sub-block (kGramSub is a multiple of kGramRows): fold it
    if (!D.sub && ((rr0 + kGramRows) % kGramSub == 0 || rr0 + kGramRows >= rows))
      fold(rr0 < kGramSub);
  }
  if (D.sub || kBlkRegs) {
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
      for (int v = 0; v < R; ++v) {
        const int a = a0 + ty * R + u, c = c0 + tx * R + v;
        double val = acc[u][v];
        if constexpr (kBlkRegs) val = D.sub ? acc[u][v] : blk[u][v];
        if (a < k && c < k && a <= c) P[(int64_t)c * n_ld + a] = val;
      }
  }
}

__device__ __forceinline__ void gram_partial_body(int64_t tile, const GramDesc& D) {
  __shared__ GramStage Xa, Xc;
  if (*D.status != kOk) return;
  if (D.tile == 8)
    gram_partial_tile<8>(tile, D, Xa, Xc);
  else if (D.tile == 16)
    gram_partial_tile<16>(tile, D, Xa, Xc);
  else
    gram_partial_tile<kGramTile>(tile, D, Xa, Xc);
}

// accumulate: the sum starts from G's upper entry instead of +0.0 (row
// panels: G holds the ascending block sum of the panels before this one)
__device__ __forceinline__ void gram_combine_body(int64_t tile, const GramDesc& D,
                                                  bool accumulate = false) {
  if (*D.status != kOk) return;
  const int k = (int)*D.k_dev;
  const int n_ld = D.n_ld;
  const int64_t nblocks = gram_nblocks(D.m);
  const int64_t idx = tile * kCombineThreads + threadIdx.x;
  if (idx >= (int64_t)k * k) return;
  const int c = (int)(idx / k), a = (int)(idx - (int64_t)c * k);
  if (a > c) return;
  const int64_t off = (int64_t)c * n_ld + a;
  double tsum = accumulate ? D.G[(int64_t)c * D.ldg + a] : 0.0;
  if (D.sub) {  // sub-block partials: each block's sum first
    const int64_t nsub = gram_nsub(D.m);
    constexpr int64_t kPer = kRowBlock / kGramSub;
    for (int64_t b = 0; b < nblocks; ++b) {
      double pb = 0.0;
      const int64_t s1 = min64(nsub, (b + 1) * kPer);
      for (int64_t s = b * kPer; s < s1; ++s)
        pb = __dadd_rn(pb, D.partial[s * (int64_t)n_ld * n_ld + off]);
      tsum = __dadd_rn(tsum, pb);
    }
  } else {
    for (int64_t b = 0; b < nblocks; ++b)
      tsum = __dadd_rn(tsum, D.partial[b * (int64_t)n_ld * n_ld + off]);
  }
  D.G[(int64_t)c * D.ldg + a] = tsum;
  D.G[(int64_t)a * D.ldg + c] = tsum;
}

// single problem: one instantiation per tile edge (each with its own
// register budget; 14 CTAs per SM for the 16 x 16 and 32 x 32 tiles)
template <int TILE>
__global__ void __launch_bounds__(64, TILE == 8 ? 1 : 12) gram_partial_kernel(GramDesc D) {
  __shared__ GramStage Xa, Xc;
  if (*D.status != kOk) return;
  gram_partial_tile<TILE>(blockIdx.x, D, Xa, Xc);
}
__global__ void __launch_bounds__(kCombineThreads) gram_combine_kernel(GramDesc D) {
  gram_combine_body(blockIdx.x, D);
}
__global__ void __launch_bounds__(kCombineThreads) gram_accumulate_kernel(GramDesc D) {
  gram_combine_body(blockIdx.x, D, true);
}
__global__ void __launch_bounds__(64) gram_partial_batched_kernel(const GramDesc* D,
                                                                  const int64_t* base, int np) {
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  gram_partial_body(t, D[p]);
}
__global__ void __launch_bounds__(kCombineThreads) gram_combine_batched_kernel(const GramDesc* D,
                                                                               const int64_t* base,
                                                                               int np) {
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  gram_combine_body(t, D[p]);
}

// Output tile edge of a single-problem Gram: the largest of 32, 16, 8 that
// still gives two waves of CTAs (a small problem has few 4096-row blocks, and
// the FP64 pipe of a few SMs would otherwise carry it alone).
static int gram_single_tile(int64_t m, int kmax) {
  for (int t : {kGramTile, 16})
    if (gram_partial_tiles(m, kmax, t) >= 2 * 152) return t;
  return 8;
}

cudaError_t launch_gram_partials(int64_t m, int kmax, const int64_t* k_dev, const double* X,
                                 int64_t ldx, void* work, const int* status,
                                 cudaStream_t stream) {
  const int tile = gram_single_tile(m, kmax);
  GramDesc D{m, kmax, k_dev, X, ldx, (double*)work, nullptr, 0, status, tile};
  const unsigned grid = (unsigned)gram_partial_tiles(m, kmax, tile);
  if (tile == 8)
    gram_partial_kernel<8><<<grid, 64, 0, stream>>>(D);
  else if (tile == 16)
    gram_partial_kernel<16><<<grid, 64, 0, stream>>>(D);
  else
    gram_partial_kernel<kGramTile><<<grid, 64, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram_sum(int64_t m, int kmax, const int64_t* k_dev, double* G, int64_t ldg,
                            void* work, const int* status, cudaStream_t stream, bool accumulate) {
  GramDesc D{m, kmax, k_dev, nullptr, 0, (double*)work, G, ldg, status, kGramTile};
  if (accumulate)
    gram_accumulate_kernel<<<(unsigned)gram_combine_tiles(kmax), kCombineThreads, 0, stream>>>(D);
  else
    gram_combine_kernel<<<(unsigned)gram_combine_tiles(kmax), kCombineThreads, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram(int64_t m, int kmax, const int64_t* k_dev, const double* X, int64_t ldx,
                        double* G, int64_t ldg, void* work, const int* status,
                        cudaStream_t stream, bool accumulate, bool sub_ok) {
  if (sub_ok && gram_sub_mode(m, kmax)) {
    int tile = 8;
    for (int t : {kGramTile, 16})
      if (gram_sub_partial_tiles(m, kmax, t) >= 2 * 152) {
        tile = t;
        break;
      }
    GramDesc D{m, kmax, k_dev, X, ldx, (double*)work, G, ldg, status, tile, 1};
    const unsigned grid = (unsigned)gram_sub_partial_tiles(m, kmax, tile);
    if (tile == 8)
      gram_partial_kernel<8><<<grid, 64, 0, stream>>>(D);
    else if (tile == 16)
      gram_partial_kernel<16><<<grid, 64, 0, stream>>>(D);
    else
      gram_partial_kernel<kGramTile><<<grid, 64, 0, stream>>>(D);
    if (accumulate)
      gram_accumulate_kernel<<<(unsigned)gram_combine_tiles(kmax), kCombineThreads, 0, stream>>>(D);
    else
      gram_combine_kernel<<<(unsigned)gram_combine_tiles(kmax), kCombineThreads, 0, stream>>>(D);
    count_launches(2);
    return cudaGetLastError();
  }
  cudaError_t e = launch_gram_partials(m, kmax, k_dev, X, ldx, work, status, stream);
  if (e != cudaSuccess) return e;
  return launch_gram_sum(m, kmax, k_dev, G, ldg, work, status, stream, accumulate);
}

cudaError_t launch_gram_batched(int phase, const GramDesc* D, const int64_t* base, int np,
                                int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return cudaSuccess;
  if (phase == 0)
    gram_partial_batched_kernel<<<(unsigned)total_tiles, 64, 0, stream>>>(D, base, np);
  else
    gram_combine_batched_kernel<<<(unsigned)total_tiles, kCombineThreads, 0, stream>>>(D, base, np);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
