// FP64-accurate matrix products on the BF16 tensor cores by error-free
// digit splitting (the scheme of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012; tensor-core
// use as in Mukunoki, Ozaki, Ogita & Imamura, ICCS 2020).  Used by the
// split-BF16 precision modes for Alg. 2 lines 4, 5 and 7, the O(m n^2) steps
// (the paper's two-roundoff model, Sec. 3.1, lets line 4 run in a
// different arithmetic; here all three keep FP64-level accuracy).
//
// Splitting.  Every row (or column) v of an operand gets a power-of-two
// scale 2^e with max|v| < 2^e (e = frexp exponent of the max).  Each entry
// x = sign * |x| is written, by integer operations on its bit pattern, as the
// 56-bit fixed-point number Y = floor(|x| 2^(56-e)) = sum_p y_p 2^(56-7p),
// p = 1..8, with 7-bit digits y_p in [0, 127]; the signed digits +-y_p are
// exact in BF16.  Truncation error: below 2^(e-56) per entry.
//
// Product.  C = A B = 2^(ea_i + eb_j) sum_{p,q} 2^(-7(p+q)) (D_p E_q)_{ij};
// pairs with p + q <= 9 are kept (36 BF16 products, level s = p + q); the
// dropped levels are below 9 * 2^-56 relative to the scales.  Each digit
// product is an integer of magnitude < 2^14, so an FP32 tensor-core
// accumulation of up to 1024 such terms is exact; chunk sums are combined
// exactly in integers and rounded to FP64 once per entry (twice when the
// product is subtracted from C).  The
// engine (tcgen05 + TMA + tensor memory) is in ozaki_tc.cu.  All operands
// are "K-contiguous" digit planes: A is stored as M rows of K digits per
// plane, B as N rows of K digits per plane.
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "ozaki.h"

namespace cqrrpt {

// ---------------------------------------------------------------------------
// digit extraction
// ---------------------------------------------------------------------------
__device__ __forceinline__ int frexp_exp(double amax) {
  if (amax == 0.0) return 0;
  int e;
  frexp(amax, &e);
  return e;
}

// Writes the 8 signed 7-bit digits of x relative to 2^e (|x| < 2^e).
__device__ __forceinline__ void digits8(double x, int e, __nv_bfloat16* out, int64_t plane_stride) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const bool neg = (b >> 63) != 0;
  int ex = (int)((b >> 52) & 0x7ff);
  unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  if (ex == 0) ex = 1; else mant |= (1ull << 52);
  const int sh = ex - 1019 - e;  // Y = mant * 2^(ex - 1075 + 56 - e)
  unsigned long long Y;
  if (mant == 0) Y = 0;
  else if (sh >= 0) Y = sh < 64 ? (mant << sh) : 0ull;
  else Y = (-sh) < 64 ? (mant >> (-sh)) : 0ull;
#pragma unroll
  for (int p = 1; p <= kOzDigits; ++p) {
    const int dig = (int)((Y >> (56 - 7 * p)) & 127ull);
    out[(p - 1) * plane_stride] = __float2bfloat16_rn((float)(neg ? -dig : dig));
  }
}

// Every helper step below has one body over a job and a tile index; the
// single-problem kernel runs tiles blockIdx.x of one job, the batched
// kernel maps CTA b to (job, tile) through a prefix table.

// e[c] for every column c of the column operand: scale over the column.  One
// CTA (256 threads) per column.
__device__ __forceinline__ void colexp_body(const OzColSplit& J, int64_t tile) {
  __shared__ double red[32];
  const int c = (int)tile;
  const double* col = J.X + (int64_t)c * J.ldx;
  double mx = 0.0;
  for (int64_t r = threadIdx.x; r < J.rows; r += blockDim.x) mx = fmax(mx, fabs(col[r]));
  for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
    J.e[c] = frexp_exp(mx);
  }
}

// e[r] for every row r of the row operand over its K columns (column k is
// column map[k] of X when map is given).  256 rows per CTA.
__device__ __forceinline__ void rowexp_body(const OzRowSplit& J, int64_t tile) {
  const int64_t r = tile * 256 + threadIdx.x;
  if (r >= J.rows) return;
  double mx = 0.0;
  for (int c = 0; c < J.cols; ++c)
    mx = fmax(mx, fabs(J.X[(J.map ? J.map[c] : (int64_t)c) * J.ldx + r]));
  J.e[r] = frexp_exp(mx);
}

// Column operand planes of X[k, c] (K = rows, zero past rows up to kpad),
// scale e[c].  Unblocked (kblk = 0): D[p][c][k].  Blocked (kblk = kOzChunk):
// D[p][k / 1024][c][k % 1024], so that a 128-column tile of one 1024-term
// K chunk is one contiguous 256 KB range; the Gram's planes have K = m
// (rows of the unblocked layout are 2m bytes long, and a tile would touch
// 128 rows that far apart: one DRAM page and one TLB entry per 128 bytes).
// CTA: one column, 2048 consecutive k.
constexpr int kOzColChunk = 2048;
__device__ __forceinline__ void splitcols_body(const OzColSplit& J, int64_t tile) {
  const int64_t chunks = (J.kpad + kOzColChunk - 1) / kOzColChunk;
  const int c = (int)(tile / chunks);
  const int64_t k0 = (tile % chunks) * kOzColChunk;
  const int ec = J.e[c];
  const int64_t k1 = min64(k0 + kOzColChunk, J.kpad);
  const double* col = J.X + (int64_t)c * J.ldx;
  if (J.kblk == 0) {
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
      digits8(k < J.rows ? col[k] : 0.0, ec, J.D + (int64_t)c * J.kpad + k, J.plane);
  } else {
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      const int64_t off = (k / kOzChunk) * J.cols * kOzChunk + (int64_t)c * kOzChunk + k % kOzChunk;
      digits8(k < J.rows ? col[k] : 0.0, ec, J.D + off, J.plane);
    }
  }
}

// Row operand planes D[p][r][k] of X[r, map[k]] (K = cols, zero past cols up
// to kpad), scale e[r].  One CTA per 32 rows walks the whole K range in
// 32 x 32 tiles transposed through shared memory, so that the reads of X
// coalesce and every plane row is written whole by one CTA (256 threads).
__device__ __forceinline__ void splitrows_body(const OzRowSplit& J, int64_t tile) {
  __shared__ double tl[32][33];
  const int64_t r0 = tile * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  int er[4];  // exponents of this thread's output rows r0 + ty + 8 i
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + ty + 8 * i;
    er[i] = r < J.rows ? J.e[r] : 0;
  }
  for (int k0 = 0; k0 < J.kpad; k0 += 32) {
    __syncthreads();  // the previous tile's reads of tl are done
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = ty + 8 * i;
      const int64_t r = r0 + tx;
      const int k = k0 + j;
      tl[j][tx] = (r < J.rows && k < J.cols) ? J.X[(J.map ? J.map[k] : (int64_t)k) * J.ldx + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = ty + 8 * i;
      const int64_t r = r0 + j;
      const int k = k0 + tx;
      if (r < J.rows && k < J.kpad) digits8(tl[tx][j], er[i], J.D + r * J.kpad + k, J.plane);
    }
  }
}

__global__ void __launch_bounds__(256) oz_colexp_kernel(OzColSplit J) { colexp_body(J, blockIdx.x); }
__global__ void __launch_bounds__(256) oz_rowexp_kernel(OzRowSplit J) { rowexp_body(J, blockIdx.x); }
__global__ void __launch_bounds__(256) oz_split_cols_kernel(OzColSplit J) {
  splitcols_body(J, blockIdx.x);
}
__global__ void __launch_bounds__(256) oz_split_rows_kernel(OzRowSplit J) {
  splitrows_body(J, blockIdx.x);
}
__global__ void __launch_bounds__(256) oz_colexp_batched_kernel(const OzColSplit* J,
                                                                const int64_t* base, int n) {
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  colexp_body(J[j], t);
}
__global__ void __launch_bounds__(256) oz_rowexp_batched_kernel(const OzRowSplit* J,
                                                                const int64_t* base, int n) {
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  rowexp_body(J[j], t);
}
__global__ void __launch_bounds__(256) oz_split_cols_batched_kernel(const OzColSplit* J,
                                                                    const int64_t* base, int n) {
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  splitcols_body(J[j], t);
}
__global__ void __launch_bounds__(256) oz_split_rows_batched_kernel(const OzRowSplit* J,
                                                                    const int64_t* base, int n) {
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  splitrows_body(J[j], t);
}

int64_t oz_rowexp_tiles(const OzRowSplit& J) { return (J.rows + 255) / 256; }
int64_t oz_splitrows_tiles(const OzRowSplit& J) { return (J.rows + 31) / 32; }
int64_t oz_colexp_tiles(const OzColSplit& J) { return J.cols; }
int64_t oz_splitcols_tiles(const OzColSplit& J) {
  return (int64_t)J.cols * ((J.kpad + kOzColChunk - 1) / kOzColChunk);
}

cudaError_t oz_rowsplit(const OzRowSplit& J, cudaStream_t s) {
  oz_rowexp_kernel<<<(unsigned)oz_rowexp_tiles(J), 256, 0, s>>>(J);
  oz_split_rows_kernel<<<(unsigned)oz_splitrows_tiles(J), 256, 0, s>>>(J);
  count_launches(2);
  return cudaGetLastError();
}
cudaError_t oz_colsplit(const OzColSplit& J, cudaStream_t s) {
  oz_colexp_kernel<<<(unsigned)oz_colexp_tiles(J), 256, 0, s>>>(J);
  oz_split_cols_kernel<<<(unsigned)oz_splitcols_tiles(J), 256, 0, s>>>(J);
  count_launches(2);
  return cudaGetLastError();
}
cudaError_t oz_rowsplit_batched(const OzRowSplit* jobs, const int64_t* base_exp,
                                int64_t tiles_exp, const int64_t* base_split,
                                int64_t tiles_split, int njobs, cudaStream_t s) {
  if (njobs <= 0 || tiles_exp <= 0) return cudaSuccess;
  oz_rowexp_batched_kernel<<<(unsigned)tiles_exp, 256, 0, s>>>(jobs, base_exp, njobs);
  oz_split_rows_batched_kernel<<<(unsigned)tiles_split, 256, 0, s>>>(jobs, base_split, njobs);
  count_launches(2);
  return cudaGetLastError();
}
cudaError_t oz_colsplit_batched(const OzColSplit* jobs, const int64_t* base_exp,
                                int64_t tiles_exp, const int64_t* base_split,
                                int64_t tiles_split, int njobs, cudaStream_t s) {
  if (njobs <= 0 || tiles_exp <= 0) return cudaSuccess;
  oz_colexp_batched_kernel<<<(unsigned)tiles_exp, 256, 0, s>>>(jobs, base_exp, njobs);
  oz_split_cols_batched_kernel<<<(unsigned)tiles_split, 256, 0, s>>>(jobs, base_split, njobs);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// the products (engine: ozaki_tc.cu)
// ---------------------------------------------------------------------------
constexpr int kOzKAlign = 32;  // K of every product padded to a multiple of this

// G[a, c] = sum over K slices s of P_s[a, c] (ascending s), upper triangle
// mirrored to the lower one.  256 entries per CTA.
__device__ __forceinline__ void combine_body(const OzCombine& J, int64_t tile) {
  const int64_t idx = tile * 256 + threadIdx.x;
  const int n = J.n;
  if (idx >= (int64_t)n * n) return;
  const int c = (int)(idx / n), a = (int)(idx - (int64_t)c * n);
  if (a > c) return;
  double s = 0.0;
  for (int k = 0; k < J.nslices; ++k)
    s = __dadd_rn(s, J.P[(int64_t)k * J.slice + (int64_t)c * n + a]);
  J.G[(int64_t)c * J.ldg + a] = s;
  J.G[(int64_t)a * J.ldg + c] = s;
}
__global__ void __launch_bounds__(256) oz_combine_sym_kernel(OzCombine J) {
  combine_body(J, blockIdx.x);
}
__global__ void __launch_bounds__(256) oz_combine_sym_batched_kernel(const OzCombine* J,
                                                                     const int64_t* base, int n) {
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  combine_body(J[j], t);
}
int64_t oz_combine_tiles(const OzCombine& J) { return ((int64_t)J.n * J.n + 255) / 256; }
cudaError_t oz_combine_batched(const OzCombine* jobs, const int64_t* base, int64_t tiles,
                               int njobs, cudaStream_t s) {
  if (njobs <= 0 || tiles <= 0) return cudaSuccess;
  oz_combine_sym_batched_kernel<<<(unsigned)tiles, 256, 0, s>>>(jobs, base, njobs);
  count_launches(1);
  return cudaGetLastError();
}

// Gather: X[:, j] = B[:, cols[j]] for j < k (FP64 copy, column-major).
__global__ void oz_gather_kernel(const double* __restrict__ B, int64_t ldb,
                                 const int64_t* __restrict__ cols, int64_t m, double* X,
                                 int64_t ldx) {
  const int j = blockIdx.y;
  const int64_t src = cols ? cols[j] : j;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)j * ldx + r] = B[src * ldb + r];
}

// W = T^{-1} for upper triangular T (k x k), row by row: row i of W solves
// w^T T = e_i^T left to right (w_j = 0 for j < i), so the computed W has a
// small right residual, |W T - I| <= c u |W| |T| -- the residual that enters
// M_k - M^pre R^sk_11 when line 4 is applied as M_k W.  One warp per row:
// for each j the dot product sum_{i<=t<j} w_t T[t, j] is split over the 32
// lanes (T's column j is contiguous: coalesced) and reduced by a fixed
// shuffle tree; the row being built lives in shared memory.
constexpr int kTrinvWarps = 4;  // at most (one warp per SM sub-partition); fewer when k rows do not fit
__device__ __forceinline__ void trinv_body(const OzTrinv& J, int64_t tile, double* rows) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = J.k;
  const int i = (int)(tile * (int64_t)(blockDim.x >> 5)) + warp;
  if (i >= k) return;
  double* w = rows + (int64_t)warp * k;
  for (int j = i; j < k; ++j) {
    const double* tc = J.T + (int64_t)j * J.ldt;
    double part = 0.0;
    for (int t = i + lane; t < j; t += 32) part = __fma_rn(w[t], tc[t], part);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) part = __dadd_rn(part, __shfl_xor_sync(0xffffffffu, part, off));
    if (lane == 0) w[j] = __ddiv_rn(((i == j) ? 1.0 : 0.0) - part, tc[j]);
    __syncwarp();
  }
  for (int j = lane; j < k; j += 32) J.W[(int64_t)j * J.ldw + i] = j < i ? 0.0 : w[j];
}
__global__ void __launch_bounds__(kTrinvWarps * 32) oz_trinv_rows_kernel(OzTrinv J) {
  extern __shared__ double trinv_rows[];  // [warps][k]
  trinv_body(J, blockIdx.x, trinv_rows);
}
__global__ void __launch_bounds__(kTrinvWarps * 32)
    oz_trinv_rows_batched_kernel(const OzTrinv* J, const int64_t* base, int n) {
  extern __shared__ double trinv_rows[];  // [warps][max k]
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  trinv_body(J[j], t, trinv_rows);
}
// A single problem's W: one CTA of kTrinvRowThreads threads per row i,
// right-looking.  Thread q owns the columns j = i + q + kTrinvRowThreads u
// and keeps their running sums s_j = [j = i] - sum_{t<j} w_t T[t, j] in
// shared memory.  At step t every thread adds -w_t T[t, j] to its columns
// j > t; the owner of column t+1 does its own entry first and divides it by
// T[t+1, t+1] at once, so each step costs one division and one block barrier
// (instead of a warp's dot product, shuffle tree and division), and the
// other threads' updates run beside that division.  Each w_j solves
// w T = e_i left to right, as trinv_body's rows do (the sums in ascending t,
// one fma per term), so W has the same small right residual.
constexpr int kTrinvRowThreads = 128;
constexpr int kTrinvRowMaxK = 200 * 1024 / 8;  // the row's sums in shared memory
__device__ __forceinline__ void trinv_row_body(const OzTrinv& J, int i, double* trinv_sums) {
  __shared__ double wb[2];  // w_t, by step parity
  const int k = J.k;
  if (i >= k) return;
  const int q = threadIdx.x, nt = blockDim.x;
  const double* T = J.T;
  const int64_t ldt = J.ldt;
  double* s = trinv_sums;
  for (int j = i + q; j < k; j += nt) s[j] = j == i ? 1.0 : 0.0;
  __syncthreads();
  if (q == 0) {
    const double w = __ddiv_rn(s[i], __ldg(T + (int64_t)i * ldt + i));
    s[i] = w;
    wb[i & 1] = w;
  }
  __syncthreads();
  for (int t = i; t + 1 < k; ++t) {
    const double w = wb[t & 1];
    const int own = (t + 1 - i) % nt;  // the thread owning column t+1
    if (q == own) {
      const int j = t + 1;
      const double v = __fma_rn(-w, __ldg(T + (int64_t)j * ldt + t), s[j]);
      const double w1 = __ddiv_rn(v, __ldg(T + (int64_t)j * ldt + j));
      s[j] = w1;
      wb[j & 1] = w1;
    }
    // this thread's columns j > t+1
    int j = i + q;
    if (j <= t + 1) j += ((t + 1 - j) / nt + 1) * nt;
    for (; j < k; j += nt) s[j] = __fma_rn(-w, __ldg(T + (int64_t)j * ldt + t), s[j]);
    __syncthreads();
  }
  for (int j = q; j < k; j += nt) J.W[(int64_t)j * J.ldw + i] = j < i ? 0.0 : s[j];
}
__global__ void __launch_bounds__(kTrinvRowThreads) oz_trinv_row_kernel(OzTrinv J) {
  extern __shared__ double trinv_sums[];  // [k]: s_j at index j (j >= i)
  trinv_row_body(J, blockIdx.x, trinv_sums);
}
// batched: CTA -> (job, row) through the prefix table of the jobs' k
__global__ void __launch_bounds__(kTrinvRowThreads)
    oz_trinv_row_batched_kernel(const OzTrinv* J, const int64_t* base, int n) {
  extern __shared__ double trinv_sums[];  // [max k]
  int64_t t;
  const int j = find_problem(base, n, blockIdx.x, &t);
  trinv_row_body(J[j], (int)t, trinv_sums);
}
bool oz_trinv_row_mode(int kmax) { return kmax <= kTrinvRowMaxK; }

// one row of W per warp in shared memory: as many warps as fit 200 KB
int oz_trinv_warps(int kmax) {
  int warps = (int)(200 * 1024 / ((int64_t)kmax * (int64_t)sizeof(double)));
  return warps < 1 ? 1 : (warps > kTrinvWarps ? kTrinvWarps : warps);
}
int64_t oz_trinv_tiles(const OzTrinv& J, int warps) { return (J.k + warps - 1) / warps; }
static cudaError_t trinv_smem_attr(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return raise_smem_limit(fn, bytes);
}
cudaError_t oz_trinv(const OzTrinv& J, cudaStream_t s) {
  if (J.k <= 0) return cudaSuccess;
  const size_t smem = (size_t)J.k * sizeof(double);
  if (oz_trinv_row_mode(J.k)) {  // one CTA per row
    cudaError_t e = trinv_smem_attr((const void*)oz_trinv_row_kernel, smem);
    if (e != cudaSuccess) return e;
    oz_trinv_row_kernel<<<(unsigned)J.k, kTrinvRowThreads, smem, s>>>(J);
    count_launches(1);
    return cudaGetLastError();
  }
  const int warps = oz_trinv_warps(J.k);
  const size_t smem_w = (size_t)warps * J.k * sizeof(double);
  cudaError_t e = trinv_smem_attr((const void*)oz_trinv_rows_kernel, smem_w);
  if (e != cudaSuccess) return e;
  oz_trinv_rows_kernel<<<(unsigned)oz_trinv_tiles(J, warps), warps * 32, smem_w, s>>>(J);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t oz_trinv_batched(const OzTrinv* jobs, const int64_t* base, int64_t tiles, int njobs,
                             int warps, int kmax, cudaStream_t s) {
  if (njobs <= 0 || tiles <= 0) return cudaSuccess;
  if (oz_trinv_row_mode(kmax)) {  // one CTA per row (the caller's tiles: k per job)
    const size_t smem_r = (size_t)kmax * sizeof(double);
    cudaError_t e = trinv_smem_attr((const void*)oz_trinv_row_batched_kernel, smem_r);
    if (e != cudaSuccess) return e;
    oz_trinv_row_batched_kernel<<<(unsigned)tiles, kTrinvRowThreads, smem_r, s>>>(jobs, base, njobs);
    count_launches(1);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)warps * kmax * sizeof(double);
  cudaError_t e = trinv_smem_attr((const void*)oz_trinv_rows_batched_kernel, smem);
  if (e != cudaSuccess) return e;
  oz_trinv_rows_batched_kernel<<<(unsigned)tiles, warps * 32, smem, s>>>(jobs, base, njobs);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int64_t oz_plane_bytes(int64_t rows, int64_t kpad) {
  return align256(rows * kpad * (int64_t)sizeof(__nv_bfloat16));
}

cudaError_t oz_gemm_launch(const OzGemm& G, cudaStream_t s) { return oz_gemm_tc_launch(G, s); }

// Number of K slices for `active` output tiles over `chunks` 1024-term K
// chunks: at least two waves of one CTA per SM (the engine's residency), and
// the last wave at least 90% full when possible.
static int64_t choose_slices(int64_t chunks, int64_t active) {
  const int64_t slots = 152;
  int64_t nslices = 1;
  double best = -1.0;
  for (int64_t ns = 1; ns <= chunks && ns <= 4096; ++ns) {
    const int64_t per = (chunks + ns - 1) / ns;   // chunks per slice
    const int64_t real = (chunks + per - 1) / per;  // slices actually used
    const int64_t ctas = active * real;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (ctas >= 2 * slots && eff >= 0.9) { nslices = real; best = eff; break; }
    if (eff > best) { best = eff; nslices = real; }
  }
  return nslices;
}

// Gram: G = X^T X (k x k) from X (m x k).
int64_t oz_gram_workspace(int64_t m, int k, int64_t* nslices_out) {
  const int64_t kpad = round_up(m, kOzChunk);
  const int64_t chunks = kpad / kOzChunk;
  // tiles the upper-triangle launch keeps (not strictly below the diagonal)
  // (tile shape of the tensor-core engine: 128 x 128)
  const int64_t tile = 128;
  int64_t active = 0;
  for (int64_t tn = 0; tn < (k + tile - 1) / tile; ++tn)
    for (int64_t tm = 0; tm < (k + tile - 1) / tile; ++tm)
      if (tm * tile < tn * tile + tile) ++active;
  const int64_t nslices = choose_slices(chunks, active);
  if (nslices_out) *nslices_out = nslices;
  return (int64_t)kOzDigits * oz_plane_bytes(k, kpad) + align256((int64_t)k * 4) +
         align256(nslices * (int64_t)k * k * 8);
}

int64_t oz_gram_slices(int64_t m, int k) {
  int64_t ns = 1;
  oz_gram_workspace(m, k, &ns);
  return ns;
}

cudaError_t oz_gram(int64_t m, int k, const double* X, int64_t ldx, double* Gm, int64_t ldg,
                    void* work, cudaStream_t s, int* status) {
  int64_t nslices = 1;
  oz_gram_workspace(m, k, &nslices);
  const int64_t kpad = round_up(m, kOzChunk);
  char* w = (char*)work;
  __nv_bfloat16* D = (__nv_bfloat16*)w;
  const int64_t plane = (int64_t)k * kpad;
  w += (int64_t)kOzDigits * oz_plane_bytes(k, kpad);
  int* e = (int*)w;
  w += align256((int64_t)k * 4);
  double* P = (double*)w;
  const OzColSplit cs{X, ldx, m, k, kpad, e, D, plane, kOzChunk};
  cudaError_t err0 = oz_colsplit(cs, s);
  if (err0 != cudaSuccess) return err0;
  OzGemm G{};
  G.M = k; G.N = k; G.Kpad = kpad;
  G.kslice = ((kpad / kOzChunk + nslices - 1) / nslices) * kOzChunk;
  G.A = D; G.a_plane = plane; G.B = D; G.b_plane = plane;
  G.a_kblk = kOzChunk; G.b_kblk = kOzChunk;
  G.ea = e; G.eb = e;
  G.C = P; G.ldc = k; G.c_slice = (int64_t)k * k;
  G.mode = kOzStore; G.upper_only = 1;
  G.err = status;
  cudaError_t err = oz_gemm_launch(G, s);
  if (err != cudaSuccess) return err;
  const int64_t ns = (kpad + G.kslice - 1) / G.kslice;
  const OzCombine cb{P, G.c_slice, (int)ns, k, Gm, ldg};
  oz_combine_sym_kernel<<<(unsigned)oz_combine_tiles(cb), 256, 0, s>>>(cb);
  count_launches(1);
  return cudaGetLastError();
}

// C = X^T Y (ka x kb) from X (m x ka) and Y (m x kb): the Gram's K-sliced
// product with two operands and every output tile (line 1 with a dense
// operator S: X = S^T).  Partial results per K slice are added in ascending
// slice order (oz_combine_kernel).
__global__ void __launch_bounds__(256) oz_combine_kernel(const double* P, int64_t slice,
                                                         int nslices, int ka, int kb, double* C,
                                                         int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= (int64_t)ka * kb) return;
  const int c = (int)(idx / ka), a = (int)(idx - (int64_t)c * ka);
  double v = 0.0;
  for (int q = 0; q < nslices; ++q) v = __dadd_rn(v, P[(int64_t)q * slice + idx]);
  C[(int64_t)c * ldc + a] = v;
}

int64_t oz_gemm_tn_workspace(int64_t m, int ka, int kb, int64_t* nslices_out) {
  const int64_t kpad = round_up(m, kOzChunk);
  const int64_t tiles = (int64_t)((ka + 127) / 128) * ((kb + 127) / 128);
  const int64_t nslices = choose_slices(kpad / kOzChunk, tiles);
  if (nslices_out) *nslices_out = nslices;
  return (int64_t)kOzDigits * (oz_plane_bytes(ka, kpad) + oz_plane_bytes(kb, kpad)) +
         align256((int64_t)ka * 4) + align256((int64_t)kb * 4) +
         align256(nslices * (int64_t)ka * kb * 8);
}

cudaError_t oz_gemm_tn(int64_t m, int ka, int kb, const double* X, int64_t ldx, const double* Y,
                       int64_t ldy, double* Cm, int64_t ldc, void* work, cudaStream_t s,
                       int* status) {
  int64_t nslices = 1;
  oz_gemm_tn_workspace(m, ka, kb, &nslices);
  const int64_t kpad = round_up(m, kOzChunk);
  char* w = (char*)work;
  __nv_bfloat16* DX = (__nv_bfloat16*)w;
  const int64_t px = (int64_t)ka * kpad;
  w += (int64_t)kOzDigits * oz_plane_bytes(ka, kpad);
  __nv_bfloat16* DY = (__nv_bfloat16*)w;
  const int64_t py = (int64_t)kb * kpad;
  w += (int64_t)kOzDigits * oz_plane_bytes(kb, kpad);
  int* ex = (int*)w;
  w += align256((int64_t)ka * 4);
  int* ey = (int*)w;
  w += align256((int64_t)kb * 4);
  double* P = (double*)w;
  cudaError_t e = oz_colsplit(OzColSplit{X, ldx, m, ka, kpad, ex, DX, px, kOzChunk}, s);
  if (e == cudaSuccess) e = oz_colsplit(OzColSplit{Y, ldy, m, kb, kpad, ey, DY, py, kOzChunk}, s);
  if (e != cudaSuccess) return e;
  OzGemm G{};
  G.M = ka; G.N = kb; G.Kpad = kpad;
  G.kslice = ((kpad / kOzChunk + nslices - 1) / nslices) * kOzChunk;
  G.A = DX; G.a_plane = px; G.B = DY; G.b_plane = py;
  G.a_kblk = kOzChunk; G.b_kblk = kOzChunk;
  G.ea = ex; G.eb = ey;
  G.C = P; G.ldc = ka; G.c_slice = (int64_t)ka * kb;
  G.mode = kOzStore; G.upper_only = 0;
  G.err = status;
  e = oz_gemm_launch(G, s);
  if (e != cudaSuccess) return e;
  const int ns = (int)((kpad + G.kslice - 1) / G.kslice);
  const unsigned grid = (unsigned)(((int64_t)ka * kb + 255) / 256);
  oz_combine_kernel<<<grid, 256, 0, s>>>(P, G.c_slice, ns, ka, kb, Cm, ldc);
  count_launches(1);
  return cudaGetLastError();
}

// TRSM: X = B[:, cols] T^{-1} (X m x k), recursive halving down to blocks of
// kOzTrsmNB columns: X[:, a:b] is solved as X[:, a:h] first, then
// X[:, h:b] -= X[:, a:h] T[a:h, h:b] as one split-BF16 product, then
// X[:, h:b]; the kOzTrsmNB-column diagonal blocks are solved in place by the
// FP64 row-wise substitution kernel.  Backward stable for any T: every
// update is an FP64-accurate product and every diagonal solve is a
// substitution.
__global__ void oz_widths_kernel(int k, int nb, int64_t* widths, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i * nb < k) widths[i] = min(nb, k - i * nb);
  if (i == 0) *status = kOk;
}

int64_t oz_trsm_workspace(int64_t m, int k) {
  const int64_t kp = round_up(k, kOzKAlign);
  const int64_t big = kp > 1024 ? kp : 1024;
  return (int64_t)kOzDigits * oz_plane_bytes(m, big) +  // row planes of X[:, a:h]
         (int64_t)kOzDigits * oz_plane_bytes(k, big) +  // column planes of T blocks
         align256(m * 4) + align256((int64_t)k * 4) +  // exponents
         align256(((int64_t)k / kOzTrsmNB + 2) * 8) + 256;  // block widths, status
}

namespace {
struct TrsmCtx {
  int64_t m;
  int k;
  double* X;
  int64_t ldx;
  const double* T;
  int64_t ldt;
  __nv_bfloat16* DA;
  __nv_bfloat16* DB;
  int* ea;
  int* eb;
  int64_t* widths;
  int* status;
  int* err;  // caller's status word (or null) for engine timeouts
};

void carve_trsm(TrsmCtx& c, int64_t m, int k, void* work) {
  const int64_t kp = round_up(k, kOzKAlign);
  const int64_t big = kp > 1024 ? kp : 1024;
  char* w = (char*)work;
  c.DA = (__nv_bfloat16*)w; w += (int64_t)kOzDigits * oz_plane_bytes(m, big);
  c.DB = (__nv_bfloat16*)w; w += (int64_t)kOzDigits * oz_plane_bytes(k, big);
  c.ea = (int*)w; w += align256(m * 4);
  c.eb = (int*)w; w += align256((int64_t)k * 4);
  c.widths = (int64_t*)w; w += align256(((int64_t)k / kOzTrsmNB + 2) * 8);
  c.status = (int*)w;
}

// C[:, 0:n] (m x n, ld ldc) op= Xs[:, map[0:kk]] * Ts (kk x n) (identity map
// when map is null); mode store/sub.
// ts_ready (or null): an event the column operand Ts waits for (it may be
// produced on another stream while the row operand is split).
cudaError_t oz_mul(const TrsmCtx& c, const double* Xs, int64_t ldxs, const int64_t* map, int kk,
                   const double* Ts, int64_t ldts, int n, double* C, int64_t ldc, int mode,
                   cudaStream_t s, cudaEvent_t ts_ready = nullptr) {
  const int64_t kpad = round_up(kk, kOzKAlign);
  const OzRowSplit rs{Xs, ldxs, map, c.m, kk, kpad, c.ea, c.DA, c.m * kpad};
  const OzColSplit cs{Ts, ldts, kk, n, kpad, c.eb, c.DB, (int64_t)n * kpad};
  cudaError_t e0 = oz_rowsplit(rs, s);
  if (e0 == cudaSuccess && ts_ready) e0 = cudaStreamWaitEvent(s, ts_ready, 0);
  if (e0 == cudaSuccess) e0 = oz_colsplit(cs, s);
  if (e0 != cudaSuccess) return e0;
  OzGemm G{};
  G.M = c.m; G.N = n; G.Kpad = kpad; G.kslice = kpad;
  G.A = c.DA; G.a_plane = c.m * kpad; G.B = c.DB; G.b_plane = (int64_t)n * kpad;
  G.ea = c.ea; G.eb = c.eb; G.C = C; G.ldc = ldc; G.c_slice = 0;
  G.mode = mode; G.upper_only = 0;
  G.err = c.err;
  return oz_gemm_launch(G, s);
}

cudaError_t solve(const TrsmCtx& c, int a, int b, cudaStream_t s) {
  cudaError_t e;
  if (b - a <= kOzTrsmNB) {
    // diagonal block by FP64 row-wise substitution, in place (the same
    // kernel and arithmetic as the FP64 mode's TRSM)
    return launch_trsm_rut(c.m, b - a, c.widths + a / kOzTrsmNB, c.X + (int64_t)a * c.ldx, c.ldx,
                           nullptr, c.T + (int64_t)a * c.ldt + a, c.ldt,
                           c.X + (int64_t)a * c.ldx, c.ldx, c.status, s);
  }
  int h = a + ((b - a) / 2 + kOzTrsmNB - 1) / kOzTrsmNB * kOzTrsmNB;
  if (h >= b) h = b - kOzTrsmNB;
  if ((e = solve(c, a, h, s)) != cudaSuccess) return e;
  // X[:, h:b] -= X[:, a:h] T[a:h, h:b]
  if ((e = oz_mul(c, c.X + (int64_t)a * c.ldx, c.ldx, nullptr, h - a,
                  c.T + (int64_t)h * c.ldt + a, c.ldt, b - h, c.X + (int64_t)h * c.ldx, c.ldx,
                  kOzSub, s)) != cudaSuccess)
    return e;
  return solve(c, h, b, s);
}
}  // namespace

cudaError_t oz_trsm(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                    const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                    cudaStream_t s, int* status) {
  TrsmCtx c{};
  c.m = m; c.k = k; c.X = X; c.ldx = ldx; c.T = T; c.ldt = ldt;
  carve_trsm(c, m, k, work);
  c.err = status;
  if (B != X || cols) {
    dim3 g((unsigned)min64((m + 255) / 256, 256), (unsigned)k);
    oz_gather_kernel<<<g, 256, 0, s>>>(B, ldb, cols, m, X, ldx);
    count_launches(1);
  }
  const int nblk = (k + kOzTrsmNB - 1) / kOzTrsmNB;
  oz_widths_kernel<<<(nblk + 127) / 128, 128, 0, s>>>(k, kOzTrsmNB, c.widths, c.status);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return solve(c, 0, k, s);
}

int64_t oz_trsm_inv_workspace(int64_t m, int k) {
  return oz_trsm_workspace(m, k) + align256((int64_t)k * k * 8);
}

// X := B[:, cols] T^{-1} as one split-BF16 product with W = T^{-1} computed
// row by row in FP64 (small right residual |W T - I|).  Accurate when that
// residual times the row grading of T is small: for R^pre (condition near 1,
// Theorem 3) and for the row-graded R^sk of a max-norm QRCP (R = D U with
// |U_ij| <= 1 above a unit diagonal), where |W||T| = |U^{-1}||U|.
cudaError_t oz_trsm_inv(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                        const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                        cudaStream_t s, int* status, const OzSide* side) {
  TrsmCtx c{};
  c.m = m; c.k = k; c.X = X; c.ldx = ldx; c.T = T; c.ldt = ldt;
  carve_trsm(c, m, k, work);
  c.err = status;
  double* W = (double*)((char*)work + oz_trsm_workspace(m, k));
  const OzTrinv ti{T, ldt, k, W, k};
  cudaError_t e;
  cudaEvent_t w_ready = nullptr;
  if (side) {
    // W = T^{-1} (latency-bound, a few CTAs) on the side stream while the
    // row operand is split on s (HBM-bound): disjoint buffers
    e = cudaEventRecord(side->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side->stream, side->fork, 0);
    if (e == cudaSuccess) e = oz_trinv(ti, side->stream);
    if (e == cudaSuccess) e = cudaEventRecord(side->join, side->stream);
    w_ready = side->join;
  } else {
    e = oz_trinv(ti, s);
  }
  if (e != cudaSuccess) return e;
  // the split reads B[:, cols] (the gather is fused into it) before the
  // product writes X (separate planes, so X may be B)
  return oz_mul(c, B, ldb, cols, k, W, k, k, X, ldx, kOzStore, s, w_ready);
}

}  // namespace cqrrpt
