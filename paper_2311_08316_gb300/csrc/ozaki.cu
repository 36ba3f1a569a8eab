// FP64-accurate matrix products on the BF16 tensor cores by error-free
// digit splitting (the scheme of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012; tensor-core
// use as in Mukunoki, Ozaki, Ogita & Imamura, ICCS 2020).  Used by the
// split-BF16 precision modes for Alg. 2 lines 4, 5 and 7, the O(m n^2) steps
// (the paper's two-roundoff model, Sec. 4.1, lets line 4 run in a
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
// exactly in 64-bit integers and rounded to FP64 twice per entry.  The
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

// e[c] for every column c of X (rows x cols, column-major): scale over the
// column.  One CTA per column.
__global__ void oz_colexp_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows,
                                 int* __restrict__ e) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const double* col = X + (int64_t)c * ldx;
  double mx = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) mx = fmax(mx, fabs(col[r]));
  for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
    e[c] = frexp_exp(mx);
  }
}

// e[r] for every row r over columns [0, cols) of X (column c of X is
// column map[c] of the array when map is given).
__global__ void oz_rowexp_kernel(const double* __restrict__ X, int64_t ldx, const int64_t* map,
                                 int64_t rows, int cols, int* __restrict__ e) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double mx = 0.0;
  for (int c = 0; c < cols; ++c) mx = fmax(mx, fabs(X[(map ? map[c] : (int64_t)c) * ldx + r]));
  e[r] = frexp_exp(mx);
}

// Column operand: digit planes D[p][c][k] of X[k, c] (K = rows, padded to
// kpad with zeros), scale e[c].
__global__ void oz_split_cols_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows,
                                     int cols, int64_t kpad, const int* __restrict__ e,
                                     __nv_bfloat16* __restrict__ D, int64_t plane) {
  const int c = blockIdx.y;
  const int ec = e[c];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < kpad;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x = k < rows ? X[(int64_t)c * ldx + k] : 0.0;
    digits8(x, ec, D + (int64_t)c * kpad + k, plane);
  }
}

// Row operand: digit planes D[p][r][k] of X[r, k] for k in [0, cols) (K =
// columns, padded to kpad; column k is column map[k] of the array when map
// is given), scale e[r].  32 x 32 tiles transposed through shared memory so
// that both the reads of X and the writes of D coalesce.
__global__ void oz_split_rows_kernel(const double* __restrict__ X, int64_t ldx, const int64_t* map,
                                     int64_t rows, int cols, int64_t kpad,
                                     const int* __restrict__ e, __nv_bfloat16* __restrict__ D,
                                     int64_t plane) {
  __shared__ double tile[32][33];
  const int64_t r0 = blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + tx;
    const int k = k0 + j;
    tile[j][tx] = (r < rows && k < cols) ? X[(map ? map[k] : (int64_t)k) * ldx + r] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j;
    const int k = k0 + tx;
    if (r < rows && k < kpad) digits8(tile[tx][j], e[r], D + r * kpad + k, plane);
  }
}

// ---------------------------------------------------------------------------
// the products (engine: ozaki_tc.cu)
// ---------------------------------------------------------------------------
constexpr int kOzKAlign = 32;  // K of every product padded to a multiple of this

// G[a, c] = sum over K slices s of P_s[a, c] (ascending s), upper triangle
// mirrored to the lower one.
__global__ void oz_combine_sym_kernel(const double* __restrict__ P, int64_t slice, int nslices,
                                      int n, double* __restrict__ G, int64_t ldg) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int c = (int)(idx / n), a = (int)(idx - (int64_t)c * n);
  if (a > c) return;
  double s = 0.0;
  for (int k = 0; k < nslices; ++k) s = __dadd_rn(s, P[(int64_t)k * slice + (int64_t)c * n + a]);
  G[(int64_t)c * ldg + a] = s;
  G[(int64_t)a * ldg + c] = s;
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
constexpr int kTrinvWarps = 8;  // at most; fewer when k rows do not fit
__global__ void __launch_bounds__(kTrinvWarps * 32)
    oz_trinv_rows_kernel(const double* __restrict__ T, int64_t ldt, int k, double* __restrict__ W,
                         int64_t ldw) {
  extern __shared__ double trinv_rows[];  // [warps][k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (int)(blockDim.x >> 5) + warp;
  if (i >= k) return;
  double* w = trinv_rows + (int64_t)warp * k;
  for (int j = i; j < k; ++j) {
    const double* tc = T + (int64_t)j * ldt;
    double part = 0.0;
    for (int t = i + lane; t < j; t += 32) part = __fma_rn(w[t], tc[t], part);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) part = __dadd_rn(part, __shfl_xor_sync(0xffffffffu, part, off));
    if (lane == 0) w[j] = __ddiv_rn(((i == j) ? 1.0 : 0.0) - part, tc[j]);
    __syncwarp();
  }
  for (int j = lane; j < k; j += 32) W[(int64_t)j * ldw + i] = j < i ? 0.0 : w[j];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int64_t oz_plane_bytes(int64_t rows, int64_t kpad) {
  return align256(rows * kpad * (int64_t)sizeof(__nv_bfloat16));
}

cudaError_t oz_gemm_launch(const OzGemm& G, cudaStream_t s) { return oz_gemm_tc_launch(G, s); }

// Gram: G = X^T X (k x k) from X (m x k).
int64_t oz_gram_workspace(int64_t m, int k, int64_t* nslices_out) {
  const int64_t kpad = round_up(m, kOzChunk);
  const int64_t chunks = kpad / kOzChunk;
  // tiles the upper-triangle launch keeps (not strictly below the diagonal)
  // (tile shape and residency of the tensor-core engine: 128 x 128, one CTA
  // per SM)
  const int64_t tile = 128;
  int64_t active = 0;
  for (int64_t tn = 0; tn < (k + tile - 1) / tile; ++tn)
    for (int64_t tm = 0; tm < (k + tile - 1) / tile; ++tm)
      if (tm * tile < tn * tile + tile) ++active;
  // number of K slices: at least two waves of one CTA per SM, and the last
  // wave at least 90% full when possible
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
  if (nslices_out) *nslices_out = nslices;
  return (int64_t)kOzDigits * oz_plane_bytes(k, kpad) + align256((int64_t)k * 4) +
         align256(nslices * (int64_t)k * k * 8);
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
  oz_colexp_kernel<<<k, 256, 0, s>>>(X, ldx, m, e);
  dim3 sg((unsigned)min64((kpad + 255) / 256, 1024), (unsigned)k);
  oz_split_cols_kernel<<<sg, 256, 0, s>>>(X, ldx, m, k, kpad, e, D, plane);
  OzGemm G{};
  G.M = k; G.N = k; G.Kpad = kpad;
  G.kslice = ((kpad / kOzChunk + nslices - 1) / nslices) * kOzChunk;
  G.A = D; G.a_plane = plane; G.B = D; G.b_plane = plane;
  G.ea = e; G.eb = e;
  G.C = P; G.ldc = k; G.c_slice = (int64_t)k * k;
  G.mode = kOzStore; G.upper_only = 1;
  G.err = status;
  cudaError_t err = oz_gemm_launch(G, s);
  if (err != cudaSuccess) return err;
  const int64_t ns = (kpad + G.kslice - 1) / G.kslice;
  oz_combine_sym_kernel<<<(unsigned)(((int64_t)k * k + 255) / 256), 256, 0, s>>>(P, G.c_slice, (int)ns,
                                                                                k, Gm, ldg);
  count_launches(3);
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
cudaError_t oz_mul(const TrsmCtx& c, const double* Xs, int64_t ldxs, const int64_t* map, int kk,
                   const double* Ts, int64_t ldts, int n, double* C, int64_t ldc, int mode,
                   cudaStream_t s) {
  const int64_t kpad = round_up(kk, kOzKAlign);
  oz_rowexp_kernel<<<(unsigned)((c.m + 255) / 256), 256, 0, s>>>(Xs, ldxs, map, c.m, kk, c.ea);
  dim3 gr((unsigned)((c.m + 31) / 32), (unsigned)((kpad + 31) / 32));
  oz_split_rows_kernel<<<gr, 256, 0, s>>>(Xs, ldxs, map, c.m, kk, kpad, c.ea, c.DA, c.m * kpad);
  oz_colexp_kernel<<<n, 128, 0, s>>>(Ts, ldts, kk, c.eb);
  dim3 gc((unsigned)((kpad + 255) / 256), (unsigned)n);
  oz_split_cols_kernel<<<gc, 256, 0, s>>>(Ts, ldts, kk, n, kpad, c.eb, c.DB, (int64_t)n * kpad);
  count_launches(4);
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
// Theorem 2) and for the row-graded R^sk of a max-norm QRCP (R = D U with
// |U_ij| <= 1 above a unit diagonal), where |W||T| = |U^{-1}||U|.
cudaError_t oz_trsm_inv(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                        const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                        cudaStream_t s, int* status) {
  TrsmCtx c{};
  c.m = m; c.k = k; c.X = X; c.ldx = ldx; c.T = T; c.ldt = ldt;
  carve_trsm(c, m, k, work);
  c.err = status;
  double* W = (double*)((char*)work + oz_trsm_workspace(m, k));
  // one row of W per warp in shared memory: as many warps as fit 200 KB
  int warps = (int)(200 * 1024 / ((int64_t)k * (int64_t)sizeof(double)));
  warps = warps < 1 ? 1 : (warps > kTrinvWarps ? kTrinvWarps : warps);
  const size_t trinv_smem = (size_t)warps * k * sizeof(double);
  if (trinv_smem > 48 * 1024) {
    cudaError_t ea = cudaFuncSetAttribute(oz_trinv_rows_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)trinv_smem);
    if (ea != cudaSuccess) return ea;
  }
  oz_trinv_rows_kernel<<<(k + warps - 1) / warps, warps * 32, trinv_smem, s>>>(T, ldt, k, W, k);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the split reads B[:, cols] (the gather is fused into it) before the
  // product writes X (separate planes, so X may be B)
  return oz_mul(c, B, ldb, cols, k, W, k, k, X, ldx, kOzStore, s);
}

}  // namespace cqrrpt
