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
// pairs with p + q <= 9 are kept (36 BF16 products, taken level by level,
// level s = p + q); the dropped levels are below 9 * 2^-56 relative to the
// scales.  Each digit product is an integer of magnitude < 2^14, so an FP32
// tensor-core accumulation of up to 1024 such terms is exact.  After every
// chunk of at most 1024 K-terms the FP32 accumulator is converted exactly to
// an integer and added to a 64-bit integer accumulator of the level (exact);
// when a level is complete its integer sum T_s (< 2^53) is converted exactly
// and added, scaled by 2^(-7s), to an FP64 accumulator.  The roundings are
// those eight FP64 additions and the final scaling.  No FP64 arithmetic runs
// in the inner loop (the FP64 pipe is scarce on GB300).
//
// The tensor-core engine is warp-level mma.sync m16n8k16 (bf16 x bf16 ->
// f32): CTA tile 64 x 128, 8 warps of 32 x 32, K staged 32 at a time through
// a 4-stage cp.async pipeline, ldmatrix fragment loads double-buffered over
// the two k16 steps of a stage; the FP64 accumulators of the tile live in
// shared memory.  All operands are "K-contiguous": A is stored as M rows of K
// digits, B as N rows of K digits.
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

// e[r] for every row r over columns [0, cols) of X.
__global__ void oz_rowexp_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int cols,
                                 int* __restrict__ e) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double mx = 0.0;
  for (int c = 0; c < cols; ++c) mx = fmax(mx, fabs(X[(int64_t)c * ldx + r]));
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
// columns, padded to kpad), scale e[r].  32 x 32 tiles transposed through
// shared memory so that both the reads of X and the writes of D coalesce.
__global__ void oz_split_rows_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows,
                                     int cols, int64_t kpad, const int* __restrict__ e,
                                     __nv_bfloat16* __restrict__ D, int64_t plane) {
  __shared__ double tile[32][33];
  const int64_t r0 = blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + tx;
    const int k = k0 + j;
    tile[j][tx] = (r < rows && k < cols) ? X[(int64_t)k * ldx + r] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j;
    const int k = k0 + tx;
    if (r < rows && k < kpad) digits8(tile[tx][j], e[r], D + r * kpad + k, plane);
  }
}

// ---------------------------------------------------------------------------
// the GEMM engine
// ---------------------------------------------------------------------------
constexpr int kBM = 64, kBN = 128, kBK = 32, kStages = 3, kPad = 8;
constexpr int kLdS = kBK + kPad;  // shared row stride (bf16)
constexpr int kLdC = kBN + 1;     // FP64 tile row stride (doubles)
constexpr size_t kOzSmem = (size_t)kStages * (kBM + kBN) * kLdS * 2 + (size_t)kBM * kLdC * 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                            const void* smem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// pair index -> (p, q) in level order: level s = p + q = 2, 3, ..., 9; inside
// a level p ascends.  Level s starts at index (s-2)(s-1)/2.
__device__ __forceinline__ void pair_of(int idx, int& p, int& q, int& s, bool& level_end) {
  s = 2;
  while ((s - 1) * s / 2 <= idx) ++s;
  const int first = (s - 2) * (s - 1) / 2;
  p = idx - first + 1;
  q = s - p;
  level_end = (p == s - 1);
}

struct Frag {
  unsigned a[2][4];
  unsigned b[4][2];
};

__device__ __forceinline__ void load_frags(Frag& f, const __nv_bfloat16 (*As)[kLdS],
                                           const __nv_bfloat16 (*Bs)[kLdS], int wm, int wn,
                                           int kk, int lane) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int row = wm * 32 + i * 16 + (lane & 15);
    const int col = kk + (lane >> 4) * 8;
    ldmatrix_x4(f.a[i][0], f.a[i][1], f.a[i][2], f.a[i][3], &As[row][col]);
  }
#pragma unroll
  for (int j2 = 0; j2 < 2; ++j2) {
    const int row = wn * 32 + j2 * 16 + (lane & 7) + ((lane >> 4) << 3);
    const int col = kk + ((lane >> 3) & 1) * 8;
    unsigned r0, r1, r2, r3;
    ldmatrix_x4(r0, r1, r2, r3, &Bs[row][col]);
    f.b[2 * j2][0] = r0; f.b[2 * j2][1] = r1;
    f.b[2 * j2 + 1][0] = r2; f.b[2 * j2 + 1][1] = r3;
  }
}

__global__ void __launch_bounds__(256, 2) oz_gemm_kernel(OzGemm G) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  typedef __nv_bfloat16 RowA[kLdS];
  RowA* As = (RowA*)oz_smem;                                  // [kStages * kBM]
  RowA* Bs = (RowA*)(oz_smem + (size_t)kStages * kBM * kLdS * 2);  // [kStages * kBN]
  double* Cs = (double*)(oz_smem + (size_t)kStages * (kBM + kBN) * kLdS * 2);  // [kBM][kLdC]

  const int tiles_m = (int)((G.M + kBM - 1) / kBM);
  const int tiles_n = (G.N + kBN - 1) / kBN;
  const int tile = blockIdx.x;
  const int tm = tile % tiles_m, tn = (tile / tiles_m) % tiles_n;
  const int ks = tile / (tiles_m * tiles_n);  // K slice
  const int64_t m0 = (int64_t)tm * kBM;
  const int n0 = tn * kBN;
  if (G.upper_only && m0 >= n0 + kBN) return;
  const int64_t kbeg = (int64_t)ks * G.kslice;
  const int64_t kend = min64(kbeg + G.kslice, G.Kpad);
  if (kbeg >= kend) return;
  const int nstage_k = (int)((kend - kbeg) / kBK);  // Kpad and kslice are multiples of kBK
  const int total = nstage_k * kOzPairs;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps, each 32 x 32
  for (int e = threadIdx.x; e < kBM * kLdC; e += 256) Cs[e] = 0.0;
  float acc[2][4][4];
  long long lev[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 4; ++v) { acc[i][j][v] = 0.f; lev[i][j][v] = 0; }

  auto load_stage = [&](int it, int buf) {
    int p, q, s;
    bool le;
    pair_of(it / nstage_k, p, q, s, le);
    const int64_t k0 = kbeg + (int64_t)(it % nstage_k) * kBK;
    const __nv_bfloat16* Ap = G.A + (int64_t)(p - 1) * G.a_plane;
    const __nv_bfloat16* Bq = G.B + (int64_t)(q - 1) * G.b_plane;
    {  // A: 64 rows x 32 k = 256 chunks of 16 B
      const int row = threadIdx.x >> 2, ch = threadIdx.x & 3;
      const int64_t gm = m0 + row;
      const bool ok = gm < G.M;
      cp_async16(&As[buf * kBM + row][ch * 8], Ap + (ok ? gm : 0) * G.Kpad + k0 + ch * 8, ok);
    }
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {  // B: 128 rows x 32 k = 512 chunks
      const int idx = threadIdx.x + rep * 256;
      const int row = idx >> 2, ch = idx & 3;
      const int gn = n0 + row;
      const bool ok = gn < G.N;
      cp_async16(&Bs[buf * kBN + row][ch * 8], Bq + (int64_t)(ok ? gn : 0) * G.Kpad + k0 + ch * 8,
                 ok);
    }
  };

  // prologue
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < total) load_stage(s, s);
    cp_async_commit();
  }
  const int g = lane >> 2, t4 = lane & 3;
  for (int it = 0; it < total; ++it) {
    cp_async_wait<kStages - 2>();
    __syncthreads();
    const int nxt = it + kStages - 1;
    if (nxt < total) load_stage(nxt, nxt % kStages);
    cp_async_commit();
    const int buf = it % kStages;
    const RowA* Ab = As + buf * kBM;
    const RowA* Bb = Bs + buf * kBN;
    Frag f0, f1;
    load_frags(f0, Ab, Bb, wm, wn, 0, lane);
    load_frags(f1, Ab, Bb, wm, wn, 16, lane);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], f0.a[i], f0.b[j]);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], f1.a[i], f1.b[j]);
    // FP32 -> exact integer after every chunk of kOzChunk K-terms and at the
    // end of a pair; integer level sum -> FP64 tile at the end of a level
    const int sk = it % nstage_k;
    const bool pair_end = (sk == nstage_k - 1);
    if (pair_end || ((sk + 1) * kBK) % kOzChunk == 0) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            lev[i][j][v] += (long long)__float2int_rn(acc[i][j][v]);
            acc[i][j][v] = 0.f;
          }
      int p, q, s;
      bool level_end;
      pair_of(it / nstage_k, p, q, s, level_end);
      if (pair_end && level_end) {
        const double scale = ldexp(1.0, -7 * s);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int row = wm * 32 + i * 16 + g + ((v >> 1) << 3);
              const int col = wn * 32 + j * 8 + 2 * t4 + (v & 1);
              double* c = &Cs[row * kLdC + col];
              *c = __fma_rn((double)lev[i][j][v], scale, *c);
              lev[i][j][v] = 0;
            }
      }
    }
  }
  cp_async_wait<0>();

  // epilogue: scale by 2^(ea_i + eb_j) and store / subtract / write partial
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int lr = wm * 32 + i * 16 + g + ((v >> 1) << 3);
        const int lc = wn * 32 + j * 8 + 2 * t4 + (v & 1);
        const int64_t row = m0 + lr;
        const int col = n0 + lc;
        if (row >= G.M || col >= G.N) continue;
        const double val = ldexp(Cs[lr * kLdC + lc], G.ea[row] + G.eb[col]);
        double* c = G.C + (int64_t)ks * G.c_slice + (int64_t)col * G.ldc + row;
        if (G.mode == kOzStore) *c = val;
        else *c = __dsub_rn(*c, val);
      }
}

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
// M_k - M^pre R^sk_11 when line 4 is applied as M_k W.  One thread per row.
__global__ void oz_trinv_rows_kernel(const double* __restrict__ T, int64_t ldt, int k,
                                     double* __restrict__ W, int64_t ldw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  for (int j = 0; j < i; ++j) W[(int64_t)j * ldw + i] = 0.0;
  for (int j = i; j < k; ++j) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int t = i; t < j; ++t)
      s = __fma_rn(-W[(int64_t)t * ldw + i], T[(int64_t)j * ldt + t], s);
    W[(int64_t)j * ldw + i] = __ddiv_rn(s, T[(int64_t)j * ldt + j]);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int64_t oz_plane_bytes(int64_t rows, int64_t kpad) {
  return align256(rows * kpad * (int64_t)sizeof(__nv_bfloat16));
}

cudaError_t oz_gemm_launch(const OzGemm& G, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t tiles_m = (G.M + kBM - 1) / kBM;
  const int64_t tiles_n = (G.N + kBN - 1) / kBN;
  const int64_t nks = (G.Kpad + G.kslice - 1) / G.kslice;
  oz_gemm_kernel<<<(unsigned)(tiles_m * tiles_n * nks), 256, kOzSmem, s>>>(G);
  count_launches(1);
  return cudaGetLastError();
}

// Gram: G = X^T X (k x k) from X (m x k).
int64_t oz_gram_workspace(int64_t m, int k, int64_t* nslices_out) {
  const int64_t kpad = round_up(m, kOzChunk);
  const int64_t chunks = kpad / kOzChunk;
  // tiles the upper-triangle launch keeps (not strictly below the diagonal)
  int64_t active = 0;
  for (int64_t tn = 0; tn < (k + kBN - 1) / kBN; ++tn)
    for (int64_t tm = 0; tm < (k + kBM - 1) / kBM; ++tm)
      if (tm * kBM < tn * kBN + kBN) ++active;
  // number of K slices: at least two waves of 2 CTAs per SM, and the last
  // wave at least 90% full when possible
  const int64_t slots = 152 * 2;
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
                    void* work, cudaStream_t s) {
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
  const int64_t kp = round_up(k, kBK);
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
};

void carve_trsm(TrsmCtx& c, int64_t m, int k, void* work) {
  const int64_t kp = round_up(k, kBK);
  const int64_t big = kp > 1024 ? kp : 1024;
  char* w = (char*)work;
  c.DA = (__nv_bfloat16*)w; w += (int64_t)kOzDigits * oz_plane_bytes(m, big);
  c.DB = (__nv_bfloat16*)w; w += (int64_t)kOzDigits * oz_plane_bytes(k, big);
  c.ea = (int*)w; w += align256(m * 4);
  c.eb = (int*)w; w += align256((int64_t)k * 4);
  c.widths = (int64_t*)w; w += align256(((int64_t)k / kOzTrsmNB + 2) * 8);
  c.status = (int*)w;
}

// C[:, 0:n] (m x n, ld ldc) op= Xs[:, 0:kk] * Ts (kk x n); mode store/sub.
cudaError_t oz_mul(const TrsmCtx& c, const double* Xs, int64_t ldxs, int kk, const double* Ts,
                   int64_t ldts, int n, double* C, int64_t ldc, int mode, cudaStream_t s) {
  const int64_t kpad = round_up(kk, kBK);
  oz_rowexp_kernel<<<(unsigned)((c.m + 255) / 256), 256, 0, s>>>(Xs, ldxs, c.m, kk, c.ea);
  dim3 gr((unsigned)((c.m + 31) / 32), (unsigned)((kpad + 31) / 32));
  oz_split_rows_kernel<<<gr, 256, 0, s>>>(Xs, ldxs, c.m, kk, kpad, c.ea, c.DA, c.m * kpad);
  oz_colexp_kernel<<<n, 128, 0, s>>>(Ts, ldts, kk, c.eb);
  dim3 gc((unsigned)((kpad + 255) / 256), (unsigned)n);
  oz_split_cols_kernel<<<gc, 256, 0, s>>>(Ts, ldts, kk, n, kpad, c.eb, c.DB, (int64_t)n * kpad);
  count_launches(4);
  OzGemm G{};
  G.M = c.m; G.N = n; G.Kpad = kpad; G.kslice = kpad;
  G.A = c.DA; G.a_plane = c.m * kpad; G.B = c.DB; G.b_plane = (int64_t)n * kpad;
  G.ea = c.ea; G.eb = c.eb; G.C = C; G.ldc = ldc; G.c_slice = 0;
  G.mode = mode; G.upper_only = 0;
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
  if ((e = oz_mul(c, c.X + (int64_t)a * c.ldx, c.ldx, h - a, c.T + (int64_t)h * c.ldt + a, c.ldt,
                  b - h, c.X + (int64_t)h * c.ldx, c.ldx, kOzSub, s)) != cudaSuccess)
    return e;
  return solve(c, h, b, s);
}
}  // namespace

cudaError_t oz_trsm(int64_t m, int k, const double* B, int64_t ldb, const int64_t* cols,
                    const double* T, int64_t ldt, double* X, int64_t ldx, void* work,
                    cudaStream_t s) {
  TrsmCtx c{};
  c.m = m; c.k = k; c.X = X; c.ldx = ldx; c.T = T; c.ldt = ldt;
  carve_trsm(c, m, k, work);
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
                        cudaStream_t s) {
  TrsmCtx c{};
  c.m = m; c.k = k; c.X = X; c.ldx = ldx; c.T = T; c.ldt = ldt;
  carve_trsm(c, m, k, work);
  double* W = (double*)((char*)work + oz_trsm_workspace(m, k));
  if (B != X || cols) {
    dim3 g((unsigned)min64((m + 255) / 256, 256), (unsigned)k);
    oz_gather_kernel<<<g, 256, 0, s>>>(B, ldb, cols, m, X, ldx);
    count_launches(1);
  }
  oz_trinv_rows_kernel<<<(k + 127) / 128, 128, 0, s>>>(T, ldt, k, W, k);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the split reads X before the product overwrites it (separate planes)
  return oz_mul(c, X, ldx, k, W, k, k, X, ldx, kOzStore, s);
}

}  // namespace cqrrpt
