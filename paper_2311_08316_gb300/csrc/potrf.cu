// Alg. 2 line 6: R^pre = chol(G), upper (G = R^T R), with the failure rule
// of Remark 4 (Sec. 3.3): if the pivot of column j is not positive the
// factorisation stops, records fail = j, and the leading j x j block of R is
// the valid factor of G[0:j, 0:j].
//
// Every entry follows the unblocked recurrence
//   R[j, c] = (G[j, c] - sum_{t<j} R[t, j] R[t, c]) / R[j, j],
//   R[j, j] = sqrt(G[j, j] - sum_{t<j} R[t, j]^2),
// each sum in ascending t with one fma per term.  It is evaluated
// right-looking in panels of kCholNB columns, which keeps that order: G is
// used as working storage S and receives the terms t of earlier panels in
// ascending order (update step), the terms of the current panel are added
// by the diagonal-block and panel steps, again in ascending t.
//
// Single problem: three launches per panel (diagonal block, panel rows,
// trailing update); a factor of at most 128 columns runs on one CTA, as a
// batch's problems do.  Inside the diagonal block and the panel the sums run
// right-looking (registers hold every running sum of a column), which keeps
// each entry's ascending-t order but shortens the dependent chain.  Batch: one CTA per problem runs every panel with block
// barriers between the steps; same bodies, same arithmetic.
#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

// Diagonal block [jb, jb + nb) by one warp, lane = column c = jb + lane.
// Right-looking inside the block: lane c keeps the running sums acc[j] of
// its entries (j, c), j <= c, in registers; once row t is final, every sum
// of a later row receives its term -R[t, j] R[t, c] (ascending t, one fma,
// as the recurrence), so the critical path is one square root, one division
// and one fma per row instead of the whole dot product.  Returns false (and
// records sc->fail) on a non-positive pivot.
__device__ __forceinline__ bool potrf_diag_body(int jb, const PotrfDesc& D) {
  DeviceScalars* sc = D.sc;
  const double* S = D.G;
  double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int lane = threadIdx.x & 31;
  const int c = jb + lane;
  const bool mine = lane < nb;
  double acc[kCholNB];
#pragma unroll
  for (int j = 0; j < kCholNB; ++j)
    acc[j] = (mine && j <= lane) ? S[(int64_t)c * lds + jb + j] : 0.0;
#pragma unroll
  for (int t = 0; t < kCholNB; ++t) {
    if (t < nb) {
      const double piv = __shfl_sync(0xffffffffu, acc[t], t);
      if (!(piv > 0.0)) {
        if (lane == 0) sc->fail = jb + t;
        return false;
      }
      const double rd = __dsqrt_rn(piv);
      double rt = 0.0;  // R[jb + t, c]
      if (lane == t) {
        rt = rd;
        R[(int64_t)c * ldr + jb + t] = rd;
      } else if (mine && lane > t) {
        rt = __ddiv_rn(acc[t], rd);
        R[(int64_t)c * ldr + jb + t] = rt;
      }
#pragma unroll
      for (int j = t + 1; j < kCholNB; ++j) {
        const double rtj = __shfl_sync(0xffffffffu, rt, j);  // R[jb + t, jb + j]
        if (mine && j <= lane) acc[j] = __fma_rn(-rtj, rt, acc[j]);
      }
    }
  }
  return true;
}

// Panel rows [jb, jb + nb) of column c >= jb + nb, right-looking as the
// diagonal block: acc[j] holds the running sum of entry (jb + j, c).
__device__ __forceinline__ void potrf_panel_col(int jb, int nb, int c, const PotrfDesc& D) {
  const double* S = D.G;
  double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  double acc[kCholNB];
#pragma unroll
  for (int j = 0; j < kCholNB; ++j) acc[j] = j < nb ? S[(int64_t)c * lds + jb + j] : 0.0;
#pragma unroll
  for (int t = 0; t < kCholNB; ++t) {
    if (t < nb) {
      const double rt = __ddiv_rn(acc[t], R[(int64_t)(jb + t) * ldr + jb + t]);
      R[(int64_t)c * ldr + jb + t] = rt;
#pragma unroll
      for (int j = t + 1; j < kCholNB; ++j)
        if (j < nb) acc[j] = __fma_rn(-R[(int64_t)(jb + j) * ldr + jb + t], rt, acc[j]);
    }
  }
}

// The same as a separate function: inlined into the batched kernel's loop
// the unrolled body lost its register array to local memory.
__device__ __noinline__ void potrf_panel_col_call(int jb, int nb, int c, const PotrfDesc& D) {
  potrf_panel_col(jb, nb, c, D);
}

// Trailing update of S[a, c] (a <= c, both >= jb + nb) by the panel's rows.
__device__ __forceinline__ void potrf_update_elem(int jb, int base, int a, int c,
                                                  const PotrfDesc& D) {
  double* S = D.G;
  const double* R = D.R;
  const int64_t lds = D.ldg, ldr = D.ldr;
  double s = S[(int64_t)c * lds + a];
  for (int t = jb; t < base; ++t) s = __fma_rn(-R[(int64_t)a * ldr + t], R[(int64_t)c * ldr + t], s);
  S[(int64_t)c * lds + a] = s;
}

// ---- single problem: one launch per step ------------------------------------
__global__ void potrf_diag_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  if (jb >= (int)sc->k) return;
  potrf_diag_body(jb, D);
}

__global__ void potrf_panel_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int c = jb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (jb >= k || c >= k) return;
  potrf_panel_col(jb, nb, c, D);
}

__global__ void potrf_update_kernel(int jb, PotrfDesc D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  const int nb = min(kCholNB, k - jb);
  const int base = jb + nb;
  if (jb >= k || base >= k) return;
  const int a = base + blockIdx.y * 16 + threadIdx.y;
  const int c = base + blockIdx.x * 16 + threadIdx.x;
  if (a >= k || c >= k || a > c) return;
  potrf_update_elem(jb, base, a, c, D);
}

// ---- one CTA per problem (a batch, or a small single problem) -----------------
__device__ __forceinline__ void potrf_cta_body(const PotrfDesc& D) {
  DeviceScalars* sc = D.sc;
  __shared__ int go;
  for (int jb = 0; jb < D.kmax; jb += kCholNB) {
    if (threadIdx.x == 0)
      go = (*(volatile int*)&sc->status == kOk && *(volatile int64_t*)&sc->fail < 0 &&
            jb < (int)sc->k);
    __syncthreads();
    if (!go) return;
    const int k = (int)sc->k;
    const int nb = min(kCholNB, k - jb);
    const int base = jb + nb;
    if (threadIdx.x < 32) potrf_diag_body(jb, D);
    __syncthreads();
    if (threadIdx.x == 0) go = (*(volatile int64_t*)&sc->fail < 0);
    __syncthreads();
    if (!go) return;
    for (int c = base + threadIdx.x; c < k; c += blockDim.x) potrf_panel_col_call(jb, nb, c, D);
    __syncthreads();
    const int w = k - base;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int a = base + e / w, c = base + e % w;
      if (a <= c) potrf_update_elem(jb, base, a, c, D);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) potrf_batched_kernel(const PotrfDesc* Dv) {
  potrf_cta_body(Dv[blockIdx.x]);
}

// A small factor (k <= kPotrfSmallMax): one CTA of 1024 threads, fully
// right-looking.  Step t: thread 0 takes R[t, t] = sqrt(S[t, t]) (or records
// the Remark 4 failure at t); the threads divide row t, R[t, c] = S[t, c] /
// R[t, t] for c > t, in parallel; then every trailing entry S[j, c]
// (t < j <= c) receives its term -R[t, j] R[t, c] with one fma.  Each entry
// still receives its terms in ascending t and the same division and square
// root as the recurrence, but every step spreads its work over 32 warps (a
// single warp issues one FP64 instruction per 64 cycles).  S lives in shared
// memory (k <= 64: 32 KB).
constexpr int kPotrfSmallMax = 64;
constexpr int kPotrfSmallThreads = 1024;
__global__ void __launch_bounds__(kPotrfSmallThreads) potrf_small_kernel(PotrfDesc D) {
  __shared__ double S[kPotrfSmallMax * kPotrfSmallMax];  // column-major, ld kPotrfSmallMax
  __shared__ int fail_at;
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk || sc->fail >= 0) return;
  const int k = (int)sc->k;
  if (k <= 0) return;
  const int ld = kPotrfSmallMax;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int c = e / k, j = e - c * k;
    S[c * ld + j] = j <= c ? D.G[(int64_t)c * D.ldg + j] : 0.0;
  }
  __syncthreads();
  // thread 0 takes each pivot's square root one step ahead: at step t, right
  // after the divisions of column t, it applies step t's update to
  // (t+1, t+1) (the same fma the trailing update would) and takes the root,
  // while warps 1.. update the rest of the trailing block
  auto pivot = [&](int t) {  // thread 0: S[t, t] holds the updated pivot
    const double piv = S[t * ld + t];
    if (!(piv > 0.0)) {
      fail_at = t;
    } else {
      const double r = __dsqrt_rn(piv);
      S[t * ld + t] = r;
      D.R[(int64_t)t * D.ldr + t] = r;
    }
  };
  if (threadIdx.x == 0) {
    fail_at = -1;
    pivot(0);
  }
  __syncthreads();
  const int upd_threads = (int)blockDim.x - 32;
  for (int t = 0; t < k; ++t) {
    if (fail_at >= 0) break;  // uniform
    const double rtt = S[t * ld + t];
    // column t's divisions (threads 0 .. k-t-2: warps 0 and 1); warp 0 then
    // signals barrier 1 and thread 0 goes on to the next pivot while warps
    // 1.. (after barrier 1) update the trailing block
    double v1 = 0.0;
    for (int c = t + 1 + (int)threadIdx.x; c < k; c += blockDim.x) {
      const double v = __ddiv_rn(S[c * ld + t], rtt);
      S[c * ld + t] = v;
      D.R[(int64_t)c * D.ldr + t] = v;
      if (c == t + 1) v1 = v;
    }
    if (threadIdx.x < 32) {
      asm volatile("barrier.arrive 1, %0;" ::"r"((int)blockDim.x) : "memory");
      if (threadIdx.x == 0 && t + 1 < k) {  // the next pivot
        const int c = t + 1;
        S[c * ld + c] = __fma_rn(-v1, v1, S[c * ld + c]);
        pivot(c);
      }
    } else {
      asm volatile("barrier.sync 1, %0;" ::"r"((int)blockDim.x) : "memory");
    }
    // trailing update by warps 1..: entries (j, c), t < j <= c < k, but
    // (t+1, t+1), which thread 0 did
    if (threadIdx.x >= 32) {
      const int w = k - 1 - t;
      for (int e = (int)threadIdx.x - 32; e < w * w; e += upd_threads) {
        const int c = t + 1 + e / w, j = t + 1 + e % w;
        if (j <= c && c > t + 1)
          S[c * ld + j] = __fma_rn(-S[j * ld + t], S[c * ld + t], S[c * ld + j]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && fail_at >= 0) sc->fail = fail_at;
}

// A factor of kPotrfSmallMax < k <= kPotrfSingleCtaMax: every panel in one
// launch on one CTA (block barriers instead of three launches per panel);
// the batched body.
constexpr int kPotrfSingleCtaMax = 128;
__global__ void __launch_bounds__(256) potrf_single_cta_kernel(PotrfDesc D) {
  potrf_cta_body(D);
}

cudaError_t launch_potrf(int kmax, double* G, int64_t ldg, double* R, int64_t ldr,
                         DeviceScalars* sc, cudaStream_t stream) {
  PotrfDesc D{kmax, G, ldg, R, ldr, sc};
  if (kmax <= kPotrfSmallMax) {
    potrf_small_kernel<<<1, kPotrfSmallThreads, 0, stream>>>(D);
    count_launches(1);
    return cudaGetLastError();
  }
  if (kmax <= kPotrfSingleCtaMax) {
    potrf_single_cta_kernel<<<1, 256, 0, stream>>>(D);
    count_launches(1);
    return cudaGetLastError();
  }
  for (int jb = 0; jb < kmax; jb += kCholNB) {
    potrf_diag_kernel<<<1, 32, 0, stream>>>(jb, D);
    count_launches(1);
    const int rest = kmax - jb - kCholNB;
    if (rest > 0) {
      count_launches(2);
      potrf_panel_kernel<<<(rest + 127) / 128, 128, 0, stream>>>(jb, D);
      dim3 grid((rest + 15) / 16, (rest + 15) / 16);
      potrf_update_kernel<<<grid, dim3(16, 16), 0, stream>>>(jb, D);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_potrf_batched(const PotrfDesc* D, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  potrf_batched_kernel<<<nprob, 256, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
