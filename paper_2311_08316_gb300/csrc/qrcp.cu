// Alg. 2 lines 2-3: column-pivoted Householder QR of the d x n sketch
// (Businger-Golub max-norm pivoting, as LAPACK GEQP3 which the paper uses,
// Sec. 2.1 and Appendix A.1) and the rank rule of Sec. 3.3.
//
// The QRCP of one problem runs on G CTAs that stay resident for all n steps
// (one cooperative launch for a single large problem; G = 1 and one CTA per
// problem for a batch).  Physical columns never move: CTA b owns the physical
// columns b, b+G, b+2G, ... for the whole factorisation (one warp per
// column) and a position <-> column map (phys/posof) records the swaps, so a
// pivot exchange moves no data.  Each of the n steps is:
//   1. every CTA reduces the per-CTA candidates (largest partial norm,
//      lowest position on exact ties) to the same pivot column P;
//   2. the owner of P forms the reflector H = I - tau v v^T as LAPACK's
//      dlarfg: beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
//      v = x * (1 / (alpha - beta)) (v written over the column below the
//      diagonal, beta on it); CTA 0 records the swap;
//      -- barrier --
//   3. every CTA applies H to its unpivoted columns (w = v^T x by dot32,
//      x += v (-tau w) with one fma per element) and downdates their norms
//      (LAPACK dlaqp2 rule with the Drmac-Bujanovic recompute safeguard),
//      then publishes its candidate;  -- barrier --
// All reads of data written by other CTAs bypass L1 (ld.global.cg).  Grid
// barriers spin a bounded number of times (status kTimeout on expiry).
#include <algorithm>
#include <cstdlib>

#include <cooperative_groups.h>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace cqrrpt {

// Polls of a grid barrier before it gives up (kTimeout); lowered only by
// cqrrpt_set_wait_limits, a test hook for the timeout path.
__device__ unsigned long long g_grid_spin_limit = kSpinLimit;

cudaError_t qrcp_set_spin_limit(unsigned long long spins) {
  const unsigned long long v = spins ? spins : kSpinLimit;
  return cudaMemcpyToSymbol(g_grid_spin_limit, &v, sizeof(v));
}

// Candidate records of the multi-CTA QRCP: two slots (step parity) of
// kCandSlot CTAs each (G <= kCandSlot; G is at most one CTA per SM).
constexpr int kCandSlot = 256;

QrcpWork qrcp_carve(void* work, int n) {
  char* p = (char*)work;
  QrcpWork w;
  w.vn1 = (double*)p; p += align256((int64_t)n * 8);
  w.vn2 = (double*)p; p += align256((int64_t)n * 8);
  w.tau = (double*)p; p += align256((int64_t)n * 8);
  w.phys = (int*)p; p += align256((int64_t)n * 4);
  w.posof = (int*)p; p += align256((int64_t)n * 4);
  w.cand_val = (double*)p; p += align256(2 * kCandSlot * 8);
  w.cand_pos = (int*)p; p += align256(2 * kCandSlot * 4);
  w.cand_col = (int*)p; p += align256(2 * kCandSlot * 4);
  w.cand_refl = (double*)p; p += align256(2 * kCandSlot * 4 * 8);
  return w;
}

int64_t qrcp_workspace_bytes(int64_t n) {
  return 3 * align256(n * 8) + 2 * align256(n * 4) + align256(2 * kCandSlot * 8) +
         2 * align256(2 * kCandSlot * 4) + align256(2 * kCandSlot * 4 * 8);
}

// dot32 of x[0..len) with itself, by one warp (result in every lane).
__device__ __forceinline__ double warp_dot32_self(const double* x, int len) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int i = lane; i < len; i += 32) {
    const double v = __ldcg(x + i);
    acc = __fma_rn(v, v, acc);
  }
  return warp_tree_sum32(acc);
}

// candidate order: larger value first, then lower position
__device__ __forceinline__ bool cand_better(double va, int pa, double vb, int pb) {
  return va > vb || (va == vb && pa < pb);
}

__device__ __forceinline__ void qrcp_body(const int G, const int bid, const QrcpDesc& D,
                                          double tol3z) {
  const int d = D.d, n = D.n;
  double* X = D.X;
  const int64_t ldx = D.ldx;
  const QrcpWork& w = D.w;
  DeviceScalars* sc = D.sc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  int* status = &sc->status;
  __shared__ int sh_P, sh_p;
  __shared__ double sh_tau, sh_beta, sh_denom;  // sh_denom: 1 / (alpha - beta)
  __shared__ int sh_nz;
  __shared__ double red_val[32];
  __shared__ int red_pos[32];
  __shared__ int red_col[32];

  if (*(volatile int*)status != kOk) return;  // set before launch: uniform over CTAs
  const unsigned long long spins = g_grid_spin_limit;

  // initial norms of owned columns
  for (int q = warp;; q += nwarps) {
    const int c = bid + G * q;
    if (c >= n) break;
    const double s = warp_dot32_self(X + (int64_t)c * ldx, d);
    if (lane == 0) {
      const double v = __dsqrt_rn(s);
      w.vn1[c] = v;
      w.vn2[c] = v;
      w.phys[c] = c;
      w.posof[c] = c;
    }
  }

  // each warp scans its owned columns (all lanes alike), then thread 0
  // reduces the warps and publishes the CTA's candidate
  auto publish_candidate = [&](int j_done) {
    double bv = -1.0;
    int bp = 0x7fffffff, bc = -1;
    for (int q = warp;; q += nwarps) {
      const int c = bid + G * q;
      if (c >= n) break;
      const int pc = __ldcg(w.posof + c);
      if (pc <= j_done) continue;
      // without pivoting the key is n - position: the lowest position wins
      const double v = D.nopivot ? (double)(n - pc) : __ldcg(w.vn1 + c);
      if (cand_better(v, pc, bv, bp)) { bv = v; bp = pc; bc = c; }
    }
    if (lane == 0) { red_val[warp] = bv; red_pos[warp] = bp; red_col[warp] = bc; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < nwarps; ++i)
        if (cand_better(red_val[i], red_pos[i], bv, bp)) { bv = red_val[i]; bp = red_pos[i]; bc = red_col[i]; }
      w.cand_val[bid] = bv;
      w.cand_pos[bid] = bp;
      w.cand_col[bid] = bc;
    }
  };
  __syncthreads();
  publish_candidate(-1);
  if (!grid_sync(&sc->bar, G, status, spins)) return;

  for (int j = 0; j < n; ++j) {
    // 1. global pivot
    if (warp == 0) {
      double bv = -1.0;
      int bp = 0x7fffffff, bc = -1;
      for (int i = lane; i < G; i += 32) {
        const double v = __ldcg(w.cand_val + i);
        const int p = __ldcg(w.cand_pos + i);
        const int c = __ldcg(w.cand_col + i);
        if (c >= 0 && cand_better(v, p, bv, bp)) { bv = v; bp = p; bc = c; }
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const int op = __shfl_down_sync(0xffffffffu, bp, off);
        const int oc = __shfl_down_sync(0xffffffffu, bc, off);
        if (oc >= 0 && cand_better(ov, op, bv, bp)) { bv = ov; bp = op; bc = oc; }
      }
      if (lane == 0) { sh_P = bc; sh_p = bp; }
    }
    __syncthreads();
    const int P = sh_P, p = sh_p;
    if (P < 0) {
      // no finite candidate anywhere (overflow to Inf/NaN inside the
      // factorisation); every CTA sees the same P and leaves together
      if (bid == 0 && threadIdx.x == 0) atomicExch(status, kNonFinite);
      return;
    }
    double* colP = X + (int64_t)P * ldx;
    // 2. reflector by the owner of P; swap record by CTA 0
    if (P % G == bid) {
      if (warp == 0) {
        const double alpha = __ldcg(colP + j);
        const double sumsq = (j + 1 < d) ? warp_dot32_self(colP + j + 1, d - j - 1) : 0.0;
        if (lane == 0) {
          if (sumsq == 0.0) {
            sh_tau = 0.0;
            sh_nz = 0;
          } else {
            const double nrm = __dsqrt_rn(__fma_rn(alpha, alpha, sumsq));
            const double beta = (alpha >= 0.0) ? -nrm : nrm;
            sh_tau = __ddiv_rn(__dsub_rn(beta, alpha), beta);
            sh_beta = beta;
            sh_denom = __ddiv_rn(1.0, __dsub_rn(alpha, beta));  // 1 / (alpha - beta)
            sh_nz = 1;
          }
        }
      }
      __syncthreads();
      if (sh_nz) {
        const double rden = sh_denom;
        for (int r = j + 1 + threadIdx.x; r < d; r += blockDim.x)
          colP[r] = __dmul_rn(__ldcg(colP + r), rden);
        if (threadIdx.x == 0) colP[j] = sh_beta;
      }
      if (threadIdx.x == 0) w.tau[j] = sh_tau;
    }
    if (bid == 0 && threadIdx.x == 0) {
      const int Pj = __ldcg(w.phys + j);
      w.phys[p] = Pj;
      w.posof[Pj] = p;
      w.phys[j] = P;
      w.posof[P] = j;
    }
    if (!grid_sync(&sc->bar, G, status, spins)) return;

    // 3. apply H to owned unpivoted columns, downdate norms
    const double tau = __ldcg(w.tau + j);
    const int len = d - j;
    for (int q = warp;; q += nwarps) {
      const int c = bid + G * q;
      if (c >= n) break;
      if (__ldcg(w.posof + c) <= j) continue;
      double* colc = X + (int64_t)c * ldx + j;
      double acc = 0.0;
      for (int i = lane; i < len; i += 32) {
        const double vi = (i == 0) ? 1.0 : __ldcg(colP + j + i);
        acc = __fma_rn(vi, __ldcg(colc + i), acc);
      }
      const double wsum = warp_tree_sum32(acc);
      const double t = __dmul_rn(-tau, wsum);
      for (int i = lane; i < len; i += 32) {
        const double vi = (i == 0) ? 1.0 : __ldcg(colP + j + i);
        colc[i] = __fma_rn(vi, t, __ldcg(colc + i));
      }
      __syncwarp();
      const double v1 = __ldcg(w.vn1 + c);
      if (v1 != 0.0) {
        const double v2 = __ldcg(w.vn2 + c);
        double temp = __ddiv_rn(fabs(__ldcg(colc)), v1);
        temp = __dsub_rn(1.0, __dmul_rn(temp, temp));
        temp = temp > 0.0 ? temp : 0.0;
        const double ratio = __ddiv_rn(v1, v2);
        const double temp2 = __dmul_rn(temp, __dmul_rn(ratio, ratio));
        if (temp2 <= tol3z) {
          const double s = (j + 1 < d) ? warp_dot32_self(colc + 1, d - j - 1) : 0.0;
          if (lane == 0) {
            const double nv = (j + 1 < d) ? __dsqrt_rn(s) : 0.0;
            w.vn1[c] = nv;
            w.vn2[c] = nv;
          }
        } else if (lane == 0) {
          w.vn1[c] = __dmul_rn(v1, __dsqrt_rn(temp));
        }
      }
      __syncwarp();
    }
    __syncthreads();
    publish_candidate(j);
    if (!grid_sync(&sc->bar, G, status, spins)) return;
  }
}

__global__ void __launch_bounds__(kQrcpThreads) qrcp_kernel(QrcpDesc D, double tol3z) {
  qrcp_body(gridDim.x, blockIdx.x, D, tol3z);
  __syncthreads();
  grid_release(&D.sc->bar, gridDim.x);
}

__global__ void __launch_bounds__(1024) qrcp_batched_kernel(const QrcpDesc* D, double tol3z) {
  qrcp_body(1, 0, D[blockIdx.x], tol3z);
}

// dot32 of x[0..len) with itself (shared memory, or an owned column in
// global memory: eight loads in flight per lane), by one warp.
__device__ __forceinline__ double warp_dot32_self_smem(const double* x, int len,
                                                       bool global = false) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  int i = lane;
  if (global)
    for (; i + 32 * 7 < len; i += 32 * 8) {
    double xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x[i + 32 * u];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = __fma_rn(xv[u], xv[u], acc);
  }
#pragma unroll 8
  for (; i < len; i += 32) acc = __fma_rn(x[i], x[i], acc);
  return warp_tree_sum32(acc);
}

// The reflector of a column for step jn (LAPACK's dlarfg on rows jn.., as
// above), by one warp; every lane returns the same values.  The two
// divisions run at once on lanes 0 and 1 (the same correctly rounded
// quotients as one after the other; a warp pays for each FP64 instruction
// whatever its lanes do).  nz = 0 when the rows below jn are all zero
// (H = I, tau = 0).
__device__ __forceinline__ void warp_reflector(const double* col, int jn, int d, bool global,
                                               double& tau, double& beta, double& rden,
                                               int& nz) {
  const int lane = threadIdx.x & 31;
  const double alpha = col[jn];
  const double sumsq = (jn + 1 < d) ? warp_dot32_self_smem(col + jn + 1, d - jn - 1, global) : 0.0;
  if (sumsq == 0.0) {
    tau = 0.0;
    beta = alpha;
    rden = 1.0;
    nz = 0;
    return;
  }
  const double nrm = __dsqrt_rn(__fma_rn(alpha, alpha, sumsq));
  beta = (alpha >= 0.0) ? -nrm : nrm;
  const double num = lane == 1 ? 1.0 : __dsub_rn(beta, alpha);  // tau = (beta - alpha) / beta
  const double den = lane == 1 ? __dsub_rn(alpha, beta) : beta;  // 1 / (alpha - beta)
  const double q = __ddiv_rn(num, den);
  tau = __shfl_sync(0xffffffffu, q, 0);
  rden = __shfl_sync(0xffffffffu, q, 1);
  nz = 1;
}

// LAPACK dlaqp2's norm downdate of one column after step j (a0 = |x_j|
// after the update; `below` holds rows j+1..), by one warp; the new norms
// go to *vn1q / *vn2q from lane 0.  |x_j| / vn1 and vn1 / vn2 are formed at
// once on lanes 0 and 1.
__device__ __forceinline__ void warp_downdate(double* vn1q, double* vn2q, double a0,
                                              const double* below, int len_below, bool global,
                                              double tol3z) {
  const int lane = threadIdx.x & 31;
  const double v1 = *vn1q;
  if (v1 == 0.0) return;
  const double v2 = *vn2q;
  const double qq = __ddiv_rn(lane == 1 ? v1 : a0, lane == 1 ? v2 : v1);
  double temp = __shfl_sync(0xffffffffu, qq, 0);         // |x_j| / vn1
  const double ratio = __shfl_sync(0xffffffffu, qq, 1);  // vn1 / vn2
  temp = __dsub_rn(1.0, __dmul_rn(temp, temp));
  temp = temp > 0.0 ? temp : 0.0;
  const double temp2 = __dmul_rn(temp, __dmul_rn(ratio, ratio));
  if (temp2 <= tol3z) {
    const double s2 = len_below > 0 ? warp_dot32_self_smem(below, len_below, global) : 0.0;
    if (lane == 0) {
      const double nv = len_below > 0 ? __dsqrt_rn(s2) : 0.0;
      *vn1q = nv;
      *vn2q = nv;
    }
  } else if (lane == 0) {
    *vn1q = __dmul_rn(v1, __dsqrt_rn(temp));
  }
}

// The best candidate of the calling warp's lanes below `width` (a power of
// two at most 32); every lane of the warp ends with it (lane 0's result is
// broadcast when width < 32, so that the whole warp takes the same branch
// afterwards).  A butterfly in
// the candidate order (larger value, then lower position).  Lanes without a
// candidate hold value -1, position INT_MAX and c < 0, which every finite
// candidate beats; a NaN value never wins (as in the sequential scans).  The
// order is total over distinct positions, so the result does not depend on
// the combination order.
struct Cand {
  double v;
  int p, c, i;  // position, column (or owned index), record
  double tau, beta, rden;
  int nz;
};
__device__ __forceinline__ void warp_best(Cand& a, int width, bool carry) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off >= width) continue;
    Cand o = a;
    o.v = __shfl_xor_sync(0xffffffffu, a.v, off);
    o.p = __shfl_xor_sync(0xffffffffu, a.p, off);
    o.c = __shfl_xor_sync(0xffffffffu, a.c, off);
    o.i = __shfl_xor_sync(0xffffffffu, a.i, off);
    if (carry) {
      o.tau = __shfl_xor_sync(0xffffffffu, a.tau, off);
      o.beta = __shfl_xor_sync(0xffffffffu, a.beta, off);
      o.rden = __shfl_xor_sync(0xffffffffu, a.rden, off);
      o.nz = __shfl_xor_sync(0xffffffffu, a.nz, off);
    }
    if (o.c >= 0 && cand_better(o.v, o.p, a.v, a.p)) a = o;
  }
  if (width < 32) {  // lanes at and above width combined only among themselves
    a.v = __shfl_sync(0xffffffffu, a.v, 0);
    a.p = __shfl_sync(0xffffffffu, a.p, 0);
    a.c = __shfl_sync(0xffffffffu, a.c, 0);
    a.i = __shfl_sync(0xffffffffu, a.i, 0);
    if (carry) {
      a.tau = __shfl_sync(0xffffffffu, a.tau, 0);
      a.beta = __shfl_sync(0xffffffffu, a.beta, 0);
      a.rden = __shfl_sync(0xffffffffu, a.rden, 0);
      a.nz = __shfl_sync(0xffffffffu, a.nz, 0);
    }
  }
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int w = 1;
  while (w < x && w < 32) w <<= 1;
  return w;
}

// Named barrier 1 (0 is __syncthreads): arrive signals without
// waiting, sync waits until `nthreads` threads have arrived or synced.  The
// non-.aligned forms, so that a warp's threads may reach them apart (after
// a branch taken by one lane).
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Same arithmetic as qrcp_body, one grid barrier per step instead of two.
// Every CTA keeps its first qc owned columns (cache[q * d + r] is row r of
// physical column bid + G q), the partial norms of all of them and its own
// copy of the position <-> column maps in shared memory for the whole
// factorisation; owned columns q >= qc (when the sketch is too large for
// the SMs' shared memory) stay in X, which only their owner writes.
// At the end of step j each CTA picks its best unpivoted column (its
// candidate for step j + 1), forms that column's reflector for step j + 1
// itself (one warp, while the other warps copy the column's rows j+1.. to
// X) and publishes candidate and reflector (tau, beta, 1 / (alpha - beta))
// in its record, two slots by step parity.  After the barrier every CTA
// picks the same pivot P from the records, reads P's rows below the
// diagonal from X scaled by the published 1 / (alpha - beta) (the same
// products as the owner would form), updates its maps with the same swap
// and applies the reflector to its columns.  The owner of a cached P keeps
// beta and v in its column; a P in X gets beta written into X after the
// next barrier and keeps its rows below (only R^sk is read afterwards).
// All owned columns are written back at the end; CTA 0 writes the maps and
// tau.  G = 1 (one CTA per problem, the batched form) keeps the candidate
// and its reflector in shared memory: no global memory round trip per step.
__device__ __forceinline__ void qrcp_cached_body(const QrcpDesc& D, double tol3z, int qc, int G,
                                                 int bid, double* cache) {
  const int d = D.d, n = D.n;
  double* X = D.X;
  const int64_t ldx = D.ldx;
  const QrcpWork& w = D.w;
  DeviceScalars* sc = D.sc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  int* status = &sc->status;
  const int nown = bid < n ? (n - bid + G - 1) / G : 0;
  const int ncached = nown < qc ? nown : qc;
  double* vbuf = cache + (int64_t)ncached * d;       // d
  double* vn1 = vbuf + d;                             // nown
  double* vn2 = vn1 + nown;                           // nown
  int* phys = (int*)(vn2 + nown);                     // n
  int* posof = phys + n;                              // n
  __shared__ int sh_P, sh_p, sh_q;
  __shared__ double sh_tau, sh_beta, sh_rden;
  __shared__ int sh_nz;
  __shared__ double* sh_pend;  // beta of a pivot column in X, written after the barrier
  __shared__ double sh_pend_val;
  __shared__ double red_val[32];
  __shared__ int red_pos[32];
  __shared__ int red_col[32];

  if (*(volatile int*)status != kOk) return;  // set before launch: uniform over CTAs
  const unsigned long long spins = g_grid_spin_limit;

  // owned column q: shared memory for q < ncached, else its column of X
  auto colptr = [&](int q) -> double* {
    return q < ncached ? cache + (int64_t)q * d : X + (int64_t)(bid + G * q) * ldx;
  };
  for (int q = 0; q < ncached; ++q) {
    const double* src = X + (int64_t)(bid + G * q) * ldx;
    for (int r = threadIdx.x; r < d; r += blockDim.x) cache[(int64_t)q * d + r] = src[r];
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    phys[c] = c;
    posof[c] = c;
  }
  if (threadIdx.x == 0) sh_pend = nullptr;
  __syncthreads();
  for (int q = warp; q < nown; q += nwarps) {
    const double s = warp_dot32_self_smem(colptr(q), d, q >= ncached);
    if (lane == 0) {
      const double v = __dsqrt_rn(s);
      vn1[q] = v;
      vn2[q] = v;
    }
  }
  __syncthreads();

  // the CTA's best unpivoted column after step j_done and its reflector for
  // step j_done + 1, into record slot (j_done + 1) & 1 (G = 1: shared memory)
  auto publish_candidate = [&](int j_done) {
    const int jn = j_done + 1;
    double bv = -1.0;
    int bp = 0x7fffffff, bq = -1;
    for (int q = warp; q < nown; q += nwarps) {
      const int c = bid + G * q;
      const int pc = posof[c];
      if (pc <= j_done) continue;
      // without pivoting the key is n - position: the lowest position wins
      const double v = D.nopivot ? (double)(n - pc) : vn1[q];
      if (cand_better(v, pc, bv, bp)) { bv = v; bp = pc; bq = q; }
    }
    if (lane == 0) { red_val[warp] = bv; red_pos[warp] = bp; red_col[warp] = bq; }
    __syncthreads();
    if (warp == 0) {
      Cand a;
      a.v = lane < nwarps ? red_val[lane] : -1.0;
      a.p = lane < nwarps ? red_pos[lane] : 0x7fffffff;
      a.c = lane < nwarps ? red_col[lane] : -1;
      a.i = 0;
      a.tau = a.beta = 0.0;
      a.rden = 1.0;
      a.nz = 0;
      warp_best(a, pow2_at_least(nwarps), false);
      const int q = a.c;
      if (lane == 0) sh_q = q;
      if (G > 1) named_arrive(1, blockDim.x);  // the other warps copy the column meanwhile
      double tau = 0.0, beta = 0.0, rden = 1.0;
      int nz = 0;
      if (q >= 0 && jn < n) warp_reflector(colptr(q), jn, d, q >= ncached, tau, beta, rden, nz);
      if (lane == 0) {
        if (G > 1) {
          const int idx = (jn & 1) * kCandSlot + bid;
          w.cand_val[idx] = a.v;
          w.cand_pos[idx] = a.p;
          w.cand_col[idx] = q >= 0 ? bid + G * q : -1;
          double* r = w.cand_refl + 4 * (int64_t)idx;
          r[0] = tau;
          r[1] = beta;
          r[2] = rden;
          r[3] = (double)nz;
        } else {  // G = 1: owned index q is physical column q
          sh_P = q;
          sh_p = a.p;
          sh_tau = tau;
          sh_beta = beta;
          sh_rden = rden;
          sh_nz = nz;
        }
      }
    } else if (G > 1) {
      named_sync(1, blockDim.x);
      const int q = sh_q;
      if (q >= 0 && q < ncached) {  // a column in X is already there
        double* dst = X + (int64_t)(bid + G * q) * ldx;
        const double* src = cache + (int64_t)q * d;
        for (int r = jn + threadIdx.x - 32; r < d; r += blockDim.x - 32) dst[r] = src[r];
      }
    }
  };
  publish_candidate(-1);
  bool ok = grid_sync(&sc->bar, G, status, spins);

  for (int j = 0; ok && j < n; ++j) {
    // beta of the previous pivot, if its column lives in X: every CTA has
    // read that column by now
    if (threadIdx.x == 0 && sh_pend) {
      *sh_pend = sh_pend_val;
      sh_pend = nullptr;
    }
    // 1. global pivot and its reflector from the records (every CTA alike)
    if (G > 1 && warp == 0) {
      const int slot = (j & 1) * kCandSlot;
      Cand a;
      a.v = -1.0;
      a.p = 0x7fffffff;
      a.c = -1;
      a.i = 0;
      a.tau = 0.0;
      a.beta = 0.0;
      a.rden = 1.0;
      a.nz = 0;
      // lane l reads records l, l + 32, ... with their reflectors (all
      // loads in flight at once) and keeps its best; the butterfly then
      // moves only the keys, and the winner's reflector comes from the lane
      // that read it
      for (int i = lane; i < G; i += 32) {
        const double v = __ldcg(w.cand_val + slot + i);
        const int p = __ldcg(w.cand_pos + slot + i);
        const int c = __ldcg(w.cand_col + slot + i);
        const double2 r01 = __ldcg((const double2*)(w.cand_refl + 4 * (int64_t)(slot + i)));
        const double2 r23 = __ldcg((const double2*)(w.cand_refl + 4 * (int64_t)(slot + i)) + 1);
        if (c >= 0 && cand_better(v, p, a.v, a.p)) {
          a.v = v;
          a.p = p;
          a.c = c;
          a.i = i;
          a.tau = r01.x;
          a.beta = r01.y;
          a.rden = r23.x;
          a.nz = r23.y != 0.0;
        }
      }
      warp_best(a, 32, false);
      {
        const int src = a.i & 31;  // the lane that read record a.i
        a.tau = __shfl_sync(0xffffffffu, a.tau, src);
        a.beta = __shfl_sync(0xffffffffu, a.beta, src);
        a.rden = __shfl_sync(0xffffffffu, a.rden, src);
        a.nz = __shfl_sync(0xffffffffu, a.nz, src);
      }
      if (lane == 0) {
        sh_P = a.c;
        sh_p = a.p;
        sh_tau = a.tau;
        sh_beta = a.beta;
        sh_rden = a.rden;
        sh_nz = a.nz;
      }
    }
    __syncthreads();
    const int P = sh_P, p = sh_p;
    if (P < 0) {
      if (bid == 0 && threadIdx.x == 0) atomicExch(status, kNonFinite);
      ok = false;
      break;
    }
    // 2. v = (1, x_{j+1..} / (alpha - beta)) into vbuf; the owner of a
    // cached P keeps v and beta in its column
    const double tau = sh_tau;
    const bool nz = sh_nz != 0;
    const double rden = sh_rden;
    const int len = d - j;
    const bool owner = (P % G == bid);
    const int qP = (P - bid) / G;
    const bool owner_cached = owner && qP < ncached;
    double* cP = owner_cached ? cache + (int64_t)qP * d : nullptr;
    const double* src = owner_cached ? cP : X + (int64_t)P * ldx;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      double v = 1.0;
      if (i > 0) {
        const double x = owner_cached ? src[j + i] : __ldcg(src + j + i);
        v = nz ? __dmul_rn(x, rden) : x;
        if (owner_cached) cP[j + i] = v;
      }
      vbuf[i] = v;
    }
    if (threadIdx.x == 0) {
      if (owner_cached && nz) cP[j] = sh_beta;
      if (owner && !owner_cached && nz) {
        sh_pend = X + (int64_t)P * ldx + j;
        sh_pend_val = sh_beta;
      }
      const int Pj = phys[j];
      phys[p] = Pj;
      posof[Pj] = p;
      phys[j] = P;
      posof[P] = j;
      if (bid == 0) w.tau[j] = tau;
    }
    __syncthreads();

    // 3. apply H to owned unpivoted columns, downdate norms
    for (int q = warp; q < nown; q += nwarps) {
      const int c = bid + G * q;
      if (posof[c] <= j) continue;
      double* colc = colptr(q) + j;
      // eight loads in flight per lane (a column in X sits in L2), the fmas
      // still in ascending order
      double acc = 0.0;
      int i = lane;
      if (q >= ncached)
        for (; i + 32 * 7 < len; i += 32 * 8) {
          double xv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) xv[u] = colc[i + 32 * u];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc = __fma_rn(vbuf[i + 32 * u], xv[u], acc);
        }
#pragma unroll 8
      for (; i < len; i += 32) acc = __fma_rn(vbuf[i], colc[i], acc);
      const double wsum = warp_tree_sum32(acc);
      const double t = __dmul_rn(-tau, wsum);
#pragma unroll 8
      for (int i2 = lane; i2 < len; i2 += 32) colc[i2] = __fma_rn(vbuf[i2], t, colc[i2]);
      __syncwarp();
      warp_downdate(vn1 + q, vn2 + q, fabs(colc[0]), colc + 1, d - j - 1, q >= ncached, tol3z);
      __syncwarp();
    }
    __syncthreads();
    publish_candidate(j);
    if (!grid_sync(&sc->bar, G, status, spins)) { ok = false; break; }
  }
  // write the owned columns back (also after an early exit, so that global
  // memory holds this CTA's last state) and, from CTA 0, the maps
  __syncthreads();
  grid_release(&sc->bar, G);
  if (threadIdx.x == 0 && sh_pend) *sh_pend = sh_pend_val;  // after the last barrier
  for (int q = 0; q < ncached; ++q) {
    double* dst = X + (int64_t)(bid + G * q) * ldx;
    for (int r = threadIdx.x; r < d; r += blockDim.x) dst[r] = cache[(int64_t)q * d + r];
  }
  if (bid == 0)
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      w.phys[c] = phys[c];
      w.posof[c] = posof[c];
    }
}

__global__ void __launch_bounds__(kQrcpThreads) qrcp_cached_kernel(QrcpDesc D, double tol3z,
                                                                   int qc) {
  extern __shared__ double cache[];
  qrcp_cached_body(D, tol3z, qc, gridDim.x, blockIdx.x, cache);
}

// A small sketch (n <= kQrcpClusterMaxN) on one thread-block cluster of G
// CTAs (G <= 16, four columns each, every column in shared memory): the
// same steps and arithmetic as qrcp_cached_body, with the exchange inside
// the cluster.  At the end of a step each CTA writes its candidate and that
// column's reflector for the next step into its own shared memory (two
// slots by step parity), and the cluster barrier (barrier.cluster arrive
// with release, wait with acquire) replaces the grid barrier; every CTA then
// reads the G records and the pivot column straight from the owner CTA's
// shared memory (distributed shared memory), with no round trip through
// global memory.  The owner writes beta into its column's row j only after
// the next barrier (the others read that column during the step); the
// Householder vector itself is not kept, as only the upper triangle (R^sk)
// is read afterwards.  Every CTA runs the same sequence of barriers (the
// exits depend only on data every CTA holds alike), and a last barrier
// keeps each CTA's shared memory alive until no peer reads it.
constexpr int kQrcpClusterMaxN = 64;
constexpr int kQrcpClusterMaxG = 16;
__global__ void __launch_bounds__(kQrcpThreads) qrcp_cluster_kernel(QrcpDesc D, double tol3z) {
  extern __shared__ double cache[];
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int G = (int)cluster.num_blocks();
  const int bid = (int)cluster.block_rank();
  const int d = D.d, n = D.n;
  double* X = D.X;
  const int64_t ldx = D.ldx;
  const QrcpWork& w = D.w;
  DeviceScalars* sc = D.sc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  int* status = &sc->status;
  const int nown = bid < n ? (n - bid + G - 1) / G : 0;
  double* vbuf = cache + (int64_t)nown * d;  // d
  double* vn1 = vbuf + d;                    // nown
  double* vn2 = vn1 + nown;                  // nown
  int* phys = (int*)(vn2 + nown);            // n
  int* posof = phys + n;                     // n
  __shared__ double rec_val[2], rec_tau[2], rec_beta[2], rec_rden[2];
  __shared__ int rec_pos[2], rec_col[2], rec_nz[2];
  __shared__ int sh_P, sh_p;
  __shared__ double sh_tau, sh_beta, sh_rden;
  __shared__ int sh_nz;
  __shared__ int sh_pend_q, sh_pend_row;  // beta into row sh_pend_row of column sh_pend_q
  __shared__ double sh_pend_val;
  __shared__ double red_val[32];
  __shared__ int red_pos[32];
  __shared__ int red_col[32];

  if (*(volatile int*)status != kOk) return;  // set before launch: uniform over CTAs

  for (int q = 0; q < nown; ++q) {
    const double* src = X + (int64_t)(bid + G * q) * ldx;
    for (int r = threadIdx.x; r < d; r += blockDim.x) cache[(int64_t)q * d + r] = src[r];
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    phys[c] = c;
    posof[c] = c;
  }
  if (threadIdx.x == 0) sh_pend_q = -1;
  __syncthreads();
  for (int q = warp; q < nown; q += nwarps) {
    const double s = warp_dot32_self_smem(cache + (int64_t)q * d, d);
    if (lane == 0) {
      const double v = __dsqrt_rn(s);
      vn1[q] = v;
      vn2[q] = v;
    }
  }
  __syncthreads();

  // the CTA's best unpivoted column after step j_done and its reflector for
  // step j_done + 1, into record slot (j_done + 1) & 1
  auto publish_candidate = [&](int j_done) {
    const int jn = j_done + 1;
    double bv = -1.0;
    int bp = 0x7fffffff, bq = -1;
    for (int q = warp; q < nown; q += nwarps) {
      const int c = bid + G * q;
      const int pc = posof[c];
      if (pc <= j_done) continue;
      const double v = D.nopivot ? (double)(n - pc) : vn1[q];
      if (cand_better(v, pc, bv, bp)) { bv = v; bp = pc; bq = q; }
    }
    if (lane == 0) { red_val[warp] = bv; red_pos[warp] = bp; red_col[warp] = bq; }
    __syncthreads();
    if (warp == 0) {
      Cand a;
      a.v = lane < nwarps ? red_val[lane] : -1.0;
      a.p = lane < nwarps ? red_pos[lane] : 0x7fffffff;
      a.c = lane < nwarps ? red_col[lane] : -1;
      a.i = 0;
      a.tau = a.beta = 0.0;
      a.rden = 1.0;
      a.nz = 0;
      warp_best(a, pow2_at_least(nwarps), false);
      const int q = a.c;
      double tau = 0.0, beta = 0.0, rden = 1.0;
      int nz = 0;
      if (q >= 0 && jn < n)
        warp_reflector(cache + (int64_t)q * d, jn, d, false, tau, beta, rden, nz);
      if (lane == 0) {
        const int slot = jn & 1;
        rec_val[slot] = a.v;
        rec_pos[slot] = a.p;
        rec_col[slot] = q >= 0 ? bid + G * q : -1;
        rec_tau[slot] = tau;
        rec_beta[slot] = beta;
        rec_rden[slot] = rden;
        rec_nz[slot] = nz;
      }
    }
    cluster.sync();
  };
  publish_candidate(-1);

  bool ok = true;
  for (int j = 0; j < n; ++j) {
    // beta of the previous pivot into its owner's column: every CTA has read
    // that column (it passed the barrier after reading it)
    if (threadIdx.x == 0 && sh_pend_q >= 0) {
      cache[(int64_t)sh_pend_q * d + sh_pend_row] = sh_pend_val;
      sh_pend_q = -1;
    }
    // 1. global pivot and its reflector from the G records (every CTA alike)
    if (warp == 0) {
      const int slot = j & 1;
      Cand a;
      a.v = -1.0;
      a.p = 0x7fffffff;
      a.c = -1;
      a.i = 0;
      a.tau = 0.0;
      a.beta = 0.0;
      a.rden = 1.0;
      a.nz = 0;
      if (lane < G) {
        const int c = *cluster.map_shared_rank(&rec_col[slot], lane);
        const double v = *cluster.map_shared_rank(&rec_val[slot], lane);
        const int pp = *cluster.map_shared_rank(&rec_pos[slot], lane);
        if (c >= 0 && cand_better(v, pp, a.v, a.p)) {
          a.v = v;
          a.p = pp;
          a.c = c;
          a.tau = *cluster.map_shared_rank(&rec_tau[slot], lane);
          a.beta = *cluster.map_shared_rank(&rec_beta[slot], lane);
          a.rden = *cluster.map_shared_rank(&rec_rden[slot], lane);
          a.nz = *cluster.map_shared_rank(&rec_nz[slot], lane);
        }
      }
      warp_best(a, pow2_at_least(G), true);
      if (lane == 0) {
        sh_P = a.c;
        sh_p = a.p;
        sh_tau = a.tau;
        sh_beta = a.beta;
        sh_rden = a.rden;
        sh_nz = a.nz;
      }
    }
    __syncthreads();
    const int P = sh_P, p = sh_p;
    if (P < 0) {  // no finite candidate anywhere: every CTA sees the same
      if (bid == 0 && threadIdx.x == 0) atomicExch(status, kNonFinite);
      ok = false;
      break;
    }
    // 2. v = (1, x_{j+1..} / (alpha - beta)) from the owner's shared memory
    const int owner = P % G, qP = P / G;
    const int len = d - j;
    const double tau = sh_tau;
    const bool nz = sh_nz != 0;
    const double rden = sh_rden;
    {
      const double* src = cluster.map_shared_rank(cache + (int64_t)qP * d + j, owner);
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        double v = 1.0;
        if (i > 0) {
          const double x = src[i];
          v = nz ? __dmul_rn(x, rden) : x;
        }
        vbuf[i] = v;
      }
    }
    if (threadIdx.x == 0) {
      if (owner == bid && nz) {
        sh_pend_q = qP;
        sh_pend_row = j;
        sh_pend_val = sh_beta;
      }
      const int Pj = phys[j];
      phys[p] = Pj;
      posof[Pj] = p;
      phys[j] = P;
      posof[P] = j;
      if (bid == 0) w.tau[j] = tau;
    }
    __syncthreads();
    // 3. apply H to the owned unpivoted columns, downdate their norms
    for (int q = warp; q < nown; q += nwarps) {
      const int c = bid + G * q;
      if (posof[c] <= j) continue;
      double* colc = cache + (int64_t)q * d + j;
      double acc = 0.0;
#pragma unroll 8
      for (int i = lane; i < len; i += 32) acc = __fma_rn(vbuf[i], colc[i], acc);
      const double wsum = warp_tree_sum32(acc);
      const double t = __dmul_rn(-tau, wsum);
#pragma unroll 8
      for (int i2 = lane; i2 < len; i2 += 32) colc[i2] = __fma_rn(vbuf[i2], t, colc[i2]);
      __syncwarp();
      warp_downdate(vn1 + q, vn2 + q, fabs(colc[0]), colc + 1, d - j - 1, false, tol3z);
      __syncwarp();
    }
    __syncthreads();
    publish_candidate(j);
  }
  // no peer reads this CTA's shared memory once every CTA is past here
  cluster.sync();
  if (threadIdx.x == 0 && sh_pend_q >= 0 && ok)
    cache[(int64_t)sh_pend_q * d + sh_pend_row] = sh_pend_val;
  __syncthreads();
  for (int q = 0; q < nown; ++q) {
    double* dst = X + (int64_t)(bid + G * q) * ldx;
    for (int r = threadIdx.x; r < d; r += blockDim.x) dst[r] = cache[(int64_t)q * d + r];
  }
  if (bid == 0)
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      w.phys[c] = phys[c];
      w.posof[c] = posof[c];
    }
}

// One CTA per problem (G = 1), the problems in the table's order (the batch
// planner puts the largest first); smem_bytes of dynamic shared memory hold
// the maps, norms and reflector buffer and as many columns as fit.
constexpr int kQrcpBatchThreads = 512;
__global__ void __launch_bounds__(kQrcpBatchThreads)
    qrcp_cached_batched_kernel(const QrcpDesc* Ds, double tol3z, int64_t smem_bytes) {
  extern __shared__ double cache[];
  const QrcpDesc& D = Ds[blockIdx.x];
  const int64_t fixed = (int64_t)(D.d + 2 * D.n) * 8 + (int64_t)2 * D.n * 4;  // vbuf, norms, maps
  if (fixed > smem_bytes) {  // the maps alone do not fit: the global-memory body
    qrcp_body(1, 0, D, tol3z);
    return;
  }
  const int64_t qc = (smem_bytes - fixed) / ((int64_t)D.d * 8);
  qrcp_cached_body(D, tol3z, (int)(qc < D.n ? qc : D.n), 1, 0, cache);
}

// R^sk[i, q] = s_i X[i, phys[q]] for i <= q < n (0 below), s_i = -1 when the
// diagonal X[i, phys[i]] is negative; J[q] = phys[q].
__device__ __forceinline__ void qrcp_gather_body(int q, const QrcpDesc& D) {
  if (D.sc->status != kOk) return;
  const int n = D.n;
  const int* phys = D.w.phys;
  const int pq = phys[q];
  if (threadIdx.x == 0) D.J[q] = pq;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = 0.0;
    if (i <= q) {
      const double diag = D.X[(int64_t)phys[i] * D.ldx + i];
      v = D.X[(int64_t)pq * D.ldx + i];
      if (diag < 0.0) v = -v;
    }
    D.Rsk[(int64_t)q * D.ldr + i] = v;
  }
}

__global__ void qrcp_gather_kernel(QrcpDesc D) { qrcp_gather_body(blockIdx.x, D); }

__global__ void qrcp_gather_batched_kernel(const QrcpDesc* D, const int64_t* base, int np) {
  int64_t t;
  const int p = find_problem(base, np, blockIdx.x, &t);
  qrcp_gather_body((int)t, D[p]);
}

static double tol3z_value() { return sqrt(ldexp(1.0, -53)); }

// Cooperative QRCP grids of one device run one at a time.  Each needs all
// its CTAs resident at once (they wait on one another at the grid barrier);
// two such grids issued from different streams (several handles, threads or
// server lanes) could each hold part of the SMs and wait for the rest.  So
// every cooperative launch waits, on the GPU, for the previous one on the
// same device (an event, recorded after each launch under a lock): the host
// never blocks, and other kernels still run beside the grid.  Not applied
// while the stream is being captured into a graph.
namespace {
struct CoopFence {
  std::mutex mu;
  cudaEvent_t ev = nullptr;
  bool recorded = false;
};
CoopFence g_coop[64];
}  // namespace

static cudaError_t coop_launch(const void* fn, int G, void** args, size_t smem,
                               cudaStream_t stream) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  int dev = 0;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone ||
      cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kQrcpThreads), args, smem, stream);
  }
  CoopFence& f = g_coop[dev];
  std::lock_guard<std::mutex> lock(f.mu);
  cudaError_t e = cudaSuccess;
  if (f.ev && f.recorded && cudaStreamWaitEvent(stream, f.ev, 0) != cudaSuccess) {
    // the event died with its context (cudaDeviceReset): start afresh
    cudaGetLastError();
    f.ev = nullptr;
    f.recorded = false;
  }
  if (!f.ev) e = cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kQrcpThreads), args, smem, stream);
  if (e == cudaSuccess) {
    e = cudaEventRecord(f.ev, stream);
    f.recorded = e == cudaSuccess;
  }
  return e;
}

cudaError_t launch_qrcp(int d, int n, double* X, int64_t ldx, int64_t* J, double* Rsk,
                        int64_t ldr, void* work, DeviceScalars* sc, int num_sms,
                        cudaStream_t stream, bool nopivot) {
  QrcpDesc D{d, n, X, ldx, qrcp_carve(work, n), J, Rsk, ldr, sc, nopivot ? 1 : 0};
  // CQRRPT_QRCP_CLUSTER = 1: a small sketch on one cluster of up to 16 CTAs,
  // four columns each (as the cooperative grid below), exchanging through
  // distributed shared memory and the cluster barrier.  Same bits; at n = 64
  // it measured 0.81 ms against 0.55 ms for the cooperative grid with its
  // counter barrier, so the grid is the default.  A cluster that cannot be
  // placed falls back to the grid.
  {
    const int Gc = (n + 3) / 4;
    const int64_t nown_c = (n + Gc - 1) / Gc;  // CTA 0 owns the most columns
    // the columns, the reflector buffer, two norms per column, the two maps
    const int64_t smem_c = nown_c * d * 8 + (d + 2 * nown_c) * 8 + (int64_t)2 * n * 4;
    bool use = n <= kQrcpClusterMaxN && Gc <= kQrcpClusterMaxG && smem_c <= kQrcpSmemCap;
    const char* f = std::getenv("CQRRPT_QRCP_CLUSTER");
    use = use && f && f[0] == '1';
    cudaError_t e1 = cudaSuccess;
    if (use) {
      e1 = raise_smem_limit((const void*)qrcp_cluster_kernel, (size_t)smem_c);
      if (e1 != cudaSuccess) return e1;
      if (Gc > 8)  // clusters above 8 CTAs are opt-in
        e1 = cudaFuncSetAttribute(qrcp_cluster_kernel,
                                  cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      use = e1 == cudaSuccess;
      cudaGetLastError();
    }
    if (use) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(Gc);
      cfg.blockDim = dim3(kQrcpThreads);
      cfg.dynamicSmemBytes = (size_t)smem_c;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = Gc;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, qrcp_cluster_kernel, &cfg) != cudaSuccess)
        nclusters = 0;
      cudaGetLastError();
      if (nclusters >= 1) {
        const double tz = tol3z_value();
        e1 = cudaLaunchKernelEx(&cfg, qrcp_cluster_kernel, D, tz);
        if (e1 != cudaSuccess) return e1;
        qrcp_gather_kernel<<<n, 128, 0, stream>>>(D);
        count_launches(2);
        return cudaGetLastError();
      }
    }
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qrcp_kernel, kQrcpThreads, 0);
  if (e != cudaSuccess) return e;
  // four columns per CTA (one CTA per SM at most): measured at n = 64, 512
  // and 1024 against 8 columns per CTA, 2-6% less time per step (the
  // update of a step spreads over more SMs; the exchange costs about the
  // same)
  int G = (n + 3) / 4;
  if (G > num_sms * per_sm) G = num_sms * per_sm;
  if (G > num_sms) G = num_sms;
  if (G > kCandSlot) G = kCandSlot;
  if (G < 1) G = 1;
  const double tol3z = tol3z_value();
  void* args[] = {&D, (void*)&tol3z};
  // the maps, norms and reflector buffer in shared memory, and as many
  // owned columns as fit beside them (all of them for most sketches)
  const int64_t nown = (n + G - 1) / G;
  const int64_t kSmemCap = kQrcpSmemCap;
  const int64_t fixed = (int64_t)(d + 2 * nown) * 8 + (int64_t)2 * n * 4;
  int64_t qc = fixed < kSmemCap ? std::min<int64_t>(nown, (kSmemCap - fixed) / ((int64_t)d * 8)) : 0;
  // CQRRPT_QRCP_CACHED_COLUMNS caps the columns kept in shared memory per
  // CTA (tests of the mixed storage on small sketches); the result is the
  // same whatever the cap
  if (const char* cap = std::getenv("CQRRPT_QRCP_CACHED_COLUMNS")) {
    const long v = std::strtol(cap, nullptr, 10);
    if (v >= 0 && v < qc) qc = v;
  }
  const size_t smem = (size_t)(fixed + qc * d * 8);
  bool cached = fixed < kSmemCap;
  int qci = (int)qc;
  void* args_c[] = {&D, (void*)&tol3z, &qci};
  if (cached) {
    e = raise_smem_limit((const void*)qrcp_cached_kernel, smem);
    int per_sm_c = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, qrcp_cached_kernel,
                                                        kQrcpThreads, smem);
    cached = (e == cudaSuccess && per_sm_c >= 1 && G <= num_sms * per_sm_c);
    cudaGetLastError();
  }
  if (cached)
    e = coop_launch((const void*)qrcp_cached_kernel, G, args_c, smem, stream);
  else
    e = coop_launch((const void*)qrcp_kernel, G, args, 0, stream);
  if (e != cudaSuccess) return e;
  qrcp_gather_kernel<<<n, 128, 0, stream>>>(D);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_qrcp_batched(const QrcpDesc* D, int nprob, const int64_t* gather_base,
                                int64_t gather_tiles, int64_t qrcp_smem_bytes,
                                cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  if (qrcp_smem_bytes > 0) {
    cudaError_t e = raise_smem_limit((const void*)qrcp_cached_batched_kernel,
                                     (size_t)qrcp_smem_bytes);
    if (e != cudaSuccess) return e;
    qrcp_cached_batched_kernel<<<nprob, kQrcpBatchThreads, (size_t)qrcp_smem_bytes, stream>>>(
        D, tol3z_value(), qrcp_smem_bytes);
  } else {
    qrcp_batched_kernel<<<nprob, 512, 0, stream>>>(D, tol3z_value());
  }
  qrcp_gather_batched_kernel<<<(unsigned)gather_tiles, 128, 0, stream>>>(D, gather_base, nprob);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rank (Sec. 3.3).  tol > 0: k = number of leading j with R_jj > tol R_00.
// tol <= 0: stage 1, k_o = min{l : ||C_l||_F <= u max|R|}, with
// ||C_l||^2 = ||R[l, l:]||^2 + ||C_{l+1}||^2 (row sums ascending by fma).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rank_body(const RankDesc& D) {
  __shared__ double sh_max[1024];
  __shared__ int sh_k;
  DeviceScalars* sc = D.sc;
  const int n = D.n;
  const double* Rsk = D.Rsk;
  const int64_t ldr = D.ldr;
  double* f2 = D.f2;
  if (sc->status != kOk) {
    if (threadIdx.x == 0) sc->k = 0;
    return;
  }
  if (D.tol > 0.0) {
    if (threadIdx.x == 0) sh_k = n;
    __syncthreads();
    const double thresh = __dmul_rn(D.tol, Rsk[0]);
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      if (!(Rsk[(int64_t)j * ldr + j] > thresh)) atomicMin(&sh_k, j);
    __syncthreads();
    if (threadIdx.x == 0) sc->k = sh_k;
    return;
  }
  // stage 1
  double mx = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double rs = 0.0;
    for (int c = l; c < n; ++c) {
      const double v = Rsk[(int64_t)c * ldr + l];
      rs = __fma_rn(v, v, rs);
      const double a = fabs(v);
      mx = a > mx ? a : mx;
    }
    f2[l] = rs;
  }
  sh_max[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) smax = sh_max[i] > smax ? sh_max[i] : smax;
    const double thresh = __dmul_rn(ldexp(1.0, -53), smax);
    // suffix sums f2[l] = f2[l+1] + rs_l
    double acc = 0.0;
    f2[n] = 0.0;
    for (int l = n - 1; l >= 0; --l) {
      acc = __dadd_rn(acc, f2[l]);
      f2[l] = acc;
    }
    int ko = n;
    for (int l = 0; l <= n; ++l)
      if (__dsqrt_rn(f2[l]) <= thresh) { ko = l; break; }
    sc->k = ko;
  }
}

__global__ void __launch_bounds__(1024) rank_kernel(RankDesc D) { rank_body(D); }
__global__ void __launch_bounds__(1024) rank_batched_kernel(const RankDesc* D) {
  rank_body(D[blockIdx.x]);
}

cudaError_t launch_rank(int n, const double* Rsk, int64_t ldr, double tol, DeviceScalars* sc,
                        double* f2, cudaStream_t stream) {
  RankDesc D{n, Rsk, ldr, tol, f2, sc};
  rank_kernel<<<1, 1024, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rank_batched(const RankDesc* D, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  rank_batched_kernel<<<nprob, 1024, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

// Stage 2: k := min(k, fail) (Remark 4), then if requested the largest
// l <= k with max/min of diag(R^pre)[0:l] <= 10.
__device__ __forceinline__ void stage2_body(const Stage2Desc& D) {
  DeviceScalars* sc = D.sc;
  if (sc->status != kOk) { sc->k = 0; return; }
  int64_t k = sc->k;
  if (sc->fail >= 0 && sc->fail < k) k = sc->fail;
  if (D.stage2 && k > 0) {
    int64_t kk = 0;
    double mx = 0.0, mn = 0.0;
    for (int64_t l = 1; l <= k; ++l) {
      const double dl = D.Rpre[(l - 1) * D.ldp + (l - 1)];
      if (l == 1) { mx = dl; mn = dl; }
      else { mx = dl > mx ? dl : mx; mn = dl < mn ? dl : mn; }
      if (__ddiv_rn(mx, mn) <= 10.0) kk = l; else break;
    }
    k = kk;
  }
  sc->k = k;
}

__global__ void rank_stage2_kernel(Stage2Desc D) { stage2_body(D); }
__global__ void rank_stage2_batched_kernel(const Stage2Desc* D, int np) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) stage2_body(D[p]);
}

cudaError_t launch_rank_stage2(const double* Rpre, int64_t ldp, bool stage2, DeviceScalars* sc,
                               cudaStream_t stream) {
  Stage2Desc D{Rpre, ldp, stage2 ? 1 : 0, sc};
  rank_stage2_kernel<<<1, 1, 0, stream>>>(D);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rank_stage2_batched(const Stage2Desc* D, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  rank_stage2_batched_kernel<<<(nprob + 127) / 128, 128, 0, stream>>>(D, nprob);
  count_launches(1);
  return cudaGetLastError();
}

__device__ __forceinline__ void init_scalars_body(DeviceScalars* sc, int64_t k) {
  sc->k = k;
  sc->fail = -1;
  sc->status = kOk;
  sc->pad = 0;
  sc->bar.count = 0;
  sc->bar.released = 0;
}

__global__ void init_scalars_kernel(DeviceScalars* sc, int64_t k) { init_scalars_body(sc, k); }
__global__ void init_scalars_batched_kernel(DeviceScalars* sc, int np) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) init_scalars_body(sc + p, 0);
}

cudaError_t launch_init_scalars(DeviceScalars* sc, int64_t k, cudaStream_t stream) {
  init_scalars_kernel<<<1, 1, 0, stream>>>(sc, k);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars_batched(DeviceScalars* sc, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  init_scalars_batched_kernel<<<(nprob + 127) / 128, 128, 0, stream>>>(sc, nprob);
  count_launches(1);
  return cudaGetLastError();
}

__device__ __forceinline__ void finalize_body(DeviceScalars* sc, int64_t* k_out, int* status_out) {
  int st = sc->status;
  if (st == kOk && sc->k == 0) st = kRankZero;
  if (st != kOk && st != kRankZero) sc->k = 0;
  if (k_out) *k_out = sc->k;
  if (status_out) *status_out = st;
}

__global__ void finalize_kernel(DeviceScalars* sc, int64_t* k_out, int* status_out) {
  finalize_body(sc, k_out, status_out);
}
__global__ void finalize_batched_kernel(const FinalDesc* D, int np) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) finalize_body(D[p].sc, D[p].k_out, D[p].status_out);
}

cudaError_t launch_finalize(DeviceScalars* sc, int64_t* k_out, int* status_out,
                            cudaStream_t stream) {
  finalize_kernel<<<1, 1, 0, stream>>>(sc, k_out, status_out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_finalize_batched(const FinalDesc* D, int nprob, cudaStream_t stream) {
  if (nprob <= 0) return cudaSuccess;
  finalize_batched_kernel<<<(nprob + 127) / 128, 128, 0, stream>>>(D, nprob);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cqrrpt
