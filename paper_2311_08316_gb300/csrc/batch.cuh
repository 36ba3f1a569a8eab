// Per-kernel problem descriptors and the CTA -> problem map used by the
// batched launches: one launch covers every problem of a batch; CTA b
// belongs to problem p with base[p] <= b < base[p+1] (base = prefix sums of
// the per-problem tile counts, in device memory) and works on tile
// b - base[p] of that problem, exactly as the single-problem kernel would.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace cqrrpt {

// Device scalars of one factorisation.
struct DeviceScalars {
  int64_t k;         // current rank (rank rule, then Remark 4, then stage 2)
  int64_t fail;      // Cholesky failure column or -1
  int status;        // kOk / kNonFinite / kTimeout ...
  int pad;
  GridBarrier bar;
};

struct SketchDesc {
  int64_t m, n;
  int d, s;
  uint64_t seed;
  int64_t row0;  // index in the whole matrix of M's first row (column row0 + r of S)
  double scale;
  const double* M;
  int64_t ldm;
  int* seg_start;
  uint32_t* entries;
  double* partial;
  double* Msk;
  int64_t ldsk;
  int* status;
};

struct QrcpWork {
  double* vn1;
  double* vn2;
  double* tau;
  int* phys;
  int* posof;
  double* cand_val;
  int* cand_pos;
  int* cand_col;
  double* cand_refl;  // per record: tau, beta, 1 / (alpha - beta), nz (as 0.0 / 1.0)
};

struct QrcpDesc {
  int d, n;
  double* X;
  int64_t ldx;
  QrcpWork w;
  int64_t* J;
  double* Rsk;
  int64_t ldr;
  DeviceScalars* sc;
  int nopivot;  // 1: plain Householder QR (the column at position j is step j's pivot)
};

struct RankDesc {
  int n;
  const double* Rsk;
  int64_t ldr;
  double tol;
  double* f2;
  DeviceScalars* sc;
};

struct TrsmDesc {
  int64_t m;
  const int64_t* k_dev;
  const double* B;
  int64_t ldb;
  const int64_t* cols;
  const double* T;
  int64_t ldt;
  double* X;
  int64_t ldx;
  const int* status;
  int jb;  // widest register block of columns: 16 or 32 (0 = 32)
};

struct GramDesc {
  int64_t m;
  int n_ld;
  const int64_t* k_dev;
  const double* X;
  int64_t ldx;
  double* partial;
  double* G;
  int64_t ldg;
  const int* status;
  int tile;  // output tile edge: 8, 16 or 32 (0 = 32)
  int sub;   // 1: partials per kGramSub-row sub-block (else per kRowBlock block)
};

struct PotrfDesc {
  int kmax;
  double* G;
  int64_t ldg;
  double* R;
  int64_t ldr;
  DeviceScalars* sc;
};

struct Stage2Desc {
  const double* Rpre;
  int64_t ldp;
  int stage2;
  DeviceScalars* sc;
};

struct TrmmDesc {
  int n;
  const int64_t* k_dev;
  const double* Rp;
  int64_t ldp;
  const double* Rs;
  int64_t lds;
  double* R;
  int64_t ldr;
  const int* status;
};

struct FinalDesc {
  DeviceScalars* sc;
  int64_t* k_out;
  int* status_out;
};

// largest p with base[p] <= b (binary search; base[0] = 0, base[nprob] = total)
__device__ __forceinline__ int find_problem(const int64_t* __restrict__ base, int nprob,
                                            int64_t b, int64_t* local) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= b) lo = mid; else hi = mid - 1;
  }
  *local = b - base[lo];
  return lo;
}

}  // namespace cqrrpt
