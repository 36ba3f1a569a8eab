// Host-side planning of a batched CQRRPT (see batched.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "kernels.h"

namespace cqrrpt {

// One problem of a batch (all pointers are device pointers).
struct BatchProblem {
  int64_t m, n, d;
  int nnz;
  double tol;
  uint64_t seed;
  const double* A;
  int64_t lda;
  double* Q;
  int64_t ldq;
  double* R;
  int64_t ldr;
  int64_t* J;
  int64_t* k_out;     // device, may be null
  int* status_out;    // device, may be null
};

struct BatchPlan {
  int nprob = 0, max_d = 1;
  int64_t qrcp_smem = 0;  // dynamic shared memory of the batched QRCP
  int64_t tiles_list = 0, tiles_part = 0, tiles_comb = 0, tiles_gath = 0, tiles_trsm = 0,
          tiles_gp = 0, tiles_gc = 0, tiles_tm = 0;
  DeviceScalars* scalars = nullptr;  // device, nprob entries
  char* tables = nullptr;            // device image of `image`
  std::vector<char> image;           // host image of the tables
  const SketchDesc* sk = nullptr;
  const QrcpDesc* qr = nullptr;
  const RankDesc* rk = nullptr;
  const TrsmDesc* t1 = nullptr;
  const TrsmDesc* t2 = nullptr;
  const GramDesc* gr = nullptr;
  const PotrfDesc* po = nullptr;
  const Stage2Desc* s2 = nullptr;
  const TrmmDesc* tm = nullptr;
  const FinalDesc* fi = nullptr;
  const int64_t *base_list = nullptr, *base_part = nullptr, *base_comb = nullptr,
                *base_gath = nullptr, *base_trsm = nullptr, *base_gp = nullptr,
                *base_gc = nullptr, *base_tm = nullptr;
  // each problem's R^sk, G and R^pre inside its workspace (ld n)
  std::vector<double*> rsk, g, rpre;
};

// Tile shapes of the batched O(m n^2) kernels, per problem width bucket
// b = min((n - 1) / 32, kTuneBuckets - 1): the TRSM's widest register block
// (16 or 32 columns) and the Gram's output tile edge (16 or 32).  Only the
// blocking changes, never the arithmetic.
constexpr int kTuneBuckets = 16;
struct BatchTuning {
  int trsm_jb[kTuneBuckets];
  int gram_tile[kTuneBuckets];
};
inline int tune_bucket(int64_t n) {
  const int64_t b = (n - 1) / 32;
  return (int)(b < kTuneBuckets - 1 ? b : kTuneBuckets - 1);
}
// untuned shapes: 32-column TRSM blocks; 16 x 16 Gram tiles up to n = 64
BatchTuning default_tuning();

// workspace of one problem inside a batch
int64_t problem_workspace_bytes(int64_t m, int64_t n, int64_t d, int nnz);
// upper bound of the table image for `batch` problems
inline int64_t batch_table_bytes(int batch) {
  const int64_t descs = 10 * 256 + (int64_t)batch * (sizeof(SketchDesc) + sizeof(QrcpDesc) +
                                                      sizeof(RankDesc) + 2 * sizeof(TrsmDesc) +
                                                      sizeof(GramDesc) + sizeof(PotrfDesc) +
                                                      sizeof(Stage2Desc) + sizeof(TrmmDesc) +
                                                      sizeof(FinalDesc));
  const int64_t bases = 8 * (256 + (int64_t)(batch + 1) * 8);
  return align256(descs + bases + 256);
}
// Fills P (P.scalars and P.tables must be set by the caller beforehand) and
// carves every problem's workspace from ws_base onward, or, when ws_each is
// given, problem p's workspace (problem_workspace_bytes) from ws_each[p].
// Problem p uses the device scalars P.scalars[p], or P.scalars[scalar_index[p]]
// when scalar_index is given; tile shapes come from `tune` (NULL: defaults).
int batch_plan(BatchPlan& P, int batch, const BatchProblem* probs, char* ws_base,
               char* const* ws_each = nullptr, const BatchTuning* tune = nullptr,
               const int* scalar_index = nullptr);
// Enqueues the 14 batched launches.
cudaError_t batch_launch(const BatchPlan& P, cudaStream_t s);
// The first six of them: scalars, sketch (3), QRCP, rank rule.
cudaError_t batch_launch_front(const BatchPlan& P, cudaStream_t s);
cudaError_t sketch_set_attributes(int max_d);

}  // namespace cqrrpt
