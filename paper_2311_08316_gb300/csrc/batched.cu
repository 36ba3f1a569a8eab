// Batched CQRRPT: many independent, uneven problems factored by one batched
// launch per phase of Alg. 2 (14 launches for the whole batch, replayed as
// one CUDA graph when the batch's launch shapes repeat).
//
// Each batched kernel maps CTA b to (problem p, tile t) through a prefix
// table of per-problem tile counts and runs the same body as the
// single-problem kernel, so every problem's J, k, Q and R are bit-identical
// to a standalone cqrrpt_d call on the same inputs, whatever else shares the
// batch.  The QRCP and the Cholesky give one CTA to each problem (block
// barriers only: nothing waits on another CTA).
//
// The per-phase descriptor tables and tile prefix tables are written into a
// pinned host staging buffer and copied to the workspace with one
// cudaMemcpyAsync per call; the copy is ordered before the launches on the
// caller's stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/cqrrpt.h"
#include "batched.h"
#include "kernels.h"

namespace cqrrpt {

namespace {

struct Layout {
  // byte offsets inside the batch region
  size_t tables, scalars, per_problem;
  size_t total;
};

template <class T>
size_t push_table(std::vector<char>& buf, const std::vector<T>& v) {
  const size_t off = (buf.size() + 255) & ~size_t(255);
  buf.resize(off + v.size() * sizeof(T));
  if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

}  // namespace

int64_t problem_workspace_bytes(int64_t m, int64_t n, int64_t d, int nnz) {
  const int64_t a = sketch_workspace_bytes(m, n, (int)d, nnz);
  const int64_t b = gram_block_workspace_bytes(m, n);
  int64_t t = (a > b ? a : b);
  t += align256(d * n * 8);
  t += qrcp_workspace_bytes(n);
  t += 3 * align256(n * n * 8);
  t += align256((n + 1) * 8);
  return t;
}

BatchTuning default_tuning() {
  BatchTuning t;
  for (int b = 0; b < kTuneBuckets; ++b) {
    t.trsm_jb[b] = 32;
    t.gram_tile[b] = b < 8 ? 8 : 32;  // the autotuner's choice on uneven batches up to n = 256
  }
  return t;
}

int batch_plan(BatchPlan& P, int batch, const BatchProblem* probs, char* ws_base,
               char* const* ws_each, const BatchTuning* tune, const int* scalar_index) {
  const BatchTuning TU = tune ? *tune : default_tuning();
  DeviceScalars* scalars = P.scalars;
  char* tables = P.tables;
  P = BatchPlan();
  P.scalars = scalars;
  P.tables = tables;
  P.nprob = batch;
  P.rsk.assign((size_t)batch, nullptr);
  P.g.assign((size_t)batch, nullptr);
  P.rpre.assign((size_t)batch, nullptr);
  // per-problem workspace
  char* w = ws_base;
  std::vector<SketchDesc> sk(batch);
  std::vector<QrcpDesc> qr(batch);
  std::vector<RankDesc> rk(batch);
  std::vector<TrsmDesc> t1(batch), t2(batch);
  std::vector<GramDesc> gr(batch);
  std::vector<PotrfDesc> po(batch);
  std::vector<Stage2Desc> s2(batch);
  std::vector<TrmmDesc> tm(batch);
  std::vector<FinalDesc> fi(batch);
  std::vector<int64_t> b_list(batch + 1), b_part(batch + 1), b_comb(batch + 1),
      b_gath(batch + 1), b_trsm(batch + 1), b_gp(batch + 1), b_gc(batch + 1), b_tm(batch + 1);
  DeviceScalars* sc = P.scalars;
  b_list[0] = b_part[0] = b_comb[0] = b_gath[0] = b_trsm[0] = b_gp[0] = b_gc[0] = b_tm[0] = 0;
  int max_d = 1;
  int64_t qrcp_smem = 0;
  for (int p = 0; p < batch; ++p) {
    const BatchProblem& q = probs[p];
    const int64_t m = q.m, n = q.n, d = q.d;
    if (d > max_d) max_d = (int)d;
    const int64_t a = sketch_workspace_bytes(m, n, (int)d, q.nnz);
    const int64_t b = gram_block_workspace_bytes(m, n);
    if (ws_each) w = ws_each[p];  // problem p's own workspace
    char* region = w;
    w += (a > b ? a : b);
    double* X = (double*)w; w += align256(d * n * 8);
    void* qw = w; w += qrcp_workspace_bytes(n);
    double* Rsk = (double*)w; w += align256(n * n * 8);
    double* G = (double*)w; w += align256(n * n * 8);
    double* Rpre = (double*)w; w += align256(n * n * 8);
    double* f2 = (double*)w; w += align256((n + 1) * 8);
    P.rsk[(size_t)p] = Rsk;
    P.g[(size_t)p] = G;
    P.rpre[(size_t)p] = Rpre;
    DeviceScalars* s = sc + (scalar_index ? scalar_index[p] : p);
    const int bucket = tune_bucket(n);
    const int jb = TU.trsm_jb[bucket] == 16 ? 16 : 32;
    const int gt = TU.gram_tile[bucket] == 8 ? 8 : TU.gram_tile[bucket] == 16 ? 16 : 32;
    SketchDesc& S = sk[p];
    S = SketchDesc{};
    S.m = m; S.n = n; S.d = (int)d; S.s = q.nnz; S.seed = q.seed;
    S.scale = 1.0 / std::sqrt((double)q.nnz);
    S.M = q.A; S.ldm = q.lda; S.Msk = X; S.ldsk = d; S.status = &s->status;
    sketch_carve(S, region);
    qr[p] = QrcpDesc{(int)d, (int)n, X, d, qrcp_carve(qw, (int)n), q.J, Rsk, n, s};
    {  // shared memory the batched QRCP would like for this problem
      const int64_t want = (d + 2 * n) * 8 + 2 * n * 4 + n * d * 8;
      if (want > qrcp_smem) qrcp_smem = want;
    }
    rk[p] = RankDesc{(int)n, Rsk, n, q.tol, f2, s};
    t1[p] = TrsmDesc{m, &s->k, q.A, q.lda, q.J, Rsk, n, q.Q, q.ldq, &s->status, jb};
    gr[p] = GramDesc{m, (int)n, &s->k, q.Q, q.ldq, (double*)region, G, n, &s->status, gt};
    po[p] = PotrfDesc{(int)n, G, n, Rpre, n, s};
    s2[p] = Stage2Desc{Rpre, n, q.tol > 0.0 ? 0 : 1, s};
    t2[p] = TrsmDesc{m, &s->k, q.Q, q.ldq, nullptr, Rpre, n, q.Q, q.ldq, &s->status, jb};
    tm[p] = TrmmDesc{(int)n, &s->k, Rpre, n, Rsk, n, q.R, q.ldr, &s->status};
    fi[p] = FinalDesc{s, q.k_out, q.status_out};
    b_list[p + 1] = b_list[p] + sketch_list_tiles(S);
    b_part[p + 1] = b_part[p] + sketch_partial_tiles(S);
    b_comb[p + 1] = b_comb[p] + sketch_combine_tiles(S);

    b_trsm[p + 1] = b_trsm[p] + trsm_tiles(m);
    b_gp[p + 1] = b_gp[p] + gram_partial_tiles(m, (int)n, gt);
    b_gc[p + 1] = b_gc[p] + gram_combine_tiles((int)n);
    b_tm[p + 1] = b_tm[p] + trmm_tiles((int)n);
  }
  P.max_d = max_d;
  P.qrcp_smem = qrcp_smem < kQrcpSmemCap ? qrcp_smem : kQrcpSmemCap;
  // the QRCP takes one CTA per problem: largest work (n^2 d) first, so that
  // the long factorisations do not start last; the gather follows the same
  // order
  {
    std::vector<int> order((size_t)batch);
    for (int p = 0; p < batch; ++p) order[(size_t)p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const double wa = (double)probs[a].n * probs[a].n * probs[a].d;
      const double wb = (double)probs[b].n * probs[b].n * probs[b].d;
      return wa > wb;
    });
    std::vector<QrcpDesc> sorted((size_t)batch);
    for (int i = 0; i < batch; ++i) {
      sorted[(size_t)i] = qr[(size_t)order[(size_t)i]];
      b_gath[i + 1] = b_gath[i] + sorted[(size_t)i].n;
    }
    qr.swap(sorted);
  }
  P.tiles_list = b_list[batch];
  P.tiles_part = b_part[batch];
  P.tiles_comb = b_comb[batch];
  P.tiles_gath = b_gath[batch];
  P.tiles_trsm = b_trsm[batch];
  P.tiles_gp = b_gp[batch];
  P.tiles_gc = b_gc[batch];
  P.tiles_tm = b_tm[batch];
  // table image (host), then offsets become device pointers into P.tables
  std::vector<char>& img = P.image;
  img.clear();
  const size_t o_sk = push_table(img, sk), o_qr = push_table(img, qr), o_rk = push_table(img, rk),
               o_t1 = push_table(img, t1), o_t2 = push_table(img, t2), o_gr = push_table(img, gr),
               o_po = push_table(img, po), o_s2 = push_table(img, s2), o_tm = push_table(img, tm),
               o_fi = push_table(img, fi);
  const size_t o_bl = push_table(img, b_list), o_bp = push_table(img, b_part),
               o_bc = push_table(img, b_comb), o_bg = push_table(img, b_gath),
               o_bt = push_table(img, b_trsm), o_bgp = push_table(img, b_gp),
               o_bgc = push_table(img, b_gc), o_btm = push_table(img, b_tm);
  char* T = P.tables;
  P.sk = (const SketchDesc*)(T + o_sk);
  P.qr = (const QrcpDesc*)(T + o_qr);
  P.rk = (const RankDesc*)(T + o_rk);
  P.t1 = (const TrsmDesc*)(T + o_t1);
  P.t2 = (const TrsmDesc*)(T + o_t2);
  P.gr = (const GramDesc*)(T + o_gr);
  P.po = (const PotrfDesc*)(T + o_po);
  P.s2 = (const Stage2Desc*)(T + o_s2);
  P.tm = (const TrmmDesc*)(T + o_tm);
  P.fi = (const FinalDesc*)(T + o_fi);
  P.base_list = (const int64_t*)(T + o_bl);
  P.base_part = (const int64_t*)(T + o_bp);
  P.base_comb = (const int64_t*)(T + o_bc);
  P.base_gath = (const int64_t*)(T + o_bg);
  P.base_trsm = (const int64_t*)(T + o_bt);
  P.base_gp = (const int64_t*)(T + o_bgp);
  P.base_gc = (const int64_t*)(T + o_bgc);
  P.base_tm = (const int64_t*)(T + o_btm);
  return 0;
}

cudaError_t batch_launch_front(const BatchPlan& P, cudaStream_t s) {
  const int np = P.nprob;
  cudaError_t e = launch_init_scalars_batched(P.scalars, np, s);
  if (e == cudaSuccess) e = launch_sketch_batched(0, P.sk, P.base_list, np, P.tiles_list, P.max_d, s);
  if (e == cudaSuccess) e = launch_sketch_batched(1, P.sk, P.base_part, np, P.tiles_part, P.max_d, s);
  if (e == cudaSuccess) e = launch_sketch_batched(2, P.sk, P.base_comb, np, P.tiles_comb, P.max_d, s);
  if (e == cudaSuccess)
    e = launch_qrcp_batched(P.qr, np, P.base_gath, P.tiles_gath, P.qrcp_smem, s);
  if (e == cudaSuccess) e = launch_rank_batched(P.rk, np, s);
  return e;
}

cudaError_t batch_launch(const BatchPlan& P, cudaStream_t s) {
  const int np = P.nprob;
  cudaError_t e = batch_launch_front(P, s);
  if (e == cudaSuccess) e = launch_trsm_rut_batched(P.t1, P.base_trsm, np, P.tiles_trsm, s);
  if (e == cudaSuccess) e = launch_gram_batched(0, P.gr, P.base_gp, np, P.tiles_gp, s);
  if (e == cudaSuccess) e = launch_gram_batched(1, P.gr, P.base_gc, np, P.tiles_gc, s);
  if (e == cudaSuccess) e = launch_potrf_batched(P.po, np, s);
  if (e == cudaSuccess) e = launch_rank_stage2_batched(P.s2, np, s);
  if (e == cudaSuccess) e = launch_trsm_rut_batched(P.t2, P.base_trsm, np, P.tiles_trsm, s);
  if (e == cudaSuccess) e = launch_trmm_batched(P.tm, P.base_tm, np, P.tiles_tm, s);
  if (e == cudaSuccess) e = launch_finalize_batched(P.fi, np, s);
  return e;
}

}  // namespace cqrrpt
