// C ABI of the CQRRPT library (declared in include/cqrrpt.h): argument
// checking, workspace planning and the stream-ordered pipeline of Alg. 2.
// No entry point synchronises unless it is given a host output pointer.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cqrrpt.h"
#include "batched.h"
#include "kernels.h"
#include "ozaki.h"
#include "saso.cuh"

using namespace cqrrpt;

constexpr int kPhases = 8;  // sketch, qrcp, rank, trsm(M^pre), gram, chol, trsm(Q), trmm

struct cqrrpt_ctx {
  int device = 0;
  int num_sms = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  DeviceScalars* sc = nullptr;  // per-call device scalars
  int64_t* pinned = nullptr;    // host-pinned readback (k, status)
  int profiling = 0;
  cudaEvent_t ev[kPhases + 1] = {};
  // batched path: pinned staging of the launch tables, graph cache
  void* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t stage_ev = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_key[12] = {};
  int graph_kernels = 0;
  int use_graphs = 1;
  BatchTuning tune = default_tuning();  // tile shapes of the batched kernels
  // batched split-BF16 path: its own device workspace, pinned read-back of
  // every problem's device scalars
  void* split_ws = nullptr;
  size_t split_ws_bytes = 0;
  DeviceScalars* pinned_sc = nullptr;
  int pinned_sc_count = 0;
  // host pipeline: double-buffered device copies of A, Q, R, J for an
  // m x n shape, copy-in and copy-out streams, events (in, compute, out per
  // buffer), device and pinned slots for k and status
  double* pipe_a[2] = {};
  double* pipe_q[2] = {};
  double* pipe_r[2] = {};
  int64_t* pipe_j[2] = {};
  int64_t pipe_m = 0, pipe_n = 0;
  int64_t* pipe_slots = nullptr;  // device: k[2], then status[2] as int
  int64_t* pipe_pin = nullptr;    // pinned copy of the same 32 bytes
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev[6] = {};
  // split path: side stream and fork/join events (inverses beside splits)
  cudaStream_t side = nullptr;
  cudaEvent_t side_ev[2] = {};
  // row-partitioned form (cqrrpt_shard_*): this rank's rows and the state
  // carried from one phase to the next
  struct {
    const double* A = nullptr;
    int64_t lda = 0, m = 0, rows = 0, row0 = 0, n = 0, d = 0;
    int nnz = 0;
    double tol = 0.0;
    const int64_t* J = nullptr;
    int phase = 0;  // 1 sketched, 2 factored the sketch, 3 Gram block sums
  } shard;
};

static std::atomic<long long> g_launches{0};

namespace cqrrpt {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// The dynamic shared-memory limit of a kernel is one attribute per device,
// shared by every thread and stream: it is only ever raised (to the largest
// size any launch has asked for), under a lock, so that a launch on one
// stream never finds the limit lowered below its own size by another.
cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[std::make_pair(dev, fn)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
// k and status of the handle's last call into caller slots, stream-ordered
int handle_finalize(cqrrpt_handle h, int64_t* k_out, int* status_out, cudaStream_t s) {
  return launch_finalize(h->sc, k_out, status_out, s) == cudaSuccess ? kOk : kCudaError;
}
const BatchTuning* handle_tuning(cqrrpt_handle h) { return &h->tune; }
}  // namespace cqrrpt

namespace {

inline void mark(cqrrpt_handle h, int i, cudaStream_t s) {
  if (h->profiling) cudaEventRecord(h->ev[i], s);
}

struct Plan {
  int64_t d, nb;
  size_t region, x, qrcp, rsk, g, rpre, f2, total;
};

Plan plan_fp64(int64_t m, int64_t n, int64_t d, int nnz) {
  Plan p;
  p.d = d;
  p.nb = (m + kRowBlock - 1) / kRowBlock;
  const int64_t a = sketch_workspace_bytes(m, n, (int)d, nnz);
  const int64_t b = gram_workspace_bytes(m, n);
  p.region = (size_t)(a > b ? a : b);
  p.x = (size_t)align256(d * n * 8);
  p.qrcp = (size_t)qrcp_workspace_bytes(n);
  p.rsk = (size_t)align256(n * n * 8);
  p.g = p.rsk;
  p.rpre = p.rsk;
  p.f2 = (size_t)align256((n + 1) * 8);
  p.total = p.region + p.x + p.qrcp + p.rsk + p.g + p.rpre + p.f2;
  return p;
}

int ensure_ws(cqrrpt_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return kOk;
  if (h->ws) {
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return kNoMemory;
  }
  h->ws_bytes = bytes;
  return kOk;
}

int64_t sketch_dim(int64_t n, double gamma) { return (int64_t)std::ceil(gamma * (double)n); }

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

__global__ void copy_k_kernel(const DeviceScalars* sc, int64_t* out) { *out = sc->k; }
__global__ void copy_fail_kernel(const DeviceScalars* sc, int64_t* out) { *out = sc->fail; }

bool precision_ok(int p) {
  return p == CQRRPT_FP64 || p == CQRRPT_SPLITBF16 || p == CQRRPT_SPLITBF16_CHOLQR2;
}

// Workspace of the split-BF16 modes: the sketch scratch and the tensor-core
// scratch share one region; then M^sk, QRCP work, R^sk, G, R^pre, f2, a copy
// of the first-pass R and the device scalars of the second pass.
Plan plan_for(int64_t m, int64_t n, int64_t d, int nnz, int precision) {
  if (precision == CQRRPT_FP64) return plan_fp64(m, n, d, nnz);
  Plan p = plan_fp64(m, n, d, nnz);
  int64_t region = sketch_workspace_bytes(m, n, (int)d, nnz);
  const int64_t t = oz_trsm_inv_workspace(m, (int)n);
  const int64_t gw = oz_gram_workspace(m, (int)n, nullptr);
  region = region > t ? region : t;
  region = region > gw ? region : gw;
  p.region = (size_t)align256(region);
  p.total = p.region + p.x + p.qrcp + p.rsk + p.g + p.rpre + p.f2 + p.rsk +
            (size_t)align256(sizeof(DeviceScalars));
  return p;
}

int read_k(cqrrpt_handle h, DeviceScalars* sc, cudaStream_t s, int64_t* k, int* st) {
  if (launch_finalize(sc, h->pinned, (int*)(h->pinned + 1), s) != cudaSuccess) return kCudaError;
  if (cudaStreamSynchronize(s) != cudaSuccess) return kCudaError;
  *k = h->pinned[0];
  *st = *(int*)(h->pinned + 1);
  return kOk;
}

// Split-BF16 pipeline: FP64 sketch, QRCP, rank, Cholesky and TRMM; lines 4,
// 5 and 7 as FP64-accurate tensor-core products (ozaki.cu).  The recursive
// TRSM needs k on the host, so this path reads k back twice (after the rank
// rule and after the Cholesky).
int run_split(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda, int64_t d,
              int nnz, double tol, uint64_t seed, int precision, double* Q, int64_t ldq, double* R,
              int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host, cudaStream_t stream,
              const double* S_dense = nullptr, int64_t lds = 0) {
  const Plan p = plan_for(m, n, d, nnz, precision);
  // a dense operator's split-BF16 sketch may need a larger first region
  const int64_t need = S_dense ? sketch_dense_split_workspace_bytes(m, n, (int)d) : 0;
  const size_t extra = need > (int64_t)p.region ? (size_t)align256(need) - p.region : 0;
  int st = ensure_ws(h, p.total + extra);
  if (st != kOk) return st;
  char* w = (char*)h->ws;
  void* region = w; w += p.region + extra;
  double* X = (double*)w; w += p.x;
  void* qw = w; w += p.qrcp;
  double* Rsk = (double*)w; w += p.rsk;
  double* G = (double*)w; w += p.g;
  double* Rpre = (double*)w; w += p.rpre;
  double* f2 = (double*)w; w += p.f2;
  double* R1 = (double*)w; w += p.rsk;
  DeviceScalars* sc2 = (DeviceScalars*)w;
  DeviceScalars* sc = h->sc;
  int* status = &sc->status;
  const int ni = (int)n, di = (int)d;
  const double scale = 1.0 / std::sqrt((double)nnz);

  cudaError_t e = launch_init_scalars(sc, 0, stream);
  mark(h, 0, stream);
  if (e == cudaSuccess)
    e = S_dense ? launch_sketch_dense_split(m, n, S_dense, lds, A, lda, di, X, d, region, status,
                                          stream)
                : launch_sketch(m, n, A, lda, di, nnz, seed, scale, X, d, region, status, stream);
  mark(h, 1, stream);
  if (e == cudaSuccess) e = launch_qrcp(di, ni, X, d, J, Rsk, n, qw, sc, h->num_sms, stream);
  mark(h, 2, stream);
  if (e == cudaSuccess) e = launch_rank(ni, Rsk, n, tol, sc, f2, stream);
  mark(h, 3, stream);
  if (e != cudaSuccess) return kCudaError;
  int64_t k = 0;
  int dst = kOk;
  if ((st = read_k(h, sc, stream, &k, &dst)) != kOk) return st;
  // the inverses of lines 4 and 7 run on a side stream beside the splits
  const OzSide* side = nullptr;
  OzSide side_v{};
  if (!h->side && cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaEventCreateWithFlags(&h->side_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->side_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return kCudaError;
    }
  }
  cudaGetLastError();
  if (h->side && h->side_ev[0] && h->side_ev[1]) {
    side_v = OzSide{h->side, h->side_ev[0], h->side_ev[1]};
    side = &side_v;
  }
  if (dst == kOk && k > 0) {
    // line 4: M^pre = M[:, J[:k]] (R^sk_11)^{-1} into Q
    // (row-wise FP64 inverse of the row-graded R^sk_11, then one product)
    e = oz_trsm_inv(m, (int)k, A, lda, J, Rsk, n, Q, ldq, region, stream, status, side);
    mark(h, 4, stream);
    // line 5: G = M^pre^T M^pre
    if (e == cudaSuccess) e = oz_gram(m, (int)k, Q, ldq, G, n, region, stream, status);
    mark(h, 5, stream);
    // line 6 (FP64) and the rank rule's stage 2
    if (e == cudaSuccess) e = launch_potrf((int)k, G, n, Rpre, n, sc, stream);
    if (e == cudaSuccess) e = launch_rank_stage2(Rpre, n, !(tol > 0.0), sc, stream);
    if (e != cudaSuccess) return kCudaError;
    if ((st = read_k(h, sc, stream, &k, &dst)) != kOk) return st;
    mark(h, 6, stream);
    if (dst == kOk && k > 0) {
      // line 7: Q_k = M^pre (R^pre)^{-1}, in place; R^pre is well conditioned
      // (Theorem 3), so one product with its FP64 inverse
      e = oz_trsm_inv(m, (int)k, Q, ldq, nullptr, Rpre, n, Q, ldq, region, stream, status, side);
      mark(h, 7, stream);
      // line 8: R_k = R^pre R^sk_k
      double* Rout = (precision == CQRRPT_SPLITBF16_CHOLQR2) ? R1 : R;
      const int64_t ldo = (precision == CQRRPT_SPLITBF16_CHOLQR2) ? n : ldr;
      if (e == cudaSuccess) e = launch_trmm(ni, &sc->k, Rpre, n, Rsk, n, Rout, ldo, status, stream);
      if (e == cudaSuccess && precision == CQRRPT_SPLITBF16_CHOLQR2) {
        // second Cholesky-QR pass on Q: G2 = Q^T Q, R2 = chol(G2),
        // Q := Q R2^{-1}, R := R2 R1.  A breakdown here keeps the first pass.
        e = launch_init_scalars(sc2, k, stream);
        if (e == cudaSuccess) e = oz_gram(m, (int)k, Q, ldq, G, n, region, stream, status);
        if (e == cudaSuccess) e = launch_potrf((int)k, G, n, Rpre, n, sc2, stream);
        if (e == cudaSuccess) {
          copy_fail_kernel<<<1, 1, 0, stream>>>(sc2, h->pinned + 4);
          count_launches(1);
          e = cudaGetLastError();
        }
        if (e == cudaSuccess && cudaStreamSynchronize(stream) != cudaSuccess) return kCudaError;
        if (e == cudaSuccess && h->pinned[4] < 0) {
          e = oz_trsm_inv(m, (int)k, Q, ldq, nullptr, Rpre, n, Q, ldq, region, stream, status);
          if (e == cudaSuccess) e = launch_trmm(ni, &sc->k, Rpre, n, R1, n, R, ldr, status, stream);
        } else if (e == cudaSuccess) {
          // second pass broke down: keep the first pass's R
          e = cudaMemcpy2DAsync(R, ldr * sizeof(double), R1, n * sizeof(double),
                                (size_t)k * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice,
                                stream);
        }
      }
      mark(h, 8, stream);
    }
  }
  if (e == cudaSuccess) e = launch_finalize(sc, k_dev, nullptr, stream);
  if (e != cudaSuccess) return kCudaError;
  if (k_host) {
    if ((st = read_k(h, sc, stream, &k, &dst)) != kOk) return st;
    *k_host = k;
    return dst;
  }
  return kOk;
}

}  // namespace

// Alg. 2 in FP64, one stream-ordered launch sequence (no host wait unless
// k_host is given).  form_q = false stops before line 7: Q then holds
// M^pre (the implicit Q with R^pre); Rpre_out (ld ld_rpre) receives R^pre,
// else it stays in the workspace.
static int run_fp64(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                    int64_t d, int nnz, double tol, uint64_t seed, double* Q, int64_t ldq,
                    double* R, int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host,
                    cudaStream_t stream, bool form_q, double* Rpre_out, int64_t ld_rpre,
                    bool pivoting = true, const double* S_dense = nullptr, int64_t lds = 0,
                    double srrqr_f = 0.0, int64_t* swaps_out = nullptr) {
  const Plan p = plan_fp64(m, n, d, nnz);
  const size_t sr_bytes = srrqr_f > 0.0 ? (size_t)srrqr_workspace_bytes((int)n) : 0;
  int st = ensure_ws(h, p.total + sr_bytes);
  if (st != kOk) return st;
  char* w = (char*)h->ws;
  void* region = w; w += p.region;
  double* X = (double*)w; w += p.x;
  void* qw = w; w += p.qrcp;
  double* Rsk = (double*)w; w += p.rsk;
  double* G = (double*)w; w += p.g;
  double* Rpre = (double*)w; w += p.rpre;
  int64_t ldp = n;
  if (Rpre_out) {  // R^pre straight into the caller's buffer
    Rpre = Rpre_out;
    ldp = ld_rpre;
  }
  double* f2 = (double*)w;
  w += p.f2;
  void* srw = w;
  DeviceScalars* sc = h->sc;
  int* status = &sc->status;
  const int ni = (int)n, di = (int)d;
  const double scale = 1.0 / std::sqrt((double)nnz);

  cudaError_t e = launch_init_scalars(sc, 0, stream);
  mark(h, 0, stream);
  if (e == cudaSuccess)
    e = S_dense ? launch_sketch_dense(m, n, S_dense, lds, A, lda, di, X, d, region, status, stream)
                : launch_sketch(m, n, A, lda, di, nnz, seed, scale, X, d, region, status, stream);
  mark(h, 1, stream);
  if (e == cudaSuccess) e = launch_qrcp(di, ni, X, d, J, Rsk, n, qw, sc, h->num_sms, stream, !pivoting);
  mark(h, 2, stream);
  if (e == cudaSuccess) e = launch_rank(ni, Rsk, n, tol, sc, f2, stream);
  if (e == cudaSuccess && srrqr_f > 0.0) {
    // Sec. 2.2: strong RRQR exchanges at the rank of line 3 (host-driven)
    int st1 = kOk;
    int64_t kk = 0, sw = 0;
    if (cqrrpt_last_status(h, stream, &st1, &kk) != kOk) e = cudaErrorUnknown;
    if (e == cudaSuccess && st1 == kOk)
      e = srrqr_exchange(ni, (int)kk, srrqr_f, Rsk, n, J, srw, qw, sc, h->num_sms,
                         (double*)(h->pinned + 4), 64 * n, &sw, stream);
    if (swaps_out) *swaps_out = sw;
  }
  mark(h, 3, stream);
  if (e == cudaSuccess)
    e = launch_trsm_rut(m, ni, &sc->k, A, lda, J, Rsk, n, Q, ldq, status, stream);
  mark(h, 4, stream);
  if (e == cudaSuccess)  // region holds gram_workspace_bytes(m, n): either form
    e = launch_gram(m, ni, &sc->k, Q, ldq, G, n, region, status, stream, false, true);
  mark(h, 5, stream);
  if (e == cudaSuccess) e = launch_potrf(ni, G, n, Rpre, ldp, sc, stream);
  if (e == cudaSuccess) e = launch_rank_stage2(Rpre, ldp, !(tol > 0.0), sc, stream);
  mark(h, 6, stream);
  if (e == cudaSuccess && form_q)
    e = launch_trsm_rut(m, ni, &sc->k, Q, ldq, nullptr, Rpre, ldp, Q, ldq, status, stream);
  mark(h, 7, stream);
  if (e == cudaSuccess) e = launch_trmm(ni, &sc->k, Rpre, ldp, Rsk, n, R, ldr, status, stream);
  mark(h, 8, stream);
  if (e == cudaSuccess) e = launch_finalize(sc, k_dev, nullptr, stream);
  if (e != cudaSuccess) return kCudaError;
  if (k_host) {
    int st2 = kOk;
    int64_t kk = 0;
    int r = cqrrpt_last_status(h, stream, &st2, &kk);
    if (r != kOk) return r;
    *k_host = kk;
    return st2;
  }
  return kOk;
}

extern "C" {

int cqrrpt_create(cqrrpt_handle* h, int device) {
  if (!h) return -1;
  *h = nullptr;
  DevGuard g(device);
  cqrrpt_ctx* c = new (std::nothrow) cqrrpt_ctx();
  if (!c) return kNoMemory;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&c->sc, sizeof(DeviceScalars)) != cudaSuccess ||
      cudaMallocHost(&c->pinned, 64) != cudaSuccess) {
    cudaGetLastError();
    if (c->sc) cudaFree(c->sc);
    delete c;
    return kCudaError;
  }
  cudaMemset(c->sc, 0, sizeof(DeviceScalars));
  cudaDeviceSynchronize();
  *h = c;
  return kOk;
}

int cqrrpt_destroy(cqrrpt_handle h) {
  if (!h) return -1;
  DevGuard g(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->sc) cudaFree(h->sc);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (int i = 0; i <= kPhases; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->capture) cudaStreamDestroy(h->capture);
  if (h->stage_ev) cudaEventDestroy(h->stage_ev);
  if (h->stage) cudaFreeHost(h->stage);
  if (h->split_ws) cudaFree(h->split_ws);
  if (h->pinned_sc) cudaFreeHost(h->pinned_sc);
  for (int b = 0; b < 2; ++b) {
    if (h->pipe_a[b]) cudaFree(h->pipe_a[b]);
    if (h->pipe_q[b]) cudaFree(h->pipe_q[b]);
    if (h->pipe_r[b]) cudaFree(h->pipe_r[b]);
    if (h->pipe_j[b]) cudaFree(h->pipe_j[b]);
  }
  if (h->pipe_slots) cudaFree(h->pipe_slots);
  if (h->pipe_pin) cudaFreeHost(h->pipe_pin);
  if (h->side) cudaStreamDestroy(h->side);
  for (int i = 0; i < 2; ++i)
    if (h->side_ev[i]) cudaEventDestroy(h->side_ev[i]);
  if (h->pipe_in) cudaStreamDestroy(h->pipe_in);
  if (h->pipe_out) cudaStreamDestroy(h->pipe_out);
  for (int i = 0; i < 6; ++i)
    if (h->pipe_ev[i]) cudaEventDestroy(h->pipe_ev[i]);
  delete h;
  return kOk;
}

int cqrrpt_workspace_size(int64_t m, int64_t n, double gamma, int nnz, int precision,
                          size_t* bytes) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!(gamma >= 1.0)) return -3;
  const int64_t d = sketch_dim(n, gamma);
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -4;
  if (!precision_ok(precision)) return -5;
  if (!bytes) return -6;
  *bytes = plan_for(m, n, d, nnz, precision).total;
  return kOk;
}

int cqrrpt_reserve(cqrrpt_handle h, size_t bytes) {
  if (!h) return -1;
  DevGuard g(h->device);
  return ensure_ws(h, bytes);
}

int cqrrpt_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda, double gamma,
             int nnz, double tol, uint64_t seed, int precision, double* Q, int64_t ldq, double* R,
             int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -6;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (std::isnan(tol)) return -8;
  if (!precision_ok(precision)) return -10;
  if (!Q) return -11;
  if (ldq < m) return -12;
  if (!R) return -13;
  if (ldr < n) return -14;
  if (!J) return -15;

  DevGuard g(h->device);
  if (precision != CQRRPT_FP64)
    return run_split(h, m, n, A, lda, d, nnz, tol, seed, precision, Q, ldq, R, ldr, J, k_dev,
                     k_host, stream);
  return run_fp64(h, m, n, A, lda, d, nnz, tol, seed, Q, ldq, R, ldr, J, k_dev, k_host, stream,
                  true, nullptr, 0);
}

int cqrrpt_implicit_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                      double gamma, int nnz, double tol, uint64_t seed, double* Apre, int64_t ldp,
                      double* Rpre, int64_t ldrp, double* R, int64_t ldr, int64_t* J,
                      int64_t* k_dev, int64_t* k_host, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -6;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (std::isnan(tol)) return -8;
  if (!Apre) return -10;
  if (ldp < m) return -11;
  if (!Rpre) return -12;
  if (ldrp < n) return -13;
  if (!R) return -14;
  if (ldr < n) return -15;
  if (!J) return -16;
  DevGuard g(h->device);
  return run_fp64(h, m, n, A, lda, d, nnz, tol, seed, Apre, ldp, R, ldr, J, k_dev, k_host, stream,
                  false, Rpre, ldrp);
}

int cqrrpt_rcholqr_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                     double gamma, int nnz, uint64_t seed, double* Q, int64_t ldq, double* R,
                     int64_t ldr, int64_t* J, int64_t* k_dev, int64_t* k_host,
                     cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -6;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (!Q) return -9;
  if (ldq < m) return -10;
  if (!R) return -11;
  if (ldr < n) return -12;
  if (!J) return -13;
  DevGuard g(h->device);
  // k = n up to an exactly zero diagonal of R^sk: the rank rule with the
  // smallest normal tolerance
  return run_fp64(h, m, n, A, lda, d, nnz, DBL_MIN, seed, Q, ldq, R, ldr, J, k_dev, k_host,
                  stream, true, nullptr, 0, false);
}

int cqrrpt_srrqr_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                   double gamma, int nnz, double tol, uint64_t seed, double f, double* Q,
                   int64_t ldq, double* R, int64_t ldr, int64_t* J, int64_t* k_dev,
                   int64_t* k_host, int64_t* swaps_host, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -6;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (std::isnan(tol)) return -8;
  if (!(f > 1.0) || !std::isfinite(f)) return -10;
  if (!Q) return -11;
  if (ldq < m) return -12;
  if (!R) return -13;
  if (ldr < n) return -14;
  if (!J) return -15;
  DevGuard g(h->device);
  int64_t sw = 0;
  const int r = run_fp64(h, m, n, A, lda, d, nnz, tol, seed, Q, ldq, R, ldr, J, k_dev, k_host,
                         stream, true, nullptr, 0, true, nullptr, 0, f, &sw);
  if (swaps_host) *swaps_host = sw;
  return r;
}

int cqrrpt_dense_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda, int64_t d,
                   const double* S, int64_t lds, double tol, int precision, double* Q,
                   int64_t ldq, double* R, int64_t ldr, int64_t* J, int64_t* k_dev,
                   int64_t* k_host, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (d < n || d > m || d > 28000) return -6;
  if (!S) return -7;
  if (lds < d) return -8;
  if (std::isnan(tol)) return -9;
  if (!precision_ok(precision)) return -10;
  if (!Q) return -11;
  if (ldq < m) return -12;
  if (!R) return -13;
  if (ldr < n) return -14;
  if (!J) return -15;
  DevGuard g(h->device);
  if (precision != CQRRPT_FP64)
    return run_split(h, m, n, A, lda, d, 1, tol, 0, precision, Q, ldq, R, ldr, J, k_dev, k_host,
                     stream, S, lds);
  return run_fp64(h, m, n, A, lda, d, 1, tol, 0, Q, ldq, R, ldr, J, k_dev, k_host, stream, true,
                  nullptr, 0, true, S, lds);
}

int cqrrpt_sketch_dense_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                          int64_t d, const double* S, int64_t lds, double* Ask, int64_t ldsk,
                          cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (d < 1 || d > 65536) return -6;
  if (!S) return -7;
  if (lds < d) return -8;
  if (!Ask) return -9;
  if (ldsk < d) return -10;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)sketch_dense_workspace_bytes(m, n, (int)d));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  if (launch_sketch_dense(m, n, S, lds, A, lda, (int)d, Ask, ldsk, h->ws, &h->sc->status,
                          stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_sketch_dense_split_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A,
                                int64_t lda, int64_t d, const double* S, int64_t lds, double* Ask,
                                int64_t ldsk, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 65536) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (d < 1 || d > 65536) return -6;
  if (!S) return -7;
  if (lds < d) return -8;
  if (!Ask) return -9;
  if (ldsk < d) return -10;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)sketch_dense_split_workspace_bytes(m, n, (int)d));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  if (launch_sketch_dense_split(m, n, S, lds, A, lda, (int)d, Ask, ldsk, h->ws, &h->sc->status,
                                stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_apply_q_d(cqrrpt_handle h, int trans, int64_t m, int64_t k, const double* Apre,
                     int64_t ldp, const double* Rpre, int64_t ldrp, int64_t nrhs, const double* X,
                     int64_t ldx, double* Y, int64_t ldy, cudaStream_t stream) {
  if (!h) return -1;
  if (trans != 0 && trans != 1) return -2;
  if (m < 1) return -3;
  if (k < 0 || k > m || k > 16384) return -4;
  if (!Apre && k > 0) return -5;
  if (ldp < m) return -6;
  if (!Rpre && k > 0) return -7;
  if (ldrp < (k > 0 ? k : 1)) return -8;
  if (nrhs < 1 || nrhs > 65535) return -9;
  if (!X && k > 0) return -10;
  const int64_t xrows = trans ? m : k, yrows = trans ? k : m;
  if (ldx < (xrows > 0 ? xrows : 1)) return -11;
  if (!Y) return -12;
  if (ldy < (yrows > 0 ? yrows : 1)) return -13;
  DevGuard g(h->device);
  if (k == 0) {  // Q has no columns: Q X = 0 (m x r); Q^T X is empty
    if (!trans &&
        cudaMemset2DAsync(Y, (size_t)ldy * 8, 0, (size_t)m * 8, (size_t)nrhs, stream) != cudaSuccess)
      return kCudaError;
    return kOk;
  }
  int st = ensure_ws(h, (size_t)apply_q_workspace_bytes(trans, m, k, nrhs));
  if (st != kOk) return st;
  return launch_apply_q(trans, m, (int)k, Apre, ldp, Rpre, ldrp, (int)nrhs, X, ldx, Y, ldy, h->ws,
                        stream) == cudaSuccess
             ? kOk
             : kCudaError;
}

}  // extern "C"

namespace {

// Streams, events, slots and the two device buffer sets of the host
// pipeline for an m x n shape (grown, never shrunk).
int pipe_ensure(cqrrpt_handle h, int64_t m, int64_t n) {
  if (!h->pipe_in) {
    if (cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->pipe_out, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return kCudaError;
    }
    for (int i = 0; i < 6; ++i)
      if (cudaEventCreateWithFlags(&h->pipe_ev[i], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return kCudaError;
      }
    if (cudaMalloc(&h->pipe_slots, 32) != cudaSuccess ||
        cudaMallocHost(&h->pipe_pin, 32) != cudaSuccess) {
      cudaGetLastError();
      return kNoMemory;
    }
  }
  if (m <= h->pipe_m && n <= h->pipe_n && m * n <= h->pipe_m * h->pipe_n) return kOk;
  cudaDeviceSynchronize();
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->pipe_a[b]);
    cudaFree(h->pipe_q[b]);
    cudaFree(h->pipe_r[b]);
    cudaFree(h->pipe_j[b]);
    h->pipe_a[b] = h->pipe_q[b] = h->pipe_r[b] = nullptr;
    h->pipe_j[b] = nullptr;
  }
  h->pipe_m = h->pipe_n = 0;
  for (int b = 0; b < 2; ++b) {
    if (cudaMalloc(&h->pipe_a[b], (size_t)(m * n * 8)) != cudaSuccess ||
        cudaMalloc(&h->pipe_q[b], (size_t)(m * n * 8)) != cudaSuccess ||
        cudaMalloc(&h->pipe_r[b], (size_t)(n * n * 8)) != cudaSuccess ||
        cudaMalloc(&h->pipe_j[b], (size_t)(n * 8)) != cudaSuccess) {
      cudaGetLastError();
      return kNoMemory;
    }
  }
  h->pipe_m = m;
  h->pipe_n = n;
  return kOk;
}

}  // namespace

extern "C" {

// ---- row-partitioned CQRRPT (Sec. 2.1): one rank's phases ---------------
// The workspace carve of a rank: the plan of a rows-row factorisation.
static Plan shard_plan(cqrrpt_handle h) {
  return plan_fp64(h->shard.rows, h->shard.n, h->shard.d, h->shard.nnz);
}
struct ShardWs {
  void* region;
  double *X, *Rsk, *G, *Rpre, *f2;
  void* qw;
};
static ShardWs shard_ws(cqrrpt_handle h) {
  const Plan p = shard_plan(h);
  char* w = (char*)h->ws;
  ShardWs s;
  s.region = w; w += p.region;
  s.X = (double*)w; w += p.x;
  s.qw = w; w += p.qrcp;
  s.Rsk = (double*)w; w += p.rsk;
  s.G = (double*)w; w += p.g;
  s.Rpre = (double*)w; w += p.rpre;
  s.f2 = (double*)w;
  return s;
}

int cqrrpt_shard_sketch_d(cqrrpt_handle h, int64_t m, int64_t rows, int64_t row0, int64_t n,
                          const double* A, int64_t lda, double gamma, int nnz, uint64_t seed,
                          cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (rows < 1 || rows > m) return -3;
  if (row0 < 0 || row0 % kRowBlock != 0 || row0 + rows > m) return -4;
  if (n < 1 || n > 16384) return -5;
  if (!A) return -6;
  if (lda < rows) return -7;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -8;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -8;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -9;
  DevGuard g(h->device);
  h->shard.A = A;
  h->shard.lda = lda;
  h->shard.m = m;
  h->shard.rows = rows;
  h->shard.row0 = row0;
  h->shard.n = n;
  h->shard.d = d;
  h->shard.nnz = nnz;
  h->shard.phase = 0;
  int st = ensure_ws(h, shard_plan(h).total);
  if (st != kOk) return st;
  const ShardWs w = shard_ws(h);
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess ||
      launch_sketch_panel_partials(rows, n, A, lda, (int)d, nnz, seed, row0, w.region, stream) !=
          cudaSuccess)
    return kCudaError;
  h->shard.phase = 1;
  return kOk;
}

int cqrrpt_shard_sketch_accumulate_d(cqrrpt_handle h, double* acc, cudaStream_t stream) {
  if (!h) return -1;
  if (!acc) return -2;
  if (h->shard.phase != 1) return -1;
  DevGuard g(h->device);
  const ShardWs w = shard_ws(h);
  return launch_sketch_panel_accumulate(h->shard.rows, h->shard.n, (int)h->shard.d,
                                        h->shard.nnz, acc, w.region, stream) == cudaSuccess
             ? kOk
             : kCudaError;
}

int cqrrpt_shard_qrcp_d(cqrrpt_handle h, const double* acc, double tol, int64_t* J,
                        cudaStream_t stream) {
  if (!h) return -1;
  if (!acc) return -2;
  if (std::isnan(tol)) return -3;
  if (!J) return -4;
  if (h->shard.phase != 1) return -1;
  DevGuard g(h->device);
  const ShardWs w = shard_ws(h);
  const int ni = (int)h->shard.n, di = (int)h->shard.d;
  DeviceScalars* sc = h->sc;
  cudaError_t e = launch_sketch_finish(di, h->shard.n, acc, 1.0 / std::sqrt((double)h->shard.nnz),
                                       w.X, h->shard.d, &sc->status, stream);
  if (e == cudaSuccess)
    e = launch_qrcp(di, ni, w.X, h->shard.d, J, w.Rsk, h->shard.n, w.qw, sc, h->num_sms, stream);
  if (e == cudaSuccess) e = launch_rank(ni, w.Rsk, h->shard.n, tol, sc, w.f2, stream);
  if (e != cudaSuccess) return kCudaError;
  h->shard.tol = tol;
  h->shard.J = J;
  h->shard.phase = 2;
  return kOk;
}

int cqrrpt_shard_gram_d(cqrrpt_handle h, double* Q, int64_t ldq, cudaStream_t stream) {
  if (!h) return -1;
  if (!Q) return -2;
  if (ldq < h->shard.rows) return -3;
  if (h->shard.phase != 2) return -1;
  DevGuard g(h->device);
  const ShardWs w = shard_ws(h);
  const int ni = (int)h->shard.n;
  DeviceScalars* sc = h->sc;
  cudaError_t e = launch_trsm_rut(h->shard.rows, ni, &sc->k, h->shard.A, h->shard.lda,
                                  h->shard.J, w.Rsk, h->shard.n, Q, ldq, &sc->status, stream);
  if (e == cudaSuccess)
    e = launch_gram_partials(h->shard.rows, ni, &sc->k, Q, ldq, w.region, &sc->status, stream);
  if (e != cudaSuccess) return kCudaError;
  h->shard.phase = 3;
  return kOk;
}

int cqrrpt_shard_gram_accumulate_d(cqrrpt_handle h, double* G, cudaStream_t stream) {
  if (!h) return -1;
  if (!G) return -2;
  if (h->shard.phase != 3) return -1;
  DevGuard g(h->device);
  const ShardWs w = shard_ws(h);
  return launch_gram_sum(h->shard.rows, (int)h->shard.n, &h->sc->k, G, h->shard.n, w.region,
                         &h->sc->status, stream, true) == cudaSuccess
             ? kOk
             : kCudaError;
}

int cqrrpt_shard_finish_d(cqrrpt_handle h, double* G, double* Q, int64_t ldq, double* R,
                          int64_t ldr, int64_t* k_dev, int64_t* k_host, cudaStream_t stream) {
  if (!h) return -1;
  if (!G) return -2;
  if (!Q) return -3;
  if (ldq < h->shard.rows) return -4;
  if (!R) return -5;
  if (ldr < h->shard.n) return -6;
  if (h->shard.phase != 3) return -1;
  DevGuard g(h->device);
  const ShardWs w = shard_ws(h);
  const int ni = (int)h->shard.n;
  const int64_t n = h->shard.n;
  DeviceScalars* sc = h->sc;
  int* status = &sc->status;
  cudaError_t e = launch_potrf(ni, G, n, w.Rpre, n, sc, stream);
  if (e == cudaSuccess) e = launch_rank_stage2(w.Rpre, n, !(h->shard.tol > 0.0), sc, stream);
  if (e == cudaSuccess)
    e = launch_trsm_rut(h->shard.rows, ni, &sc->k, Q, ldq, nullptr, w.Rpre, n, Q, ldq, status,
                        stream);
  if (e == cudaSuccess) e = launch_trmm(ni, &sc->k, w.Rpre, n, w.Rsk, n, R, ldr, status, stream);
  if (e == cudaSuccess) e = launch_finalize(sc, k_dev, nullptr, stream);
  if (e != cudaSuccess) return kCudaError;
  h->shard.phase = 0;
  if (k_host) {
    int st2 = kOk;
    int64_t kk = 0;
    const int r = cqrrpt_last_status(h, stream, &st2, &kk);
    if (r != kOk) return r;
    *k_host = kk;
    return st2;
  }
  return kOk;
}

int cqrrpt_host_pipeline_d(cqrrpt_handle h, int count, int64_t m, int64_t n,
                           const double* const* A_host, int64_t lda, double gamma, int nnz,
                           double tol, const uint64_t* seeds, int precision,
                           double* const* Q_host, int64_t ldq, double* const* R_host, int64_t ldr,
                           int64_t* const* J_host, int64_t* k_host, int* status_host,
                           cudaStream_t stream) {
  if (!h) return -1;
  if (count < 1) return -2;
  if (m < 1) return -3;
  if (n < 1 || n > 16384) return -4;
  if (!A_host) return -5;
  if (lda < m) return -6;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -7;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -7;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -8;
  if (std::isnan(tol)) return -9;
  if (!seeds) return -10;
  if (!precision_ok(precision)) return -11;
  if (!Q_host) return -12;
  if (ldq < m) return -13;
  if (!R_host) return -14;
  if (ldr < n) return -15;
  if (!J_host) return -16;
  if (!k_host) return -17;
  if (!status_host) return -18;
  for (int i = 0; i < count; ++i) {
    if (!A_host[i]) return -5;
    if (!Q_host[i]) return -12;
    if (!R_host[i]) return -14;
    if (!J_host[i]) return -16;
  }
  DevGuard g(h->device);
  int st = pipe_ensure(h, m, n);
  if (st != kOk) return st;
  cudaEvent_t* ev_in = h->pipe_ev;
  cudaEvent_t* ev_comp = h->pipe_ev + 2;
  cudaEvent_t* ev_out = h->pipe_ev + 4;
  int64_t* ks_dev = h->pipe_slots;           // k[2]
  int* st_dev = (int*)(h->pipe_slots + 2);   // status[2]
  const int64_t* ks_pin = h->pipe_pin;
  const int* st_pin = (const int*)(h->pipe_pin + 2);
  cudaError_t e = cudaSuccess;

  // copy in matrix i (after the factorisation of i - 2 has read its buffer)
  auto copy_in = [&](int i) {
    const int b = i & 1;
    if (i >= 2 && e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_in, ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(h->pipe_a[b], (size_t)m * 8, A_host[i], (size_t)lda * 8,
                            (size_t)m * 8, (size_t)n, cudaMemcpyHostToDevice, h->pipe_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[b], h->pipe_in);
  };
  // factor matrix i on the caller's stream (after its copy-in, and after
  // the results of i - 2 have left its output buffers); k and status go to
  // the pinned slots
  int first_error = kOk;
  auto factor = [&](int i) {
    const int b = i & 1;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_in[b], 0);
    if (i >= 2 && e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_out[b], 0);
    if (e != cudaSuccess) return;
    const int r = cqrrpt_d(h, m, n, h->pipe_a[b], m, gamma, nnz, tol, seeds[i], precision,
                           h->pipe_q[b], m, h->pipe_r[b], n, h->pipe_j[b], nullptr, nullptr, stream);
    if (r != kOk && first_error == kOk) first_error = r;
    if (e == cudaSuccess && handle_finalize(h, ks_dev + b, st_dev + b, stream) != kOk)
      e = cudaErrorUnknown;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->pipe_pin + b, ks_dev + b, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((int*)(h->pipe_pin + 2) + b, st_dev + b, 4, cudaMemcpyDeviceToHost,
                          stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp[b], stream);
  };

  copy_in(0);
  factor(0);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const int b = i & 1;
    if (i + 1 < count) {  // queue the next matrix before waiting for this one
      copy_in(i + 1);
      factor(i + 1);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev_comp[b]);
    if (e != cudaSuccess) break;
    const int64_t k = ks_pin[b];
    k_host[i] = k;
    status_host[i] = st_pin[b];
    // copy out the result of matrix i: Q[:, :k], R[:k, :], J
    e = cudaStreamWaitEvent(h->pipe_out, ev_comp[b], 0);
    if (e == cudaSuccess && k > 0)
      e = cudaMemcpy2DAsync(Q_host[i], (size_t)ldq * 8, h->pipe_q[b], (size_t)m * 8,
                            (size_t)m * 8, (size_t)k, cudaMemcpyDeviceToHost, h->pipe_out);
    if (e == cudaSuccess && k > 0)
      e = cudaMemcpy2DAsync(R_host[i], (size_t)ldr * 8, h->pipe_r[b], (size_t)n * 8,
                            (size_t)k * 8, (size_t)n, cudaMemcpyDeviceToHost, h->pipe_out);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(J_host[i], h->pipe_j[b], (size_t)n * 8, cudaMemcpyDeviceToHost,
                          h->pipe_out);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[b], h->pipe_out);
  }
  const cudaError_t e1 = cudaStreamSynchronize(h->pipe_out);
  const cudaError_t e2 = cudaStreamSynchronize(h->pipe_in);
  const cudaError_t e3 = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return kCudaError;
  }
  return first_error;
}

int cqrrpt_panels_host_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A_host,
                         int64_t lda, double gamma, int nnz, double tol, uint64_t seed,
                         int64_t panel_rows, double* Q_host, int64_t ldq, double* R_host,
                         int64_t ldr, int64_t* J_host, int64_t* k_host, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1 || n > 16384) return -3;
  if (!A_host) return -4;
  if (lda < m) return -5;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -6;
  const int64_t d = sketch_dim(n, gamma);
  if (d > m || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (std::isnan(tol)) return -8;
  if (panel_rows < kRowBlock || panel_rows % kRowBlock != 0) return -10;
  if (!Q_host) return -11;
  if (ldq < m) return -12;
  if (!R_host) return -13;
  if (ldr < n) return -14;
  if (!J_host) return -15;
  if (!k_host) return -16;
  DevGuard g(h->device);
  *k_host = 0;
  const int64_t P = panel_rows < m ? panel_rows : (m + kRowBlock - 1) / kRowBlock * kRowBlock;
  const int64_t npan = (m + P - 1) / P;
  // device: two A panels and two M^pre / Q panels (P x n each), R and J,
  // the workspace of one P-row factorisation, the sketch accumulator
  int st = pipe_ensure(h, P, n);
  if (st != kOk) return st;
  const Plan p = plan_fp64(P, n, d, nnz);
  const size_t acc_bytes = (size_t)align256(d * n * 8);
  st = ensure_ws(h, p.total + acc_bytes);
  if (st != kOk) return st;
  char* w = (char*)h->ws;
  void* region = w; w += p.region;
  double* X = (double*)w; w += p.x;
  void* qw = w; w += p.qrcp;
  double* Rsk = (double*)w; w += p.rsk;
  double* G = (double*)w; w += p.g;
  double* Rpre = (double*)w; w += p.rpre;
  double* f2 = (double*)w; w += p.f2;
  double* acc = (double*)w;
  int64_t* Jd = h->pipe_j[0];
  double* Rd = h->pipe_r[0];
  DeviceScalars* sc = h->sc;
  int* status = &sc->status;
  const int ni = (int)n, di = (int)d;
  cudaEvent_t* ev_in = h->pipe_ev;
  cudaEvent_t* ev_comp = h->pipe_ev + 2;
  cudaEvent_t* ev_out = h->pipe_ev + 4;
  double** abuf = h->pipe_a;
  double** xbuf = h->pipe_q;
  cudaError_t e = cudaSuccess;
  int64_t it = 0;  // panel uses so far; slot it & 1
  auto rows_of = [&](int64_t q) { return q * P + P <= m ? P : m - q * P; };
  // rows of panel q (cols columns of a host matrix) into a device buffer of
  // slot b, after the compute and the copy-out that last used slot b
  auto copy_in = [&](double* dst, const double* src, int64_t ld, int64_t q, int64_t cols,
                     int b) {
    if (it >= 2 && e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_in, ev_comp[b], 0);
    if (it >= 2 && e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_in, ev_out[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dst, (size_t)P * 8, src + q * P, (size_t)ld * 8,
                            (size_t)rows_of(q) * 8, (size_t)cols, cudaMemcpyHostToDevice,
                            h->pipe_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[b], h->pipe_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_in[b], 0);
  };
  // the slot's compute is queued: its M^pre / Q panel (cols columns) to the
  // rows of panel q of Q_host
  auto copy_out = [&](int64_t q, int64_t cols, int b) {
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp[b], stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_out, ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Q_host + q * P, (size_t)ldq * 8, xbuf[b], (size_t)P * 8,
                            (size_t)rows_of(q) * 8, (size_t)cols, cudaMemcpyDeviceToHost,
                            h->pipe_out);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[b], h->pipe_out);
  };
  auto drain = [&]() {
    const cudaError_t e1 = cudaStreamSynchronize(h->pipe_in);
    const cudaError_t e2 = cudaStreamSynchronize(h->pipe_out);
    const cudaError_t e3 = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess;
  };

  // line 1: each panel's block sums continue the sketch's ascending sum
  if (e == cudaSuccess) e = launch_init_scalars(sc, 0, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (size_t)d * n * 8, stream);
  for (int64_t q = 0; q < npan && e == cudaSuccess; ++q, ++it) {
    const int b = (int)(it & 1);
    copy_in(abuf[b], A_host, lda, q, n, b);
    if (e == cudaSuccess)
      e = launch_sketch_panel(rows_of(q), n, abuf[b], P, di, nnz, seed, q * P, acc, region,
                              stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp[b], stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[b], stream);
  }
  if (e == cudaSuccess)
    e = launch_sketch_finish(di, n, acc, 1.0 / std::sqrt((double)nnz), X, d, status, stream);
  // lines 2 and 3
  if (e == cudaSuccess) e = launch_qrcp(di, ni, X, d, Jd, Rsk, n, qw, sc, h->num_sms, stream);
  if (e == cudaSuccess) e = launch_rank(ni, Rsk, n, tol, sc, f2, stream);
  int st1 = kOk;
  int64_t k1 = 0;
  if (e == cudaSuccess && cqrrpt_last_status(h, stream, &st1, &k1) != kOk) e = cudaErrorUnknown;
  if (e == cudaSuccess && st1 == kOk && k1 > 0) {
    // lines 4 and 5: M^pre panel by panel (parked in Q_host's first k1
    // columns), its Gram blocks continuing G's ascending sums
    e = cudaMemsetAsync(G, 0, (size_t)n * n * 8, stream);
    for (int64_t q = 0; q < npan && e == cudaSuccess; ++q, ++it) {
      const int b = (int)(it & 1);
      copy_in(abuf[b], A_host, lda, q, n, b);
      if (e == cudaSuccess)
        e = launch_trsm_rut(rows_of(q), ni, &sc->k, abuf[b], P, Jd, Rsk, n, xbuf[b], P, status,
                            stream);
      if (e == cudaSuccess)
        e = launch_gram(rows_of(q), ni, &sc->k, xbuf[b], P, G, n, region, status, stream, true);
      copy_out(q, k1, b);
    }
    // line 6 (Remark 4, stage 2)
    if (e == cudaSuccess) e = launch_potrf(ni, G, n, Rpre, n, sc, stream);
    if (e == cudaSuccess) e = launch_rank_stage2(Rpre, n, !(tol > 0.0), sc, stream);
    int st2 = kOk;
    int64_t k2 = 0;
    if (e == cudaSuccess && cqrrpt_last_status(h, stream, &st2, &k2) != kOk) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->pipe_out);  // M^pre is on the host
    // line 7: Q panel by panel, in place on the parked M^pre
    for (int64_t q = 0; q < npan && e == cudaSuccess && k2 > 0; ++q, ++it) {
      const int b = (int)(it & 1);
      copy_in(xbuf[b], Q_host, ldq, q, k2, b);
      if (e == cudaSuccess)
        e = launch_trsm_rut(rows_of(q), ni, &sc->k, xbuf[b], P, nullptr, Rpre, n, xbuf[b], P,
                            status, stream);
      copy_out(q, k2, b);
    }
    // line 8
    if (e == cudaSuccess) e = launch_trmm(ni, &sc->k, Rpre, n, Rsk, n, Rd, n, status, stream);
    if (e == cudaSuccess && k2 > 0)
      e = cudaMemcpy2DAsync(R_host, (size_t)ldr * 8, Rd, (size_t)n * 8, (size_t)k2 * 8,
                            (size_t)n, cudaMemcpyDeviceToHost, stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(J_host, Jd, (size_t)n * 8, cudaMemcpyDeviceToHost, stream);
  if (!drain()) return kCudaError;
  int st3 = kOk;
  int64_t k3 = 0;
  if (cqrrpt_last_status(h, stream, &st3, &k3) != kOk) return kCudaError;
  *k_host = k3;
  return st3;
}

static int batch_check(int batch, const int64_t* m, const int64_t* n, const double* const* A,
                       const int64_t* lda, double gamma, int nnz, const double* tol,
                       const uint64_t* seed, int precision, double* const* Q, const int64_t* ldq,
                       double* const* R, const int64_t* ldr, int64_t* const* J) {
  if (batch < 1) return -2;
  if (!m) return -3;
  if (!n) return -4;
  if (!A) return -5;
  if (!lda) return -6;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -7;
  if (!tol) return -9;
  if (!seed) return -10;
  if (precision != CQRRPT_FP64 && precision != CQRRPT_SPLITBF16) return -11;
  if (!Q) return -12;
  if (!ldq) return -13;
  if (!R) return -14;
  if (!ldr) return -15;
  if (!J) return -16;
  for (int p = 0; p < batch; ++p) {
    if (m[p] < 1) return -3;
    if (n[p] < 1 || n[p] > 16384) return -4;
    if (!A[p]) return -5;
    if (lda[p] < m[p]) return -6;
    const int64_t d = sketch_dim(n[p], gamma);
    if (d > m[p] || d > 28000) return -7;
    if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -8;
    if (std::isnan(tol[p])) return -9;
    if (!Q[p]) return -12;
    if (ldq[p] < m[p]) return -13;
    if (!R[p]) return -14;
    if (ldr[p] < n[p]) return -15;
    if (!J[p]) return -16;
  }
  return kOk;
}

int cqrrpt_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, double gamma,
                                  int nnz, size_t* bytes) {
  if (batch < 1) return -1;
  if (!m || !n) return -2;
  if (!(gamma >= 1.0)) return -4;
  if (!bytes) return -6;
  int64_t total = align256((int64_t)batch * sizeof(DeviceScalars)) + batch_table_bytes(batch);
  for (int p = 0; p < batch; ++p) {
    if (m[p] < 1 || n[p] < 1) return -2;
    const int64_t d = sketch_dim(n[p], gamma);
    if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -5;
    total += problem_workspace_bytes(m[p], n[p], d, nnz);
  }
  *bytes = (size_t)total;
  return kOk;
}

int cqrrpt_set_batch_graphs(cqrrpt_handle h, int enable) {
  if (!h) return -1;
  h->use_graphs = enable ? 1 : 0;
  return kOk;
}

}  // extern "C"

namespace {

std::vector<BatchProblem> batch_problems(int batch, const int64_t* m, const int64_t* n,
                                         const double* const* A, const int64_t* lda, double gamma,
                                         int nnz, const double* tol, const uint64_t* seed,
                                         double* const* Q, const int64_t* ldq, double* const* R,
                                         const int64_t* ldr, int64_t* const* J, int64_t* k_dev,
                                         int* status_dev) {
  std::vector<BatchProblem> probs((size_t)batch);
  for (int p = 0; p < batch; ++p) {
    BatchProblem& q = probs[(size_t)p];
    q.m = m[p]; q.n = n[p]; q.d = sketch_dim(n[p], gamma); q.nnz = nnz; q.tol = tol[p];
    q.seed = seed[p]; q.A = A[p]; q.lda = lda[p]; q.Q = Q[p]; q.ldq = ldq[p]; q.R = R[p];
    q.ldr = ldr[p]; q.J = J[p];
    q.k_out = k_dev ? k_dev + p : nullptr;
    q.status_out = status_dev ? status_dev + p : nullptr;
  }
  return probs;
}

// Workspace layout of a batched call: device scalars, tables, then each
// problem's workspace in order.
struct BatchWs {
  DeviceScalars* scalars;
  char* tables;
  char* per_problem;
};
BatchWs batch_ws(cqrrpt_handle h, int batch) {
  char* ws = (char*)h->ws;
  BatchWs b;
  b.scalars = (DeviceScalars*)ws;
  b.tables = ws + align256((int64_t)batch * sizeof(DeviceScalars));
  b.per_problem = b.tables + batch_table_bytes(batch);
  return b;
}

// Copies the plan's tables to the device through the pinned staging buffer
// (after the previous copy out of it has finished).
int stage_tables(cqrrpt_handle h, const BatchPlan& P, cudaStream_t stream) {
  const size_t img = P.image.size();
  if (!h->stage_ev && cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming) != cudaSuccess)
    return kCudaError;
  if (cudaEventSynchronize(h->stage_ev) != cudaSuccess) return kCudaError;
  if (img > h->stage_bytes) {
    if (h->stage) cudaFreeHost(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    if (cudaMallocHost(&h->stage, img) != cudaSuccess) return kNoMemory;
    h->stage_bytes = img;
  }
  memcpy(h->stage, P.image.data(), img);
  if (cudaMemcpyAsync(P.tables, h->stage, img, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return kCudaError;
  if (cudaEventRecord(h->stage_ev, stream) != cudaSuccess) return kCudaError;
  return kOk;
}

// Copies n bytes of a host image to device memory through the pinned
// staging buffer (after the previous copy out of it has finished).
int stage_bytes(cqrrpt_handle h, const void* host, size_t n, void* dev, cudaStream_t stream) {
  if (!h->stage_ev && cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming) != cudaSuccess)
    return kCudaError;
  if (cudaEventSynchronize(h->stage_ev) != cudaSuccess) return kCudaError;
  if (n > h->stage_bytes) {
    if (h->stage) cudaFreeHost(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    if (cudaMallocHost(&h->stage, n) != cudaSuccess) return kNoMemory;
    h->stage_bytes = n;
  }
  memcpy(h->stage, host, n);
  if (cudaMemcpyAsync(dev, h->stage, n, cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return kCudaError;
  if (cudaEventRecord(h->stage_ev, stream) != cudaSuccess) return kCudaError;
  return kOk;
}

// Host image of job tables: each table 256-byte aligned.
struct Image {
  std::vector<char> b;
  size_t raw(const void* p, size_t n) {
    const size_t off = (b.size() + 255) & ~size_t(255);
    b.resize(off + n);
    if (n) memcpy(b.data() + off, p, n);
    return off;
  }
  template <class T>
  size_t push(const std::vector<T>& v) {
    return raw(v.data(), v.size() * sizeof(T));
  }
};

// Prefix table of per-job CTA counts.
template <class F>
std::vector<int64_t> prefix(size_t n, F tiles) {
  std::vector<int64_t> b(n + 1, 0);
  for (size_t i = 0; i < n; ++i) b[i + 1] = b[i] + tiles(i);
  return b;
}

int read_scalars(cqrrpt_handle h, const DeviceScalars* sc, int batch, cudaStream_t stream) {
  if (batch > h->pinned_sc_count) {
    if (h->pinned_sc) cudaFreeHost(h->pinned_sc);
    h->pinned_sc = nullptr;
    h->pinned_sc_count = 0;
    if (cudaMallocHost((void**)&h->pinned_sc, (size_t)batch * sizeof(DeviceScalars)) != cudaSuccess)
      return kNoMemory;
    h->pinned_sc_count = batch;
  }
  if (cudaMemcpyAsync(h->pinned_sc, sc, (size_t)batch * sizeof(DeviceScalars),
                      cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int ensure_split_ws(cqrrpt_handle h, size_t bytes) {
  if (bytes <= h->split_ws_bytes) return kOk;
  if (h->split_ws) {
    cudaDeviceSynchronize();
    cudaFree(h->split_ws);
    h->split_ws = nullptr;
    h->split_ws_bytes = 0;
  }
  if (cudaMalloc(&h->split_ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->split_ws = nullptr;
    return kNoMemory;
  }
  h->split_ws_bytes = bytes;
  return kOk;
}

// Device memory of one problem's split steps (rank k): row planes (lines 4
// and 7) aliased with the Gram's planes (line 5), column planes of W,
// exponents, W, the Gram's K-slice partials.
struct SplitWs {
  __nv_bfloat16 *DA, *DB;
  int *ea, *eb;
  double *W, *P;
};
int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
size_t split_ws_one(int64_t m, int64_t k, SplitWs* out, char* base) {
  const int64_t kpad = rup(k, 32), kpadm = rup(m, kOzChunk);
  const int64_t ns = oz_gram_slices(m, (int)k);
  const int64_t da = std::max<int64_t>(kOzDigits * m * kpad * 2, kOzDigits * k * kpadm * 2);
  size_t off = 0;
  auto take = [&](int64_t bytes) {
    const size_t o = off;
    off += (size_t)align256(bytes);
    return base + o;
  };
  char* DA = take(da);
  char* DB = take(kOzDigits * k * kpad * 2);
  char* ea = take(std::max<int64_t>(m, k) * 4);
  char* eb = take(k * 4);
  char* W = take(k * k * 8);
  char* P = take(ns * k * k * 8);
  if (out) *out = SplitWs{(__nv_bfloat16*)DA, (__nv_bfloat16*)DB, (int*)ea, (int*)eb, (double*)W,
                          (double*)P};
  return off;
}

// One of lines 4 and 7 for every listed problem: X = B[:, cols] T^{-1} as
// row-wise FP64 inverse + one split product (as oz_trsm_inv, job by job).
int split_trsm_step(cqrrpt_handle h, const std::vector<int>& ids,
                    const std::vector<BatchProblem>& probs, const std::vector<int64_t>& k,
                    const std::vector<SplitWs>& ws, const std::vector<double*>& T, bool line4,
                    DeviceScalars* sc, char* tables, cudaStream_t stream) {
  const size_t nj = ids.size();
  if (nj == 0) return kOk;
  std::vector<OzTrinv> ti(nj);
  std::vector<OzRowSplit> rs(nj);
  std::vector<OzColSplit> cs(nj);
  std::vector<OzGemm> gm(nj);
  std::vector<char> maps(nj * 2 * kOzMapBytes);
  int kmax = 1;
  for (size_t j = 0; j < nj; ++j) {
    const int p = ids[j];
    const BatchProblem& q = probs[(size_t)p];
    const int kk = (int)k[(size_t)p];
    const int64_t kpad = rup(kk, 32);
    const SplitWs& w = ws[(size_t)p];
    kmax = std::max(kmax, kk);
    ti[j] = OzTrinv{T[(size_t)p], q.n, kk, w.W, kk};
    if (line4)
      rs[j] = OzRowSplit{q.A, q.lda, q.J, q.m, kk, kpad, w.ea, w.DA, q.m * kpad};
    else
      rs[j] = OzRowSplit{q.Q, q.ldq, nullptr, q.m, kk, kpad, w.ea, w.DA, q.m * kpad};
    cs[j] = OzColSplit{w.W, kk, kk, kk, kpad, w.eb, w.DB, (int64_t)kk * kpad};
    OzGemm G{};
    G.M = q.m; G.N = kk; G.Kpad = kpad; G.kslice = kpad;
    G.A = w.DA; G.a_plane = q.m * kpad; G.B = w.DB; G.b_plane = (int64_t)kk * kpad;
    G.ea = w.ea; G.eb = w.eb; G.C = q.Q; G.ldc = q.ldq; G.c_slice = 0;
    G.mode = kOzStore; G.upper_only = 0; G.err = &sc[p].status;
    if (!oz_gemm_valid(G) || !oz_gemm_encode_maps(G, maps.data() + j * 2 * kOzMapBytes))
      return kCudaError;
    gm[j] = G;
  }
  const int warps = oz_trinv_row_mode(kmax) ? 1 : oz_trinv_warps(kmax);
  const auto b_ti = prefix(nj, [&](size_t j) { return oz_trinv_tiles(ti[j], warps); });
  const auto b_re = prefix(nj, [&](size_t j) { return oz_rowexp_tiles(rs[j]); });
  const auto b_rs = prefix(nj, [&](size_t j) { return oz_splitrows_tiles(rs[j]); });
  const auto b_ce = prefix(nj, [&](size_t j) { return oz_colexp_tiles(cs[j]); });
  const auto b_cs = prefix(nj, [&](size_t j) { return oz_splitcols_tiles(cs[j]); });
  const auto b_gm = prefix(nj, [&](size_t j) { return oz_gemm_tiles(gm[j]); });
  Image im;
  const size_t o_maps = im.raw(maps.data(), maps.size());
  const size_t o_ti = im.push(ti), o_rs = im.push(rs), o_cs = im.push(cs), o_gm = im.push(gm);
  const size_t o_bti = im.push(b_ti), o_bre = im.push(b_re), o_brs = im.push(b_rs),
               o_bce = im.push(b_ce), o_bcs = im.push(b_cs), o_bgm = im.push(b_gm);
  int st = stage_bytes(h, im.b.data(), im.b.size(), tables, stream);
  if (st != kOk) return st;
  const int n = (int)nj;
  cudaError_t e = oz_trinv_batched((const OzTrinv*)(tables + o_ti), (const int64_t*)(tables + o_bti),
                                   b_ti[nj], n, warps, kmax, stream);
  if (e == cudaSuccess)
    e = oz_rowsplit_batched((const OzRowSplit*)(tables + o_rs), (const int64_t*)(tables + o_bre),
                            b_re[nj], (const int64_t*)(tables + o_brs), b_rs[nj], n, stream);
  if (e == cudaSuccess)
    e = oz_colsplit_batched((const OzColSplit*)(tables + o_cs), (const int64_t*)(tables + o_bce),
                            b_ce[nj], (const int64_t*)(tables + o_bcs), b_cs[nj], n, stream);
  if (e == cudaSuccess)
    e = oz_gemm_tc_batched_launch((const OzGemm*)(tables + o_gm), tables + o_maps,
                                  (const int64_t*)(tables + o_bgm), n, b_gm[nj], stream);
  return e == cudaSuccess ? kOk : kCudaError;
}

// Line 5 for every listed problem: G = Q^T Q as split products over K
// slices (as oz_gram, job by job).
int split_gram_step(cqrrpt_handle h, const std::vector<int>& ids,
                    const std::vector<BatchProblem>& probs, const std::vector<int64_t>& k,
                    const std::vector<SplitWs>& ws, const std::vector<double*>& Gout,
                    DeviceScalars* sc, char* tables, cudaStream_t stream) {
  const size_t nj = ids.size();
  if (nj == 0) return kOk;
  std::vector<OzColSplit> cs(nj);
  std::vector<OzGemm> gm(nj);
  std::vector<OzCombine> cb(nj);
  std::vector<char> maps(nj * 2 * kOzMapBytes);
  for (size_t j = 0; j < nj; ++j) {
    const int p = ids[j];
    const BatchProblem& q = probs[(size_t)p];
    const int kk = (int)k[(size_t)p];
    const SplitWs& w = ws[(size_t)p];
    const int64_t kpadm = rup(q.m, kOzChunk);
    const int64_t ns = oz_gram_slices(q.m, kk);
    cs[j] = OzColSplit{q.Q, q.ldq, q.m, kk, kpadm, w.ea, w.DA, (int64_t)kk * kpadm, kOzChunk};
    OzGemm G{};
    G.M = kk; G.N = kk; G.Kpad = kpadm;
    G.kslice = ((kpadm / kOzChunk + ns - 1) / ns) * kOzChunk;
    G.A = w.DA; G.a_plane = (int64_t)kk * kpadm; G.B = w.DA; G.b_plane = (int64_t)kk * kpadm;
    G.a_kblk = kOzChunk; G.b_kblk = kOzChunk;
    G.ea = w.ea; G.eb = w.ea; G.C = w.P; G.ldc = kk; G.c_slice = (int64_t)kk * kk;
    G.mode = kOzStore; G.upper_only = 1; G.err = &sc[p].status;
    if (!oz_gemm_valid(G) || !oz_gemm_encode_maps(G, maps.data() + j * 2 * kOzMapBytes))
      return kCudaError;
    gm[j] = G;
    const int nsr = (int)((kpadm + G.kslice - 1) / G.kslice);
    cb[j] = OzCombine{w.P, G.c_slice, nsr, kk, Gout[(size_t)p], q.n};
  }
  const auto b_ce = prefix(nj, [&](size_t j) { return oz_colexp_tiles(cs[j]); });
  const auto b_cs = prefix(nj, [&](size_t j) { return oz_splitcols_tiles(cs[j]); });
  const auto b_gm = prefix(nj, [&](size_t j) { return oz_gemm_tiles(gm[j]); });
  const auto b_cb = prefix(nj, [&](size_t j) { return oz_combine_tiles(cb[j]); });
  Image im;
  const size_t o_maps = im.raw(maps.data(), maps.size());
  const size_t o_cs = im.push(cs), o_gm = im.push(gm), o_cb = im.push(cb);
  const size_t o_bce = im.push(b_ce), o_bcs = im.push(b_cs), o_bgm = im.push(b_gm),
               o_bcb = im.push(b_cb);
  int st = stage_bytes(h, im.b.data(), im.b.size(), tables, stream);
  if (st != kOk) return st;
  const int n = (int)nj;
  cudaError_t e =
      oz_colsplit_batched((const OzColSplit*)(tables + o_cs), (const int64_t*)(tables + o_bce),
                          b_ce[nj], (const int64_t*)(tables + o_bcs), b_cs[nj], n, stream);
  if (e == cudaSuccess)
    e = oz_gemm_tc_batched_launch((const OzGemm*)(tables + o_gm), tables + o_maps,
                                  (const int64_t*)(tables + o_bgm), n, b_gm[nj], stream);
  if (e == cudaSuccess)
    e = oz_combine_batched((const OzCombine*)(tables + o_cb), (const int64_t*)(tables + o_bcb),
                           b_cb[nj], n, stream);
  return e == cudaSuccess ? kOk : kCudaError;
}

// Batched CQRRPT in the split-BF16 mode: the FP64 front (sketch, QRCP, rank
// rule) and back (Cholesky, stage 2, TRMM, finalize) as batched kernels,
// lines 4, 5 and 7 as batched split products -- every problem's job exactly
// the single-problem split path's, so results are bit-identical to
// cqrrpt_d in CQRRPT_SPLITBF16.  Waits for the stream twice (the products
// are sized by each problem's k).
}  // namespace

namespace cqrrpt {

// The batched split-BF16 steps of a planned batch whose tables are already
// on the device (in stream order): everything from the FP64 front on.
int batched_split_exec(cqrrpt_handle h, BatchPlan& P, const std::vector<BatchProblem>& probs,
                       cudaStream_t stream) {
  const int batch = (int)probs.size();
  int st = kOk;
  if (sketch_set_attributes(P.max_d) != cudaSuccess) return kCudaError;
  if (batch_launch_front(P, stream) != cudaSuccess) return kCudaError;
  if ((st = read_scalars(h, P.scalars, batch, stream)) != kOk) return st;
  std::vector<int64_t> k((size_t)batch, 0);
  std::vector<int> ids;
  for (int p = 0; p < batch; ++p) {
    k[(size_t)p] = h->pinned_sc[p].k;
    if (h->pinned_sc[p].status == kOk && k[(size_t)p] > 0) ids.push_back(p);
  }
  // split workspace: per problem at its k, then the job tables
  std::vector<SplitWs> ws((size_t)batch);
  std::vector<size_t> offs((size_t)batch, 0);
  size_t total = 0;
  for (int p : ids) {
    offs[(size_t)p] = total;
    total += split_ws_one(probs[(size_t)p].m, k[(size_t)p], nullptr, nullptr);
  }
  const size_t table_bytes = (size_t)align256((int64_t)batch * 2048 + 65536);
  if ((st = ensure_split_ws(h, total + table_bytes)) != kOk) return st;
  char* base = (char*)h->split_ws;
  char* tables = base + total;
  for (int p : ids) split_ws_one(probs[(size_t)p].m, k[(size_t)p], &ws[(size_t)p], base + offs[(size_t)p]);

  // line 4, line 5, then the FP64 Cholesky and stage 2
  if ((st = split_trsm_step(h, ids, probs, k, ws, P.rsk, true, P.scalars, tables, stream)) != kOk)
    return st;
  if ((st = split_gram_step(h, ids, probs, k, ws, P.g, P.scalars, tables, stream)) != kOk)
    return st;
  if (launch_potrf_batched(P.po, batch, stream) != cudaSuccess ||
      launch_rank_stage2_batched(P.s2, batch, stream) != cudaSuccess)
    return kCudaError;
  // line 7 at the rank after the Cholesky (Remark 4, stage 2)
  if ((st = read_scalars(h, P.scalars, batch, stream)) != kOk) return st;
  std::vector<int> ids7;
  for (int p : ids) {
    k[(size_t)p] = h->pinned_sc[p].k;
    if (h->pinned_sc[p].status == kOk && k[(size_t)p] > 0) ids7.push_back(p);
  }
  if ((st = split_trsm_step(h, ids7, probs, k, ws, P.rpre, false, P.scalars, tables, stream)) !=
      kOk)
    return st;
  if (launch_trmm_batched(P.tm, P.base_tm, batch, P.tiles_tm, stream) != cudaSuccess ||
      launch_finalize_batched(P.fi, batch, stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

}  // namespace cqrrpt

namespace {

int batched_split_run(cqrrpt_handle h, std::vector<BatchProblem>& probs, cudaStream_t stream) {
  const int batch = (int)probs.size();
  const BatchWs W = batch_ws(h, batch);
  BatchPlan P;
  P.scalars = W.scalars;
  P.tables = W.tables;
  batch_plan(P, batch, probs.data(), W.per_problem, nullptr, &h->tune);
  int st = stage_tables(h, P, stream);
  if (st != kOk) return st;
  return batched_split_exec(h, P, probs, stream);
}

int batched_run(cqrrpt_handle h, std::vector<BatchProblem>& probs, cudaStream_t stream) {
  const int batch = (int)probs.size();
  const BatchWs W = batch_ws(h, batch);
  BatchPlan P;
  P.scalars = W.scalars;
  P.tables = W.tables;
  batch_plan(P, batch, probs.data(), W.per_problem, nullptr, &h->tune);
  int st = stage_tables(h, P, stream);
  if (st != kOk) return st;
  if (sketch_set_attributes(P.max_d) != cudaSuccess) return kCudaError;

  if (!h->use_graphs) return batch_launch(P, stream) == cudaSuccess ? kOk : kCudaError;

  const int64_t key[12] = {batch, P.max_d, P.tiles_list, P.tiles_part, P.tiles_comb,
                           P.tiles_gath, P.tiles_trsm, P.tiles_gp, P.tiles_gc, P.tiles_tm,
                           (int64_t)(uintptr_t)P.tables, (int64_t)(uintptr_t)P.scalars};
  if (!h->graph_exec || memcmp(key, h->graph_key, sizeof(key)) != 0) {
    if (h->graph_exec) {
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    if (!h->capture && cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking) != cudaSuccess)
      return kCudaError;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return kCudaError;
    const long long before = g_launches.load();
    cudaError_t e = batch_launch(P, h->capture);
    const cudaError_t e2 = cudaStreamEndCapture(h->capture, &graph);
    h->graph_kernels = (int)(g_launches.load() - before);
    g_launches.store(before);  // captured, not launched
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return kCudaError;
    }
    e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->graph_exec = nullptr;
      return kCudaError;
    }
    memcpy(h->graph_key, key, sizeof(key));
  }
  if (cudaGraphLaunch(h->graph_exec, stream) != cudaSuccess) return kCudaError;
  count_launches(h->graph_kernels);
  return kOk;
}

// Times the line-4 TRSM and the Gram partial kernel of the problems in
// `sub` (indices into probs) with every problem at shape `v`; best of
// `reps` runs each (microseconds).
int time_bucket(cqrrpt_handle h, const std::vector<BatchProblem>& probs,
                const std::vector<int>& sub, int v, const BatchWs& W,
                const std::vector<char*>& ws_each, cudaStream_t stream, double* t_trsm,
                double* t_gram) {
  std::vector<BatchProblem> sp;
  std::vector<char*> sw;
  std::vector<int> si;
  for (int i : sub) {
    sp.push_back(probs[(size_t)i]);
    sw.push_back(ws_each[(size_t)i]);
    si.push_back(i);
  }
  BatchTuning T;
  for (int b = 0; b < kTuneBuckets; ++b) T.trsm_jb[b] = T.gram_tile[b] = v;
  BatchPlan P;
  P.scalars = W.scalars;
  P.tables = W.tables;
  batch_plan(P, (int)sp.size(), sp.data(), nullptr, sw.data(), &T, si.data());
  int st = stage_tables(h, P, stream);
  if (st != kOk) return st;
  cudaEvent_t ev[3];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return kCudaError;
  const int reps = 3;
  *t_trsm = *t_gram = 1e300;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(ev[0], stream);
    if (e == cudaSuccess)
      e = launch_trsm_rut_batched(P.t1, P.base_trsm, P.nprob, P.tiles_trsm, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], stream);
    if (e == cudaSuccess) e = launch_gram_batched(0, P.gr, P.base_gp, P.nprob, P.tiles_gp, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
    if (e == cudaSuccess) {
      *t_trsm = std::min(*t_trsm, 1e3 * (double)a);
      *t_gram = std::min(*t_gram, 1e3 * (double)b);
    }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  return e == cudaSuccess ? kOk : kCudaError;
}

}  // namespace

extern "C" {

int cqrrpt_batched_d(cqrrpt_handle h, int batch, const int64_t* m, const int64_t* n,
                     const double* const* A, const int64_t* lda, double gamma, int nnz,
                     const double* tol, const uint64_t* seed, int precision, double* const* Q,
                     const int64_t* ldq, double* const* R, const int64_t* ldr, int64_t* const* J,
                     int64_t* k_dev, int* status_dev, cudaStream_t stream) {
  if (!h) return -1;
  int st = batch_check(batch, m, n, A, lda, gamma, nnz, tol, seed, precision, Q, ldq, R, ldr, J);
  if (st != kOk) return st;
  DevGuard g(h->device);
  size_t need = 0;
  st = cqrrpt_batched_workspace_size(batch, m, n, gamma, nnz, &need);
  if (st != kOk) return st;
  st = ensure_ws(h, need);
  if (st != kOk) return st;
  std::vector<BatchProblem> probs = batch_problems(batch, m, n, A, lda, gamma, nnz, tol, seed, Q,
                                                   ldq, R, ldr, J, k_dev, status_dev);
  if (precision == CQRRPT_SPLITBF16) return batched_split_run(h, probs, stream);
  return batched_run(h, probs, stream);
}

int cqrrpt_batched_autotune(cqrrpt_handle h, int batch, const int64_t* m, const int64_t* n,
                            const double* const* A, const int64_t* lda, double gamma, int nnz,
                            const double* tol, const uint64_t* seed, int precision,
                            double* const* Q, const int64_t* ldq, double* const* R,
                            const int64_t* ldr, int64_t* const* J, int64_t* k_dev,
                            int* status_dev, double* times_us_host, cudaStream_t stream) {
  if (!h) return -1;
  int st = batch_check(batch, m, n, A, lda, gamma, nnz, tol, seed, precision, Q, ldq, R, ldr, J);
  if (st != kOk) return st;
  if (precision != CQRRPT_FP64) return -11;  // the tuned shapes are the FP64 kernels'
  DevGuard g(h->device);
  size_t need = 0;
  st = cqrrpt_batched_workspace_size(batch, m, n, gamma, nnz, &need);
  if (st != kOk) return st;
  st = ensure_ws(h, need);
  if (st != kOk) return st;
  std::vector<BatchProblem> probs = batch_problems(batch, m, n, A, lda, gamma, nnz, tol, seed, Q,
                                                   ldq, R, ldr, J, k_dev, status_dev);
  // 1. one pass with the current shapes: R^sk, J and k of every problem
  if ((st = batched_run(h, probs, stream)) != kOk) return st;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return kCudaError;
  // 2. per width bucket and shape: time the line-4 TRSM (it rewrites M^pre
  //    into Q from M, J and R^sk, the same values every time) and the Gram
  //    partial sums of that M^pre
  const BatchWs W = batch_ws(h, batch);
  std::vector<char*> ws_each((size_t)batch);
  char* w = W.per_problem;
  std::vector<std::vector<int>> members(kTuneBuckets);
  for (int p = 0; p < batch; ++p) {
    ws_each[(size_t)p] = w;
    w += problem_workspace_bytes(probs[(size_t)p].m, probs[(size_t)p].n, probs[(size_t)p].d, nnz);
    members[(size_t)tune_bucket(probs[(size_t)p].n)].push_back(p);
  }
  if (times_us_host)
    for (int i = 0; i < 4 * kTuneBuckets; ++i) times_us_host[i] = 0.0;
  BatchTuning T = h->tune;
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (members[(size_t)b].empty()) continue;
    double tt[3], tg[3];
    // shapes 16 and 32 for both kernels; 8 x 8 Gram tiles as well (less
    // padding of a small k; the TRSM time of that run is not used)
    const int shapes[3] = {16, 32, 8};
    for (int v = 0; v < 3; ++v) {
      st = time_bucket(h, probs, members[(size_t)b], shapes[v], W, ws_each, stream, &tt[v], &tg[v]);
      if (st != kOk) return st;
    }
    T.trsm_jb[b] = tt[0] < tt[1] ? 16 : 32;
    T.gram_tile[b] = tg[2] < std::min(tg[0], tg[1]) ? 8 : (tg[0] < tg[1] ? 16 : 32);
    if (times_us_host) {
      times_us_host[4 * b + 0] = tt[0];
      times_us_host[4 * b + 1] = tt[1];
      times_us_host[4 * b + 2] = tg[0];
      times_us_host[4 * b + 3] = tg[1];
    }
  }
  h->tune = T;
  // 3. the batch again with the chosen shapes (the outputs of the call)
  if ((st = batched_run(h, probs, stream)) != kOk) return st;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return kCudaError;
  return kOk;
}

int cqrrpt_batched_get_tuning(cqrrpt_handle h, int* trsm_jb_host, int* gram_tile_host) {
  if (!h) return -1;
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (trsm_jb_host) trsm_jb_host[b] = h->tune.trsm_jb[b];
    if (gram_tile_host) gram_tile_host[b] = h->tune.gram_tile[b];
  }
  return kOk;
}

int cqrrpt_batched_set_tuning(cqrrpt_handle h, const int* trsm_jb_host,
                              const int* gram_tile_host) {
  if (!h) return -1;
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (trsm_jb_host && trsm_jb_host[b] != 16 && trsm_jb_host[b] != 32) return -2;
    if (gram_tile_host && gram_tile_host[b] != 8 && gram_tile_host[b] != 16 &&
        gram_tile_host[b] != 32)
      return -3;
  }
  for (int b = 0; b < kTuneBuckets; ++b) {
    if (trsm_jb_host) h->tune.trsm_jb[b] = trsm_jb_host[b];
    if (gram_tile_host) h->tune.gram_tile[b] = gram_tile_host[b];
  }
  return kOk;
}

int cqrrpt_last_status(cqrrpt_handle h, cudaStream_t stream, int* status_host, int64_t* k_host) {
  if (!h) return -1;
  DevGuard g(h->device);
  int64_t* pk = h->pinned;
  int* ps = (int*)(h->pinned + 1);
  if (launch_finalize(h->sc, pk, ps, stream) != cudaSuccess) return kCudaError;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return kCudaError;
  if (status_host) *status_host = *ps;
  if (k_host) *k_host = *pk;
  return kOk;
}

int cqrrpt_set_profiling(cqrrpt_handle h, int enable) {
  if (!h) return -1;
  DevGuard g(h->device);
  if (enable && !h->ev[0]) {
    for (int i = 0; i <= kPhases; ++i)
      if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return kCudaError;
  }
  h->profiling = enable ? 1 : 0;
  return kOk;
}

int cqrrpt_phase_times(cqrrpt_handle h, float* ms_host, int nphases) {
  if (!h) return -1;
  if (!ms_host) return -2;
  if (nphases < 1 || nphases > kPhases) return -3;
  if (!h->profiling) return -1;
  DevGuard g(h->device);
  if (cudaEventSynchronize(h->ev[kPhases]) != cudaSuccess) return kCudaError;
  for (int i = 0; i < nphases; ++i)
    if (cudaEventElapsedTime(&ms_host[i], h->ev[i], h->ev[i + 1]) != cudaSuccess) return kCudaError;
  return kOk;
}

long long cqrrpt_kernel_launches(void) { return g_launches.load(); }

int cqrrpt_set_wait_limits(int64_t grid_spins, int64_t tensor_wait_ns) {
  if (grid_spins < 0) return -1;
  if (tensor_wait_ns < 0) return -2;
  if (qrcp_set_spin_limit((unsigned long long)grid_spins) != cudaSuccess ||
      oz_set_wait_ns((unsigned long long)tensor_wait_ns) != cudaSuccess) {
    cudaGetLastError();
    return kCudaError;
  }
  return kOk;
}

const char* cqrrpt_status_string(int status) {
  switch (status) {
    case kOk: return "success";
    case kRankZero: return "numerical rank is zero";
    case kNonFinite: return "non-finite values in the input (sketch)";
    case kCudaError: return "CUDA error";
    case kNoMemory: return "out of device memory";
    case kTimeout: return "device-side wait timed out";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

int cqrrpt_sketch_d(cqrrpt_handle h, int64_t m, int64_t n, const double* A, int64_t lda,
                    int64_t d, int nnz, uint64_t seed, double* Ask, int64_t ldsk,
                    cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (d < 1 || d > 28000) return -6;
  if (nnz < 1 || nnz > d || nnz > kMaxNnzInline) return -7;
  if (!Ask) return -9;
  if (ldsk < d) return -10;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)sketch_workspace_bytes(m, n, (int)d, nnz));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  if (launch_sketch(m, n, A, lda, (int)d, nnz, seed, 1.0 / std::sqrt((double)nnz), Ask, ldsk,
                    h->ws, &h->sc->status, stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_qrcp_d(cqrrpt_handle h, int64_t d, int64_t n, double* X, int64_t ldx, int64_t* J,
                  double* Rsk, int64_t ldr, cudaStream_t stream) {
  if (!h) return -1;
  if (d < 1) return -2;
  if (n < 1 || n > d || n > 16384) return -3;
  if (!X) return -4;
  if (ldx < d) return -5;
  if (!J) return -6;
  if (!Rsk) return -7;
  if (ldr < n) return -8;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)qrcp_workspace_bytes(n));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  if (launch_qrcp((int)d, (int)n, X, ldx, J, Rsk, ldr, h->ws, h->sc, h->num_sms, stream) !=
      cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_rank_d(cqrrpt_handle h, int64_t n, const double* Rsk, int64_t ldr, double tol,
                  int64_t* k_dev, cudaStream_t stream) {
  if (!h) return -1;
  if (n < 1 || n > 16384) return -2;
  if (!Rsk) return -3;
  if (ldr < n) return -4;
  if (std::isnan(tol)) return -5;
  if (!k_dev) return -6;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)align256((n + 1) * 8));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  if (launch_rank((int)n, Rsk, ldr, tol, h->sc, (double*)h->ws, stream) != cudaSuccess)
    return kCudaError;
  copy_k_kernel<<<1, 1, 0, stream>>>(h->sc, k_dev);
  return cudaGetLastError() == cudaSuccess ? kOk : kCudaError;
}

int cqrrpt_trsm_d(cqrrpt_handle h, int64_t m, int64_t k, const double* B, int64_t ldb,
                  const int64_t* cols, const double* T, int64_t ldt, double* X, int64_t ldx,
                  cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (k < 1 || k > 16384) return -3;
  if (!B) return -4;
  if (ldb < m) return -5;
  if (!T) return -7;
  if (ldt < k) return -8;
  if (!X) return -9;
  if (ldx < m) return -10;
  DevGuard g(h->device);
  if (launch_init_scalars(h->sc, k, stream) != cudaSuccess) return kCudaError;
  if (launch_trsm_rut(m, (int)k, &h->sc->k, B, ldb, cols, T, ldt, X, ldx, &h->sc->status,
                      stream) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_gram_d(cqrrpt_handle h, int64_t m, int64_t k, const double* X, int64_t ldx, double* G,
                  int64_t ldg, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (k < 1 || k > 16384) return -3;
  if (!X) return -4;
  if (ldx < m) return -5;
  if (!G) return -6;
  if (ldg < k) return -7;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)gram_workspace_bytes(m, k));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, k, stream) != cudaSuccess) return kCudaError;
  if (launch_gram(m, (int)k, &h->sc->k, X, ldx, G, ldg, h->ws, &h->sc->status, stream, false,
                  true) != cudaSuccess)
    return kCudaError;
  return kOk;
}

int cqrrpt_potrf_d(cqrrpt_handle h, int64_t k, double* G, int64_t ldg, double* R, int64_t ldr,
                   int64_t* fail_dev, cudaStream_t stream) {
  if (!h) return -1;
  if (k < 1 || k > 16384) return -2;
  if (!G) return -3;
  if (ldg < k) return -4;
  if (!R) return -5;
  if (ldr < k) return -6;
  DevGuard g(h->device);
  if (launch_init_scalars(h->sc, k, stream) != cudaSuccess) return kCudaError;
  if (launch_potrf((int)k, G, ldg, R, ldr, h->sc, stream) != cudaSuccess) return kCudaError;
  if (fail_dev) {
    copy_fail_kernel<<<1, 1, 0, stream>>>(h->sc, fail_dev);
    if (cudaGetLastError() != cudaSuccess) return kCudaError;
  }
  return kOk;
}

int cqrrpt_gram_split_d(cqrrpt_handle h, int64_t m, int64_t k, const double* X, int64_t ldx,
                        double* G, int64_t ldg, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (k < 1 || k > 16384) return -3;
  if (!X) return -4;
  if (ldx < m) return -5;
  if (!G) return -6;
  if (ldg < k) return -7;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)oz_gram_workspace(m, (int)k, nullptr));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  return oz_gram(m, (int)k, X, ldx, G, ldg, h->ws, stream, &h->sc->status) == cudaSuccess
             ? kOk
             : kCudaError;
}

int cqrrpt_trsm_split_d(cqrrpt_handle h, int64_t m, int64_t k, const double* B, int64_t ldb,
                        const int64_t* cols, const double* T, int64_t ldt, double* X,
                        int64_t ldx, cudaStream_t stream) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (k < 1 || k > 16384) return -3;
  if (!B) return -4;
  if (ldb < m) return -5;
  if (!T) return -7;
  if (ldt < k) return -8;
  if (!X) return -9;
  if (ldx < m) return -10;
  DevGuard g(h->device);
  int st = ensure_ws(h, (size_t)oz_trsm_workspace(m, (int)k));
  if (st != kOk) return st;
  if (launch_init_scalars(h->sc, 0, stream) != cudaSuccess) return kCudaError;
  return oz_trsm(m, (int)k, B, ldb, cols, T, ldt, X, ldx, h->ws, stream, &h->sc->status) ==
                 cudaSuccess
             ? kOk
             : kCudaError;
}

int cqrrpt_trmm_d(cqrrpt_handle h, int64_t k, int64_t n, const double* Rpre, int64_t ldp,
                  const double* Rsk, int64_t ldsk, double* R, int64_t ldr, cudaStream_t stream) {
  if (!h) return -1;
  if (k < 1) return -2;
  if (n < k || n > 16384) return -3;
  if (!Rpre) return -4;
  if (ldp < k) return -5;
  if (!Rsk) return -6;
  if (ldsk < k) return -7;
  if (!R) return -8;
  if (ldr < k) return -9;
  DevGuard g(h->device);
  if (launch_init_scalars(h->sc, k, stream) != cudaSuccess) return kCudaError;
  if (launch_trmm((int)n, &h->sc->k, Rpre, ldp, Rsk, ldsk, R, ldr, &h->sc->status, stream) !=
      cudaSuccess)
    return kCudaError;
  return kOk;
}

int64_t cqrrpt_sketch_dim(int64_t n, double gamma) { return sketch_dim(n, gamma); }

void cqrrpt_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const Philox4 r = philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

void cqrrpt_saso_column(uint64_t seed, int64_t r, int64_t d, int nnz, int32_t* rows,
                        uint8_t* neg) {
  int tr[kMaxNnzInline];
  uint32_t bits = 0;
  if (nnz < 1 || nnz > kMaxNnzInline || nnz > d) return;
  saso_column(seed, r, (int)d, nnz, tr, &bits);
  for (int q = 0; q < nnz; ++q) {
    rows[q] = tr[q];
    neg[q] = (uint8_t)((bits >> q) & 1u);
  }
}

}  // extern "C"
