// Continuous-batching CQRRPT server whose units of work overlap on the GPU.
//
// Requests (a host matrix plus host output buffers) are submitted from any
// thread and return a ticket at once.  The server runs its work on L lanes;
// a lane is a handle (workspace, device scalars), two compute streams (the
// highest stream priority for single-route units, whose kernels then get
// the SMs first, the lowest for batched waves), a launch table area and a
// worker thread.  One scheduler thread:
//   * admits queued requests in arrival order while their device footprint
//     (A, Q, R, J, per-problem workspace) fits the HBM budget -- a first-fit
//     arena over one allocation made at creation -- and at most max_inflight
//     are in flight; the host -> device copy of an admitted request's A is
//     issued at once on the copy-in stream, overlapping running work;
//   * hands units of work to idle lanes, the oldest arrived request first.
//     A request with n above kBatchMaxN (where the one-CTA-per-problem QRCP
//     and Cholesky of the batched kernels would serialise) or in the mode
//     with a second Cholesky-QR pass is a single-route unit: it runs alone
//     on its lane through cqrrpt_d, with the multi-CTA QRCP.  At most
//     lanes - 1 single-route units are in flight, so a lane is always left
//     for small requests.  Other requests run as batched waves: one batched
//     pass (batched.cu, or the batched split path) over the arrived requests
//     of the oldest one's precision.  A wave starts at once when the GPU is
//     idle; while any unit is in flight, arrivals gather until kMinWave are
//     waiting or the oldest has waited kMaxWaitUs.  The cooperative QRCP
//     grids of single-route units on different lanes run one after another
//     on the GPU (qrcp.cu's per-device launch fence), everything else side
//     by side;
//   * when a lane's unit completes, copies each result (Q, R, J, k, status)
//     back on the copy-out stream, frees the request's arena block when the
//     copy is done and records the completion time.
// So a large request no longer holds the GPU alone: small waves and other
// large requests run on the other lanes beside it.  The
// worker threads make the launches (the split path reads k back on the way,
// which blocks only its own lane).  Every wait of the scheduler is a
// host-side poll with a bounded sleep; the kernels contain no cross-CTA
// waits except the single-route QRCP's grid barrier, which is bounded (and
// never shared by two grids at once).
// Results are bit-identical to a standalone call on the same request,
// whatever else shares a wave or runs beside it: each lane has its own
// workspace and the kernels fix their summation orders.
#include <cstdlib>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cqrrpt.h"
#include "batched.h"
#include "kernels.h"
#include "saso.cuh"

namespace cqrrpt {

int handle_finalize(cqrrpt_handle h, int64_t* k_out, int* status_out, cudaStream_t s);
const BatchTuning* handle_tuning(cqrrpt_handle h);
int batched_split_exec(cqrrpt_handle h, BatchPlan& P, const std::vector<BatchProblem>& probs,
                       cudaStream_t stream);

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator of offsets inside one device buffer (host bookkeeping).
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t s) {
    size = s;
    free_.clear();
    free_[0] = s;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum ReqState { kPending = 0, kStaging, kRunning, kCopyBack, kDone };

struct Req {
  uint64_t ticket;
  cqrrpt_request r;
  int64_t d;
  size_t off = 0, bytes = 0;
  double *A = nullptr, *Q = nullptr, *R = nullptr;
  int64_t* J = nullptr;
  char* ws = nullptr;
  int64_t* k_dev = nullptr;
  int* st_dev = nullptr;
  int64_t* k_host = nullptr;  // pinned slots
  int* st_host = nullptr;
  cudaEvent_t h2d = nullptr, done = nullptr;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = kPending;
  cqrrpt_result res{};
};

// Widest problem a batched wave takes; wider ones (and the split-BF16 mode
// with a second Cholesky-QR pass) run alone through cqrrpt_d with the
// multi-CTA QRCP and Cholesky.
constexpr int64_t kBatchMaxN = 256;

bool single_route(const cqrrpt_request& r) {
  return r.precision == CQRRPT_SPLITBF16_CHOLQR2 || r.n > kBatchMaxN;
}

// Device bytes a request holds while in flight.  Requests on the single
// path use the handle's workspace instead of their own.
size_t footprint(const cqrrpt_request& r, int64_t d, int nnz) {
  const int64_t m = r.m, n = r.n;
  size_t b = 0;
  b += (size_t)align256(m * n * 8);      // A
  b += (size_t)align256(m * n * 8);      // Q
  b += (size_t)align256(n * n * 8);      // R
  b += (size_t)align256(n * 8);          // J
  b += 256;                              // k, status
  if (!single_route(r)) b += (size_t)problem_workspace_bytes(m, n, d, nnz);
  return b;
}

}  // namespace

// Dynamic batching: while any unit is in flight, a new wave waits until
// this many requests are ready or the oldest has waited this long.
// CQRRPT_SERVER_MAX_WAIT_US, read when a server is created, sets the wait
// (a larger one trades latency for larger waves).
constexpr int kMinWave = 4;
constexpr double kMaxWaitUs = 8000.0;

enum LaneState { kLaneIdle = 0, kLaneLaunching, kLaneRunning };

struct Lane {
  int id = 0;
  cqrrpt_handle h = nullptr;
  bool own_handle = false;
  cudaStream_t compute = nullptr;     // the current unit's stream
  cudaStream_t wave_stream = nullptr;  // batched waves
  cudaStream_t single_stream = nullptr;  // single-route units: highest priority
  cudaEvent_t done = nullptr, stage_ev = nullptr;
  char* fixed = nullptr;  // DeviceScalars[max_inflight] + batch tables
  void* stage = nullptr;  // pinned table staging
  size_t stage_bytes = 0;
  std::vector<Req*> wave;
  bool single = false;
  int state = kLaneIdle;
  bool has_work = false;
  int rc = kOk;
  std::thread th;
  std::condition_variable cv;
};

struct Server {
  cqrrpt_handle h = nullptr;
  int device = 0;
  double gamma = 1.25;
  int nnz = 4;
  int max_inflight = 64;
  char* arena_base = nullptr;
  Arena arena;
  size_t fixed_bytes = 0;
  int64_t* pinned_slots = nullptr;  // 2 words per in-flight slot
  std::vector<int> free_slots;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  std::vector<Lane*> lanes;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Req*> inflight;
  std::unordered_map<uint64_t, Req*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool stop_workers = false;
  int error = 0;
  int64_t waves = 0, completed = 0, single_units = 0, batched_units = 0, batched_reqs = 0;
  int busy = 0, max_busy = 0;
  double max_wait_us = kMaxWaitUs;
  int (*run_single)(cqrrpt_handle, const cqrrpt_request&, double, int, double*, double*, double*,
                    int64_t*, cudaStream_t) = nullptr;

  void loop();
  bool step();
  void worker(Lane* L);
  int launch_unit(Lane* L);
};

// The lane's unit: launches only (the worker records `done` after them).
int Server::launch_unit(Lane* L) {
  if (L->single) {
    Req* q = L->wave[0];
    // FP64 requests are enqueued without a host wait; the split-BF16
    // pipeline reads k back on the way (its recursive products are sized on
    // the host).  k and status land in the request's device slots.
    const int rc = run_single(L->h, q->r, gamma, nnz, q->A, q->Q, q->R, q->J, L->compute);
    if (rc != kOk && rc != kRankZero && rc != kNonFinite) {
      *q->k_host = 0;
      *q->st_host = rc;
      cudaMemcpyAsync(q->k_dev, q->k_host, sizeof(int64_t), cudaMemcpyHostToDevice, L->compute);
      cudaMemcpyAsync(q->st_dev, q->st_host, sizeof(int), cudaMemcpyHostToDevice, L->compute);
      return kOk;
    }
    return handle_finalize(L->h, q->k_dev, q->st_dev, L->compute);
  }
  const std::vector<Req*>& ready = L->wave;
  std::vector<BatchProblem> probs(ready.size());
  std::vector<char*> wss(ready.size());
  for (size_t i = 0; i < ready.size(); ++i) {
    const Req* q = ready[i];
    BatchProblem& b = probs[i];
    b.m = q->r.m; b.n = q->r.n; b.d = q->d; b.nnz = nnz; b.tol = q->r.tol;
    b.seed = q->r.seed; b.A = q->A; b.lda = q->r.m; b.Q = q->Q; b.ldq = q->r.m;
    b.R = q->R; b.ldr = q->r.n; b.J = q->J; b.k_out = q->k_dev; b.status_out = q->st_dev;
    wss[i] = q->ws;
  }
  BatchPlan P;
  P.scalars = (DeviceScalars*)L->fixed;
  P.tables = L->fixed + align256((int64_t)max_inflight * sizeof(DeviceScalars));
  batch_plan(P, (int)ready.size(), probs.data(), nullptr, wss.data(), handle_tuning(L->h));
  const size_t img = P.image.size();
  cudaEventSynchronize(L->stage_ev);
  if (img > L->stage_bytes) {
    if (L->stage) cudaFreeHost(L->stage);
    L->stage = nullptr;
    L->stage_bytes = 0;
    if (cudaMallocHost(&L->stage, img) != cudaSuccess) return kNoMemory;
    L->stage_bytes = img;
  }
  memcpy(L->stage, P.image.data(), img);
  if (cudaMemcpyAsync(P.tables, L->stage, img, cudaMemcpyHostToDevice, L->compute) != cudaSuccess)
    return kCudaError;
  cudaEventRecord(L->stage_ev, L->compute);
  if (ready[0]->r.precision != CQRRPT_FP64)
    return batched_split_exec(L->h, P, probs, L->compute);  // waits for its stream twice
  sketch_set_attributes(P.max_d);
  return batch_launch(P, L->compute) == cudaSuccess ? kOk : kCudaError;
}

void Server::worker(Lane* L) {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu);
  while (true) {
    L->cv.wait(lock, [&] { return L->has_work || stop_workers; });
    if (!L->has_work) break;
    lock.unlock();
    int rc = launch_unit(L);
    if (cudaEventRecord(L->done, L->compute) != cudaSuccess && rc == kOk) rc = kCudaError;
    lock.lock();
    L->rc = rc;
    L->has_work = false;
    L->state = kLaneRunning;
    cv.notify_all();
  }
}

bool Server::step() {
  bool progress = false;
  {
    std::lock_guard<std::mutex> lock(mu);
    // completions of copies back
    for (size_t i = 0; i < inflight.size();) {
      Req* q = inflight[i];
      if (q->state == kCopyBack && cudaEventQuery(q->done) == cudaSuccess) {
        q->t_done = now_us();
        q->res.k = *q->k_host;
        q->res.status = *q->st_host;
        q->res.latency_us = q->t_done - q->t_submit;
        q->res.queue_us = q->t_start - q->t_submit;
        q->state = kDone;
        arena.release(q->off, q->bytes);
        free_slots.push_back((int)((q->k_host - pinned_slots) / 2));
        inflight[i] = inflight.back();
        inflight.pop_back();
        ++completed;
        progress = true;
        continue;
      }
      ++i;
    }
    // units that finished on the GPU: copy their results back
    for (Lane* L : lanes) {
      if (L->state != kLaneRunning || cudaEventQuery(L->done) != cudaSuccess) continue;
      if (L->rc != kOk) {
        error = L->rc;
        return false;
      }
      cudaStreamWaitEvent(copy_out, L->done, 0);
      for (Req* q : L->wave) {
        const cqrrpt_request& r = q->r;
        cudaMemcpy2DAsync(r.Q_host, r.ldq * sizeof(double), q->Q, r.m * sizeof(double),
                          r.m * sizeof(double), r.n, cudaMemcpyDeviceToHost, copy_out);
        cudaMemcpy2DAsync(r.R_host, r.ldr * sizeof(double), q->R, r.n * sizeof(double),
                          r.n * sizeof(double), r.n, cudaMemcpyDeviceToHost, copy_out);
        cudaMemcpyAsync(r.J_host, q->J, r.n * sizeof(int64_t), cudaMemcpyDeviceToHost, copy_out);
        cudaMemcpyAsync(q->k_host, q->k_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, copy_out);
        cudaMemcpyAsync(q->st_host, q->st_dev, sizeof(int), cudaMemcpyDeviceToHost, copy_out);
        cudaEventRecord(q->done, copy_out);
        q->state = kCopyBack;
      }
      L->wave.clear();
      L->single = false;
      L->state = kLaneIdle;
      --busy;
      progress = true;
    }
    // admission
    while (!pending.empty() && (int)inflight.size() < max_inflight && !free_slots.empty()) {
      Req* q = pending.front();
      const cqrrpt_request& r = q->r;
      size_t off = 0;
      const size_t bytes = footprint(r, q->d, nnz);
      if (!arena.alloc(bytes, &off)) break;
      pending.pop_front();
      q->off = off;
      q->bytes = bytes;
      char* p = arena_base + off;
      q->A = (double*)p; p += align256(r.m * r.n * 8);
      q->Q = (double*)p; p += align256(r.m * r.n * 8);
      q->R = (double*)p; p += align256(r.n * r.n * 8);
      q->J = (int64_t*)p; p += align256(r.n * 8);
      q->k_dev = (int64_t*)p;
      q->st_dev = (int*)(p + 8);
      p += 256;
      q->ws = p;
      const int slot = free_slots.back();
      free_slots.pop_back();
      q->k_host = pinned_slots + 2 * slot;
      q->st_host = (int*)(pinned_slots + 2 * slot + 1);
      cudaMemcpy2DAsync(q->A, r.m * sizeof(double), r.A_host, r.lda * sizeof(double),
                        r.m * sizeof(double), r.n, cudaMemcpyHostToDevice, copy_in);
      cudaEventRecord(q->h2d, copy_in);
      q->state = kStaging;
      q->t_start = now_us();
      inflight.push_back(q);
      progress = true;
    }
    // hand units to idle lanes
    std::vector<Req*> arrived;
    for (Req* q : inflight)
      if (q->state == kStaging && cudaEventQuery(q->h2d) == cudaSuccess) arrived.push_back(q);
    std::sort(arrived.begin(), arrived.end(),
              [](const Req* a, const Req* b) { return a->t_submit < b->t_submit; });
    int singles_busy = 0, waves_busy = 0;
    for (Lane* L : lanes)
      if (L->state != kLaneIdle) {
        if (L->single) ++singles_busy;
        else ++waves_busy;
      }
    // single-route units in flight at most: all lanes but one, so that a
    // lane is always left for the batched waves of small requests
    const int max_singles = lanes.size() > 1 ? (int)lanes.size() - 1 : 1;
    const double now = now_us();
    for (Lane* L : lanes) {
      if (L->state != kLaneIdle || arrived.empty()) continue;
      std::vector<Req*> unit;
      bool single = false;
      Req* oldest_single = nullptr;
      Req* oldest_batched = nullptr;
      for (Req* q : arrived) {
        if (single_route(q->r)) {
          if (!oldest_single) oldest_single = q;
        } else if (!oldest_batched) {
          oldest_batched = q;
        }
      }
      const bool can_single = oldest_single && singles_busy < max_singles;
      if (can_single && (!oldest_batched || oldest_single->t_submit < oldest_batched->t_submit)) {
        unit.push_back(oldest_single);
        single = true;
      } else if (oldest_batched) {
        for (Req* q : arrived)
          if (!single_route(q->r) && q->r.precision == oldest_batched->r.precision)
            unit.push_back(q);
        if (waves_busy + singles_busy > 0 && (int)unit.size() < kMinWave &&
            now - oldest_batched->t_start < max_wait_us) {
          unit.clear();  // gather more while another wave runs
          if (can_single) {
            unit.push_back(oldest_single);
            single = true;
          }
        }
      } else if (can_single) {
        unit.push_back(oldest_single);
        single = true;
      }
      if (unit.empty()) continue;
      for (Req* q : unit) {
        q->state = kRunning;
        arrived.erase(std::find(arrived.begin(), arrived.end(), q));
      }
      L->wave = unit;
      L->single = single;
      // a large request's kernels get the SMs first (it sets the tail
      // latency); small waves fill what it leaves
      L->compute = single ? L->single_stream : L->wave_stream;
      L->state = kLaneLaunching;
      L->has_work = true;
      ++busy;
      if (busy > max_busy) max_busy = busy;
      ++waves;
      if (single) {
        ++single_units;
        ++singles_busy;
      } else {
        ++batched_units;
        batched_reqs += (int64_t)unit.size();
        ++waves_busy;
      }
      L->cv.notify_all();
      progress = true;
    }
  }
  if (progress) cv.notify_all();
  return progress;
}

void Server::loop() {
  cudaSetDevice(device);
  while (true) {
    {
      std::lock_guard<std::mutex> lock(mu);
      if (stop && pending.empty() && inflight.empty() && busy == 0) break;
    }
    const bool progress = step();
    if (error) {
      std::lock_guard<std::mutex> lock(mu);
      cv.notify_all();
      break;
    }
    if (!progress) {
      std::unique_lock<std::mutex> lock(mu);
      cv.wait_for(lock, std::chrono::microseconds(50));
    }
  }
}

}  // namespace cqrrpt

using namespace cqrrpt;

struct cqrrpt_server_s {
  Server s;
};

namespace {

int run_single_impl(cqrrpt_handle h, const cqrrpt_request& r, double gamma, int nnz, double* A,
                    double* Q, double* R, int64_t* J, cudaStream_t s) {
  return cqrrpt_d(h, r.m, r.n, A, r.m, gamma, nnz, r.tol, r.seed, r.precision, Q, r.m, R, r.n, J,
                  nullptr, nullptr, s);
}

}  // namespace

extern "C" {

int cqrrpt_server_create_lanes(cqrrpt_handle h, size_t hbm_budget_bytes, int max_inflight,
                                double gamma, int nnz_per_col, int lanes, cqrrpt_server* out) {
  if (!h) return -1;
  if (hbm_budget_bytes < (1u << 20)) return -2;
  if (max_inflight < 1 || max_inflight > 4096) return -3;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -4;
  if (nnz_per_col < 1 || nnz_per_col > kMaxNnzInline) return -5;
  if (lanes < 1 || lanes > 8) return -6;
  if (!out) return -7;
  *out = nullptr;
  cqrrpt_server_s* S = new cqrrpt_server_s();
  Server& s = S->s;
  if (const char* e = std::getenv("CQRRPT_SERVER_MAX_WAIT_US")) {
    const double v = std::strtod(e, nullptr);
    if (v >= 0.0 && v <= 10e6) s.max_wait_us = v;
  }
  s.h = h;
  s.gamma = gamma;
  s.nnz = nnz_per_col;
  s.max_inflight = max_inflight;
  s.run_single = run_single_impl;
  if (cudaGetDevice(&s.device) != cudaSuccess) { delete S; return kCudaError; }
  s.fixed_bytes = (size_t)(align256((int64_t)max_inflight * sizeof(DeviceScalars)) +
                           batch_table_bytes(max_inflight));
  int jb[16], gt[16];
  bool ok = cudaMalloc((void**)&s.arena_base, hbm_budget_bytes) == cudaSuccess &&
            cudaMallocHost((void**)&s.pinned_slots, (size_t)max_inflight * 16) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s.copy_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s.copy_out, cudaStreamNonBlocking) == cudaSuccess &&
            cqrrpt_batched_get_tuning(h, jb, gt) == kOk;
  for (int i = 0; ok && i < lanes; ++i) {
    Lane* L = new Lane();
    L->id = i;
    s.lanes.push_back(L);
    if (i == 0) {
      L->h = h;
    } else {
      ok = cqrrpt_create(&L->h, s.device) == kOk && cqrrpt_batched_set_tuning(L->h, jb, gt) == kOk;
      L->own_handle = L->h != nullptr;
    }
    int lo = 0, hi = 0;
    ok = ok && cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
         cudaStreamCreateWithPriority(&L->wave_stream, cudaStreamNonBlocking, lo) == cudaSuccess &&
         cudaStreamCreateWithPriority(&L->single_stream, cudaStreamNonBlocking, hi) ==
             cudaSuccess &&
         cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&L->stage_ev, cudaEventDisableTiming) == cudaSuccess &&
         cudaMalloc((void**)&L->fixed, s.fixed_bytes) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (Lane* L : s.lanes) {
      if (L->fixed) cudaFree(L->fixed);
      if (L->done) cudaEventDestroy(L->done);
      if (L->stage_ev) cudaEventDestroy(L->stage_ev);
      if (L->wave_stream) cudaStreamDestroy(L->wave_stream);
      if (L->single_stream) cudaStreamDestroy(L->single_stream);
      if (L->own_handle) cqrrpt_destroy(L->h);
      delete L;
    }
    if (s.copy_in) cudaStreamDestroy(s.copy_in);
    if (s.copy_out) cudaStreamDestroy(s.copy_out);
    if (s.pinned_slots) cudaFreeHost(s.pinned_slots);
    if (s.arena_base) cudaFree(s.arena_base);
    delete S;
    return kNoMemory;
  }
  s.arena.init(hbm_budget_bytes);
  for (int i = max_inflight - 1; i >= 0; --i) s.free_slots.push_back(i);
  for (Lane* L : s.lanes) L->th = std::thread([S, L] { S->s.worker(L); });
  s.th = std::thread([S] { S->s.loop(); });
  *out = S;
  return kOk;
}

int cqrrpt_server_create(cqrrpt_handle h, size_t hbm_budget_bytes, int max_inflight, double gamma,
                         int nnz_per_col, cqrrpt_server* out) {
  if (!out) return -6;
  const int rc = cqrrpt_server_create_lanes(h, hbm_budget_bytes, max_inflight, gamma,
                                            nnz_per_col, 3, out);
  return rc == -7 ? -6 : rc;
}

int cqrrpt_server_submit(cqrrpt_server S, const cqrrpt_request* r, uint64_t* ticket) {
  if (!S) return -1;
  if (!r) return -2;
  if (!ticket) return -3;
  Server& s = S->s;
  if (r->m < 1 || r->n < 1 || r->n > 16384 || !r->A_host || r->lda < r->m || !r->Q_host ||
      r->ldq < r->m || !r->R_host || r->ldr < r->n || !r->J_host || std::isnan(r->tol))
    return -2;
  if (r->precision != CQRRPT_FP64 && r->precision != CQRRPT_SPLITBF16 &&
      r->precision != CQRRPT_SPLITBF16_CHOLQR2)
    return -2;
  const int64_t d = (int64_t)std::ceil(s.gamma * (double)r->n);
  if (d > r->m || d > 28000 || s.nnz > d) return -2;
  if (footprint(*r, d, s.nnz) > s.arena.size) return kNoMemory;
  Req* q = new Req();
  q->r = *r;
  q->d = d;
  q->t_submit = now_us();
  if (cudaEventCreateWithFlags(&q->h2d, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming) != cudaSuccess) {
    delete q;
    return kCudaError;
  }
  {
    std::lock_guard<std::mutex> lock(s.mu);
    if (s.error) { delete q; return s.error; }
    q->ticket = s.next_ticket++;
    s.pending.push_back(q);
    s.all[q->ticket] = q;
  }
  s.cv.notify_all();
  *ticket = q->ticket;
  return kOk;
}

int cqrrpt_server_poll(cqrrpt_server S, uint64_t ticket, int* done, cqrrpt_result* out) {
  if (!S) return -1;
  if (!done) return -3;
  Server& s = S->s;
  std::lock_guard<std::mutex> lock(s.mu);
  auto it = s.all.find(ticket);
  if (it == s.all.end()) return -2;
  Req* q = it->second;
  *done = q->state == kDone;
  if (*done && out) *out = q->res;
  if (*done) {
    cudaEventDestroy(q->h2d);
    cudaEventDestroy(q->done);
    s.all.erase(it);
    delete q;
  }
  return s.error;
}

int cqrrpt_server_drain(cqrrpt_server S, int64_t timeout_us) {
  if (!S) return -1;
  Server& s = S->s;
  const double t_end = now_us() + (double)timeout_us;
  std::unique_lock<std::mutex> lock(s.mu);
  while (!(s.pending.empty() && s.inflight.empty())) {
    if (s.error) return s.error;
    if (timeout_us >= 0 && now_us() > t_end) return kTimeout;
    s.cv.wait_for(lock, std::chrono::microseconds(200));
  }
  return s.error;
}

int cqrrpt_server_stats(cqrrpt_server S, int64_t* waves, int64_t* completed, int64_t* inflight,
                        int64_t* queued) {
  if (!S) return -1;
  Server& s = S->s;
  std::lock_guard<std::mutex> lock(s.mu);
  if (waves) *waves = s.waves;
  if (completed) *completed = s.completed;
  if (inflight) *inflight = (int64_t)s.inflight.size();
  if (queued) *queued = (int64_t)s.pending.size();
  return kOk;
}

int cqrrpt_server_stats_ex(cqrrpt_server S, int64_t* out, int count) {
  if (!S) return -1;
  if (!out || count < 0) return -2;
  Server& s = S->s;
  std::lock_guard<std::mutex> lock(s.mu);
  const int64_t v[10] = {s.waves,         s.completed,       (int64_t)s.inflight.size(),
                         (int64_t)s.pending.size(), (int64_t)s.lanes.size(), s.max_busy,
                         s.single_units,  s.batched_units,   s.batched_reqs, s.busy};
  for (int i = 0; i < count && i < 10; ++i) out[i] = v[i];
  return kOk;
}

int cqrrpt_server_destroy(cqrrpt_server S) {
  if (!S) return -1;
  Server& s = S->s;
  {
    std::lock_guard<std::mutex> lock(s.mu);
    s.stop = true;
  }
  s.cv.notify_all();
  if (s.th.joinable()) s.th.join();
  {
    std::lock_guard<std::mutex> lock(s.mu);
    s.stop_workers = true;
  }
  for (Lane* L : s.lanes) {
    L->cv.notify_all();
    if (L->th.joinable()) L->th.join();
  }
  for (Lane* L : s.lanes) {
    cudaStreamSynchronize(L->wave_stream);
    cudaStreamSynchronize(L->single_stream);
  }
  cudaStreamSynchronize(s.copy_in);
  cudaStreamSynchronize(s.copy_out);
  for (auto& kv : s.all) {
    cudaEventDestroy(kv.second->h2d);
    cudaEventDestroy(kv.second->done);
    delete kv.second;
  }
  for (Lane* L : s.lanes) {
    cudaFree(L->fixed);
    if (L->stage) cudaFreeHost(L->stage);
    cudaEventDestroy(L->done);
    cudaEventDestroy(L->stage_ev);
    cudaStreamDestroy(L->wave_stream);
    cudaStreamDestroy(L->single_stream);
    if (L->own_handle) cqrrpt_destroy(L->h);
    delete L;
  }
  cudaFree(s.arena_base);
  cudaFreeHost(s.pinned_slots);
  cudaStreamDestroy(s.copy_in);
  cudaStreamDestroy(s.copy_out);
  delete S;
  return kOk;
}

}  // extern "C"
