// Continuous-batching CQRRPT server.
//
// Requests (a host matrix plus host output buffers) are submitted from any
// thread and return a ticket at once.  One scheduler thread per server:
//   * admits queued requests in arrival order while their device footprint
//     (A, Q, R, J, per-problem workspace) fits the HBM budget -- a first-fit
//     arena over one allocation made at creation -- and at most max_inflight
//     are in flight; the host -> device copy of an admitted request's A is
//     issued at once on a copy stream, overlapping the running wave;
//   * whenever no wave is running, starts the next unit of work, chosen by
//     the oldest request whose input has arrived: one batched pass over
//     every arrived request of its kind (FP64 waves run the batched kernels
//     of batched.cu, split-BF16 waves the batched split path) -- requests
//     that arrived while the previous wave ran join the next one -- or, for
//     a request routed to the single-problem path (n above kBatchMaxN, where
//     the one-CTA-per-problem QRCP and Cholesky of the batched kernels would
//     serialise, or the mode with a second Cholesky-QR pass), that request
//     alone on the whole GPU;
//   * when a wave completes, copies each result (Q, R, J, k, status) back on
//     the copy stream, frees the request's arena block when the copy is done
//     and records the completion time.
// Every wait of the scheduler is a host-side poll with a bounded sleep; the
// kernels contain no cross-CTA waits.  Results are bit-identical to a
// standalone call on the same request, whatever else shares a wave.
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

struct Server {
  cqrrpt_handle h = nullptr;
  int device = 0;
  double gamma = 1.25;
  int nnz = 4;
  int max_inflight = 64;
  char* arena_base = nullptr;
  Arena arena;
  char* fixed = nullptr;  // DeviceScalars[max_inflight] + tables
  size_t fixed_bytes = 0;
  void* stage = nullptr;  // pinned table staging
  size_t stage_bytes = 0;
  int64_t* pinned_slots = nullptr;  // 2 words per in-flight slot
  std::vector<int> free_slots;
  cudaStream_t compute = nullptr, copy = nullptr;
  cudaEvent_t wave_done = nullptr, stage_ev = nullptr;
  bool wave_running = false;
  std::vector<Req*> wave;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Req*> inflight;
  std::unordered_map<uint64_t, Req*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  int error = 0;
  int64_t waves = 0, completed = 0;
  int (*run_single)(cqrrpt_handle, const cqrrpt_request&, double, int, double*, double*, double*,
                    int64_t*, cudaStream_t) = nullptr;

  void loop();
  bool step();
};

bool Server::step() {
  bool progress = false;
  std::vector<Req*> finished;
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
  }
  if (progress) cv.notify_all();
  // wave completion: copy results back
  if (wave_running && cudaEventQuery(wave_done) == cudaSuccess) {
    std::lock_guard<std::mutex> lock(mu);
    cudaStreamWaitEvent(copy, wave_done, 0);
    for (Req* q : wave) {
      const cqrrpt_request& r = q->r;
      cudaMemcpy2DAsync(r.Q_host, r.ldq * sizeof(double), q->Q, r.m * sizeof(double),
                        r.m * sizeof(double), r.n, cudaMemcpyDeviceToHost, copy);
      cudaMemcpy2DAsync(r.R_host, r.ldr * sizeof(double), q->R, r.n * sizeof(double),
                        r.n * sizeof(double), r.n, cudaMemcpyDeviceToHost, copy);
      cudaMemcpyAsync(r.J_host, q->J, r.n * sizeof(int64_t), cudaMemcpyDeviceToHost, copy);
      cudaMemcpyAsync(q->k_host, q->k_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, copy);
      cudaMemcpyAsync(q->st_host, q->st_dev, sizeof(int), cudaMemcpyDeviceToHost, copy);
      cudaEventRecord(q->done, copy);
      q->state = kCopyBack;
    }
    wave.clear();
    wave_running = false;
    progress = true;
  }
  // admission
  {
    std::lock_guard<std::mutex> lock(mu);
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
                        r.m * sizeof(double), r.n, cudaMemcpyHostToDevice, copy);
      cudaEventRecord(q->h2d, copy);
      q->state = kStaging;
      q->t_start = now_us();
      inflight.push_back(q);
      progress = true;
    }
  }
  // launch the next unit of work: the oldest arrived request decides
  // between a batched wave and a single-path run
  if (!wave_running) {
    // arrived requests: single route, or one of the two batched routes
    // (FP64 waves and split-BF16 waves); the oldest decides what runs
    std::vector<Req*> ready;
    Req* solo = nullptr;
    Req* oldest = nullptr;
    {
      std::lock_guard<std::mutex> lock(mu);
      for (Req* q : inflight) {
        if (q->state != kStaging || cudaEventQuery(q->h2d) != cudaSuccess) continue;
        if (!oldest || q->t_submit < oldest->t_submit) oldest = q;
        if (single_route(q->r) && (!solo || q->t_submit < solo->t_submit)) solo = q;
      }
      if (oldest && !single_route(oldest->r))
        for (Req* q : inflight)
          if (q->state == kStaging && !single_route(q->r) &&
              q->r.precision == oldest->r.precision && cudaEventQuery(q->h2d) == cudaSuccess)
            ready.push_back(q);
    }
    const bool split_wave = !ready.empty() && oldest->r.precision != CQRRPT_FP64;
    if (!ready.empty()) {
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
      P.scalars = (DeviceScalars*)fixed;
      P.tables = fixed + align256((int64_t)max_inflight * sizeof(DeviceScalars));
      batch_plan(P, (int)ready.size(), probs.data(), nullptr, wss.data(), handle_tuning(h));
      const size_t img = P.image.size();
      cudaEventSynchronize(stage_ev);
      if (img > stage_bytes) {
        if (stage) cudaFreeHost(stage);
        stage = nullptr;
        stage_bytes = 0;
        if (cudaMallocHost(&stage, img) != cudaSuccess) { error = kNoMemory; return false; }
        stage_bytes = img;
      }
      memcpy(stage, P.image.data(), img);
      cudaMemcpyAsync(P.tables, stage, img, cudaMemcpyHostToDevice, compute);
      cudaEventRecord(stage_ev, compute);
      {
        std::lock_guard<std::mutex> lock(mu);
        for (Req* q : ready) q->state = kRunning;
        wave = ready;
      }
      if (split_wave) {
        // the split products are sized by each problem's k: this waits for
        // the compute stream twice
        if (batched_split_exec(h, P, probs, compute) != kOk) { error = kCudaError; return false; }
      } else {
        sketch_set_attributes(P.max_d);
        if (batch_launch(P, compute) != cudaSuccess) { error = kCudaError; return false; }
      }
      cudaEventRecord(wave_done, compute);
      wave_running = true;
      ++waves;
      progress = true;
    } else if (solo) {
      Req* q = solo;
      {
        std::lock_guard<std::mutex> lock(mu);
        q->state = kRunning;
        wave.assign(1, q);
      }
      // FP64 requests are enqueued without a host wait; the split-BF16
      // pipeline reads k back on the way (its recursive products are sized
      // on the host).  k and status land in the request's device slots.
      const int rc = run_single(h, q->r, gamma, nnz, q->A, q->Q, q->R, q->J, compute);
      if (rc != kOk && rc != kRankZero && rc != kNonFinite) {
        *q->k_host = 0;
        *q->st_host = rc;
        cudaMemcpyAsync(q->k_dev, q->k_host, sizeof(int64_t), cudaMemcpyHostToDevice, compute);
        cudaMemcpyAsync(q->st_dev, q->st_host, sizeof(int), cudaMemcpyHostToDevice, compute);
      } else if (handle_finalize(h, q->k_dev, q->st_dev, compute) != kOk) {
        error = kCudaError;
        return false;
      }
      cudaEventRecord(wave_done, compute);
      wave_running = true;
      ++waves;
      progress = true;
    }
  }
  return progress;
}

void Server::loop() {
  cudaSetDevice(device);
  while (true) {
    {
      std::lock_guard<std::mutex> lock(mu);
      if (stop && pending.empty() && inflight.empty() && !wave_running) break;
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

int cqrrpt_server_create(cqrrpt_handle h, size_t hbm_budget_bytes, int max_inflight, double gamma,
                         int nnz_per_col, cqrrpt_server* out) {
  if (!h) return -1;
  if (hbm_budget_bytes < (1u << 20)) return -2;
  if (max_inflight < 1 || max_inflight > 4096) return -3;
  if (!(gamma >= 1.0) || !std::isfinite(gamma)) return -4;
  if (nnz_per_col < 1 || nnz_per_col > kMaxNnzInline) return -5;
  if (!out) return -6;
  *out = nullptr;
  cqrrpt_server_s* S = new cqrrpt_server_s();
  Server& s = S->s;
  s.h = h;
  s.gamma = gamma;
  s.nnz = nnz_per_col;
  s.max_inflight = max_inflight;
  s.run_single = run_single_impl;
  if (cudaGetDevice(&s.device) != cudaSuccess) { delete S; return kCudaError; }
  s.fixed_bytes = (size_t)(align256((int64_t)max_inflight * sizeof(DeviceScalars)) +
                           batch_table_bytes(max_inflight));
  if (cudaMalloc((void**)&s.arena_base, hbm_budget_bytes) != cudaSuccess ||
      cudaMalloc((void**)&s.fixed, s.fixed_bytes) != cudaSuccess ||
      cudaMallocHost((void**)&s.pinned_slots, (size_t)max_inflight * 16) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s.compute, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s.copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s.wave_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s.stage_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (s.arena_base) cudaFree(s.arena_base);
    if (s.fixed) cudaFree(s.fixed);
    delete S;
    return kNoMemory;
  }
  s.arena.init(hbm_budget_bytes);
  for (int i = max_inflight - 1; i >= 0; --i) s.free_slots.push_back(i);
  s.th = std::thread([S] { S->s.loop(); });
  *out = S;
  return kOk;
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

int cqrrpt_server_destroy(cqrrpt_server S) {
  if (!S) return -1;
  Server& s = S->s;
  {
    std::lock_guard<std::mutex> lock(s.mu);
    s.stop = true;
  }
  s.cv.notify_all();
  if (s.th.joinable()) s.th.join();
  cudaStreamSynchronize(s.compute);
  cudaStreamSynchronize(s.copy);
  for (auto& kv : s.all) {
    cudaEventDestroy(kv.second->h2d);
    cudaEventDestroy(kv.second->done);
    delete kv.second;
  }
  cudaFree(s.arena_base);
  cudaFree(s.fixed);
  cudaFreeHost(s.pinned_slots);
  if (s.stage) cudaFreeHost(s.stage);
  cudaEventDestroy(s.wave_done);
  cudaEventDestroy(s.stage_ev);
  cudaStreamDestroy(s.compute);
  cudaStreamDestroy(s.copy);
  delete S;
  return kOk;
}

}  // extern "C"
