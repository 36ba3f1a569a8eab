// Allocation-free variant of the sketch entry point (the sketch S A).
//
// Some callers cannot allocate device memory at the time they need a
// sketch: code running inside a memory pool that is already sized and
// locked, allocators that forbid cudaMalloc after start-up, or hosts that
// must not create library handles (each handle owns a workspace).  For them
// cqrrpt_sketch_noalloc_d computes exactly what cqrrpt_sketch_d computes,
// with the same kernels, but keeps its scratch (the per-block SASO lists,
// the per-block partial sketches and the status word) in one file-scope
// device array of kNoAllocScratchBytes bytes instead of a handle's
// workspace.  Every GPU that loads the library holds that array until the
// process exits.
//
// Host code may not use the array's name as a device address (in host code
// it names a host-side stand-in); the device address is obtained with
// cudaGetSymbolAddress, with the device current, on the first call made in
// each CUDA context of a device.  The address is cached per device together
// with the context's unique id, so a context that was destroyed and created
// again (cudaDeviceReset) is looked up afresh.  That first call should
// come before any stream capture.  All calls on a device share the one
// array and it keeps the contents of the last call; the status word is
// cleared at the start of every call, the other scratch is fully
// overwritten.  Calls whose executions overlap on the GPU (different
// streams without ordering) race on the array and must not be issued.
#include <cmath>
#include <mutex>

#include <cuda.h>

#include "../../include/cqrrpt.h"
#include "kernels.h"
#include "saso.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr size_t kStatusBytes = 256;                       // status word + padding
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Unique id of the current context (cuCtxGetId through the runtime's driver
// entry point, so the library needs no link against libcuda for it); 0 if
// unavailable, which disables the cache.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)p;
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device (looked up on
// the first call in each context of the device).  Returns nullptr on failure.
void* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long ctx = current_context_id();
  if (g_scratch_ptr[device] && ctx != 0 && ctx == g_scratch_ctx[device])
    return g_scratch_ptr[device];
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_scratch_ptr[device] = p;
  // the lookup has made the runtime create and bind the context if it did
  // not exist yet; a context id of 0 (unknown) keeps the cache off
  g_scratch_ctx[device] = current_context_id();
  return p;
}

}  // namespace

extern "C" {

size_t cqrrpt_sketch_noalloc_max_bytes(void) { return kNoAllocScratchBytes - kStatusBytes; }

int cqrrpt_sketch_noalloc_d(int64_t m, int64_t n, const double* A, int64_t lda, int64_t d,
                            int nnz_per_col, uint64_t seed, double* Ask, int64_t ldsk,
                            cudaStream_t stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (d < 1 || d > 28000) return -5;
  if (nnz_per_col < 1 || nnz_per_col > d || nnz_per_col > cqrrpt::kMaxNnzInline) return -6;
  if (!Ask) return -8;
  if (ldsk < d) return -9;
  const int64_t need = cqrrpt::sketch_workspace_bytes(m, n, (int)d, nnz_per_col);
  if (need > (int64_t)(kNoAllocScratchBytes - kStatusBytes)) return CQRRPT_TOO_LARGE;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return CQRRPT_CUDA_ERROR;
  unsigned char* base = (unsigned char*)scratch_address(device);
  if (!base) return CQRRPT_CUDA_ERROR;
  int* status = (int*)base;
  if (cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess) return CQRRPT_CUDA_ERROR;
  const double scale = 1.0 / std::sqrt((double)nnz_per_col);
  if (cqrrpt::launch_sketch(m, n, A, lda, (int)d, nnz_per_col, seed, scale, Ask, ldsk,
                            base + kStatusBytes, status, stream) != cudaSuccess)
    return CQRRPT_CUDA_ERROR;
  return CQRRPT_OK;
}

int cqrrpt_sketch_noalloc_status(cudaStream_t stream, int* status_host) {
  if (!status_host) return -2;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return CQRRPT_CUDA_ERROR;
  unsigned char* base = (unsigned char*)scratch_address(device);
  if (!base) return CQRRPT_CUDA_ERROR;
  if (cudaMemcpyAsync(status_host, base, sizeof(int), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return CQRRPT_CUDA_ERROR;
  }
  return CQRRPT_OK;
}

}  // extern "C"
