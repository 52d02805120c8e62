// voila_belief_update_noalloc: the SIR belief update for callers that cannot
// allocate device memory. Its scratch is one fixed array compiled into the
// library instead of a caller workspace.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/voila.h"

namespace {

// The scratch every call of voila_belief_update_noalloc uses. It lives in the
// library's device image, so each GPU that loads the library holds these
// bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[VOILA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // the context the address above belongs to

// The CUDA driver API's cuCtxGetCurrent through the runtime's entry-point query (the
// library does not link libcuda itself).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  return fn;
}

// Device address of g_noalloc_scratch on the current device. On the host the
// symbol is only a stand-in for the device array, so the address must come
// from the runtime: looked up once per device, with that device current, and
// again if the device's context has changed since (after cudaDeviceReset the
// library's device image is loaded anew and the array may have moved).
voila_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VOILA_ERR_CUDA;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return VOILA_ERR_CUDA;
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return VOILA_ERR_CUDA;  // NULL before this thread's first runtime work
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!ctx || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
    // the lookup also makes the device's context current in this thread
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VOILA_ERR_CUDA;
    if (get(&ctx) != CUDA_SUCCESS || !ctx) return VOILA_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return VOILA_OK;
}

}  // namespace

extern "C" voila_status voila_belief_update_noalloc(
    const voila_mlp* g_T, const voila_likelihood* ell, const float* particles_in,
    const double* logw_in, int32_t N, int32_t d_s, const float* action, const float* obs,
    int32_t d_a, int32_t d_o, int32_t d_omega, float lambda, uint64_t seed, uint32_t step,
    uint32_t planner_id, float* particles_out, int32_t* idx_out, double* w_out, double* logZ_out,
    double* ess_out, int32_t* status_out, voila_stream_t stream) {
  size_t need = 0;
  voila_status st = voila_belief_update_workspace_size(g_T, ell, N, &need);
  if (st != VOILA_OK) return st;
  if (need > (size_t)VOILA_NOALLOC_SCRATCH_BYTES) return VOILA_ERR_WORKSPACE;
  void* ws = nullptr;
  st = scratch_for_current_device(&ws);
  if (st != VOILA_OK) return st;
  // The update clears the status word at the start of the array itself and
  // writes every other scratch byte it reads, so stale contents from the
  // previous call do not matter.
  st = voila_belief_update(g_T, ell, particles_in, logw_in, N, d_s, action, obs, d_a, d_o, d_omega,
                           lambda, seed, step, planner_id, particles_out, idx_out, w_out, logZ_out,
                           ess_out, ws, (size_t)VOILA_NOALLOC_SCRATCH_BYTES, stream);
  if (st != VOILA_OK || !status_out) return st;
  if (N == 0)
    return cudaMemsetAsync(status_out, 0, sizeof(int32_t), (cudaStream_t)stream) == cudaSuccess
               ? VOILA_OK
               : VOILA_ERR_CUDA;
  // The device-side status word (first 4 bytes of the scratch) for the caller.
  if (cudaMemcpyAsync(status_out, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return VOILA_ERR_CUDA;
  return VOILA_OK;
}
