// ap_noalloc.cu -- batched gather + push whose scratch lives in a static
// device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they push
// particles: a host application whose framework allocator has already
// reserved all of the GPU's memory, or a time-stepping loop that must not
// make calls that can synchronise the device or fail for lack of memory in
// the middle of a step.  ap_gather_push_batched asks such callers for a
// workspace; this entry point instead keeps that scratch (the tile-queue
// counter of the persistent launch) in a file-scope __device__ array that
// every GPU loading the library holds until the process exits.
#include <cuda.h>  // driver types only: the two driver calls are resolved at run time
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ap_internal.h"

// Scratch of the batched persistent launch, AP_STATIC_SCRATCH_BYTES bytes.
// In host code `g_batch_scratch` is only a stand-in for the symbol; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_batch_scratch[AP_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_context_id[kMaxDevices] = {0};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Process-unique id of the calling thread's current CUDA context, 0 when it
// cannot be read.  The driver functions are resolved through the runtime,
// so the library does not link the driver library.  Called under g_mutex.
unsigned long long current_context_id() {
  static bool resolved = false;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!resolved) {
    resolved = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

// Device address of the scratch array on the current device.  It is looked
// up once per device with that device current, and again whenever the
// device's context is not the one the cached address belongs to (a context
// re-created after cudaDeviceReset loads the module afresh, at a new
// address); where the context cannot be identified it is looked up on every
// call.
int scratch_for_current_device(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_context_id[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_batch_scratch) != cudaSuccess || !p) return AP_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    g_context_id[dev] = current_context_id();  // current now, if it was not before the lookup
  }
  *out = g_scratch_ptr[dev];
  return AP_OK;
}

}  // namespace

extern "C" int ap_gather_push_batched_static(ap_handle h, const ap_particles *p, const ap_grid *g,
                                             double t0, double dt, int64_t n_steps,
                                             int32_t precision, const ap_diag *diag,
                                             void *stream) {
  if (!h) return AP_ERR_ARG;
  const size_t need = ap_batch_workspace_bytes(h);
  if (need > (size_t)AP_STATIC_SCRATCH_BYTES) return AP_ERR_WORKSPACE;
  void *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != AP_OK) return rc;
  // The batched call zeroes the counter it uses on `stream` before its launch.
  return ap_gather_push_batched(h, p, g, t0, dt, n_steps, precision, diag, scratch,
                                (size_t)AP_STATIC_SCRATCH_BYTES, stream);
}
