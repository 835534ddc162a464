// psfsim_forward_static: the FP32 forward product with its partial sums kept
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory when they simulate an image and have no spare buffer
// to pass as scratch.  The paper has no counterpart.
//
// The array is a file-scope __device__ variable.  It is reserved on a device
// when the library's device code is loaded there (with CUDA's default lazy
// module loading: at the first psfsim_forward_static call on that device) and
// stays reserved until the process exits.  In host code its name is only a
// host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress, with the device current.  The lookup is cached per
// CUDA context, keyed on the context's process-unique ID, so that a device
// reset (a new primary context, the module loaded afresh) makes the next call
// look the address up again instead of using a stale one.
#include <cudaTypedefs.h>

#include <mutex>

#include "psfsim_internal.cuh"

namespace {

constexpr size_t kStaticFloats = PSFSIM_STATIC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_forward_scratch[kStaticFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct CachedAddress {
  unsigned long long ctx_id;
  void *ptr;
};
CachedAddress g_cache[kMaxDevices] = {};

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

bool driver_entry(const char *name, int version, void **fn) {
  cudaDriverEntryPointQueryResult q;
  *fn = nullptr;
  return cudaGetDriverEntryPointByVersion(name, fn, version, cudaEnableDefault, &q) == cudaSuccess &&
         q == cudaDriverEntryPointSuccess && *fn;
}

// ID of the context current on this thread (the device's primary context once
// cudaSetDevice has run); 0 when it cannot be determined.
unsigned long long current_context_id() {
  if (!g_ctx_current || !g_ctx_id) {
    void *a = nullptr, *b = nullptr;
    if (!driver_entry("cuCtxGetCurrent", 4000, &a) || !driver_entry("cuCtxGetId", 12000, &b)) return 0;
    g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(a);
    g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(b);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_forward_scratch on `device` (which must be current).
int scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return PSFSIM_ERR_UNSUPPORTED;
  // Makes the device's primary context current on this thread (it exists: the
  // plan was built on this device); allocates nothing.
  if (cudaSetDevice(device) != cudaSuccess) return PSFSIM_ERR_CUDA;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  CachedAddress &c = g_cache[device];
  if (!c.ptr || id == 0 || c.ctx_id != id) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_forward_scratch) != cudaSuccess || !ptr) return PSFSIM_ERR_CUDA;
    c.ptr = ptr;
    c.ctx_id = id;
  }
  *out = c.ptr;
  return PSFSIM_OK;
}

}  // namespace

extern "C" int psfsim_forward_static(psfsim_t h, const float *d_x, int B, float *d_y, void *stream) {
  if (!h || !d_x || !d_y || B < 1) return PSFSIM_ERR_ARG;
  if (h->storage != PSFSIM_FP32) return PSFSIM_ERR_UNSUPPORTED;
  if (psfsim_forward_fp32_scratch(h, B) > PSFSIM_STATIC_SCRATCH_BYTES) return PSFSIM_ERR_WORKSPACE;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return PSFSIM_ERR_CUDA;
  if (device != h->device) return PSFSIM_ERR_ARG;
  void *scratch = nullptr;
  if (int rc = scratch_address(device, &scratch)) return rc;
  // Every launch overwrites all the partial sums it later reads, so the
  // previous call's contents never need clearing.
  return psfsim_launch_forward_fp32(h, d_x, B, d_y, scratch, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PSFSIM_OK
             : PSFSIM_ERR_CUDA;
}
