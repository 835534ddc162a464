// psfsim_forward_static: the FP32 forward product with its partial sums kept
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory when they simulate an image and have no spare buffer
// to pass as scratch.  The paper has no counterpart.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds PSFSIM_STATIC_SCRATCH_BYTES of it until the process exits.  In
// host code its name is only a host-side stand-in, so the device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on it.
#include <mutex>

#include "psfsim_internal.cuh"

namespace {

constexpr size_t kStaticFloats = PSFSIM_STATIC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_forward_scratch[kStaticFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_forward_scratch on `device` (which must be current).
int scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return PSFSIM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_forward_scratch) != cudaSuccess || !ptr) return PSFSIM_ERR_CUDA;
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
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
