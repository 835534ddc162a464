// C-ABI entry points of libpsfsim: argument validation, workspace layout, dispatch.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "psfsim_internal.cuh"
#include "../../include/psfsim_testing.h"

namespace {

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int check_radii(const double *r, int n_r) {
  if (!r) return PSFSIM_ERR_ARG;
  if (n_r < 2 || n_r > PSFSIM_MAX_RADII) return PSFSIM_ERR_RADII;
  for (int i = 0; i < n_r; ++i) {
    if (!std::isfinite(r[i])) return PSFSIM_ERR_RADII;
    if (i > 0 && !(r[i] > r[i - 1])) return PSFSIM_ERR_RADII;
  }
  return PSFSIM_OK;
}

bool storage_ok(int storage) {
  return storage == PSFSIM_FP32 || storage == PSFSIM_SPLIT_BF16 || storage == PSFSIM_BF16 ||
         storage == PSFSIM_FP32_SYM || storage == PSFSIM_FUSED || storage == PSFSIM_SPLIT_BF16_SYM;
}

int common_build(const float *d_lib, const double *h_radii, int n_r, int n, double s, int N, double S,
                 const double *h_xy, int64_t K, int storage, int interp, void *d_ws, size_t ws_bytes,
                 void *stream, psfsim_t *out) {
  if (!out) return PSFSIM_ERR_ARG;
  *out = nullptr;
  if (!d_lib || !d_ws || n < 1 || n > 4096 || K < 1 || K > (int64_t)1 << 30) return PSFSIM_ERR_ARG;
  if (!(s > 0.0) || !std::isfinite(s)) return PSFSIM_ERR_ARG;
  if (!storage_ok(storage) || (interp != PSFSIM_LINEAR && interp != PSFSIM_NEAREST)) return PSFSIM_ERR_ARG;
  if (!aligned(d_lib, 16)) return PSFSIM_ERR_ARG;
  if (int rc = check_radii(h_radii, n_r)) return rc;
  // FUSED and FP32_SYM use the exact quarter-turn symmetry of an even N x N scene grid.
  const bool quadrant =
      storage == PSFSIM_FUSED || storage == PSFSIM_FP32_SYM || storage == PSFSIM_SPLIT_BF16_SYM;
  if (quadrant && (h_xy || N < 2 || (N & 1))) return PSFSIM_ERR_UNSUPPORTED;
  const WsLayout L = psfsim_layout(n, K, storage, n_r);
  if (!aligned(d_ws, 256) || ws_bytes < (size_t)L.total) return PSFSIM_ERR_WORKSPACE;

  psfsim_plan *h = new (std::nothrow) psfsim_plan;
  if (!h) return PSFSIM_ERR_ARG;
  std::memset(h, 0, sizeof(*h));
  h->storage = storage;
  h->interp = interp;
  h->n = n;
  h->n_r = n_r;
  h->M = (int64_t)n * n;
  h->K = K;
  h->ld = L.ld;
  h->N = N;
  h->S = S;
  h->quadrant = quadrant;
  h->Kg = h->quadrant ? K / 4 : K;
  h->d_lib = d_lib;
  for (int i = 0; i < n_r; ++i) h->radii[i] = h_radii[i];
  h->ws = static_cast<char *>(d_ws);
  h->ws_bytes = ws_bytes;
  h->a_off = L.a_off;
  h->lo_off = L.lo_off;
  h->scale_off = L.scale_off;
  h->geom_off = L.geom_off;
  h->order_off = L.order_off;
  h->bstart_off = L.bstart_off;
  h->pts_off = L.pts_off;
  h->status_off = L.status_off;
  h->libmax_off = L.libmax_off;
  h->plib_off = L.plib_off;
  h->cols_off = L.cols_off;
  h->mtorder_off = L.mtorder_off;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = PSFSIM_OK;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    rc = PSFSIM_ERR_CUDA;
  } else if (h_xy) {
    // Synchronous copy of the field points into the workspace.
    if (cudaMemcpyAsync(h->ws + h->pts_off, h_xy, (size_t)K * 16, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = PSFSIM_ERR_CUDA;
  }
  if (rc == PSFSIM_OK && psfsim_launch_build(h, st) != cudaSuccess) rc = PSFSIM_ERR_CUDA;
  if (rc != PSFSIM_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return PSFSIM_OK;
}

}  // namespace

extern "C" {

const char *psfsim_status_string(int status) {
  switch (status) {
    case PSFSIM_OK: return "ok";
    case PSFSIM_ERR_ARG: return "invalid argument";
    case PSFSIM_ERR_RADII: return "radii must be finite and strictly increasing (2..256 of them)";
    case PSFSIM_ERR_WORKSPACE: return "workspace or scratch too small or misaligned";
    case PSFSIM_ERR_CUDA: return "CUDA runtime error";
    case PSFSIM_ERR_UNSUPPORTED: return "unsupported in this build";
    case PSFSIM_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

int psfsim_workspace_bytes(int n, int n_r, int64_t K, int storage, size_t *bytes) {
  if (!bytes || n < 1 || n > 4096 || n_r < 2 || n_r > PSFSIM_MAX_RADII || K < 1 || K > (int64_t)1 << 30 ||
      !storage_ok(storage))
    return PSFSIM_ERR_ARG;
  *bytes = (size_t)psfsim_layout(n, K, storage, n_r).total;
  return PSFSIM_OK;
}

int psfsim_build(const float *d_lib, const double *h_radii, int n_r, int n, double s, int N, double S,
                 int storage, int interp, void *d_workspace, size_t workspace_bytes, void *stream,
                 psfsim_t *out) {
  if (N < 1 || N > 32768 || !(S > 0.0) || !std::isfinite(S)) {
    if (out) *out = nullptr;
    return PSFSIM_ERR_ARG;
  }
  return common_build(d_lib, h_radii, n_r, n, s, N, S, nullptr, (int64_t)N * N, storage, interp, d_workspace,
                      workspace_bytes, stream, out);
}

int psfsim_build_points(const float *d_lib, const double *h_radii, int n_r, int n, double s, const double *h_xy,
                        int64_t K, int storage, int interp, void *d_workspace, size_t workspace_bytes,
                        void *stream, psfsim_t *out) {
  if (!h_xy) {
    if (out) *out = nullptr;
    return PSFSIM_ERR_ARG;
  }
  for (int64_t j = 0; j < 2 * K; ++j)
    if (!std::isfinite(h_xy[j])) {
      if (out) *out = nullptr;
      return PSFSIM_ERR_ARG;
    }
  return common_build(d_lib, h_radii, n_r, n, s, 0, 0.0, h_xy, K, storage, interp, d_workspace, workspace_bytes,
                      stream, out);
}

int psfsim_info(psfsim_t h, psfsim_info_t *info) {
  if (!h || !info) return PSFSIM_ERR_ARG;
  info->storage = h->storage;
  info->interp = h->interp;
  info->n = h->n;
  info->n_r = h->n_r;
  info->M = h->M;
  info->K = h->K;
  info->ld = h->ld;
  info->a_offset = h->a_off;
  info->lo_offset = h->lo_off;
  info->scale_offset = h->scale_off;
  info->workspace_bytes = (int64_t)h->ws_bytes;
  info->K_stored = h->quadrant ? h->K_valid : h->K;
  return PSFSIM_OK;
}

int psfsim_forward_scratch_bytes(psfsim_t h, int B, size_t *bytes) {
  if (!h || !bytes || B < 1) return PSFSIM_ERR_ARG;
  if (h->storage == PSFSIM_FP32) {
    *bytes = psfsim_forward_fp32_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16) {
    *bytes = psfsim_forward_tc_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_FUSED) {
    *bytes = psfsim_forward_fused_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_FP32_SYM) {
    *bytes = psfsim_forward_sym_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_SPLIT_BF16_SYM) {
    *bytes = psfsim_forward_split_sym_scratch(h, B);
    return PSFSIM_OK;
  }
  return PSFSIM_ERR_UNSUPPORTED;
}

int psfsim_adjoint_scratch_bytes(psfsim_t h, int B, size_t *bytes) {
  if (!h || !bytes || B < 1) return PSFSIM_ERR_ARG;
  if (h->storage == PSFSIM_FP32) {
    *bytes = 0;
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16) {
    *bytes = psfsim_adjoint_split_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_FP32_SYM) {
    *bytes = psfsim_adjoint_sym_scratch(h, B);
    return PSFSIM_OK;
  }
  if (h->storage == PSFSIM_SPLIT_BF16_SYM) {
    *bytes = psfsim_adjoint_split_sym_scratch(h, B);
    return PSFSIM_OK;
  }
  return PSFSIM_ERR_UNSUPPORTED;
}

int psfsim_forward(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch, size_t scratch_bytes,
                   void *stream) {
  if (!h || !d_x || !d_y || B < 1) return PSFSIM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->storage == PSFSIM_FP32) {
    const size_t need = psfsim_forward_fp32_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_fp32(h, d_x, B, d_y, d_scratch, st) == cudaSuccess ? PSFSIM_OK
                                                                                    : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16) {
    const size_t need = psfsim_forward_tc_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_tc(h, d_x, B, d_y, d_scratch, st) == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_FP32_SYM) {
    const size_t need = psfsim_forward_sym_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_sym(h, d_x, B, d_y, d_scratch, st) == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_SPLIT_BF16_SYM) {
    const size_t need = psfsim_forward_split_sym_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_split_sym(h, d_x, B, d_y, d_scratch, st) == cudaSuccess ? PSFSIM_OK
                                                                                         : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_FUSED) {
    const size_t need = psfsim_forward_fused_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_fused(h, d_x, B, d_y, d_scratch, st) == cudaSuccess ? PSFSIM_OK
                                                                                     : PSFSIM_ERR_CUDA;
  }
  return PSFSIM_ERR_UNSUPPORTED;
}

int psfsim_forward_sparse_scratch_bytes(psfsim_t h, int B, size_t *bytes) {
  if (!h || !bytes || B < 1) return PSFSIM_ERR_ARG;
  if (h->storage != PSFSIM_FP32) return PSFSIM_ERR_UNSUPPORTED;
  *bytes = psfsim_forward_sparse_scratch(h, B);
  return PSFSIM_OK;
}

int psfsim_forward_sparse(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch, size_t scratch_bytes,
                          void *stream) {
  if (!h || !d_x || !d_y || B < 1) return PSFSIM_ERR_ARG;
  if (h->storage != PSFSIM_FP32) return PSFSIM_ERR_UNSUPPORTED;
  const size_t need = psfsim_forward_sparse_scratch(h, B);
  if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
  return psfsim_launch_forward_sparse(h, d_x, B, d_y, d_scratch, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PSFSIM_OK
             : PSFSIM_ERR_CUDA;
}

int psfsim_adjoint(psfsim_t h, const float *d_g, int B, float *d_gx, void *d_scratch, size_t scratch_bytes,
                   void *stream) {
  if (!h || !d_g || !d_gx || B < 1) return PSFSIM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (h->storage == PSFSIM_FP32)
    return psfsim_launch_adjoint_fp32(h, d_g, B, d_gx, st) == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
  if (h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16) {
    const size_t need = psfsim_adjoint_split_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_adjoint_split(h, d_g, B, d_gx, d_scratch, st) == cudaSuccess ? PSFSIM_OK
                                                                                      : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_FP32_SYM) {
    const size_t need = psfsim_adjoint_sym_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_adjoint_sym(h, d_g, B, d_gx, d_scratch, st) == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
  }
  if (h->storage == PSFSIM_SPLIT_BF16_SYM) {
    const size_t need = psfsim_adjoint_split_sym_scratch(h, B);
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_adjoint_split_sym(h, d_g, B, d_gx, d_scratch, st) == cudaSuccess ? PSFSIM_OK
                                                                                          : PSFSIM_ERR_CUDA;
  }
  return PSFSIM_ERR_UNSUPPORTED;
}

int psfsim_forward_multi_scratch_bytes(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tuning,
                                       size_t *bytes) {
  if (!bytes) return PSFSIM_ERR_ARG;
  if (int rc = psfsim_multi_validate(jobs, njobs)) return rc;
  *bytes = psfsim_forward_multi_scratch(jobs, njobs, tuning);
  return PSFSIM_OK;
}

int psfsim_forward_multi(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tuning, void *d_scratch,
                         size_t scratch_bytes, void *stream) {
  if (int rc = psfsim_multi_validate(jobs, njobs)) return rc;
  if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < psfsim_forward_multi_scratch(jobs, njobs, tuning))
    return PSFSIM_ERR_WORKSPACE;
  return psfsim_launch_forward_multi(jobs, njobs, tuning, d_scratch, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PSFSIM_OK
             : PSFSIM_ERR_CUDA;
}

int psfsim_sync_status(psfsim_t h, void *stream) {
  if (!h) return PSFSIM_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return PSFSIM_ERR_CUDA;
  int status = 0;
  if (cudaMemcpy(&status, h->ws + h->status_off, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PSFSIM_ERR_CUDA;
  return status;
}

int psfsim_reset_status(psfsim_t h, void *stream) {
  if (!h) return PSFSIM_ERR_ARG;
  return cudaMemsetAsync(h->ws + h->status_off, 0, sizeof(int), static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PSFSIM_OK
             : PSFSIM_ERR_CUDA;
}

int psfsim_debug_forward_stall(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch,
                               size_t scratch_bytes, uint64_t wait_ns, int64_t stall_load, void *stream) {
  if (!h || !d_x || !d_y || B < 1 || B > 80) return PSFSIM_ERR_ARG;
  if (wait_ns < 1000 || wait_ns > 2000000000ull || stall_load < -1) return PSFSIM_ERR_ARG;
  if (h->storage == PSFSIM_FUSED) {
    if (B > 64) return PSFSIM_ERR_ARG;
    if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < psfsim_forward_fused_scratch(h, B))
      return PSFSIM_ERR_WORKSPACE;
    return psfsim_launch_forward_fused_stall(h, d_x, B, d_y, d_scratch, wait_ns, stall_load,
                                             static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? PSFSIM_OK
               : PSFSIM_ERR_CUDA;
  }
  if (h->storage != PSFSIM_SPLIT_BF16 && h->storage != PSFSIM_BF16) return PSFSIM_ERR_UNSUPPORTED;
  const size_t need = psfsim_forward_tc_scratch(h, B);
  if (!d_scratch || !aligned(d_scratch, 256) || scratch_bytes < need) return PSFSIM_ERR_WORKSPACE;
  return psfsim_launch_forward_tc_stall(h, d_x, B, d_y, d_scratch, wait_ns, stall_load,
                                        static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PSFSIM_OK
             : PSFSIM_ERR_CUDA;
}

void psfsim_free(psfsim_t h) { delete h; }

}  // extern "C"
