// Internal declarations shared by the psfsim CUDA translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/psfsim.h"

#define PSFSIM_MAX_RADII 256
#define PSFSIM_FRAC_BITS 40  // fixed-point fraction bits of the rotation coordinates
#define PSFSIM_THETA_BINS 16 // angle bins per radial bracket when ordering columns
// Column-ordering buckets: (bracket, angle bin) for valid columns, one more for zero columns.
static inline __host__ __device__ int psfsim_num_buckets(int n_r) { return (n_r - 1) * PSFSIM_THETA_BINS + 1; }

// Per-column geometry, computed once per build on the device (FP64, Sec. 2):
// radial bracket k (-1: beyond the last radius, zero column), the two lerp
// weights, and cos/sin of the polar angle as fixed-point integers
// round(v * 2^PSFSIM_FRAC_BITS).  Exact integer arithmetic on these makes
// theta = 0 the identity and quarter turns exact permutations.
struct ColGeom {
  int k;
  int bin;        // polar-angle bin (0..PSFSIM_THETA_BINS-1), for column ordering only
  float w0, w1;  // weights of L[k] and L[k+1]
  long long C, Sn;
};
static_assert(sizeof(ColGeom) == 32, "ColGeom layout");

struct psfsim_plan {
  int storage, interp, n, n_r;
  int64_t M, K, ld;
  int N;          // scene side for grid builds, 0 for point builds
  bool quadrant;  // FUSED: columns are the x > 0, y > 0 quadrant of the N x N grid
  int64_t Kg;     // columns with geometry tables (K, or K/4 for the quadrant)
  int64_t K_valid;  // FUSED: columns inside the last radius (host copy, read back at build)
  double S;
  const float *d_lib;
  double radii[PSFSIM_MAX_RADII];
  char *ws;
  size_t ws_bytes;
  int64_t a_off, lo_off, scale_off, geom_off, order_off, bstart_off, pts_off, status_off, libmax_off, plib_off,
      cols_off, mtorder_off;
  int device, num_sms;
  int fit_ks;           // column splits of the fit-gradient forward, fixed at first use (0: not yet)
  CUtensorMap lib_map;  // 3D tensor map over the library for TMA staging
};

// Workspace layout for a given shape; returns total bytes.
struct WsLayout {
  int64_t ld, a_off, lo_off, scale_off, geom_off, order_off, bstart_off, pts_off, status_off, libmax_off, plib_off,
      cols_off, mtorder_off, total;
};
WsLayout psfsim_layout(int n, int64_t K, int storage, int n_r);
// FUSED storage's copy of the library: one 32-byte pair entry per bracket
// pair and padded pixel, plus a zero entry; psfsim_launch_pair_library also
// writes the column table (fused.cu).
int64_t psfsim_pair_library_bytes(int n, int n_r);
// ... and its column table: the generators' (angle-sorted) columns, with
// their starting coordinates, steps and weights, padded to whole k-tiles.
int64_t psfsim_fused_columns_bytes(int64_t K);
// ... and its M-tile order (the image's 8 x 16 pixel tiles, nearest the centre first).
int64_t psfsim_fused_mtile_order_bytes(int n);
cudaError_t psfsim_launch_pair_library(psfsim_plan *h, cudaStream_t st);

// Kernel launchers (return cudaError_t of the launch).
cudaError_t psfsim_launch_build(psfsim_plan *h, cudaStream_t st);
cudaError_t psfsim_launch_forward_fp32(const psfsim_plan *h, const float *x, int B, float *y,
                                       void *scratch, cudaStream_t st);
size_t psfsim_forward_fp32_scratch(const psfsim_plan *h, int B);
// FP32 forward over the scene pixels that are non-zero in some scene of the batch.
size_t psfsim_forward_sparse_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_forward_sparse(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                         cudaStream_t st);
cudaError_t psfsim_launch_adjoint_fp32(const psfsim_plan *h, const float *g, int B, float *gx,
                                       cudaStream_t st);
// y[b, i] = sum_ks part[(ks * B + b) * ld + i], fixed order.
// Slots b >= *count (when count is not NULL) are skipped.
cudaError_t psfsim_launch_reduce_partials(const float *part, int KS, int B, int64_t ld, int64_t M, float *y,
                                          const int *count, cudaStream_t st);
// Split-BF16 storage: build, tensor-core forward, CUDA-core adjoint.
cudaError_t psfsim_launch_split_build(psfsim_plan *h, cudaStream_t st);
size_t psfsim_forward_tc_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_forward_tc(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                     cudaStream_t st);
size_t psfsim_adjoint_split_scratch(const psfsim_plan *h, int B);
// Test hook: the tensor-core forward of <= 80 scenes on one CTA with every
// wait bounded by wait_ns and load number stall_it never issued.
cudaError_t psfsim_launch_forward_tc_stall(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                           uint64_t wait_ns, int64_t stall_it, cudaStream_t st);
// Multi-job persistent tensor-core forward (several split-BF16 plans, one launch).
int psfsim_multi_validate(const psfsim_job_t *jobs, int njobs);
size_t psfsim_forward_multi_scratch(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tune);
cudaError_t psfsim_launch_forward_multi(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tune,
                                        void *scratch, cudaStream_t st);
// Generic FP32 GEMV pieces (column-major A) used by several storages.
int psfsim_gemv_splits(int64_t ld, int64_t K, int num_sms);
cudaError_t psfsim_launch_gemv_partials(const float *A, int64_t ld, int64_t K, const float *x, int B, float *part,
                                        int KS, cudaStream_t st);
cudaError_t psfsim_launch_adjoint_cols(const float *A, int64_t ld, int64_t M, int64_t K, const float *g, int B,
                                       float *gx, int num_sms, cudaStream_t st);
// FP32 storage compacted by the quarter-turn symmetry and zero columns.
size_t psfsim_forward_sym_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_forward_sym(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                      cudaStream_t st);
size_t psfsim_adjoint_sym_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_adjoint_sym(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                      cudaStream_t st);
// Fused (A regenerated on chip) forward.
size_t psfsim_forward_fused_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_forward_fused(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                        cudaStream_t st);
// Test hook: the fused forward of <= 32 scenes on one CTA with every wait
// bounded by wait_ns and the x load of k-tile number stall_load never issued.
cudaError_t psfsim_launch_forward_fused_stall(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                              uint64_t wait_ns, int64_t stall_load, cudaStream_t st);
cudaError_t psfsim_launch_adjoint_split(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                        cudaStream_t st);

static inline int64_t psfsim_round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Columns stored in A: the quadrant's valid columns for the compacted storages.
static inline int64_t psfsim_cols(const psfsim_plan *h) { return h->quadrant ? h->K_valid : h->K; }

// Split-BF16 storage compacted by the quarter-turn symmetry (sym.cu).
size_t psfsim_forward_split_sym_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_forward_split_sym(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                            cudaStream_t st);
size_t psfsim_adjoint_split_sym_scratch(const psfsim_plan *h, int B);
cudaError_t psfsim_launch_adjoint_split_sym(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                            cudaStream_t st);

// Launch configuration with programmatic stream serialization: the kernel may
// be scheduled while the previous kernel in the stream finishes; it calls
// griddep_wait before touching that kernel's results.
inline cudaLaunchConfig_t psfsim_pdl_config(dim3 grid, int threads, cudaStream_t st, cudaLaunchAttribute (&attr)[1]) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Fit gradient on FP32_SYM storage (the compact quadrant matrix), three
// launches; the C-ABI calls in fit_gradient.cu dispatch here.
struct RingParams;
size_t psfsim_sym_gradient_scratch(psfsim_plan *h);
cudaError_t psfsim_sym_forward_loss(psfsim_plan *h, const RingParams &P, const float *d, double sigma, float *z,
                                    float *y, float *r, void *scratch, cudaStream_t st);
cudaError_t psfsim_sym_adjoint_chain(psfsim_plan *h, const float *r, float *gz, double *out, void *scratch,
                                     cudaStream_t st);
