// Fit operators (include/psfsim_fit.h): ring scene model, its parameter
// chain rule, and the image-space loss with its residual.  Per-pixel model
// arithmetic is float32; reductions are float64 over a fixed grid and a fixed
// tree, so results are deterministic.
#include <cmath>

#include "../../include/psfsim_fit.h"
#include "psfsim_internal.cuh"
#include "ring_model.cuh"

namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

__global__ void ring_scene_kernel(const RingParams P, float *z) {
  const int64_t K = (int64_t)P.N * P.N;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x)
    z[j] = ring_eval<false>(P, j, nullptr);
}

// Fixed-tree block reduction of NV doubles; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
  __shared__ double red[kRedThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NV; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < NV; ++m) red[warp][m] = v[m];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      double t = red[0][m];
      for (int w = 1; w < kRedThreads / 32; ++w) t += red[w][m];
      v[m] = t;
    }
}

__global__ void __launch_bounds__(kRedThreads) ring_chain_partial(const RingParams P, const float *gz, double *part) {
  const int64_t K = (int64_t)P.N * P.N;
  double acc[5] = {0, 0, 0, 0, 0};
  float J[5];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < K; j += (int64_t)gridDim.x * blockDim.x) {
    ring_eval<true>(P, j, J);
    const double gj = (double)gz[j];
#pragma unroll
    for (int m = 0; m < 5; ++m) acc[m] += gj * (double)J[m];
  }
  block_reduce<5>(acc);
  if (threadIdx.x == 0)
    for (int m = 0; m < 5; ++m) part[blockIdx.x * 5 + m] = acc[m];
}

template <int NV>
__global__ void __launch_bounds__(kRedThreads) finish_sum(const double *part, int nblocks, double scale, double *out) {
  double acc[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) acc[m] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int m = 0; m < NV; ++m) acc[m] += part[b * NV + m];
  block_reduce<NV>(acc);
  if (threadIdx.x == 0)
    for (int m = 0; m < NV; ++m) out[m] = scale * acc[m];
}

__global__ void __launch_bounds__(kRedThreads) loss_partial(const float *y, const float *d, int64_t M, double sigma,
                                                           float inv_s2, float *r, double *part) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const float diff = y[i] - d[i];
    if (r) r[i] = diff * inv_s2;
    const double t = (double)diff / sigma;
    acc[0] += t * t;
  }
  block_reduce<1>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

}  // namespace

extern "C" {

int psfsim_ring_chain_scratch_bytes(int N, size_t *bytes) {
  if (!bytes || N < 1) return PSFSIM_ERR_ARG;
  *bytes = (size_t)kRedBlocks * 5 * sizeof(double);
  return PSFSIM_OK;
}

int psfsim_loss_scratch_bytes(int64_t M, size_t *bytes) {
  if (!bytes || M < 1) return PSFSIM_ERR_ARG;
  *bytes = (size_t)kRedBlocks * sizeof(double);
  return PSFSIM_OK;
}

int psfsim_ring_scene(int N, double S, double r_max, const double *h_theta, float *d_z, void *stream) {
  RingParams P;
  if (!d_z || !ring_params(N, S, r_max, h_theta, &P)) return PSFSIM_ERR_ARG;
  const int64_t K = (int64_t)N * N;
  const unsigned grid = (unsigned)((K + 255) / 256 < 4096 ? (K + 255) / 256 : 4096);
  ring_scene_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(P, d_z);
  return cudaGetLastError() == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
}

int psfsim_ring_chain(int N, double S, double r_max, const double *h_theta, const float *d_gz, double *d_dtheta,
                      void *d_scratch, size_t scratch_bytes, void *stream) {
  RingParams P;
  if (!d_gz || !d_dtheta || !ring_params(N, S, r_max, h_theta, &P)) return PSFSIM_ERR_ARG;
  if (!d_scratch || !aligned256(d_scratch) || scratch_bytes < (size_t)kRedBlocks * 5 * sizeof(double))
    return PSFSIM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *part = static_cast<double *>(d_scratch);
  ring_chain_partial<<<kRedBlocks, kRedThreads, 0, st>>>(P, d_gz, part);
  finish_sum<5><<<1, kRedThreads, 0, st>>>(part, kRedBlocks, 1.0, d_dtheta);
  return cudaGetLastError() == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
}

int psfsim_residual_loss(const float *d_y, const float *d_d, int64_t M, double sigma, float *d_r, double *d_loss,
                         void *d_scratch, size_t scratch_bytes, void *stream) {
  if (!d_y || !d_d || !d_loss || M < 1 || !(sigma > 0.0) || !std::isfinite(sigma)) return PSFSIM_ERR_ARG;
  if (!d_scratch || !aligned256(d_scratch) || scratch_bytes < (size_t)kRedBlocks * sizeof(double))
    return PSFSIM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *part = static_cast<double *>(d_scratch);
  loss_partial<<<kRedBlocks, kRedThreads, 0, st>>>(d_y, d_d, M, sigma, (float)(1.0 / (sigma * sigma)), d_r, part);
  finish_sum<1><<<1, kRedThreads, 0, st>>>(part, kRedBlocks, 0.5, d_loss);
  return cudaGetLastError() == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
}

}  // extern "C"
