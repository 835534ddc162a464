// Products with a stored FP32 A (column-major, each PSF contiguous):
//   forward  S = A Z   (Eq. 6): row-parallel, split over columns, partials in
//            caller scratch, then a fixed-order reduction (deterministic);
//   adjoint  A^T g:            contiguous column ranges per CTA, rows split
//            across the CTA, fixed-order reduction.
#include "gemv_device.cuh"
#include "psfsim_internal.cuh"

using namespace psfsim_gemv;

namespace {

// part[(ks*B + b)*ld + r] = sum over the ks-th column chunk of A[r, j] x[b, j].
template <int BB>
__global__ void __launch_bounds__(kFwdThreads) fwd_partial_kernel(const float *__restrict__ A, int64_t ld,
                                                                  int64_t K, const float *__restrict__ x,
                                                                  int B, int b0, float *__restrict__ part) {
  const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + 4 * threadIdx.x;
  const int KS = gridDim.y, ks = blockIdx.y;
  if (r >= ld) return;
  float acc[BB][4];
  fwd_accumulate<BB>(A, ld, K, x, b0, r, K * ks / KS, K * (ks + 1) / KS, acc);
#pragma unroll
  for (int b = 0; b < BB; ++b)
    *reinterpret_cast<float4 *>(part + ((int64_t)ks * B + b0 + b) * ld + r) =
        make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
}

// y[b, i] = sum_ks part[ks, b, i] in a fixed order.  A CTA covers 128 rows;
// its 8 warps split the KS partials (ks = warp, warp + 8, ...) and combine
// through shared memory, so every output needs only ~KS/8 loads per thread.
constexpr int kRedRows = 128;
__global__ void __launch_bounds__(256) fwd_reduce_kernel(const float *__restrict__ part, int KS, int B,
                                                         int64_t ld, int64_t M, float *__restrict__ y,
                                                         const int *__restrict__ count) {
  __shared__ float4 red[8][32];
  const int c4 = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t r = ((int64_t)blockIdx.x * 32 + c4) * 4;
  const int b = blockIdx.y;
  if (count && b >= *count) return;  // scene slot not present in this call
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r < ld) {
    const float *p = part + (int64_t)b * ld + r;
    const int64_t step = (int64_t)B * ld;
    int ks = grp;
#pragma unroll 4
    for (; ks < KS; ks += 8) {
      const float4 v = *reinterpret_cast<const float4 *>(p + ks * step);
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
  }
  red[grp][c4] = s;
  __syncthreads();
  if (grp == 0 && r < M) {
    float4 t = red[0][c4];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      const float4 v = red[k][c4];
      t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
    }
    float *out = y + (int64_t)b * M + r;
    out[0] = t.x;
    if (r + 1 < M) out[1] = t.y;
    if (r + 2 < M) out[2] = t.z;
    if (r + 3 < M) out[3] = t.w;
  }
}

// Resident fwd_partial_kernel CTAs per SM (registers decide it), queried once.
int fwd_ctas_per_sm() {
  static const int per_sm = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fwd_partial_kernel<1>, kFwdThreads, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      n = 0;
    }
    return n > 0 ? n : 1;
  }();
  return per_sm;
}

int forward_splits(const psfsim_plan *h) { return psfsim_gemv_splits(h->ld, h->K, h->num_sms); }

// gx[b, j] = sum_i A[i, j] g[b, i]; CTA c owns the contiguous column range
// [K c / G, K (c+1) / G).
template <int BB, bool kVec>
__global__ void __launch_bounds__(kAdjThreads) adj_kernel(const float *__restrict__ A, int64_t ld, int64_t M,
                                                          int64_t K, const float *__restrict__ g, int b0,
                                                          float *__restrict__ gx) {
  adj_columns<BB, kVec>(A, ld, M, K, g, b0, gx, K * blockIdx.x / gridDim.x, K * (blockIdx.x + 1) / gridDim.x);
}

template <int BB>
cudaError_t fwd_group(const psfsim_plan *h, const float *x, int B, int b0, float *part, int KS,
                      cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  dim3 grid((unsigned)((h->ld + kRowsPerCta - 1) / kRowsPerCta), (unsigned)KS);
  fwd_partial_kernel<BB><<<grid, kFwdThreads, 0, st>>>(A, h->ld, h->K, x, B, b0, part);
  return cudaGetLastError();
}

template <int BB>
cudaError_t adj_group(const psfsim_plan *h, const float *g, int b0, float *gx, bool vec, cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  auto kern = vec ? adj_kernel<BB, true> : adj_kernel<BB, false>;
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)h->num_sms * (per_sm < 1 ? 1 : per_sm);
  if (grid > h->K) grid = h->K;
  kern<<<(unsigned)grid, kAdjThreads, 0, st>>>(A, h->ld, h->M, h->K, g, b0, gx);
  return cudaGetLastError();
}

}  // namespace

cudaError_t psfsim_launch_gemv_partials(const float *A, int64_t ld, int64_t K, const float *x, int B, float *part,
                                        int KS, cudaStream_t st) {
  dim3 grid((unsigned)((ld + kRowsPerCta - 1) / kRowsPerCta), (unsigned)KS);
  int b0 = 0;
  while (b0 < B) {
    const int left = B - b0;
    if (left >= 8) { fwd_partial_kernel<8><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 8; }
    else if (left >= 4) { fwd_partial_kernel<4><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 4; }
    else if (left >= 2) { fwd_partial_kernel<2><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 2; }
    else { fwd_partial_kernel<1><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 1; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Column splits: one wave of resident CTAs over the row tiles (at least 8
// columns per split).
int psfsim_gemv_splits(int64_t ld, int64_t K, int num_sms) {
  const int64_t row_blocks = (ld + kRowsPerCta - 1) / kRowsPerCta;
  int64_t ks = (int64_t)num_sms * fwd_ctas_per_sm() / row_blocks;
  ks = ks < 1 ? 1 : ks;
  const int64_t max_ks = K / 8 > 0 ? K / 8 : 1;
  return (int)(ks < max_ks ? ks : max_ks);
}

cudaError_t psfsim_launch_adjoint_cols(const float *A, int64_t ld, int64_t M, int64_t K, const float *g, int B,
                                       float *gx, int num_sms, cudaStream_t st) {
  const bool vec = (M % 4 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
  int b0 = 0;
  while (b0 < B) {
    const int left = B - b0;
    const int bb = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    auto launch = [&](auto kern) -> cudaError_t {
      int per_sm = 1;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, 0);
      if (e != cudaSuccess) return e;
      int64_t grid = (int64_t)num_sms * (per_sm < 1 ? 1 : per_sm);
      if (grid > K) grid = K;
      kern<<<(unsigned)grid, kAdjThreads, 0, st>>>(A, ld, M, K, g, b0, gx);
      return cudaGetLastError();
    };
    cudaError_t e;
    if (bb == 8) e = vec ? launch(adj_kernel<8, true>) : launch(adj_kernel<8, false>);
    else if (bb == 4) e = vec ? launch(adj_kernel<4, true>) : launch(adj_kernel<4, false>);
    else if (bb == 2) e = vec ? launch(adj_kernel<2, true>) : launch(adj_kernel<2, false>);
    else e = vec ? launch(adj_kernel<1, true>) : launch(adj_kernel<1, false>);
    if (e != cudaSuccess) return e;
    b0 += bb;
  }
  return cudaSuccess;
}

size_t psfsim_forward_fp32_scratch(const psfsim_plan *h, int B) {
  return (size_t)forward_splits(h) * (size_t)B * (size_t)h->ld * 4;
}

cudaError_t psfsim_launch_forward_fp32(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                       cudaStream_t st) {
  const int KS = forward_splits(h);
  float *part = reinterpret_cast<float *>(scratch);
  cudaError_t e = cudaSuccess;
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 8) { e = fwd_group<8>(h, x, B, b0, part, KS, st); b0 += 8; }
    else if (left >= 4) { e = fwd_group<4>(h, x, B, b0, part, KS, st); b0 += 4; }
    else if (left >= 2) { e = fwd_group<2>(h, x, B, b0, part, KS, st); b0 += 2; }
    else { e = fwd_group<1>(h, x, B, b0, part, KS, st); b0 += 1; }
  }
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((h->ld + kRedRows - 1) / kRedRows), (unsigned)B);
  fwd_reduce_kernel<<<grid, 256, 0, st>>>(part, KS, B, h->ld, h->M, y, nullptr);
  return cudaGetLastError();
}

cudaError_t psfsim_launch_reduce_partials(const float *part, int KS, int B, int64_t ld, int64_t M, float *y,
                                          const int *count, cudaStream_t st) {
  dim3 grid((unsigned)((ld + kRedRows - 1) / kRedRows), (unsigned)B);
  fwd_reduce_kernel<<<grid, 256, 0, st>>>(part, KS, B, ld, M, y, count);
  return cudaGetLastError();
}

cudaError_t psfsim_launch_adjoint_fp32(const psfsim_plan *h, const float *g, int B, float *gx, cudaStream_t st) {
  const bool vec = (h->M % 4 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
  cudaError_t e = cudaSuccess;
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 8) { e = adj_group<8>(h, g, b0, gx, vec, st); b0 += 8; }
    else if (left >= 4) { e = adj_group<4>(h, g, b0, gx, vec, st); b0 += 4; }
    else if (left >= 2) { e = adj_group<2>(h, g, b0, gx, vec, st); b0 += 2; }
    else { e = adj_group<1>(h, g, b0, gx, vec, st); b0 += 1; }
  }
  return e;
}
