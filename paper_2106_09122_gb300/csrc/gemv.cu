// Products with a stored FP32 A (column-major, each PSF contiguous):
//   forward  S = A Z   (Eq. 6): row-parallel, split over columns, partials in
//            caller scratch, then a fixed-order reduction (deterministic);
//   adjoint  A^T g:            contiguous column ranges per CTA, rows split
//            across the CTA, fixed-order reduction.
// Both stream A once from HBM with 128-bit loads that bypass L1.
#include "psfsim_internal.cuh"

namespace {

__device__ __forceinline__ float4 ld_stream4(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

constexpr int kFwdThreads = 256;
constexpr int kRowsPerCta = kFwdThreads * 4;

// part[(ks*B + b)*ld + r] = sum over the ks-th column chunk of A[r, j] x[b, j].
template <int BB>
__global__ void __launch_bounds__(kFwdThreads) fwd_partial_kernel(const float *__restrict__ A, int64_t ld,
                                                                  int64_t K, const float *__restrict__ x,
                                                                  int B, int b0, float *__restrict__ part) {
  const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + 4 * threadIdx.x;
  const int KS = gridDim.y, ks = blockIdx.y;
  const int64_t j0 = K * ks / KS, j1 = K * (ks + 1) / KS;
  if (r >= ld) return;
  float acc[BB][4];
#pragma unroll
  for (int b = 0; b < BB; ++b) acc[b][0] = acc[b][1] = acc[b][2] = acc[b][3] = 0.f;
  const float *a = A + j0 * ld + r;
  const float *xb = x + (int64_t)b0 * K;
  int64_t j = j0;
  for (; j + 4 <= j1; j += 4, a += 4 * ld) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ld_stream4(a + u * ld);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int b = 0; b < BB; ++b) {
        const float xv = __ldg(xb + (int64_t)b * K + j + u);
        acc[b][0] = fmaf(v[u].x, xv, acc[b][0]);
        acc[b][1] = fmaf(v[u].y, xv, acc[b][1]);
        acc[b][2] = fmaf(v[u].z, xv, acc[b][2]);
        acc[b][3] = fmaf(v[u].w, xv, acc[b][3]);
      }
    }
  }
  for (; j < j1; ++j, a += ld) {
    const float4 v = ld_stream4(a);
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      const float xv = __ldg(xb + (int64_t)b * K + j);
      acc[b][0] = fmaf(v.x, xv, acc[b][0]);
      acc[b][1] = fmaf(v.y, xv, acc[b][1]);
      acc[b][2] = fmaf(v.z, xv, acc[b][2]);
      acc[b][3] = fmaf(v.w, xv, acc[b][3]);
    }
  }
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

// One image: y[i] = sum_ks part[ks][i] (fixed order) fused with the fit's
// residual r = (y - d) / sigma^2 and FP64 loss partials sum ((y - d)/sigma)^2
// per block (same layout as fwd_reduce_kernel, 128 rows per CTA).
__global__ void __launch_bounds__(256) fwd_reduce_loss_kernel(const float *__restrict__ part, int KS, int64_t ld,
                                                              int64_t M, const float *__restrict__ d, double sigma,
                                                              float inv_s2, float *__restrict__ y,
                                                              float *__restrict__ r, double *__restrict__ loss_part) {
  __shared__ float4 red[8][32];
  const int c4 = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t row = ((int64_t)blockIdx.x * 32 + c4) * 4;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (row < ld) {
#pragma unroll 4
    for (int ks = grp; ks < KS; ks += 8) {
      const float4 v = *reinterpret_cast<const float4 *>(part + (int64_t)ks * ld + row);
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
  }
  red[grp][c4] = s;
  __syncthreads();
  if (grp == 0) {
    double acc = 0.0;
    if (row < M) {
      float4 t = red[0][c4];
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        const float4 v = red[k][c4];
        t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
      }
      const float vals[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (row + e < M) {
          y[row + e] = vals[e];
          const float diff = vals[e] - d[row + e];
          r[row + e] = diff * inv_s2;
          const double q = (double)diff / sigma;
          acc += q * q;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (c4 == 0) loss_part[blockIdx.x] = acc;
  }
}

int forward_splits(const psfsim_plan *h) {
  const int64_t row_blocks = (h->ld + kRowsPerCta - 1) / kRowsPerCta;
  int64_t ks = (int64_t)h->num_sms * 8 / row_blocks;
  ks = ks < 1 ? 1 : ks;
  const int64_t max_ks = h->K / 8 > 0 ? h->K / 8 : 1;
  return (int)(ks < max_ks ? ks : max_ks);
}

constexpr int kAdjThreads = 256;

// gx[b, j] = sum_i A[i, j] g[b, i].  CTA c owns the contiguous column range
// [K c / G, K (c+1) / G); for each column its 256 threads split the rows
// (float4 strided), reduce in registers, then across warps through a
// double-buffered shared array.  Fixed assignment and order: deterministic.
template <int BB, bool kVec>
__global__ void __launch_bounds__(kAdjThreads) adj_kernel(const float *__restrict__ A, int64_t ld, int64_t M,
                                                          int64_t K, const float *__restrict__ g, int b0,
                                                          float *__restrict__ gx) {
  __shared__ float red[2][kAdjThreads / 32][BB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0 = K * blockIdx.x / gridDim.x, j1 = K * (blockIdx.x + 1) / gridDim.x;
  const float *gb = g + (int64_t)b0 * M;
  int parity = 0;
  for (int64_t j = j0; j < j1; ++j, parity ^= 1) {
    const float *col = A + j * ld;
    float acc[BB];
#pragma unroll
    for (int b = 0; b < BB; ++b) acc[b] = 0.f;
    if (kVec) {
      const int64_t M4 = M >> 2;
      int64_t i4 = threadIdx.x;
      constexpr int T = kAdjThreads;
      for (; i4 + 3 * T < M4; i4 += 4 * T) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ld_stream4(col + 4 * (i4 + T * u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int b = 0; b < BB; ++b) {
            const float4 gv = __ldg(reinterpret_cast<const float4 *>(gb + (int64_t)b * M) + i4 + T * u);
            acc[b] = fmaf(v[u].x, gv.x, acc[b]);
            acc[b] = fmaf(v[u].y, gv.y, acc[b]);
            acc[b] = fmaf(v[u].z, gv.z, acc[b]);
            acc[b] = fmaf(v[u].w, gv.w, acc[b]);
          }
        }
      }
      for (; i4 < M4; i4 += T) {
        const float4 v = ld_stream4(col + 4 * i4);
#pragma unroll
        for (int b = 0; b < BB; ++b) {
          const float4 gv = __ldg(reinterpret_cast<const float4 *>(gb + (int64_t)b * M) + i4);
          acc[b] = fmaf(v.x, gv.x, acc[b]);
          acc[b] = fmaf(v.y, gv.y, acc[b]);
          acc[b] = fmaf(v.z, gv.z, acc[b]);
          acc[b] = fmaf(v.w, gv.w, acc[b]);
        }
      }
    } else {
      for (int64_t i = threadIdx.x; i < M; i += kAdjThreads) {
        const float v = __ldg(col + i);
#pragma unroll
        for (int b = 0; b < BB; ++b) acc[b] = fmaf(v, __ldg(gb + (int64_t)b * M + i), acc[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      float s = acc[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[parity][warp][b] = s;
    }
    __syncthreads();
    if (threadIdx.x < BB) {
      float t = red[parity][0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < kAdjThreads / 32; ++w) t += red[parity][w][threadIdx.x];
      gx[(int64_t)(b0 + threadIdx.x) * K + j] = t;
    }
  }
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

int psfsim_gemv_splits(int64_t ld, int64_t K, int num_sms) {
  const int64_t row_blocks = (ld + kRowsPerCta - 1) / kRowsPerCta;
  int64_t ks = (int64_t)num_sms * 8 / row_blocks;
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

int psfsim_reduce_loss_blocks(const psfsim_plan *h) { return (int)((h->ld + kRedRows - 1) / kRedRows); }

cudaError_t psfsim_launch_forward_loss(const psfsim_plan *h, const float *x, const float *d, double sigma, float *y,
                                       float *r, void *scratch, double *loss_part, cudaStream_t st) {
  const int KS = forward_splits(h);
  float *part = reinterpret_cast<float *>(scratch);
  cudaError_t e = fwd_group<1>(h, x, 1, 0, part, KS, st);
  if (e != cudaSuccess) return e;
  fwd_reduce_loss_kernel<<<psfsim_reduce_loss_blocks(h), 256, 0, st>>>(part, KS, h->ld, h->M, d, sigma,
                                                                       (float)(1.0 / (sigma * sigma)), y, r, loss_part);
  return cudaGetLastError();
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
