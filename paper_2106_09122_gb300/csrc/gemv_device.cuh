// Device building blocks of the FP32 products with a stored A (column-major,
// each PSF contiguous), shared by the plain forward/adjoint kernels (gemv.cu)
// and the fit-gradient kernels (fit_gradient.cu).  Both directions stream A
// once from HBM with 128-bit loads that bypass L1.
#pragma once

#include <stdint.h>

namespace psfsim_gemv {

__device__ __forceinline__ float4 ld_stream4(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

constexpr int kFwdThreads = 256;
constexpr int kRowsPerCta = kFwdThreads * 4;

// acc[b][e] = sum_{j0 <= j < j1} A[r + e, j] x_b[j] for the thread's 4 rows,
// where x_b[j] = x[(b0 + b) K + j] (kSmemX false: global scene vectors) or
// x[b kXStride + j - j0] (kSmemX true: the range's scene values in shared
// memory, kXStride apart).
template <int BB, bool kSmemX = false, int kXStride = 0>
__device__ __forceinline__ void fwd_accumulate(const float *__restrict__ A, int64_t ld, int64_t K,
                                               const float *__restrict__ x, int b0, int64_t r, int64_t j0,
                                               int64_t j1, float (&acc)[BB][4]) {
#pragma unroll
  for (int b = 0; b < BB; ++b) acc[b][0] = acc[b][1] = acc[b][2] = acc[b][3] = 0.f;
  const float *a = A + j0 * ld + r;
  auto xval = [&](int b, int64_t j) -> float {
    if (kSmemX) return x[b * kXStride + (j - j0)];
    return __ldg(x + (int64_t)(b0 + b) * K + j);
  };
  int64_t j = j0;
  for (; j + 4 <= j1; j += 4, a += 4 * ld) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ld_stream4(a + u * ld);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int b = 0; b < BB; ++b) {
        const float xv = xval(b, j + u);
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
      const float xv = xval(b, j);
      acc[b][0] = fmaf(v.x, xv, acc[b][0]);
      acc[b][1] = fmaf(v.y, xv, acc[b][1]);
      acc[b][2] = fmaf(v.z, xv, acc[b][2]);
      acc[b][3] = fmaf(v.w, xv, acc[b][3]);
    }
  }
}

// As fwd_accumulate<BB> over the listed columns idx[t0..t1) (ascending).
template <int BB>
__device__ __forceinline__ void fwd_accumulate_idx(const float *__restrict__ A, int64_t ld, int64_t K,
                                                   const float *__restrict__ x, int b0, int64_t r,
                                                   const int *__restrict__ idx, int64_t t0, int64_t t1,
                                                   float (&acc)[BB][4]) {
#pragma unroll
  for (int b = 0; b < BB; ++b) acc[b][0] = acc[b][1] = acc[b][2] = acc[b][3] = 0.f;
  const float *xb = x + (int64_t)b0 * K;
  int64_t t = t0;
  for (; t + 4 <= t1; t += 4) {
    int j[4];
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = __ldg(idx + t + u);
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ld_stream4(A + (int64_t)j[u] * ld + r);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int b = 0; b < BB; ++b) {
        const float xv = __ldg(xb + (int64_t)b * K + j[u]);
        acc[b][0] = fmaf(v[u].x, xv, acc[b][0]);
        acc[b][1] = fmaf(v[u].y, xv, acc[b][1]);
        acc[b][2] = fmaf(v[u].z, xv, acc[b][2]);
        acc[b][3] = fmaf(v[u].w, xv, acc[b][3]);
      }
    }
  }
  for (; t < t1; ++t) {
    const int j = __ldg(idx + t);
    const float4 v = ld_stream4(A + (int64_t)j * ld + r);
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      const float xv = __ldg(xb + (int64_t)b * K + j);
      acc[b][0] = fmaf(v.x, xv, acc[b][0]);
      acc[b][1] = fmaf(v.y, xv, acc[b][1]);
      acc[b][2] = fmaf(v.z, xv, acc[b][2]);
      acc[b][3] = fmaf(v.w, xv, acc[b][3]);
    }
  }
}

constexpr int kAdjThreads = 256;
constexpr int kStashCols = 128;

// gx[b, j] = sum_i A[i, j] g[b, i] for j0 <= j < j1: for each column the
// CTA's 256 threads split the rows (float4 strided), reduce in registers, then
// across warps through a double-buffered shared array.  Fixed assignment and
// order: deterministic.  stash (shared memory, may be null): stash[j - j0] =
// gx[b0][j] for the first kStashCols columns, for a tail that reuses them.
template <int BB, bool kVec>
__device__ __forceinline__ void adj_columns(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K,
                                            const float *__restrict__ g, int b0, float *__restrict__ gx, int64_t j0,
                                            int64_t j1, float *stash = nullptr) {
  __shared__ float red[2][kAdjThreads / 32][BB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
      if (stash != nullptr && threadIdx.x == 0 && j - j0 < kStashCols) stash[j - j0] = t;
    }
  }
}

}  // namespace psfsim_gemv
