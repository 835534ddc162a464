// Adjoint A^T g for split-BF16 and BF16 storage (row-major hi[/lo],
// per-column scale): gx[b, j] = sigma_j sum_i (hi_ij + lo_ij) g[b, i] (lo = 0
// for BF16).  Each thread owns 8 consecutive columns (one 16-byte load of hi,
// and of lo, per row); the rows are split KS ways into partial sums in caller
// scratch, reduced in a fixed order afterwards (deterministic).
#include <cuda_bf16.h>

#include "psfsim_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kColsPerCta = kThreads * 8;

__device__ __forceinline__ uint4 ld_stream16(const void *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ void unpack8(uint4 h, float (&a)[8]) {
  const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    a[2 * t] = __uint_as_float(hw[t] << 16);
    a[2 * t + 1] = __uint_as_float(hw[t] & 0xFFFF0000u);
  }
}

__device__ __forceinline__ void unpack8(uint4 h, uint4 l, float (&a)[8]) {
  const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    a[2 * t] = __uint_as_float(hw[t] << 16) + __uint_as_float(lw[t] << 16);
    a[2 * t + 1] = __uint_as_float(hw[t] & 0xFFFF0000u) + __uint_as_float(lw[t] & 0xFFFF0000u);
  }
}

// Row i's 8 columns from j: hi + lo (kLo) or hi alone.
template <bool kLo>
__device__ __forceinline__ void load8(const __nv_bfloat16 *hi, const __nv_bfloat16 *lo, int64_t off, float (&a)[8]) {
  if (kLo)
    unpack8(ld_stream16(hi + off), ld_stream16(lo + off), a);
  else
    unpack8(ld_stream16(hi + off), a);
}

template <int BB, bool kLo>
__global__ void __launch_bounds__(kThreads) adj_split_partial(const __nv_bfloat16 *__restrict__ hi,
                                                              const __nv_bfloat16 *__restrict__ lo,
                                                              const float *__restrict__ scale, int64_t ld,
                                                              int64_t M, const float *__restrict__ g, int B, int b0,
                                                              float *__restrict__ part) {
  const int64_t j = (int64_t)blockIdx.x * kColsPerCta + 8 * threadIdx.x;
  const int KS = gridDim.y, ks = blockIdx.y;
  if (j >= ld) return;
  const int64_t i0 = M * ks / KS, i1 = M * (ks + 1) / KS;
  float acc[BB][8];
#pragma unroll
  for (int b = 0; b < BB; ++b)
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[b][t] = 0.f;
  const float *gb = g + (int64_t)b0 * M;
  int64_t i = i0;
  for (; i + 2 <= i1; i += 2) {
    float a0[8], a1[8];
    load8<kLo>(hi, lo, i * ld + j, a0);
    load8<kLo>(hi, lo, (i + 1) * ld + j, a1);
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      const float g0 = __ldg(gb + (int64_t)b * M + i), g1 = __ldg(gb + (int64_t)b * M + i + 1);
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[b][t] = fmaf(a1[t], g1, fmaf(a0[t], g0, acc[b][t]));
    }
  }
  for (; i < i1; ++i) {
    float a0[8];
    load8<kLo>(hi, lo, i * ld + j, a0);
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      const float g0 = __ldg(gb + (int64_t)b * M + i);
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[b][t] = fmaf(a0[t], g0, acc[b][t]);
    }
  }
  float sc[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) sc[t] = scale[j + t];
#pragma unroll
  for (int b = 0; b < BB; ++b) {
    float *out = part + ((int64_t)ks * B + b0 + b) * ld + j;
    *reinterpret_cast<float4 *>(out) =
        make_float4(acc[b][0] * sc[0], acc[b][1] * sc[1], acc[b][2] * sc[2], acc[b][3] * sc[3]);
    *reinterpret_cast<float4 *>(out + 4) =
        make_float4(acc[b][4] * sc[4], acc[b][5] * sc[5], acc[b][6] * sc[6], acc[b][7] * sc[7]);
  }
}

int adjoint_splits(const psfsim_plan *h) {
  const int64_t col_blocks = (h->ld + kColsPerCta - 1) / kColsPerCta;
  int64_t ks = (int64_t)h->num_sms * 8 / col_blocks;
  ks = ks < 1 ? 1 : ks;
  const int64_t max_ks = h->M / 8 > 0 ? h->M / 8 : 1;
  return (int)(ks < max_ks ? ks : max_ks);
}

template <int BB>
cudaError_t group(const psfsim_plan *h, const float *g, int B, int b0, float *part, int KS, cudaStream_t st) {
  const __nv_bfloat16 *hi = reinterpret_cast<const __nv_bfloat16 *>(h->ws + h->a_off);
  const float *scale = reinterpret_cast<const float *>(h->ws + h->scale_off);
  dim3 grid((unsigned)((h->ld + kColsPerCta - 1) / kColsPerCta), (unsigned)KS);
  if (h->lo_off >= 0)
    adj_split_partial<BB, true><<<grid, kThreads, 0, st>>>(
        hi, reinterpret_cast<const __nv_bfloat16 *>(h->ws + h->lo_off), scale, h->ld, h->M, g, B, b0, part);
  else
    adj_split_partial<BB, false><<<grid, kThreads, 0, st>>>(hi, nullptr, scale, h->ld, h->M, g, B, b0, part);
  return cudaGetLastError();
}

}  // namespace

size_t psfsim_adjoint_split_scratch(const psfsim_plan *h, int B) {
  return (size_t)adjoint_splits(h) * (size_t)B * (size_t)h->ld * 4;
}

cudaError_t psfsim_launch_adjoint_split(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                        cudaStream_t st) {
  const int KS = adjoint_splits(h);
  float *part = reinterpret_cast<float *>(scratch);
  cudaError_t e = cudaSuccess;
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 4) { e = group<4>(h, g, B, b0, part, KS, st); b0 += 4; }
    else if (left >= 2) { e = group<2>(h, g, B, b0, part, KS, st); b0 += 2; }
    else { e = group<1>(h, g, B, b0, part, KS, st); b0 += 1; }
  }
  if (e != cudaSuccess) return e;
  return psfsim_launch_reduce_partials(part, KS, B, h->ld, psfsim_cols(h), gx, nullptr, st);
}
