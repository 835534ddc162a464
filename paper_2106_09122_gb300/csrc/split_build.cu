// Split-BF16 and BF16 storage of A for the tensor-core path.
//
// A_ij (the same lerp + bilinear-rotation element as the FP32 build, Sec. 2)
// is stored as sigma_j (hi_ij + lo_ij): sigma_j is the smallest power of two
// >= max(max|L_k|, max|L_{k+1}|) over the column's radial bracket (an exact
// bound on |A_ij|, since the lerp and bilinear weights are convex), hi =
// RN_bf16(A_ij / sigma_j), lo = RN_bf16(A_ij / sigma_j - hi); BF16 storage
// keeps hi alone.  hi and lo are row-major [rows][ld] (each image pixel's row
// contiguous along the scene pixels: K-major for the MMA), ld = K rounded up
// to 64, rows = M rounded up to 128; padding is zero.
#include <cuda_bf16.h>

#include "psfsim_internal.cuh"

namespace {

constexpr int kTileRows = 128;
constexpr int kTileCols = 64;

__global__ void libmax_kernel(const float *lib, int64_t M, float *libmax) {
  const float *L = lib + (int64_t)blockIdx.x * M;
  float m = 0.f;
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) m = fmaxf(m, fabsf(L[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    m = fmaxf(m, red[0]);
    libmax[blockIdx.x] = m;
  }
}

__device__ __forceinline__ float pow2_at_least(float m) {
  if (!(m > 0.f)) return 1.f;
  int e;
  const float f = frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return f == 0.5f ? m : ldexpf(1.f, e);
}

struct SplitParams {
  int n, pad;
  int64_t K, ld, M, rows;
  const ColGeom *geom;
  const int *order;  // compacted storage: column j is geometry entry order[j] (else null: entry j)
  const float *lib;
  const float *libmax;
  __nv_bfloat16 *hi;
  __nv_bfloat16 *lo;  // null for BF16 storage
  float *scale;
};

__device__ __forceinline__ float element(const float *L0, const float *L1, int n, long long a2, long long b2,
                                         float w0, float w1) {
  constexpr int kShift = PSFSIM_FRAC_BITS + 1;
  const int q0 = (int)(a2 >> kShift);
  const int p0 = (int)(b2 >> kShift);
  if (q0 < -1 || q0 > n - 1 || p0 < -1 || p0 > n - 1) return 0.f;
  const unsigned fa = (unsigned)((unsigned long long)a2 >> (kShift - 32));
  const unsigned fb = (unsigned)((unsigned long long)b2 >> (kShift - 32));
  constexpr float kInv32 = 2.3283064365386963e-10f;
  const float wa1 = __uint2float_rn(fa) * kInv32;
  const float wa0 = fa ? __uint2float_rn(0u - fa) * kInv32 : 1.f;
  const float wb1 = __uint2float_rn(fb) * kInv32;
  const float wb0 = fb ? __uint2float_rn(0u - fb) * kInv32 : 1.f;
  auto tap = [&](const float *L, int r, int c) -> float {
    return (r < 0 || r >= n || c < 0 || c >= n) ? 0.f : __ldg(L + r * n + c);
  };
  const float v0 = wb0 * (wa0 * tap(L0, p0, q0) + wa1 * tap(L0, p0, q0 + 1)) +
                   wb1 * (wa0 * tap(L0, p0 + 1, q0) + wa1 * tap(L0, p0 + 1, q0 + 1));
  float v1 = 0.f;
  if (w1 != 0.f)
    v1 = wb0 * (wa0 * tap(L1, p0, q0) + wa1 * tap(L1, p0, q0 + 1)) +
         wb1 * (wa0 * tap(L1, p0 + 1, q0) + wa1 * tap(L1, p0 + 1, q0 + 1));
  return w0 * v0 + w1 * v1;
}

// One 128 x 64 tile per iteration: thread t builds column t/4 for rows
// 32*(t%4) .. +31 into shared memory, then the tile leaves as 128-byte rows.
__global__ void __launch_bounds__(256) split_build_kernel(const SplitParams P) {
  __shared__ __align__(16) __nv_bfloat16 thi[kTileRows][kTileCols + 8];
  __shared__ __align__(16) __nv_bfloat16 tlo[kTileRows][kTileCols + 8];
  const int jj = threadIdx.x >> 2, rq = (threadIdx.x & 3) * 32;
  const int64_t ktiles = P.ld / kTileCols, mtiles = P.rows / kTileRows;
  const int n = P.n;
  const long long h = n - 1;
  const long long base = h << PSFSIM_FRAC_BITS;
  for (int64_t t = blockIdx.x; t < ktiles * mtiles; t += gridDim.x) {
    const int64_t mt = t / ktiles, kt = t % ktiles;
    const int64_t j = kt * kTileCols + jj;
    ColGeom g;
    g.k = -1;
    if (j < P.K) g = P.geom[P.order ? P.order[j] : j];
    float inv = 1.f, sigma = 1.f;
    const float *L0 = P.lib, *L1 = P.lib;
    if (g.k >= 0) {
      sigma = pow2_at_least(fmaxf(P.libmax[g.k], P.libmax[g.k + 1]));
      inv = 1.f / sigma;  // exact: sigma is a power of two
      L0 = P.lib + (int64_t)g.k * P.M;
      L1 = L0 + P.M;
    }
    if (mt == 0 && (threadIdx.x & 3) == 0) P.scale[j] = sigma;
    int64_t i = mt * kTileRows + rq;
    int p = (int)(i / n), q = (int)(i % n);
    for (int r = 0; r < 32; ++r, ++i) {
      float v = 0.f;
      if (g.k >= 0 && i < P.M) {
        const long long a2 = base + g.C * (2 * q - h) + g.Sn * (2 * p - h);
        const long long b2 = base - g.Sn * (2 * q - h) + g.C * (2 * p - h);
        v = element(L0, L1, n, a2, b2, g.w0, g.w1) * inv;
      }
      const __nv_bfloat16 vh = __float2bfloat16_rn(v);
      thi[rq + r][jj] = vh;
      tlo[rq + r][jj] = __float2bfloat16_rn(v - __bfloat162float(vh));
      if (++q == n) { q = 0; ++p; }
    }
    __syncthreads();
    // 128 rows x 128 bytes per matrix = 1024 16-byte chunks; 4 per thread per matrix.
    for (int c = threadIdx.x; c < kTileRows * 8; c += blockDim.x) {
      const int row = c >> 3, part = c & 7;
      const int64_t off = (mt * kTileRows + row) * P.ld + kt * kTileCols + part * 8;
      *reinterpret_cast<uint4 *>(P.hi + off) = *reinterpret_cast<const uint4 *>(&thi[row][part * 8]);
      if (P.lo) *reinterpret_cast<uint4 *>(P.lo + off) = *reinterpret_cast<const uint4 *>(&tlo[row][part * 8]);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t psfsim_launch_split_build(psfsim_plan *h, cudaStream_t st) {
  float *libmax = reinterpret_cast<float *>(h->ws + h->libmax_off);
  libmax_kernel<<<h->n_r, 256, 0, st>>>(h->d_lib, h->M, libmax);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SplitParams P;
  P.n = h->n;
  P.pad = 0;
  P.K = psfsim_cols(h);
  P.order = h->quadrant ? reinterpret_cast<const int *>(h->ws + h->order_off) : nullptr;
  P.ld = h->ld;
  P.M = h->M;
  P.rows = psfsim_round_up(h->M, kTileRows);
  P.geom = reinterpret_cast<const ColGeom *>(h->ws + h->geom_off);
  P.lib = h->d_lib;
  P.libmax = libmax;
  P.hi = reinterpret_cast<__nv_bfloat16 *>(h->ws + h->a_off);
  P.lo = h->lo_off >= 0 ? reinterpret_cast<__nv_bfloat16 *>(h->ws + h->lo_off) : nullptr;
  P.scale = reinterpret_cast<float *>(h->ws + h->scale_off);
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_build_kernel, 256, 0)) != cudaSuccess)
    return e;
  split_build_kernel<<<h->num_sms * (per_sm < 1 ? 1 : per_sm), 256, 0, st>>>(P);
  return cudaGetLastError();
}
