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
  // The 2 x 2 footprint of both PSFs; taps outside the library are zero.  A
  // footprint wholly inside (the common case) is read without tests.
  const bool inner = q0 >= 0 && q0 < n - 1 && p0 >= 0 && p0 < n - 1;
  float t[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    if (w == 1 && w1 == 0.f) break;
    const float *L = w ? L1 : L0;
    if (inner) {
      const float *f = L + p0 * n + q0;
      t[w][0] = __ldg(f);
      t[w][1] = __ldg(f + 1);
      t[w][2] = __ldg(f + n);
      t[w][3] = __ldg(f + n + 1);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = p0 + (e >> 1), c = q0 + (e & 1);
        if (r >= 0 && r < n && c >= 0 && c < n) t[w][e] = __ldg(L + r * n + c);
      }
    }
  }
  const float v0 = wb0 * (wa0 * t[0][0] + wa1 * t[0][1]) + wb1 * (wa0 * t[0][2] + wa1 * t[0][3]);
  float v1 = 0.f;
  if (w1 != 0.f) v1 = wb0 * (wa0 * t[1][0] + wa1 * t[1][1]) + wb1 * (wa0 * t[1][2] + wa1 * t[1][3]);
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

// Dense storage of an even N x N scene grid, through the exact quarter-turn
// symmetry.  The quarter turn R(ix, iy) = (N-1-iy, ix) of the scene, (x, y) ->
// (-y, x), and P(p, q) = (q, n-1-p) of the image leave the source coordinates
// unchanged: with the fixed-point geometry, column R(j) has (C, Sn) = (-Sn_j,
// C_j), the same radius, bracket, weights and scale, so at pixel P(i) it holds
// A_ij bit for bit.  Only the x > 0, y > 0 quadrant (ix, iy >= N/2) is
// generated, and every element is written to its four positions
// A[P^m(i), R^m(j)], m = 0..3.
//
// Tile: 32 consecutive image pixels x a 16 x 16 block of quadrant pixels (256
// columns), generated into shared memory; then each of the four copies leaves
// as, per pixel, 16 runs of 16 columns (the rotated block's rows, 32 bytes of
// hi and of lo each).
constexpr int kQB = 16;                // quadrant block side (scene pixels)
constexpr int kQCols = kQB * kQB;      // columns per tile
constexpr int kQPix = 32;              // image pixels per tile
constexpr int kQPitch = kQCols + 16;   // shared row pitch in bf16: consecutive rows 8 banks apart

struct SymSplitParams {
  int n, N, H, nqb;  // image side, scene side, N / 2, quadrant blocks per side
  int vec;           // whole blocks can leave as 16-byte stores (N % 16 == 0)
  int vec32;         // ... and as 32-byte stores (N % 32 == 0)
  int64_t M, K, ld, tiles;
  const ColGeom *geom;
  const float *lib;
  const float *libmax;
  __nv_bfloat16 *hi;
  __nv_bfloat16 *lo;  // null for BF16 storage
  float *scale;
};

// One 32-byte global store (the address must be 32-byte aligned).
__device__ __forceinline__ void store32(void *p, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

// Image pixel P^m(p, q), as a row index.
__device__ __forceinline__ int64_t turn_pixel(int m, int p, int q, int n) {
  int pp = p, qq = q;
  for (int t = 0; t < m; ++t) {
    const int nq = n - 1 - pp;
    pp = qq;
    qq = nq;
  }
  return (int64_t)pp * n + qq;
}

__global__ void __launch_bounds__(256, 3) split_sym_build_kernel(const SymSplitParams P) {
  __shared__ __align__(16) __nv_bfloat16 thi[kQPix][kQPitch];
  __shared__ __align__(16) __nv_bfloat16 tlo[kQPix][kQPitch];
  const int n = P.n, N = P.N;
  const long long h = n - 1;
  const long long base = h << PSFSIM_FRAC_BITS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = P.nqb * P.nqb;
  if (blockIdx.x == 0)  // padding columns carry scale 1, as in the direct build
    for (int64_t j = P.K + threadIdx.x; j < P.ld; j += blockDim.x) P.scale[j] = 1.f;
  for (int64_t t = blockIdx.x; t < P.tiles; t += gridDim.x) {
    // Consecutive tiles: neighbouring quadrant blocks of the same pixels.
    const int64_t i0 = (t / nblk) * kQPix;
    const int jb = (int)(t % nblk);
    const int bx = P.H + (jb % P.nqb) * kQB, by = P.H + (jb / P.nqb) * kQB;
    const int bw = min(kQB, N - bx), bh = min(kQB, N - by);
    // Warp w generates block columns 32 w .. +31 (block rows 2 w, 2 w + 1): lane
    // l takes column 32 w + 4 g + l % 4 for the pixels l / 4 + 8 t, so one
    // load covers 8 neighbouring pixels of 4 neighbouring columns (nearby
    // footprints in the same or an adjacent bracket).
    // this lane's 4 pixels: offsets 2 du, 2 dv from the image centre (doubled)
    int du2[kQPix / 8], dv2[kQPix / 8];
#pragma unroll
    for (int t = 0; t < kQPix / 8; ++t) {
      const int i = (int)i0 + (lane >> 2) + 8 * t;  // < M < 2^31
      const int p = i / n;
      du2[t] = 2 * (i - p * n) - (int)h;
      dv2[t] = 2 * p - (int)h;
    }
    for (int g = 0; g < 8; ++g) {
      const int c = 32 * warp + 4 * g + (lane & 3), cu = c % kQB, cv = c / kQB;
      ColGeom gm;
      gm.k = -1;
      gm.C = gm.Sn = 0;
      gm.w0 = gm.w1 = 0.f;
      const int ix = bx + cu, iy = by + cv;
      const bool valid = cu < bw && cv < bh;
      if (valid) gm = P.geom[(int64_t)(iy - P.H) * P.H + (ix - P.H)];  // quadrant entry
      float inv = 1.f, sigma = 1.f;
      const float *L0 = P.lib, *L1 = P.lib;
      if (gm.k >= 0) {
        sigma = pow2_at_least(fmaxf(P.libmax[gm.k], P.libmax[gm.k + 1]));
        inv = 1.f / sigma;  // exact: sigma is a power of two
        L0 = P.lib + (int64_t)gm.k * P.M;
        L1 = L0 + P.M;
      }
      if (i0 == 0 && valid && lane < 4) {
        P.scale[(int64_t)iy * N + ix] = sigma;
        P.scale[(int64_t)ix * N + (N - 1 - iy)] = sigma;
        P.scale[(int64_t)(N - 1 - iy) * N + (N - 1 - ix)] = sigma;
        P.scale[(int64_t)(N - 1 - ix) * N + iy] = sigma;
      }
#pragma unroll
      for (int t = 0; t < kQPix / 8; ++t) {
        const int r = (lane >> 2) + 8 * t;
        const int64_t i = i0 + r;
        float v = 0.f;
        if (gm.k >= 0 && i < P.M) {
          const long long a2 = base + gm.C * du2[t] + gm.Sn * dv2[t];
          const long long b2 = base - gm.Sn * du2[t] + gm.C * dv2[t];
          v = element(L0, L1, n, a2, b2, gm.w0, gm.w1) * inv;
        }
        const __nv_bfloat16 vh = __float2bfloat16_rn(v);
        thi[r][c] = vh;
        tlo[r][c] = __float2bfloat16_rn(v - __bfloat162float(vh));
      }
    }
    __syncthreads();
    // Copy m, pixel r, rotated-block row vd: destination row P^m(i0 + r),
    // columns (oy + vd) N + ox + ud, ud = 0..15; its source in the tile is
    // block position (su, sv) of the generated block.
    const int vd = lane & 15;
    for (int k = 0; k < 4 * kQPix / 16; ++k) {
      const int m = k & 3;
      const int r = 2 * (warp + 8 * (k >> 2)) + (lane >> 4);
      const int64_t i = i0 + r;
      if (i >= P.M) continue;
      const int ii = (int)i, pi = ii / n;
      const int64_t row = turn_pixel(m, pi, ii - pi * n, n);
      int ox, oy;
      if (m == 0) { ox = bx; oy = by; }
      else if (m == 1) { ox = N - kQB - by; oy = bx; }
      else if (m == 2) { ox = N - kQB - bx; oy = N - kQB - by; }
      else { ox = by; oy = N - kQB - bx; }
      const __nv_bfloat16 *sh = thi[r], *sl = tlo[r];
      __nv_bfloat16 *dh = P.hi + row * P.ld + (int64_t)(oy + vd) * N + ox;
      __nv_bfloat16 *dl = P.lo ? P.lo + row * P.ld + (int64_t)(oy + vd) * N + ox : nullptr;
      // source column (in the tile) of destination position ud of this run
      auto src = [&](int ud) -> int {
        if (m == 0) return vd * kQB + ud;
        if (m == 1) return (kQB - 1 - ud) * kQB + vd;
        if (m == 2) return (kQB - 1 - vd) * kQB + (kQB - 1 - ud);
        return ud * kQB + (kQB - 1 - vd);
      };
      if (P.vec && bw == kQB && bh == kQB) {
        uint32_t wh[8], wl[8];
        if (m == 0 || m == 2) {
          const int s0 = (m == 0 ? vd : kQB - 1 - vd) * kQB;
          const uint4 h0 = *reinterpret_cast<const uint4 *>(sh + s0);
          const uint4 h1 = *reinterpret_cast<const uint4 *>(sh + s0 + 8);
          const uint4 l0 = *reinterpret_cast<const uint4 *>(sl + s0);
          const uint4 l1 = *reinterpret_cast<const uint4 *>(sl + s0 + 8);
          const uint32_t ah[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
          const uint32_t al[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            // m = 2 runs backwards: word w holds source positions 15 - 2w, 14 - 2w
            wh[w] = m == 0 ? ah[w] : __byte_perm(ah[7 - w], 0u, 0x1032);
            wl[w] = m == 0 ? al[w] : __byte_perm(al[7 - w], 0u, 0x1032);
          }
        } else {
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            const int a = src(2 * w), b = src(2 * w + 1);
            wh[w] = (uint32_t)__bfloat16_as_ushort(sh[a]) | ((uint32_t)__bfloat16_as_ushort(sh[b]) << 16);
            wl[w] = (uint32_t)__bfloat16_as_ushort(sl[a]) | ((uint32_t)__bfloat16_as_ushort(sl[b]) << 16);
          }
        }
        if (P.vec32) {  // 32-byte aligned runs: one store each
          store32(dh, wh);
          if (dl) store32(dl, wl);
        } else {
          reinterpret_cast<uint4 *>(dh)[0] = make_uint4(wh[0], wh[1], wh[2], wh[3]);
          reinterpret_cast<uint4 *>(dh)[1] = make_uint4(wh[4], wh[5], wh[6], wh[7]);
          if (dl) {
            reinterpret_cast<uint4 *>(dl)[0] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
            reinterpret_cast<uint4 *>(dl)[1] = make_uint4(wl[4], wl[5], wl[6], wl[7]);
          }
        }
      } else {
        // A block at the quadrant's outer edge (or N % 16 != 0): element by
        // element, only positions whose source lies inside the block.
        for (int ud = 0; ud < kQB; ++ud) {
          const int s = src(ud), su = s % kQB, sv = s / kQB;
          if (su >= bw || sv >= bh) continue;
          dh[ud] = sh[s];
          if (dl) dl[ud] = sl[s];
        }
      }
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
  if (h->N > 0 && h->N % 2 == 0 && !h->quadrant) {
    // Dense storage of an even grid: the quadrant's columns, four copies each.
    // The padding (rows M.. and columns K.. of every row) is zeroed first.
    const size_t row_bytes = (size_t)P.ld * 2;
    for (__nv_bfloat16 *a : {P.hi, P.lo}) {
      if (!a) continue;
      if ((e = cudaMemsetAsync(a + P.M * P.ld, 0, (size_t)(P.rows - P.M) * row_bytes, st)) != cudaSuccess) return e;
      if (P.ld > P.K &&
          (e = cudaMemset2DAsync(a + P.K, row_bytes, 0, (size_t)(P.ld - P.K) * 2, (size_t)P.M, st)) != cudaSuccess)
        return e;
    }
    SymSplitParams Q;
    Q.n = h->n;
    Q.N = h->N;
    Q.H = h->N / 2;
    Q.nqb = (Q.H + kQB - 1) / kQB;
    Q.vec = h->N % 16 == 0;
    Q.vec32 = h->N % 32 == 0;
    Q.M = h->M;
    Q.K = h->K;
    Q.ld = h->ld;
    Q.tiles = (h->M + kQPix - 1) / kQPix * (int64_t)Q.nqb * Q.nqb;
    Q.geom = P.geom;
    Q.lib = P.lib;
    Q.libmax = libmax;
    Q.hi = P.hi;
    Q.lo = P.lo;
    Q.scale = P.scale;
    int per_sm = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_sym_build_kernel, 256, 0)) != cudaSuccess)
      return e;
    split_sym_build_kernel<<<h->num_sms * (per_sm < 1 ? 1 : per_sm), 256, 0, st>>>(Q);
    return cudaGetLastError();
  }
  int per_sm = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_build_kernel, 256, 0)) != cudaSuccess)
    return e;
  split_build_kernel<<<h->num_sms * (per_sm < 1 ? 1 : per_sm), 256, 0, st>>>(P);
  return cudaGetLastError();
}
