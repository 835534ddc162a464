// Fused on-the-fly S = A Z: A is never stored.  Tiles of A are regenerated
// from the radial library (lerp + bilinear rotation, Sec. 2) straight into
// shared memory in the layout the tensor cores read, and multiplied there —
// the paper's "standard interpolation method" (rebuild every time, Table 4)
// done on chip, for scenes whose A does not fit in memory.
//
// Exact quadrant symmetry: with fixed-point rotation coordinates the column of
// scene pixel R(j) = (-y, x) is bit-exactly the quarter-turned column of
// pixel j = (x, y).  Only the x > 0, y > 0 quadrant Q0 is generated (columns
// beyond the last radius are skipped), and
//     S = sum_{m=0..3} P^m (A_Q0 X^(m)),   X^(m)_j = x_{R^m(j)},
// where P permutes image pixels by a quarter turn.  The four rotated copies of
// each scene ride along the MMA's N dimension; x is split exactly into two
// bf16 parts (x1 | x2) and A into hi + lo, so per k-step
//     D[:, 0:8Bp] += hi [x1 x2]^T,  D[:, 0:4Bp] += lo [x1]^T.
// The epilogue applies P^m as a scatter into per-rotation partial images that
// are summed in a fixed order afterwards.
//
// Warps: 0 TMA producer (x tiles), 1 tcgen05.mma issuer, 2..17 generators.
// Generator g = w - 2 builds 8 columns of a 64-row half of every 128 x 64
// tile, two rows per lane (a column's entry and coordinates serve both), and
// also drains the TMEM accumulator of rotation g/4 for rows 32*(w%4)..+31
// into FP32 registers every kChunk k-tiles (the tensor core's FP32
// accumulation is not round-to-nearest, so long accumulations drift).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "psfsim_internal.cuh"
#include "ptx_util.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kGenWarps = 16;
constexpr int kThreads = (2 + kGenWarps) * 32;
constexpr int kMaxStages = 6;
constexpr int kChunk = 8;
constexpr int kMaxBp = 32;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint32_t kTileBytes = BM * BK * 2;

// An M-tile is a 16 x 8 block of image pixels (tile row r -> pixel
// (p0 + r / 16, q0 + r % 16)), so a warp's 32 rows form a 16 x 2 patch and its
// bilinear taps touch few cache lines.
constexpr int kBlockQ = 16, kBlockP = 8;
constexpr int kTabTiles = 4;  // k-tiles per column table (one generator barrier per table)

struct FusedParams {
  int n, N, Bp, B, KS, m_tiles, k_tiles, stages, tiles_q;
  int64_t M, rows, K0v, psz;  // psz: float4 entries per quad-layout PSF, (n + 1)^2
  uint32_t stage_bytes;
  const ColGeom *geom;
  const int *order;
  const float4 *qlib; // quad-layout library, [n_r][(n+1)^2]
  float *part;        // [KS][4][B][M]
  int *status;
};

// Per-column constants of one k-tile, shared by the generator warps: the
// fixed-point source coordinates of the tile's origin pixel and the steps.
// The steps C = cos and S = sin (fixed point) are kept as (lo, hi) 32-bit
// pieces so that offsets u >= 0 inside a tile cost one wide and one narrow
// integer multiply-add each (exact modulo 2^64).
struct ColEntry {
  long long A0, B0;
  uint32_t Clo, Slo, NSlo;
  int32_t Chi, Shi, NShi;
  int64_t off;  // offset of L[k] in the quad-layout library (0 for padding columns)
  float w0, w1;
};

__device__ __forceinline__ long long fx_mad(long long base, uint32_t lo, int32_t hi, uint32_t u) {
  uint64_t r = (uint64_t)base + (uint64_t)lo * u;
  r += (uint64_t)(uint32_t)(hi * (int32_t)u) << 32;
  return (long long)r;
}

__device__ __forceinline__ void split64(long long v, uint32_t &lo, int32_t &hi) {
  lo = (uint32_t)(unsigned long long)v;
  hi = (int32_t)(v >> 32);
}

// The two bilinear weights of one axis from the 32-bit fixed-point fraction,
// in units of 2^-32: the smaller one is converted (relative accuracy 2^-24),
// the larger one is 2^32 - smaller, exact because the smaller is at most 2^31.
// The two factors 2^-32 are applied as exact power-of-two scalings elsewhere:
// one in the column weights w0, w1 of the table, one in the epilogue.
__device__ __forceinline__ void axis_weights(unsigned f, float &w_lo_tap, float &w_hi_tap) {
  const bool low = f <= 0x80000000u;
  const float small = __uint2float_rn(low ? f : 0u - f);
  const float large = 4294967296.f - small;
  w_hi_tap = low ? small : large;
  w_lo_tap = low ? large : small;
}

// Library in "quad" layout: for every padded pixel (p, q), p, q in [-1, n-1],
// the float4 (L[p][q], L[p][q+1], L[p+1][q], L[p+1][q+1]) with zeros outside
// the PSF, so the whole bilinear footprint of a sample is one aligned 16-byte
// load.  Indexed [k][(p+1)(n+1) + (q+1)].
__global__ void quad_library_kernel(const float *__restrict__ lib, int n, int n_r, float4 *__restrict__ qlib) {
  const int nq = n + 1;
  const int64_t total = (int64_t)n_r * nq * nq;
  auto at = [&](int64_t k, int p, int q) -> float {
    return (p >= 0 && p < n && q >= 0 && q < n) ? lib[(k * n + p) * n + q] : 0.f;
  };
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / ((int64_t)nq * nq);
    const int rem = (int)(t % ((int64_t)nq * nq));
    const int p = rem / nq - 1, q = rem % nq - 1;
    qlib[t] = make_float4(at(k, p, q), at(k, p, q + 1), at(k, p + 1, q), at(k, p + 1, q + 1));
  }
}

// xs[(part * 4Bp + m Bp + b) * ldx + t] = part of x_b at scene pixel R^m(order[t]).
__global__ void fused_xgather(const float *__restrict__ x, int B, int Bp, int N, int64_t K0v, int64_t ldx,
                              const int *__restrict__ order, __nv_bfloat16 *__restrict__ xs) {
  const int64_t total = (int64_t)4 * Bp * ldx;
  const int H = N / 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int mb = (int)(idx / ldx);
    const int64_t t = idx % ldx;
    const int m = mb / Bp, b = mb % Bp;
    float v = 0.f;
    if (b < B && t < K0v) {
      const int j0 = order[t];
      int ix = H + j0 % H, iy = H + j0 / H;
      for (int r = 0; r < m; ++r) {  // R(ix, iy) = (N-1-iy, ix): (x, y) -> (-y, x)
        const int nx = N - 1 - iy;
        iy = ix;
        ix = nx;
      }
      v = x[(int64_t)b * N * N + (int64_t)iy * N + ix];
    }
    const __nv_bfloat16 x1 = __float2bfloat16_rn(v);
    xs[idx] = x1;
    xs[total + idx] = __float2bfloat16_rn(v - __bfloat162float(x1));
  }
}

// One A element, times 2^32, from a column-table entry and the pixel's
// fixed-point source coordinates (a2, b2).  The 2 x 2 footprint of each PSF
// is one float4 of the quad-layout library, so only the footprint position
// (q0, p0 in [-1, n-1]) needs a check.  Padding columns have weights 0 and an
// in-range footprint, so they give 0 without a test of their own.
__device__ __forceinline__ float gen_element(const ColEntry &e, const float4 *__restrict__ qlib, int n,
                                             int64_t qsz, long long a2, long long b2) {
  constexpr int kShift = PSFSIM_FRAC_BITS + 1;
  const int q0 = (int)(a2 >> kShift);
  const int p0 = (int)(b2 >> kShift);
  if ((unsigned)(q0 + 1) > (unsigned)n || (unsigned)(p0 + 1) > (unsigned)n) return 0.f;
  float wa0, wa1, wb0, wb1;
  axis_weights((unsigned)((unsigned long long)a2 >> (kShift - 32)), wa0, wa1);
  axis_weights((unsigned)((unsigned long long)b2 >> (kShift - 32)), wb0, wb1);
  const float4 *Q0 = qlib + e.off + (int64_t)(p0 + 1) * (n + 1) + (q0 + 1);
  const float4 t0 = __ldg(Q0);
  const float v0 = wb0 * (wa0 * t0.x + wa1 * t0.y) + wb1 * (wa0 * t0.z + wa1 * t0.w);
  float v1 = 0.f;
  if (e.w1 != 0.f) {
    const float4 t1 = __ldg(Q0 + qsz);
    v1 = wb0 * (wa0 * t1.x + wa1 * t1.y) + wb1 * (wa0 * t1.z + wa1 * t1.w);
  }
  return e.w0 * v0 + e.w1 * v1;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
}

__device__ __forceinline__ void set_abort(volatile int *flag, int *status) {
  *flag = 1;
  atomicExch(status, PSFSIM_ERR_TIMEOUT);
}

// Warp-uniform bounded wait: lane 0 decides, every lane then takes the acquire.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status) {
  const int lane = threadIdx.x & 31;
  int ok = 0;
  if (lane == 0) {
    ok = !*abort_flag && ptx::mbar_wait_bounded(bar, parity);
    if (!ok) set_abort(abort_flag, status);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && !ptx::mbar_wait_bounded(bar, parity)) set_abort(abort_flag, status);
  return ok != 0;
}

// Named barrier over the generator warps that also ANDs a flag across them,
// so every generator leaves the pipeline at the same point after a timeout.
__device__ __forceinline__ bool gen_barrier_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(kGenWarps * 32)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ int unit_k0(const FusedParams &P, int ks) { return (int)((int64_t)P.k_tiles * ks / P.KS); }

__global__ void __launch_bounds__(kThreads, 1)
    fused_kernel(const __grid_constant__ CUtensorMap map_x, const FusedParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t xfull[kMaxStages], gfull[kMaxStages], empty[kMaxStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ ColEntry ctab[2][kTabTiles * BK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      ptx::mbar_init(&xfull[s], 1);
      ptx::mbar_init(&gfull[s], kGenWarps);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], kGenWarps);
    }
    abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&map_x);
  }
  if (warp == 0) {
    ptx::tmem_alloc(&tmem_base_sh, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  const int units = P.m_tiles * P.KS;
  const int Bp = P.Bp;

  if (warp == 0) {
    if (lane == 0) {  // ---- TMA producer: x tiles ----
      uint32_t it = 0;
      const uint32_t tx = (uint32_t)(8 * Bp) * BK * 2;
      for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
        const int ks = u / P.m_tiles;
        const int k0 = unit_k0(P, ks), k1 = unit_k0(P, ks + 1);
        for (int kt = k0; kt < k1; ++kt, ++it) {
          const int s = (int)(it % P.stages);
          if (!ptx::mbar_wait_bounded(&empty[s], ((it / P.stages) & 1) ^ 1)) {
            set_abort(&abort_flag, P.status);
            break;
          }
          ptx::mbar_arrive_expect_tx(&xfull[s], tx);
          ptx::tma_load_2d(smem + (size_t)s * P.stage_bytes + 2 * kTileBytes, &map_x, kt * BK, 0, &xfull[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer ----
      const uint32_t idesc_hi = ptx::idesc_bf16_f32(BM, 8 * Bp);
      const uint32_t idesc_lo = ptx::idesc_bf16_f32(BM, 4 * Bp);
      uint32_t it = 0, c = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok && !abort_flag; u += gridDim.x) {
        const int ks = u / P.m_tiles;
        const int k0 = unit_k0(P, ks), k1 = unit_k0(P, ks + 1);
        for (int kc = k0; kc < k1 && ok; kc += kChunk, ++c) {
          const int kc1 = min(kc + kChunk, k1);
          const uint32_t acc = c & 1;
          if (!ptx::mbar_wait_bounded(&tempty[acc], ((c >> 1) & 1) ^ 1)) {
            set_abort(&abort_flag, P.status);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d_tmem = tbase + acc * kAccStride;
          for (int kt = kc; kt < kc1; ++kt, ++it) {
            const int s = (int)(it % P.stages);
            const uint32_t par = (it / P.stages) & 1;
            if (!ptx::mbar_wait_bounded(&xfull[s], par) || !ptx::mbar_wait_bounded(&gfull[s], par)) {
              set_abort(&abort_flag, P.status);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint8_t *st = smem + (size_t)s * P.stage_bytes;
            const uint64_t dh = ptx::smem_desc_sw128(st);
            const uint64_t dl = ptx::smem_desc_sw128(st + kTileBytes);
            const uint64_t dx = ptx::smem_desc_sw128(st + 2 * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t adv = (uint64_t)(kk * 32) >> 4;
              ptx::mma_bf16(d_tmem, dh + adv, dx + adv, idesc_hi, (kt > kc || kk > 0) ? 1u : 0u);
              ptx::mma_bf16(d_tmem, dl + adv, dx + adv, idesc_lo, 1u);
            }
            ptx::mma_commit(&empty[s]);
          }
          if (ok) ptx::mma_commit(&tfull[acc]);
        }
      }
    }
  } else {
    // ---- generators (+ accumulator drain) ----
    const int g = warp - 2;              // 0..15
    const int gtid = g * 32 + lane;      // 0..511
    const int quarter = warp & 3;        // TMEM lane quarter this warp may access
    const int rot = g >> 2;              // rotation whose accumulator columns this warp drains
    const int r = quarter * 32 + lane;   // tile row this lane drains
    // Generation: this warp builds 8 columns (group g / 2) of the tile's 64-row
    // half g % 2, two rows per lane: rA and rB = rA + 32, i.e. two image rows
    // further down, whose source coordinates are rA's plus 2 (S, C) per column.
    const int gc8 = g >> 1;
    const int rA = 64 * (g & 1) + lane, rB = rA + 32;
    const int n = P.n;
    const long long h = n - 1;
    const long long base = h << PSFSIM_FRAC_BITS;
    const uint32_t du2 = 2 * (rA % kBlockQ), dv2 = 2 * (rA / kBlockQ);
    uint32_t it = 0, c = 0, tg = 0;
    const ColEntry *cur = ctab[0];
    bool ok = true;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const int ks = u / P.m_tiles, mt = u % P.m_tiles;
      const int k0 = unit_k0(P, ks), k1 = unit_k0(P, ks + 1);
      const int po = (mt / P.tiles_q) * kBlockP, qo = (mt % P.tiles_q) * kBlockQ;
      const int p = po + r / kBlockQ, q = qo + r % kBlockQ;
      const bool row_ok = p < n && q < n;
      const bool okA = po + rA / kBlockQ < n && qo + rA % kBlockQ < n;
      const bool okB = po + rB / kBlockQ < n && qo + rB % kBlockQ < n;
      const long long uo = 2 * qo - h, vo = 2 * po - h;
      float sum[kMaxBp];
#pragma unroll
      for (int t = 0; t < kMaxBp; ++t) sum[t] = 0.f;
      auto drain = [&](uint32_t cc) -> bool {
        const uint32_t acc = cc & 1;
        if (!warp_wait(&tfull[acc], (cc >> 1) & 1, &abort_flag, P.status)) return false;
        ptx::tc_fence_after();
        const uint32_t tacc = tbase + ((uint32_t)(quarter * 32) << 16) + acc * kAccStride + rot * Bp;
#pragma unroll
        for (int qq = 0; qq < kMaxBp / 16; ++qq) {
          if (qq * 16 < Bp) {
            float v1[16], v2[16];
            ptx::tmem_ld16(tacc + qq * 16, v1);
            ptx::tmem_ld16(tacc + 4 * Bp + qq * 16, v2);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < 16; ++t) sum[qq * 16 + t] += v1[t] + v2[t];
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
        return true;
      };
      // Every exit from this loop happens right after gen_barrier_and, which
      // all generator warps reach the same number of times.
      bool stop = false;
      for (int kc = k0; kc < k1 && !stop; kc += kChunk, ++c) {
        const int kc1 = min(kc + kChunk, k1);
        for (int kt = kc; kt < kc1; ++kt, ++it) {
          // Column table for the next kTabTiles k-tiles (double-buffered; one
          // named barrier per table, which also carries the abort decision).
          if (((kt - k0) % kTabTiles) == 0) {
            ColEntry *tab = ctab[tg & 1];
            for (int c = gtid; c < kTabTiles * BK; c += kGenWarps * 32) {
              const int64_t t = (int64_t)kt * BK + c;
              ColEntry e;  // padding: zero steps from the centre pixel, zero weights
              e.off = 0;
              e.A0 = e.B0 = base;
              e.Clo = e.Slo = e.NSlo = 0;
              e.Chi = e.Shi = e.NShi = 0;
              e.w0 = e.w1 = 0.f;
              if (t < P.K0v && kt + c / BK < k1) {
                const ColGeom gm = P.geom[P.order[t]];
                e.A0 = base + gm.C * uo + gm.Sn * vo;
                e.B0 = base - gm.Sn * uo + gm.C * vo;
                split64(gm.C, e.Clo, e.Chi);
                split64(gm.Sn, e.Slo, e.Shi);
                split64(-gm.Sn, e.NSlo, e.NShi);
                e.off = (int64_t)gm.k * P.psz;
                e.w0 = gm.w0 * 0x1p-32f;
                e.w1 = gm.w1 * 0x1p-32f;
              }
              tab[c] = e;
            }
            if (!gen_barrier_and(ok)) {
              stop = true;
              break;
            }
            cur = tab;
            ++tg;
          }
          if (!ok) continue;  // after a timeout: no more work until the next barrier exits
          const ColEntry *tab = cur + ((kt - k0) % kTabTiles) * BK;
          const int s = (int)(it % P.stages);
          if (!warp_wait(&empty[s], ((it / P.stages) & 1) ^ 1, &abort_flag, P.status)) {
            ok = false;
            continue;
          }
          uint8_t *st = smem + (size_t)s * P.stage_bytes;
          uint32_t hw[2][4], lw[2][4];
#pragma unroll
          for (int cc = 0; cc < 8; cc += 2) {
            float vA[2], vB[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const ColEntry &ce = tab[gc8 * 8 + cc + e];
              const long long a2 = fx_mad(fx_mad(ce.A0, ce.Clo, ce.Chi, du2), ce.Slo, ce.Shi, dv2);
              const long long b2 = fx_mad(fx_mad(ce.B0, ce.NSlo, ce.NShi, du2), ce.Clo, ce.Chi, dv2);
              vA[e] = okA ? gen_element(ce, P.qlib, n, P.psz, a2, b2) : 0.f;
              vB[e] = okB ? gen_element(ce, P.qlib, n, P.psz, fx_mad(a2, ce.Slo, ce.Shi, 4u),
                                        fx_mad(b2, ce.Clo, ce.Chi, 4u))
                          : 0.f;
            }
            uint32_t hp = pack_bf16(vA[0], vA[1]);
            hw[0][cc >> 1] = hp;
            lw[0][cc >> 1] =
                pack_bf16(vA[0] - __uint_as_float(hp << 16), vA[1] - __uint_as_float(hp & 0xFFFF0000u));
            hp = pack_bf16(vB[0], vB[1]);
            hw[1][cc >> 1] = hp;
            lw[1][cc >> 1] =
                pack_bf16(vB[0] - __uint_as_float(hp << 16), vB[1] - __uint_as_float(hp & 0xFFFF0000u));
          }
          // 128-byte swizzle: 16-byte chunk index XOR (row % 8) inside each 1024-byte row group.
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) {
            const int rr = hr ? rB : rA;
            const uint32_t row_off = (uint32_t)(rr >> 3) * 1024 + (uint32_t)(rr & 7) * 128;
            const uint32_t chunk = (uint32_t)gc8 ^ (uint32_t)(rr & 7);
            *reinterpret_cast<uint4 *>(st + row_off + chunk * 16) =
                make_uint4(hw[hr][0], hw[hr][1], hw[hr][2], hw[hr][3]);
            *reinterpret_cast<uint4 *>(st + kTileBytes + row_off + chunk * 16) =
                make_uint4(lw[hr][0], lw[hr][1], lw[hr][2], lw[hr][3]);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&gfull[s]);
        }
        if (!stop && ok && kc > k0 && !drain(c - 1)) ok = false;
      }
      if (stop) break;
      if (ok && !drain(c - 1)) ok = false;
      if (!ok) continue;  // the next unit's first barrier takes every generator out
      if (row_ok) {
        int pp = p, qp = q;  // P^rot: (p, q) -> (q, n-1-p), applied rot times
        for (int t = 0; t < rot; ++t) {
          const int nxt = qp;
          qp = n - 1 - pp;
          pp = nxt;
        }
        float *out = P.part + ((int64_t)(ks * 4 + rot) * P.B) * P.rows + (int64_t)pp * n + qp;
#pragma unroll
        for (int t = 0; t < kMaxBp; ++t)
          if (t < P.B) out[(int64_t)t * P.rows] = sum[t] * 0x1p-32f;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tbase, kTmemCols);
  }
}

bool encode_x_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint32_t box_outer) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult qr;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
            cudaSuccess ||
        qr != cudaDriverEntryPointSuccess)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {BK, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct FusedPlanInfo {
  int Bp, KS, m_tiles, k_tiles, stages, tiles_q;
  int64_t rows, ldx;
  uint32_t stage_bytes;
  size_t smem, xs_bytes, part_bytes;
};

FusedPlanInfo fused_info(const psfsim_plan *h, int Bc) {
  FusedPlanInfo f;
  f.Bp = Bc <= 16 ? 16 : 32;
  f.rows = psfsim_round_up(h->M, BM);
  f.tiles_q = (h->n + kBlockQ - 1) / kBlockQ;
  f.m_tiles = f.tiles_q * ((h->n + kBlockP - 1) / kBlockP);
  f.k_tiles = (int)((h->K_valid + BK - 1) / BK);
  if (f.k_tiles < 1) f.k_tiles = 1;
  f.ldx = (int64_t)f.k_tiles * BK;
  f.KS = 1;
  while ((int64_t)f.m_tiles * f.KS < 2 * h->num_sms && f.KS * 2 <= f.k_tiles) f.KS *= 2;
  f.stage_bytes = (uint32_t)psfsim_round_up(2 * kTileBytes + 8 * f.Bp * BK * 2, 1024);
  f.stages = (int)((200 * 1024) / f.stage_bytes);
  if (f.stages > kMaxStages) f.stages = kMaxStages;
  f.smem = (size_t)f.stages * f.stage_bytes + 1024;
  f.xs_bytes = (size_t)psfsim_round_up(8ll * f.Bp * f.ldx * 2, 256);
  f.part_bytes = (size_t)4 * f.KS * Bc * f.rows * 4;
  return f;
}

}  // namespace

cudaError_t psfsim_launch_quad_library(psfsim_plan *h, cudaStream_t st) {
  quad_library_kernel<<<h->num_sms * 4, 256, 0, st>>>(h->d_lib, h->n, h->n_r,
                                                      reinterpret_cast<float4 *>(h->ws + h->plib_off));
  return cudaGetLastError();
}

size_t psfsim_forward_fused_scratch(const psfsim_plan *h, int B) {
  const int Bc = B < kMaxBp ? B : kMaxBp;
  const FusedPlanInfo f = fused_info(h, Bc);
  return f.xs_bytes + f.part_bytes;
}

cudaError_t psfsim_launch_forward_fused(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                        cudaStream_t st) {
  int *status = reinterpret_cast<int *>(h->ws + h->status_off);
  for (int b0 = 0; b0 < B; b0 += kMaxBp) {
    const int Bc = (B - b0) < kMaxBp ? (B - b0) : kMaxBp;
    const FusedPlanInfo f = fused_info(h, Bc);
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(scratch);
    float *part = reinterpret_cast<float *>(static_cast<char *>(scratch) + f.xs_bytes);
    const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
    fused_xgather<<<h->num_sms * 8, 256, 0, st>>>(x + (int64_t)b0 * h->K, Bc, f.Bp, h->N, h->K_valid, f.ldx, order,
                                                  xs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap mx;
    if (!encode_x_map(&mx, xs, (uint64_t)f.ldx, (uint64_t)(8 * f.Bp), (uint32_t)(8 * f.Bp)))
      return cudaErrorInvalidValue;
    FusedParams P;
    P.n = h->n;
    P.N = h->N;
    P.Bp = f.Bp;
    P.B = Bc;
    P.KS = f.KS;
    P.m_tiles = f.m_tiles;
    P.tiles_q = f.tiles_q;
    P.psz = (int64_t)(h->n + 1) * (h->n + 1);
    P.k_tiles = f.k_tiles;
    P.stages = f.stages;
    P.M = h->M;
    P.rows = f.rows;
    P.K0v = h->K_valid;
    P.stage_bytes = f.stage_bytes;
    P.geom = reinterpret_cast<const ColGeom *>(h->ws + h->geom_off);
    P.order = order;
    P.qlib = reinterpret_cast<const float4 *>(h->ws + h->plib_off);
    P.part = part;
    P.status = status;
    if ((e = cudaFuncSetAttribute(fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem)) !=
        cudaSuccess)
      return e;
    const int units = f.m_tiles * f.KS;
    fused_kernel<<<units < h->num_sms ? units : h->num_sms, kThreads, f.smem, st>>>(mx, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = psfsim_launch_reduce_partials(part, 4 * f.KS, Bc, f.rows, h->M, y + (int64_t)b0 * h->M, nullptr, st)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}
