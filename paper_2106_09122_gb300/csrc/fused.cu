// Fused on-the-fly S = A Z: A is never stored.  Tiles of A are regenerated
// from the radial library (lerp + bilinear rotation, Sec. 2) straight into
// shared memory in the layout the tensor cores read, and multiplied there --
// the paper's "standard interpolation method" (rebuild every time, Table 4)
// done on chip, for scenes whose A does not fit in memory.
//
// Exact quadrant symmetry: with fixed-point rotation coordinates the column of
// scene pixel R(j) = (-y, x) is exactly the quarter-turned column of pixel
// j = (x, y).  Only the x > 0, y > 0 quadrant Q0 is generated (columns beyond
// the last radius are skipped), and
//     S = sum_{m=0..3} P^m (A_Q0 X^(m)),   X^(m)_j = x_{R^m(j)},
// where P permutes image pixels by a quarter turn.  The four rotated copies of
// each scene ride along the MMA's N dimension; x is split exactly into two
// bf16 parts x1 + x2 and A into hi + lo, so per k-step three MMAs of N = 4Bp
// accumulate into one TMEM accumulator D:
//     D += hi x1^T,  D += hi x2^T,  D += lo x1^T
// (only lo x2, < 2^-18 relative, is dropped).  The epilogue applies P^m as a
// scatter into per-rotation partial images that are summed in a fixed order
// afterwards.
//
// Generation.  The library is kept as "pair entries": for every bracket pair
// (L[k], L[k+1]) and padded pixel (p, q) in [-1, n-1]^2, one 32-byte entry
// holding the 2 x 2 bilinear footprint of both PSFs, tap by tap,
//     (L00, L00'), (L01, L01'), (L10, L10'), (L11, L11')
// (L01 = L[p][q+1], L10 = L[p+1][q], primes for L[k+1]), so one 256-bit load
// fetches everything an element needs.  Source coordinates are 64-bit
// fixed point in units of 2^-41 pixel (the geometry's cos and sin are exact
// integers in those units, so moving by whole pixels is exact): a per-(tile,
// column) origin plus multiples of cos and sin.  The bilinear weights of each
// axis come from the coordinate's fraction rounded to 32 bits, f, as two
// floats, f and 2^32 - f, each converted from the exact integer, so every
// weight -- also a tiny one next to the edge of a footprint -- is accurate
// relative to itself up to the 2^-32 rounding of the coordinate; with all
// four taps and weights non-negative an element carries no cancellation,
// which keeps the faint pixels at the image's corners, built only from such
// edge samples, within their bound.  The two PSFs of the pair are
// interpolated at once with paired FP32 operations.
//
// Warps: 16, all generators (four per scheduler partition, so each thread
// may hold 128 registers).  Thread 0 also issues the x tiles' TMA loads, and
// for each stage the warp that finishes its part last issues the stage's
// tcgen05.mma (one lane).  An M-tile is an 8 x 16 block of image pixels.
// Warp g builds columns 4g .. 4g+3 of every 128 x 64 tile: lane l takes
// column 4g + l % 4 for the pixels du = l / 4 of all 16 rows dv, so one warp
// load covers 8 neighbouring pixels x 4 neighbouring columns (columns are
// sorted by angle within each radial bracket, and neighbouring columns often
// need the same footprint entry for a pixel: the request touches fewer
// sectors).  The A tiles are M-major (the MMA's transposed-A form), with tile
// row 16 sigma(du) + dv for pixel (du, dv): a lane's 16 values of a k-tile
// are two runs of 8 contiguous bf16, written as 16-byte stores after pairs of
// rows are rounded together, and sigma spreads each 8-lane group's stores
// over 8 bank groups.  Each lane starts its column itself from the plan's
// column table (origin terms, steps and weights of every column in the
// angle-sorted order, prepared at build time), so the warps share no table
// and meet at no block-wide barrier: stages, accumulators and running sums
// are handed over through mbarriers only.  A lane keeps four rows' footprint
// loads in flight, and the stream runs on across the k-tiles of an
// accumulation chunk: while a k-tile's last rows are finished, the next
// k-tile's first rows are already loading.  A k-tile in which every lane's
// 16 rows lie beyond one edge of the library (the image corners at many
// angles) is written as zeros without loads.  CTAs take their work units in
// order of the M-tile's distance from the image centre (a table built with
// the plan), so the M-tiles in flight at once read the same annulus of the
// library and share it in L2.  Warps also drain the TMEM
// accumulator of rotation g / 4 for rows 32 (g % 4) .. +31 every kChunk
// k-tiles into a running FP32 sum kept in a third TMEM region (the tensor
// core's FP32 accumulation is not round-to-nearest, so long accumulations
// drift; the sums are added on the CUDA cores, and keeping them in TMEM leaves
// the registers to generation).  A launch carries 16, 32 or 64 scenes; with 64
// (N = 256) TMEM holds a single accumulator beside the sums, and a chunk's
// drain comes right after the next chunk's first k-tile is generated.  Every wait is bounded; after a timeout every
// later wait fails at once, each warp leaves its loop, and each role waits
// (bounded) for the asynchronous work it issued before the CTA releases its
// memory.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "psfsim_internal.cuh"
#include "ptx_util.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kWarps = 16;                   // every warp generates; see the file comment for roles
constexpr int kThreads = kWarps * 32;
constexpr int kStages = 2;
constexpr int kChunk = 5;                    // k-tiles per accumulation: 5 x 4 x 3 = 60 MMAs
constexpr int kMaxBp = 64;                   // scenes per launch: 16, 32 or 64 (padded)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 128;         // Bp <= 32: two accumulators of 4Bp <= 128 columns
constexpr uint32_t kSumCol = 256;            // running sums: columns 256 .. 256 + 4Bp
// Bp = 64 ("wide"): one accumulator of 256 columns, the sums beside it.
constexpr uint32_t kTileBytes = BM * BK * 2;
constexpr int kTileW = 8, kTileH = 16;       // M-tile: 8 x 16 image pixels
constexpr int kCols = BK / kWarps;           // columns per generator warp per k-tile
constexpr int kDepth = 4;                    // rows whose footprint loads a lane keeps in flight
static_assert(kTileW * kTileH == BM && kCols == 4 && kWarps == 16 && kTileH % kDepth == 0, "tile shape");
constexpr int kFixShift = PSFSIM_FRAC_BITS + 1;  // fraction bits of the source coordinates a and b

// One column of the generators' (angle-sorted) order, prepared at build
// time.  With X = q0 + du and Y = p0 + dv for tile pixel (du, dv) of the
// M-tile whose origin pixel is (p0, q0), the source column (+1) and row (+1)
// in units of 2^-41 are
//     a = A00 + C2 X + S2 Y,   b = B00 - S2 X + C2 Y
// (Eq. 2-3's rotation about the library centre (n-1)/2, in fixed point; the
// half unit of 2^-32 that rounds the weights' fraction is folded into A00
// and B00).  Padding columns have an origin far outside the library, zero
// steps and zero weights.
struct __align__(16) FusedCol {
  long long A00, B00;
  unsigned long long C2, S2;  // cos, sin (both in [0, 1) for the quadrant) in units of 2^-41
  uint32_t off;               // first pair entry of the column's bracket
  float w0, w1;               // lerp weights of L[k] and L[k+1], times 2^-64
  uint32_t pad;
};
static_assert(sizeof(FusedCol) == 48, "FusedCol layout");

struct FusedParams {
  int n, Bp, B, KS, m_tiles, k_tiles, tiles_q;
  int64_t rows;
  uint32_t stage_bytes;
  uint32_t zero_entry;    // index of the all-zero entry after the last bracket pair's (n + 1)^2 entries
  const FusedCol *cols;   // the angle-sorted columns, padded to whole k-tiles
  const int *mt_order;    // M-tiles nearest the image centre first
  const float *plib;      // pair entries, 8 floats each
  float *part;            // [KS][4][B][rows]
  int *status;
  uint64_t wait_ns;
  int64_t stall_load;     // test hook: the x load of this k-tile (CTA issue order) is never issued; -1: none
};

// A lane's column in the current k-tile: the source coordinates a and b of
// its pixel in the current tile row (advanced one row, dv, at a time), the
// steps, the column's first pair entry and its lerp weights (x 2^-64).
struct LaneCol {
  unsigned long long a, b, C2, S2;
  uint32_t off;
  float w0, w1;
};

__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Two FP32 multiplies (round to nearest) on register pairs.
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Two FP32 fused multiply-adds (round to nearest) on register pairs.
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// One 32-byte pair entry (read-only path): the four taps, each as the pair
// (L[k], L[k+1]).
struct Entry {
  uint64_t t00, t01, t10, t11;
};

__device__ __forceinline__ Entry load_entry(const float *p) {
  Entry e;
  asm volatile("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
               : "=l"(e.t00), "=l"(e.t01), "=l"(e.t10), "=l"(e.t11)
               : "l"(p));
  return e;
}

// Pair entries of the library (see the file comment); entry (k, p, q) at
// k (n+1)^2 + (p+1)(n+1) + (q+1), plus one all-zero entry at the end.
__global__ void pair_library_kernel(const float *__restrict__ lib, int n, int n_r, float *__restrict__ plib) {
  const int nq = n + 1;
  const int64_t per = (int64_t)nq * nq;
  const int64_t total = (int64_t)(n_r - 1) * per + 1;
  auto at = [&](int64_t k, int p, int q) -> float {
    return (p >= 0 && p < n && q >= 0 && q < n) ? lib[(k * n + p) * n + q] : 0.f;
  };
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (t < total - 1) {
      const int64_t k = t / per;
      const int rem = (int)(t % per);
      const int p = rem / nq - 1, q = rem % nq - 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        e[h] = at(k + h, p, q);
        e[2 + h] = at(k + h, p, q + 1);
        e[4 + h] = at(k + h, p + 1, q);
        e[6 + h] = at(k + h, p + 1, q + 1);
      }
    }
    float4 *dst = reinterpret_cast<float4 *>(plib + 8 * t);
    dst[0] = make_float4(e[0], e[1], e[2], e[3]);
    dst[1] = make_float4(e[4], e[5], e[6], e[7]);
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

// order[rank] = M-tile: M-tiles sorted by the squared distance of their
// centre from the image centre (in half pixels, so exactly), ties by index.
__global__ void mtile_order_kernel(int n, int tiles_q, int m_tiles, int *__restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m_tiles) return;
  auto dist2 = [&](int mt) -> long long {
    const long long dp = 2ll * (mt / tiles_q) * kTileH + (kTileH - 1) - (n - 1);
    const long long dq = 2ll * (mt % tiles_q) * kTileW + (kTileW - 1) - (n - 1);
    return dp * dp + dq * dq;
  };
  const long long di = dist2(i);
  int rank = 0;
  for (int j = 0; j < m_tiles; ++j) {
    const long long dj = dist2(j);
    rank += (dj < di) || (dj == di && j < i);
  }
  order[rank] = i;
}

// cols[t] from the geometry of column order[t] (the generators' order);
// entries from K0v up to the next whole k-tile are padding.
__global__ void fused_columns_kernel(const ColGeom *__restrict__ geom, const int *__restrict__ order, int n,
                                     uint32_t pair_entries, int64_t K0v, int64_t Kpad, FusedCol *__restrict__ cols) {
  const long long h = n - 1;
  // 2a and 2b in units of 2^-PSFSIM_FRAC_BITS, i.e. a and b in units of
  // 2^-41; +1 pixel (2^42) for the padded index; half a unit of 2^-32 (2^8)
  // rounds the fraction the weights use.
  const long long base = ((h + 2) << PSFSIM_FRAC_BITS) + (1ll << (kFixShift - 33));
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Kpad; t += (int64_t)gridDim.x * blockDim.x) {
    FusedCol c;
    c.A00 = c.B00 = -(1ll << 62);
    c.C2 = c.S2 = 0ull;
    c.off = 0u;
    c.w0 = c.w1 = 0.f;
    c.pad = 0u;
    if (t < K0v) {
      const ColGeom gm = geom[order[t]];
      // Tile pixel (du, dv) of the M-tile at (p0, q0) is image pixel
      // (p0 + dv, q0 + du); its source coordinates are
      //     a = base + C (2 X - h) + Sn (2 Y - h),  b = base - Sn (2 X - h) + C (2 Y - h).
      c.A00 = base - h * (gm.C + gm.Sn);
      c.B00 = base + h * (gm.Sn - gm.C);
      c.C2 = (unsigned long long)(2 * gm.C);
      c.S2 = (unsigned long long)(2 * gm.Sn);
      c.off = (uint32_t)gm.k * pair_entries;
      c.w0 = gm.w0 * 0x1p-64f;
      c.w1 = gm.w1 * 0x1p-64f;
    }
    cols[t] = c;
  }
}

__device__ __forceinline__ void set_abort(volatile int *flag, int *status) {
  *flag = 1;
  atomicExch(status, PSFSIM_ERR_TIMEOUT);
}

// Warp-uniform bounded wait: lane 0 decides, every lane then takes the acquire.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status,
                                          uint64_t lim) {
  const int lane = threadIdx.x & 31;
  int ok = 0;
  if (lane == 0) {
    ok = !*abort_flag && ptx::mbar_wait_bounded(bar, parity, lim);
    if (!ok) set_abort(abort_flag, status);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && !ptx::mbar_wait_bounded(bar, parity, lim)) set_abort(abort_flag, status);
  return ok != 0;
}

// Bounded wait by lane 0 alone: the warp's later accesses are ordered after
// its acquire by __syncwarp.
__device__ __forceinline__ bool warp_wait_lane0(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status,
                                                uint64_t lim) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) {
    ok = !*abort_flag && ptx::mbar_wait_bounded(bar, parity, lim);
    if (!ok) set_abort(abort_flag, status);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

__device__ __forceinline__ int unit_k0(const FusedParams &P, int ks) { return (int)((int64_t)P.k_tiles * ks / P.KS); }

// Start of a lane's column for the M-tile whose origin pixel is (p0, q0), at
// its pixel (du, 0).
__device__ __forceinline__ void lane_start(const FusedCol &c, int p0, int q0, uint32_t du, LaneCol &L) {
  const uint32_t X = (uint32_t)q0 + du, Y = (uint32_t)p0;
  L.C2 = c.C2;
  L.S2 = c.S2;
  L.a = (unsigned long long)c.A00 + c.C2 * X + c.S2 * Y;
  L.b = (unsigned long long)c.B00 - c.S2 * X + c.C2 * Y;
  L.off = c.off;
  L.w0 = c.w0;
  L.w1 = c.w1;
}

// True when all 16 rows of a lane's column, from its current start L, fall
// beyond one edge of the library (their footprints are all zero): a and b
// only grow along the rows (C2, S2 >= 0 in the quadrant), so the first and
// the last row decide.
__device__ __forceinline__ bool rows_outside(const LaneCol &L, uint32_t un) {
  const long long a0 = (long long)L.a, b0 = (long long)L.b;
  const long long a15 = a0 + (long long)(kTileH - 1) * (long long)L.S2;
  const long long b15 = b0 + (long long)(kTileH - 1) * (long long)L.C2;
  const long long lim = (long long)(un + 1u) << kFixShift;  // padded index > n
  return a15 < 0 || a0 >= lim || b15 < 0 || b0 >= lim;
}

// The two bilinear weights of one axis, in units of 2^-32, from the 32-bit
// fraction f of a source coordinate: (2^32 - f, f), each from its exact
// integer, so each is accurate relative to itself however small: f converts
// with one rounding, 2^32 - f as (2^32 - 1 - f) + 1 with two (the + 1 is
// exact below 2^24 and under half an ulp above).
__device__ __forceinline__ void axis_weights(uint32_t f, float &w_near, float &w_far) {
  w_far = __uint2float_rn(f);
  w_near = __uint2float_rn(~f) + 1.0f;
}

// The A tiles (hi, lo) are M-major: K groups of 8 columns, each two 1024-byte
// swizzle atoms of 64 tile rows (128-byte swizzle), the atoms of a group 1024
// bytes apart (leading byte offset), the groups 2048 bytes apart (stride byte
// offset).  The descriptor's other fields are those of the K-major one.
constexpr uint32_t kAtomMN = 1024, kGroupK = 2048;

__device__ __forceinline__ uint64_t smem_desc_mn_sw128(const void *tile) {
  const uint64_t addr = ptx::smem_u32(tile);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;
  d |= (uint64_t)(kAtomMN >> 4) << 16;
  d |= (uint64_t)(kGroupK >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Tile-row block of pixel column du: rows 16 sigma(du) .. +15 (sigma swaps
// bits 0 and 1), so that the two pixels of each 8-lane group (du = 2i, 2i + 1)
// have rows 32 apart modulo 64 and their 16-byte stores meet 8 different
// 16-byte bank groups.  sigma is its own inverse.
__host__ __device__ constexpr uint32_t sigma(uint32_t du) { return (du & 4u) | ((du & 1u) << 1) | ((du & 2u) >> 1); }

// MMAs of one stage (k-tile kt of chunk [kc, kc1)), issued by the generator
// lane whose warp finished the stage last: wait for all generators and for the
// x tile, and (first k-tile of a chunk) for the accumulator to be drained;
// then 4 k-steps of three N = 4Bp MMAs, a commit that frees the stage, and
// (last k-tile of the chunk) one that hands the accumulator to the drain.
template <bool kWide>
__device__ __forceinline__ void issue_stage_mmas(const FusedParams &P, uint8_t *stage, uint64_t *xfull,
                                                 uint64_t *gfull, uint64_t *empty, uint64_t *tfull, uint64_t *tempty,
                                                 uint32_t par, uint32_t c, bool first_kt, bool last_kt, uint32_t tbase,
                                                 volatile int *abort_flag) {
  const uint64_t lim = P.wait_ns;
  // Bp <= 32: accumulator c % 2, each used every other chunk; Bp = 64: the one
  // accumulator, drained after every chunk.
  const uint32_t acc = kWide ? 0u : (c & 1);
  const uint32_t drained = kWide ? ((c & 1) ^ 1) : (((c >> 1) & 1) ^ 1);
  if (!ptx::mbar_wait_bounded(gfull, par, lim) || !ptx::mbar_wait_bounded(xfull, par, lim) ||
      (first_kt && !ptx::mbar_wait_bounded(&tempty[acc], drained, lim))) {
    set_abort(abort_flag, P.status);
    return;
  }
  ptx::tc_fence_after();
  const uint32_t idesc = ptx::idesc_bf16_f32(BM, 4 * P.Bp) | (1u << 15);  // A is M-major
  const uint32_t x2_off = (uint32_t)(4 * P.Bp) * 128;  // x2 rows follow the 4Bp rows of x1
  const uint64_t dh = smem_desc_mn_sw128(stage);
  const uint64_t dl = smem_desc_mn_sw128(stage + kTileBytes);
  const uint64_t dx1 = ptx::smem_desc_sw128(stage + 2 * kTileBytes);
  const uint64_t dx2 = ptx::smem_desc_sw128(stage + 2 * kTileBytes + x2_off);
  const uint32_t d_tmem = tbase + acc * kAccStride;
#pragma unroll
  for (int kk = 0; kk < BK / 16; ++kk) {
    const uint64_t adv = (uint64_t)(kk * 32) >> 4;              // x: 16 columns along the row
    const uint64_t adva = (uint64_t)(kk * 2 * kGroupK) >> 4;     // A: two K groups
    ptx::mma_bf16(d_tmem, dh + adva, dx1 + adv, idesc, (!first_kt || kk > 0) ? 1u : 0u);
    ptx::mma_bf16(d_tmem, dh + adva, dx2 + adv, idesc, 1u);
    ptx::mma_bf16(d_tmem, dl + adva, dx1 + adv, idesc, 1u);
  }
  ptx::mma_commit(empty);
  if (last_kt) ptx::mma_commit(&tfull[acc]);
}

// kStallHook: the test hook's instantiation, the only one that reads
// P.stall_load.
// kWide: the Bp = 64 form (one accumulator, the chunk's drain moved to the
// next chunk's first k-tile).
template <bool kWide, bool kStallHook>
__global__ void __launch_bounds__(kThreads, 1)
    fused_kernel(const __grid_constant__ CUtensorMap map_x, const FusedParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t xfull[kStages], gfull[kStages], empty[kStages], tfull[2], tempty[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ int arrivals[kStages];
  __shared__ uint32_t x_last[kStages];  // test hook only: latest x load issued into each stage (k-tile + 1)
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t lim = P.wait_ns;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&xfull[s], 1);
      ptx::mbar_init(&gfull[s], kWarps);
      ptx::mbar_init(&empty[s], 1);
      arrivals[s] = 0;
      x_last[s] = 0u;
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], kWarps);
    }
    ptx::mbar_init(&drain_bar, kWarps);
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
  const bool producer = threadIdx.x == 0;  // also issues the x tiles' TMA loads
  const uint32_t x_tx = (uint32_t)(8 * Bp) * BK * 2;
  uint32_t x_issued = 0;  // x loads issued (producer only)

  const int g = warp;                  // 0..15
  const int quarter = warp & 3;        // TMEM lane quarter this warp may access
  const int rot = g >> 2;              // rotation whose accumulator columns this warp drains
  const int n = P.n;
  const uint32_t un = (uint32_t)n;
  const uint32_t nq = (uint32_t)(n + 1);
  // Lane l generates column 4g + (l % 4) for the pixel du = l / 4 of each of
  // the tile's 16 rows dv: a warp's load then covers 8 neighbouring pixels x
  // 4 neighbouring columns, and columns next to each other in the sorted
  // order often need the same footprint entry for a pixel, so the request
  // touches fewer sectors.
  const int col = g * kCols + (lane & 3);
  const uint32_t du = (uint32_t)(lane >> 2);
  // This lane's 16 values of a k-tile are tile rows 16 sigma(du) + dv of
  // column col: two runs of 8 contiguous bf16 in the M-major layout, in the
  // swizzle atom of rows 64 (sd / 4) .. +63 of K group col / 8, K row col % 8,
  // 16-byte chunk (row % 64) / 8 XOR (col % 8).
  const uint32_t sd = sigma(du), kr = (uint32_t)col & 7u;
  const uint32_t run_base = ((uint32_t)col >> 3) * kGroupK + (sd >> 2) * kAtomMN + kr * 128;
  const uint32_t run_off0 = run_base + (((2u * (sd & 3u)) ^ kr) << 4);
  const uint32_t run_off1 = run_base + (((2u * (sd & 3u) + 1u) ^ kr) << 4);
  uint32_t it = 0, c = 0;
  bool ok = true;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    // Units in order of the M-tile's distance from the image centre: the CTAs
    // of a wave then work on M-tiles at similar radii, whose footprints over a
    // bracket's angles sweep the same annulus of the library (L2 hit rate 88
    // -> 96 % at 512^2).
    const int ks = u / P.m_tiles, mt = P.mt_order[u % P.m_tiles];
    const int k0 = unit_k0(P, ks), k1 = unit_k0(P, ks + 1);
    const int p0 = (mt / P.tiles_q) * kTileH, q0 = (mt % P.tiles_q) * kTileW;
    // Running sums of this warp's rotation and lane quarter in TMEM.
    const uint32_t tsum = tbase + ((uint32_t)(quarter * 32) << 16) + kSumCol + rot * Bp;
    bool first = true;  // the unit's first drain writes the sums instead of adding
    auto drain = [&](uint32_t cc) -> bool {
      const uint32_t acc = kWide ? 0u : (cc & 1);
      if (!warp_wait(&tfull[acc], kWide ? (cc & 1) : ((cc >> 1) & 1), &abort_flag, P.status, lim)) return false;
      ptx::tc_fence_after();
      const uint32_t tacc = tbase + ((uint32_t)(quarter * 32) << 16) + acc * kAccStride + rot * Bp;
#pragma unroll
      for (int qq = 0; qq < (kWide ? 64 : 32) / 16; ++qq) {
        if (qq * 16 < Bp) {
          float v[16], sm[16];
          ptx::tmem_ld16(tacc + qq * 16, v);
          if (!first) ptx::tmem_ld16(tsum + qq * 16, sm);
          ptx::tmem_ld_wait();
          if (!first) {
#pragma unroll
            for (int t = 0; t < 16; ++t) v[t] += sm[t];
          }
          ptx::tmem_st16(tsum + qq * 16, v);
        }
      }
      ptx::tmem_st_wait();
      first = false;
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
      return true;
    };
    // Warps run independently: the stages, the accumulators and the running
    // sums are handed over through mbarriers only.  After a timeout every
    // bounded wait fails at once and each warp leaves for the final drain.
    for (int kc = k0; kc < k1 && ok; kc += kChunk, ++c) {
      const int kc1 = min(kc + kChunk, k1);
      // The loads of a chunk run as one stream: while a k-tile's last rows
      // are finished, the first rows of the next are already being loaded.
      LaneCol L;
      lane_start(P.cols[(int64_t)kc * BK + col], p0, q0, du, L);
      // A k-tile whose footprints are all zero for the whole warp is written
      // as zeros without loading anything.
      bool skip = __all_sync(0xffffffffu, rows_outside(L, un));
      Entry ent[kDepth];
      uint32_t fa[kDepth], fb[kDepth];
      auto issue = [&](int t) {
        const uint32_t qa = (uint32_t)(L.a >> kFixShift), pb = (uint32_t)(L.b >> kFixShift);
        const bool inside = qa <= un && pb <= un;
        const uint32_t idx = inside ? L.off + pb * nq + qa : P.zero_entry;
        ent[t % kDepth] = load_entry(P.plib + 8 * (size_t)idx);
        fa[t % kDepth] = (uint32_t)(L.a >> (kFixShift - 32));
        fb[t % kDepth] = (uint32_t)(L.b >> (kFixShift - 32));
        L.a += L.S2;
        L.b += L.C2;
      };
      if (!skip) {
#pragma unroll
        for (int t = 0; t < kDepth; ++t) issue(t);
      }
      for (int kt = kc; kt < kc1; ++kt, ++it) {
        const bool more = kt + 1 < kc1;
        // The next column's entry, read where its first row is issued.
        const FusedCol *next_col = P.cols + ((int64_t)(kt + 1) * BK + col);
        FusedCol cn;
        const int s = (int)(it % kStages);
        const uint32_t par = (it / kStages) & 1;
        if (!warp_wait_lane0(&empty[s], par ^ 1, &abort_flag, P.status, lim)) {
          ok = false;
          break;
        }
        uint8_t *stage = smem + (size_t)s * P.stage_bytes;
        if (producer && (!kStallHook || (int64_t)it != P.stall_load)) {
          ptx::mbar_arrive_expect_tx(&xfull[s], x_tx);
          ptx::tma_load_2d(stage + 2 * kTileBytes, &map_x, kt * BK, 0, &xfull[s]);
          if (kWide)  // 8 Bp = 512 rows: two boxes of 256
            ptx::tma_load_2d(stage + 2 * kTileBytes + 256 * 128, &map_x, kt * BK, 256, &xfull[s]);
          ++x_issued;
          if (kStallHook) x_last[s] = it + 1;
        }
        const uint32_t st = ptx::smem_u32(stage);
        if (skip) {
          const uint32_t z = 0u;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t ad = st + (h ? run_off1 : run_off0);
            asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(ad), "r"(z));
            asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(ad + kTileBytes), "r"(z));
          }
          if (more) {
            cn = *next_col;
            lane_start(cn, p0, q0, du, L);
            skip = __all_sync(0xffffffffu, rows_outside(L, un));
            if (!skip) {
#pragma unroll
              for (int t = 0; t < kDepth; ++t) issue(kTileH + t);
            }
          }
        } else {
        const float w0 = L.w0, w1 = L.w1;
        const uint32_t st = ptx::smem_u32(stage);
        uint32_t hw[4], lw[4];
        float y_even = 0.f;
        auto finish = [&](int t) {
          const int i = t % kDepth;
          float an, af, bn, bf;
          axis_weights(fa[i], an, af);
          axis_weights(fb[i], bn, bf);
          const uint64_t an2 = f2_pack(an, an), af2 = f2_pack(af, af);
          const uint64_t r0 = fma2(af2, ent[i].t01, mul2(an2, ent[i].t00));  // row p, both PSFs
          const uint64_t r1 = fma2(af2, ent[i].t11, mul2(an2, ent[i].t10));  // row p + 1
          const uint64_t v = fma2(f2_pack(bf, bf), r1, mul2(f2_pack(bn, bn), r0));
          float v0, v1;
          f2_unpack(v, v0, v1);
          const float y = fmaf(w1, v1, w0 * v0);
          if ((t & 1) == 0) {
            y_even = y;
          } else {
            // Rows t - 1 and t as one word each of hi and lo (row t - 1 in the low half).
            uint32_t h2, l2;
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h2) : "f"(y), "f"(y_even));
            const float r_even = y_even - __uint_as_float(h2 << 16);
            const float r_odd = y - __uint_as_float(h2 & 0xFFFF0000u);
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l2) : "f"(r_odd), "f"(r_even));
            hw[(t >> 1) & 3] = h2;
            lw[(t >> 1) & 3] = l2;
          }
          if ((t & 7) == 7) {
            const uint32_t ad = st + ((t >> 3) ? run_off1 : run_off0);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ad), "r"(hw[0]), "r"(hw[1]), "r"(hw[2]),
                         "r"(hw[3]));
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ad + kTileBytes), "r"(lw[0]), "r"(lw[1]),
                         "r"(lw[2]), "r"(lw[3]));
          }
        };
#pragma unroll
        for (int t = 0; t < kTileH; ++t) {
          // Rows t + kDepth >= kTileH belong to the next k-tile's column.
          if (t == kTileH - kDepth && more) {
            cn = *next_col;
            lane_start(cn, p0, q0, du, L);
            skip = __all_sync(0xffffffffu, rows_outside(L, un));
          }
          finish(t);
          if (t + kDepth < kTileH || (more && !skip)) issue(t + kDepth);
        }
        }
        // Bp = 64: the previous chunk's accumulator is drained here, after this
        // chunk's first k-tile is generated and before this warp arrives for
        // it (the first k-tile's MMAs wait for the drain; the generators do not).
        if (kWide && kt == kc && kc > k0 && !drain(c - 1)) {
          ok = false;
          break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&gfull[s]);
          // The warp that completes the stage issues its MMAs (the counter
          // only grows: every use of a stage adds kWarps).
          if ((atomicAdd(&arrivals[s], 1) & (kWarps - 1)) == kWarps - 1) {
            issue_stage_mmas<kWide>(P, stage, &xfull[s], &gfull[s], &empty[s], tfull, tempty, par, c, kt == kc,
                                    kt == kc1 - 1, tbase, &abort_flag);
          }
        }
        __syncwarp();
      }
      if (!kWide && ok && kc > k0 && !drain(c - 1)) ok = false;
    }
    if (ok && !drain(c - 1)) ok = false;
    if (!ok) break;
    // This lane drains tile row 32 quarter + lane = 16 sigma(du) + dv.  The
    // TMEM loads are warp-collective, so every lane takes part; only lanes
    // whose pixel lies inside the image store.
    const int p = p0 + (lane & 15), q = q0 + (int)sigma((uint32_t)(2 * quarter + (lane >> 4)));
    const bool inside = p < n && q < n;
    int pp = p, qp = q;  // P^rot: (p, q) -> (q, n-1-p), applied rot times
    for (int t = 0; t < rot; ++t) {
      const int nxt = qp;
      qp = n - 1 - pp;
      pp = nxt;
    }
    float *out = P.part + ((int64_t)(ks * 4 + rot) * P.B) * P.rows + (int64_t)pp * n + qp;
#pragma unroll
    for (int qq = 0; qq < (kWide ? 64 : 32) / 16; ++qq) {
      if (qq * 16 < Bp) {
        float v[16];
        ptx::tmem_ld16(tsum + qq * 16, v);
        ptx::tmem_ld_wait();
        if (inside) {
#pragma unroll
          for (int t = 0; t < 16; ++t)
            if (qq * 16 + t < P.B) out[(int64_t)(qq * 16 + t) * P.rows] = v[t];
        }
      }
    }
    ptx::tc_fence_before();
  }
  // Drain before the memory is released: every lane that issued MMAs commits
  // them to drain_bar (a thread with none arrives at once), and the copies of
  // x the producer issued land.  Without the test hook the copies alternate
  // between the stages in issue order, so the last kStages issued are the
  // ones to wait for; with it one copy may be missing, and the latest copy
  // issued into each stage is waited for (a stage's earlier copies were
  // consumed by MMAs before it was refilled).
  if (lane == 0) ptx::mma_commit(&drain_bar);
  if (producer) {
    if (kStallHook) {
      for (int st2 = 0; st2 < kStages; ++st2)
        if (x_last[st2] && !ptx::mbar_wait_bounded(&xfull[st2], ((x_last[st2] - 1) / kStages) & 1, lim))
          set_abort(&abort_flag, P.status);
    } else {
      for (uint32_t i = x_issued > (uint32_t)kStages ? x_issued - (uint32_t)kStages : 0u; i < x_issued; ++i)
        if (!ptx::mbar_wait_bounded(&xfull[i % kStages], (i / kStages) & 1, lim)) set_abort(&abort_flag, P.status);
    }
  }
  if (lane == 0 && !ptx::mbar_wait_bounded(&drain_bar, 0, lim)) set_abort(&abort_flag, P.status);
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
  int Bp, KS, m_tiles, k_tiles, tiles_q;
  int64_t rows, ldx;
  uint32_t stage_bytes;
  size_t smem, xs_bytes, part_bytes;
};

FusedPlanInfo fused_info(const psfsim_plan *h, int Bc) {
  FusedPlanInfo f;
  f.Bp = Bc <= 16 ? 16 : (Bc <= 32 ? 32 : 64);
  f.rows = psfsim_round_up(h->M, BM);
  f.tiles_q = (h->n + kTileW - 1) / kTileW;
  f.m_tiles = f.tiles_q * ((h->n + kTileH - 1) / kTileH);
  f.k_tiles = (int)((h->K_valid + BK - 1) / BK);
  if (f.k_tiles < 1) f.k_tiles = 1;
  f.ldx = (int64_t)f.k_tiles * BK;
  // Split over k: the fewest splits whose last wave of units is nearly full.
  f.KS = 1;
  double best = 0.0;
  for (int ks = 1; ks <= 8 && ks <= f.k_tiles; ++ks) {
    const int64_t units = (int64_t)f.m_tiles * ks;
    const int64_t waves = (units + h->num_sms - 1) / h->num_sms;
    const double eff = (double)units / (double)(waves * h->num_sms);
    if (eff > best + 0.02) {
      best = eff;
      f.KS = ks;
    }
  }
  f.stage_bytes = (uint32_t)psfsim_round_up(2 * kTileBytes + 8 * f.Bp * BK * 2, 1024);
  // Two stages: a stage's MMAs take a fraction of the time its generation
  // does, and the shared memory a third stage would take is worth more as
  // L1 cache for the library footprints.
  f.smem = (size_t)kStages * f.stage_bytes + 1024;
  f.xs_bytes = (size_t)psfsim_round_up(8ll * f.Bp * f.ldx * 2, 256);
  f.part_bytes = (size_t)4 * f.KS * Bc * f.rows * 4;
  return f;
}

}  // namespace

int64_t psfsim_pair_library_bytes(int n, int n_r) { return ((int64_t)(n_r - 1) * (n + 1) * (n + 1) + 1) * 32; }

int64_t psfsim_fused_columns_bytes(int64_t K) { return (psfsim_round_up(K, BK) + BK) * (int64_t)sizeof(FusedCol); }

int64_t psfsim_fused_mtile_order_bytes(int n) {
  return (int64_t)((n + kTileW - 1) / kTileW) * ((n + kTileH - 1) / kTileH) * (int64_t)sizeof(int);
}

cudaError_t psfsim_launch_pair_library(psfsim_plan *h, cudaStream_t st) {
  pair_library_kernel<<<h->num_sms * 4, 256, 0, st>>>(h->d_lib, h->n, h->n_r,
                                                      reinterpret_cast<float *>(h->ws + h->plib_off));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tiles_q = (h->n + kTileW - 1) / kTileW, m_tiles = tiles_q * ((h->n + kTileH - 1) / kTileH);
  mtile_order_kernel<<<(m_tiles + 255) / 256, 256, 0, st>>>(h->n, tiles_q, m_tiles,
                                                            reinterpret_cast<int *>(h->ws + h->mtorder_off));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // At least one whole k-tile of entries: a plan with no column inside the
  // last radius still runs one k-tile of padding.
  fused_columns_kernel<<<h->num_sms, 256, 0, st>>>(
      reinterpret_cast<const ColGeom *>(h->ws + h->geom_off), reinterpret_cast<const int *>(h->ws + h->order_off), h->n,
      (uint32_t)((h->n + 1) * (h->n + 1)), h->K_valid, psfsim_round_up(h->K_valid > 0 ? h->K_valid : 1, BK),
      reinterpret_cast<FusedCol *>(h->ws + h->cols_off));
  return cudaGetLastError();
}

size_t psfsim_forward_fused_scratch(const psfsim_plan *h, int B) {
  const int Bc = B < kMaxBp ? B : kMaxBp;
  const FusedPlanInfo f = fused_info(h, Bc);
  return f.xs_bytes + f.part_bytes;
}

// One fused forward per chunk of at most kMaxBp scenes; max_ctas, wait_ns and
// stall_load serve the test hook (all SMs, 2 s and -1 otherwise).
static cudaError_t launch_fused(const psfsim_plan *h, const float *x, int B, float *y, void *scratch, int max_ctas,
                                uint64_t wait_ns, int64_t stall_load, cudaStream_t st) {
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
    // a TMA box holds at most 256 rows; Bp = 64 loads its 512 rows as two boxes
    if (!encode_x_map(&mx, xs, (uint64_t)f.ldx, (uint64_t)(8 * f.Bp), (uint32_t)(8 * f.Bp < 256 ? 8 * f.Bp : 256)))
      return cudaErrorInvalidValue;
    FusedParams P;
    P.n = h->n;
    P.Bp = f.Bp;
    P.B = Bc;
    P.KS = f.KS;
    P.m_tiles = f.m_tiles;
    P.tiles_q = f.tiles_q;
    P.k_tiles = f.k_tiles;
    P.rows = f.rows;
    P.stage_bytes = f.stage_bytes;
    P.zero_entry = (uint32_t)(h->n_r - 1) * (uint32_t)((h->n + 1) * (h->n + 1));
    P.cols = reinterpret_cast<const FusedCol *>(h->ws + h->cols_off);
    P.mt_order = reinterpret_cast<const int *>(h->ws + h->mtorder_off);
    P.plib = reinterpret_cast<const float *>(h->ws + h->plib_off);
    P.part = part;
    P.status = status;
    P.wait_ns = wait_ns;
    P.stall_load = stall_load;
    const bool wide = f.Bp == 64;
    auto kernel = wide ? (stall_load >= 0 ? fused_kernel<true, true> : fused_kernel<true, false>)
                       : (stall_load >= 0 ? fused_kernel<false, true> : fused_kernel<false, false>);
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem)) !=
        cudaSuccess)
      return e;
    const int units = f.m_tiles * f.KS;
    kernel<<<units < max_ctas ? units : max_ctas, kThreads, f.smem, st>>>(mx, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = psfsim_launch_reduce_partials(part, 4 * f.KS, Bc, f.rows, h->M, y + (int64_t)b0 * h->M, nullptr, st)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

cudaError_t psfsim_launch_forward_fused(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                        cudaStream_t st) {
  return launch_fused(h, x, B, y, scratch, h->num_sms, 2000000000ull, -1, st);
}

cudaError_t psfsim_launch_forward_fused_stall(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                              uint64_t wait_ns, int64_t stall_load, cudaStream_t st) {
  return launch_fused(h, x, B, y, scratch, 1, wait_ns, stall_load, st);
}
