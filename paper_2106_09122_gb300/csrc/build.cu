// Library build (Sec. 2): per-column geometry, bracket sort, and the kernels
// that write every column of A = [I_1 ... I_K] (Eq. 4-5).
#include <cudaTypedefs.h>

#include <climits>
#include <cstring>

#include "psfsim_internal.cuh"
#include "ptx_util.cuh"

namespace {

constexpr double kFix = 1099511627776.0;  // 2^PSFSIM_FRAC_BITS
static_assert(PSFSIM_FRAC_BITS == 40, "kFix");

struct GeomParams {
  int n_r, N, interp, quadrant;
  int64_t K;
  double S;
  const double *pts;
  double radii[PSFSIM_MAX_RADII];
};

// a1-a2: field offset (Eq. 2-3), polar angle as x/r, y/r, radial bracket + weight.
__global__ void geom_kernel(const __grid_constant__ GeomParams P, ColGeom *geom) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= P.K) return;
  double x, y;
  if (P.pts) {
    x = P.pts[2 * j];
    y = P.pts[2 * j + 1];
  } else if (P.quadrant) {  // x > 0, y > 0 quadrant of an even N x N grid
    const int H = P.N / 2;
    const int iy = H + (int)(j / H), ix = H + (int)(j % H);
    const double half = 0.5 * (double)(P.N - 1);
    x = __dmul_rn((double)ix - half, P.S);
    y = __dmul_rn((double)iy - half, P.S);
  } else {
    const int iy = (int)(j / P.N), ix = (int)(j % P.N);
    const double half = 0.5 * (double)(P.N - 1);
    x = __dmul_rn((double)ix - half, P.S);
    y = __dmul_rn((double)iy - half, P.S);
  }
  const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = __ddiv_rn(x, r);
    s = __ddiv_rn(y, r);
  }
  ColGeom g;
  {
    const float th = atan2f((float)y, (float)x);  // ordering only
    int bin = (int)((th + 3.14159265f) * (PSFSIM_THETA_BINS / 6.2831853f));
    g.bin = bin < 0 ? 0 : (bin >= PSFSIM_THETA_BINS ? PSFSIM_THETA_BINS - 1 : bin);
  }
  g.C = __double2ll_rn(c * kFix);
  g.Sn = __double2ll_rn(s * kFix);
  if (!(r <= P.radii[P.n_r - 1])) {
    g.k = -1;
    g.w0 = 0.f;
    g.w1 = 0.f;
  } else {
    int lo = 0, hi = P.n_r - 2;  // largest k in [0, n_r-2] with radii[k] <= r
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.radii[mid] <= r) lo = mid; else hi = mid - 1;
    }
    double w = __ddiv_rn(__dsub_rn(r, P.radii[lo]), __dsub_rn(P.radii[lo + 1], P.radii[lo]));
    if (w < 0.0) w = 0.0;
    if (P.interp == PSFSIM_NEAREST) w = (w > 0.5) ? 1.0 : 0.0;
    g.k = lo;
    g.w0 = (float)(1.0 - w);
    g.w1 = (float)w;
  }
  geom[j] = g;
}

__device__ __forceinline__ int column_bucket(const ColGeom &g, int n_r) {
  return g.k < 0 ? psfsim_num_buckets(n_r) - 1 : g.k * PSFSIM_THETA_BINS + g.bin;
}

// Stable counting sort of the columns by (radial bracket, angle bin), zero
// columns last, so that a CTA can stage one bracket pair for many columns and
// neighbouring columns read nearby library pixels.  One CTA; warp w of W takes
// the w-th contiguous chunk of the columns, with its own row of bucket
// counters in shared memory (W x buckets ints): the chunks are counted, every
// bucket's cursor for chunk w starts after the bucket's earlier buckets and
// the bucket's entries of chunks < w, and each warp scatters its chunk in
// index order with match_any ranks.  The order is deterministic: by bucket,
// ties by column index.
__global__ void __launch_bounds__(1024) bracket_sort_kernel(const ColGeom *geom, int64_t K, int n_r, int W,
                                                            int *order, int *bstart) {
  extern __shared__ int cnt[];  // [W][nb]
  const int nb = psfsim_num_buckets(n_r);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < W * nb; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int64_t c0 = K * warp / W, c1 = K * (warp + 1) / W;
  if (warp < W)
    for (int64_t j = c0 + lane; j < c1; j += 32) atomicAdd(&cnt[warp * nb + column_bucket(geom[j], n_r)], 1);
  __syncthreads();
  // Per bucket: its total, then the cursors of the chunks within it.
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int t = 0;
    for (int w = 0; w < W; ++w) {
      const int c = cnt[w * nb + b];
      cnt[w * nb + b] = t;
      t += c;
    }
    bstart[b] = t;  // total for now
  }
  __syncthreads();
  // Bucket starts: exclusive prefix of the totals, in bucket order (one warp).
  if (warp == 0) {
    int run = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const int b = b0 + lane;
      const int v = b < nb ? bstart[b] : 0;
      int x = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (b < nb) bstart[b] = run + x - v;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) bstart[nb] = run;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < W * nb; i += blockDim.x) cnt[i] += bstart[i % nb];
  __syncthreads();
  if (warp < W) {
    int *cur = cnt + warp * nb;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = c0; base < c1; base += 32) {
      const int64_t j = base + lane;
      const int key = j < c1 ? column_bucket(geom[j], n_r) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      int pos0 = 0;
      if (lane == leader && key >= 0) pos0 = cur[key];
      pos0 = __shfl_sync(0xffffffffu, pos0, leader);
      if (key >= 0) order[pos0 + __popc(peers & lt)] = (int)j;
      __syncwarp();
      if (lane == leader && key >= 0) cur[key] = pos0 + __popc(peers);
      __syncwarp();
    }
  }
}

// Within each radial bracket, orders the columns by polar angle (the sine in
// fixed point, increasing over the x > 0, y > 0 quadrant; ties by column
// index, so the order is deterministic).  One CTA per bracket sorts its
// segment of the bracket-sorted list in shared memory (bitonic); a segment
// longer than kAngleSortMax keeps its (bracket, angle bin) order.  Any
// column order gives the same product; this one puts columns of nearly the
// same angle next to each other, so neighbouring columns read nearly the
// same library pixels for a given image pixel.
constexpr int kAngleSortMax = 4096;
__global__ void __launch_bounds__(1024) angle_sort_kernel(const ColGeom *geom, int n_r, int *order,
                                                          const int *bstart) {
  __shared__ long long key[kAngleSortMax];
  __shared__ int val[kAngleSortMax];
  const int k = blockIdx.x;
  const int begin = bstart[k * PSFSIM_THETA_BINS], end = bstart[(k + 1) * PSFSIM_THETA_BINS];
  const int m = end - begin;
  if (m < 2 || m > kAngleSortMax) return;
  int pow2 = 1;
  while (pow2 < m) pow2 <<= 1;
  for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
    if (i < m) {
      const int j = order[begin + i];
      key[i] = geom[j].Sn;
      val[i] = j;
    } else {
      key[i] = LLONG_MAX;
      val[i] = INT_MAX;
    }
  }
  __syncthreads();
  for (int size = 2; size <= pow2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
        const int partner = i ^ stride;
        if (partner > i) {
          const bool up = (i & size) == 0;
          const bool gt = key[i] > key[partner] || (key[i] == key[partner] && val[i] > val[partner]);
          if (gt == up) {
            const long long tk = key[i];
            key[i] = key[partner];
            key[partner] = tk;
            const int tv = val[i];
            val[i] = val[partner];
            val[partner] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) order[begin + i] = val[i];
}

struct BuildParams {
  int n, n_r, Wp, compact;  // compact: column c of the sorted list is stored at position c
  int N;                    // scene side of a grid build (0: field points)
  int64_t K, ld;
  const ColGeom *geom;
  const int *order;
  const int *bstart;
  const float *lib;
  float *A;
  int *status;
};

// One rotated + lerped element (a3-a4).  a2/b2 hold 2a and 2b in fixed point
// with PSFSIM_FRAC_BITS fraction bits; taps come from `tap(psf, row, col)`.
template <typename TapFn>
__device__ __forceinline__ float rotated_value(long long a2, long long b2, int n, float w0, float w1,
                                               TapFn tap) {
  constexpr int kShift = PSFSIM_FRAC_BITS + 1;
  const int q0 = (int)(a2 >> kShift);
  const int p0 = (int)(b2 >> kShift);
  if (q0 < -1 || q0 > n - 1 || p0 < -1 || p0 > n - 1) return 0.f;
  const unsigned fa = (unsigned)((unsigned long long)a2 >> (kShift - 32));
  const unsigned fb = (unsigned)((unsigned long long)b2 >> (kShift - 32));
  constexpr float kInv32 = 2.3283064365386963e-10f;  // 2^-32
  const float wa1 = __uint2float_rn(fa) * kInv32;
  const float wa0 = fa ? __uint2float_rn(0u - fa) * kInv32 : 1.f;
  const float wb1 = __uint2float_rn(fb) * kInv32;
  const float wb0 = fb ? __uint2float_rn(0u - fb) * kInv32 : 1.f;
  float v0 = wb0 * (wa0 * tap(0, p0, q0) + wa1 * tap(0, p0, q0 + 1)) +
             wb1 * (wa0 * tap(0, p0 + 1, q0) + wa1 * tap(0, p0 + 1, q0 + 1));
  float v1 = 0.f;
  if (w1 != 0.f)
    v1 = wb0 * (wa0 * tap(1, p0, q0) + wa1 * tap(1, p0, q0 + 1)) +
         wb1 * (wa0 * tap(1, p0 + 1, q0) + wa1 * tap(1, p0 + 1, q0 + 1));
  return w0 * v0 + w1 * v1;
}

// Writes column j of A (FP32, column-major) with one warp.
template <bool kSmem, bool kVec4>
__device__ __forceinline__ void build_column(const BuildParams &P, int j, int64_t dest, const float *s0,
                                             const float *s1, int lane) {
  const ColGeom g = P.geom[j];
  float *col = P.A + dest * P.ld;
  const int n = P.n;
  const int64_t M = (int64_t)n * n;
  if (g.k < 0) {
    for (int64_t i = lane; i < P.ld; i += 32) col[i] = 0.f;
    return;
  }
  const float *L0 = P.lib + (int64_t)g.k * M;
  const float *L1 = L0 + M;
  const int Wp = P.Wp;
  auto tap = [&](int which, int r, int c) -> float {
    if (kSmem) {
      const float *s = which ? s1 : s0;
      return s[(r + 1) * Wp + (c + 4)];
    } else {
      if (r < 0 || r >= n || c < 0 || c >= n) return 0.f;
      return __ldg((which ? L1 : L0) + r * n + c);
    }
  };
  const long long h = n - 1;
  const long long base = h << PSFSIM_FRAC_BITS;
  if (kVec4) {
    const int n4 = n >> 2;
    int q4 = lane, p = 0;
    while (q4 >= n4) { q4 -= n4; ++p; }
    const int total = (int)(M >> 2);
    for (int f = lane; f < total; f += 32) {
      const int q = q4 << 2;
      long long a2 = base + g.C * (2 * q - h) + g.Sn * (2 * p - h);
      long long b2 = base - g.Sn * (2 * q - h) + g.C * (2 * p - h);
      float4 v;
      v.x = rotated_value(a2, b2, n, g.w0, g.w1, tap);
      a2 += 2 * g.C; b2 -= 2 * g.Sn;
      v.y = rotated_value(a2, b2, n, g.w0, g.w1, tap);
      a2 += 2 * g.C; b2 -= 2 * g.Sn;
      v.z = rotated_value(a2, b2, n, g.w0, g.w1, tap);
      a2 += 2 * g.C; b2 -= 2 * g.Sn;
      v.w = rotated_value(a2, b2, n, g.w0, g.w1, tap);
      __stcs(reinterpret_cast<float4 *>(col + (int64_t)p * n + q), v);
      q4 += 32;
      while (q4 >= n4) { q4 -= n4; ++p; }
    }
  } else {
    for (int64_t i = lane; i < M; i += 32) {
      const int p = (int)(i / n), q = (int)(i % n);
      const long long a2 = base + g.C * (2 * q - h) + g.Sn * (2 * p - h);
      const long long b2 = base - g.Sn * (2 * q - h) + g.C * (2 * p - h);
      col[i] = rotated_value(a2, b2, n, g.w0, g.w1, tap);
    }
  }
  for (int64_t i = M + lane; i < P.ld; i += 32) col[i] = 0.f;
}

// Walks this CTA's contiguous range of the bracket-sorted column list group
// by group (one radial bracket, every angle bin; or the zero columns).  With
// kSmem, a group's bracket pair L[k], L[k+1] (zero-padded by one pixel) is
// staged in shared memory at s0 by one TMA tensor load whenever the bracket
// changes; then work(pos, gend) runs for the group's list positions.  The
// whole CTA calls it (it synchronizes); mbar must be initialised.  A staging
// copy that times out sets PSFSIM_ERR_TIMEOUT and ends the walk.
template <bool kSmem, class GroupWork>
__device__ __forceinline__ void for_each_bracket_group(const CUtensorMap *map, const BuildParams &P, float *s0,
                                                       uint64_t *mbar, GroupWork work) {
  const int64_t begin = P.K * blockIdx.x / gridDim.x;
  const int64_t end = P.K * (blockIdx.x + 1) / gridDim.x;
  const uint32_t tx_bytes = 2u * (uint32_t)((P.n + 2) * P.Wp) * 4u;
  int cur_k = -2;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t pos = begin; pos < end;) {
    const int j0 = P.order[pos];
    const int k = P.geom[j0].k;
    const int group_end = k < 0 ? psfsim_num_buckets(P.n_r) : (k + 1) * PSFSIM_THETA_BINS;
    const int64_t gend = min(end, (int64_t)P.bstart[group_end]);
    if (kSmem && k >= 0 && k != cur_k) {
      __syncthreads();  // every warp is done with the previous pair
      if (threadIdx.x == 0) {
        ptx::mbar_arrive_expect_tx(mbar, tx_bytes);
        ptx::tma_load_3d(s0, map, -4, -1, k, mbar);
      }
      if (!ptx::mbar_wait_bounded(mbar, phase)) failed = true;
      cur_k = k;
      if (__syncthreads_or(failed)) {
        // The copy may still be landing in shared memory: give it one more
        // bounded wait before the CTA exits.
        if (threadIdx.x == 0) {
          ptx::mbar_wait_bounded(mbar, phase);
          atomicExch(P.status, PSFSIM_ERR_TIMEOUT);
        }
        return;
      }
      phase ^= 1u;
    }
    work(pos, gend);
    pos = gend;
  }
}

// Each CTA owns a contiguous range of the bracket-sorted column list; its warps
// build whole columns, one warp per column.
template <bool kSmem, bool kVec4>
__global__ void __launch_bounds__(512) build_fp32_kernel(const __grid_constant__ CUtensorMap map,
                                                         const BuildParams P) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t mbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  float *s0 = smem;
  float *s1 = smem + (P.n + 2) * P.Wp;
  if (kSmem && threadIdx.x == 0) {
    ptx::mbar_init(&mbar, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  for_each_bracket_group<kSmem>(&map, P, s0, &mbar, [&](int64_t pos, int64_t gend) {
    for (int64_t c = pos + warp; c < gend; c += nwarps) {
      const int j = P.order[c];
      build_column<kSmem, kVec4>(P, j, P.compact ? c : (int64_t)j, s0, s1, lane);
    }
  });
}

// Dense FP32 storage of an even N x N grid through the exact quarter-turn
// symmetry: R(ix, iy) = (N-1-iy, ix) on the scene and P(p, q) = (q, n-1-p) on
// the image leave the fixed-point source coordinates unchanged, so column R(j)
// holds at pixel P(i) the bits column j holds at i.  A warp builds one 32 x 32
// pixel block of a column of the x > 0, y > 0 quadrant at a time (in shared
// memory) and writes it to its four turned places, A[P^m(block), R^m(j)]:
// every copy is 32 rows of 32 contiguous floats.
constexpr int kSymBlk = 32, kSymPitch = 33;  // block side; shared pitch (transposed reads without conflicts)

template <bool kSmem>
__device__ __forceinline__ void build_block_sym(const BuildParams &P, int jq, int p0, int q0, const float *s0,
                                                const float *s1, float *blk, int lane) {
  const int N = P.N, n = P.n, H = N / 2;
  const int iy = H + jq / H, ix = H + jq % H;  // quadrant entry jq
  const int64_t j = (int64_t)iy * N + ix;
  float *Am[4] = {P.A + j * P.ld, P.A + ((int64_t)ix * N + (N - 1 - iy)) * P.ld,
                  P.A + ((int64_t)(N - 1 - iy) * N + (N - 1 - ix)) * P.ld, P.A + ((int64_t)(N - 1 - ix) * N + iy) * P.ld};
  const ColGeom g = P.geom[jq];
  __syncwarp();  // the previous block's copies have read the buffer
  if (g.k < 0) {  // beyond the last radius: zeros
    for (int a = 0; a < kSymBlk; ++a) blk[a * kSymPitch + lane] = 0.f;
  } else {
    const int64_t M = (int64_t)n * n;
    const float *L0 = P.lib + (int64_t)g.k * M;
    const float *L1 = L0 + M;
    const int Wp = P.Wp;
    auto tap = [&](int which, int r, int c) -> float {
      if (kSmem) {
        const float *s = which ? s1 : s0;
        return s[(r + 1) * Wp + (c + 4)];
      } else {
        if (r < 0 || r >= n || c < 0 || c >= n) return 0.f;
        return __ldg((which ? L1 : L0) + r * n + c);
      }
    };
    const long long h = n - 1;
    const long long base = h << PSFSIM_FRAC_BITS;
    // lane: pixel column q0 + lane, down the block's 32 rows (exact steps)
    const int q = q0 + lane;
    long long a2 = base + g.C * (2 * q - h) + g.Sn * (2 * p0 - h);
    long long b2 = base - g.Sn * (2 * q - h) + g.C * (2 * p0 - h);
    for (int a = 0; a < kSymBlk; ++a) {
      blk[a * kSymPitch + lane] = rotated_value(a2, b2, n, g.w0, g.w1, tap);
      a2 += 2 * g.Sn;
      b2 += 2 * g.C;
    }
  }
  __syncwarp();
  // Row r of each turned block: m = 0 row p0 + r; m = 1 row q0 + r (source
  // column r, rows reversed); m = 2 row n-1-p0-r (reversed); m = 3 row
  // n-1-q0-r (source column r).  Lane l writes floats 4 (l % 8) .. +3 of row
  // r0 + l / 8, so one 16-byte store instruction covers four rows (the rows
  // are 128-byte aligned: n, p0 and q0 are multiples of 32).
  const int rr = lane >> 3, f = (lane & 7) * 4;
  for (int r0 = 0; r0 < kSymBlk; r0 += 4) {
    const int r = r0 + rr;
    float4 v0, v1, v2, v3;
    float *a0 = &v0.x, *a1 = &v1.x, *a2 = &v2.x, *a3 = &v3.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a0[i] = blk[r * kSymPitch + f + i];
      a1[i] = blk[(kSymBlk - 1 - f - i) * kSymPitch + r];
      a2[i] = blk[r * kSymPitch + (kSymBlk - 1 - f - i)];
      a3[i] = blk[(f + i) * kSymPitch + r];
    }
    __stcs(reinterpret_cast<float4 *>(Am[0] + (int64_t)(p0 + r) * n + q0 + f), v0);
    __stcs(reinterpret_cast<float4 *>(Am[1] + (int64_t)(q0 + r) * n + (n - kSymBlk - p0) + f), v1);
    __stcs(reinterpret_cast<float4 *>(Am[2] + (int64_t)(n - 1 - p0 - r) * n + (n - kSymBlk - q0) + f), v2);
    __stcs(reinterpret_cast<float4 *>(Am[3] + (int64_t)(n - 1 - q0 - r) * n + p0 + f), v3);
  }
}

// As build_fp32_kernel, over the bracket-sorted list of the quadrant's
// columns, in (column, 32 x 32 pixel block) tasks; each warp also owns a
// 32 x 33 float block buffer after the staged pair.
template <bool kSmem>
__global__ void __launch_bounds__(512, 1) build_fp32_sym_kernel(const __grid_constant__ CUtensorMap map,
                                                             const BuildParams P) {
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t mbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int pair_floats = kSmem ? 2 * (P.n + 2) * P.Wp : 0;
  float *s0 = smem;
  float *s1 = smem + (P.n + 2) * P.Wp;
  float *blk = smem + pair_floats + warp * (kSymBlk * kSymPitch);
  if (kSmem && threadIdx.x == 0) {
    ptx::mbar_init(&mbar, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  const int nbq = P.n / kSymBlk, nblocks = nbq * nbq;
  for_each_bracket_group<kSmem>(&map, P, s0, &mbar, [&](int64_t pos, int64_t gend) {
    // the group's tasks, dealt round-robin to the warps
    for (int64_t t = warp; t < (gend - pos) * nblocks; t += nwarps) {
      const int jq = P.order[pos + t / nblocks];
      const int b = (int)(t % nblocks);
      build_block_sym<kSmem>(P, jq, (b / nbq) * kSymBlk, (b % nbq) * kSymBlk, s0, s1, blk, lane);
    }
  });
}

}  // namespace

WsLayout psfsim_layout(int n, int64_t K, int storage, int n_r) {
  WsLayout L{};
  const int64_t M = (int64_t)n * n;
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t at = off;
    off = psfsim_round_up(off + bytes, 256);
    return at;
  };
  L.lo_off = L.scale_off = -1;
  if (storage == PSFSIM_FP32 || storage == PSFSIM_FP32_SYM) {
    L.ld = psfsim_round_up(M, 32);
    // FP32_SYM stores at most the x > 0, y > 0 quadrant's columns.
    L.a_off = take(L.ld * (storage == PSFSIM_FP32_SYM ? (K + 3) / 4 : K) * 4);
  } else if (storage == PSFSIM_SPLIT_BF16 || storage == PSFSIM_BF16 || storage == PSFSIM_SPLIT_BF16_SYM) {
    // SPLIT_BF16_SYM stores at most the x > 0, y > 0 quadrant's columns.
    L.ld = psfsim_round_up(storage == PSFSIM_SPLIT_BF16_SYM ? (K + 3) / 4 : K, 64);
    const int64_t rows = psfsim_round_up(M, 128);
    L.a_off = take(rows * L.ld * 2);
    if (storage != PSFSIM_BF16) L.lo_off = take(rows * L.ld * 2);
    L.scale_off = take(L.ld * 4);
  } else {  // FUSED: nothing but the tables
    L.ld = 0;
    L.a_off = -1;
  }
  L.geom_off = take(K * (int64_t)sizeof(ColGeom));
  L.order_off = take(K * 4);
  L.bstart_off = take((int64_t)(psfsim_num_buckets(PSFSIM_MAX_RADII) + 1) * 4);
  L.pts_off = take(K * 16);
  L.status_off = take(16);
  L.libmax_off = take(PSFSIM_MAX_RADII * 4);
  // FUSED keeps the library as pair entries (both PSFs of a radial bracket,
  // each pixel's 2 x 2 bilinear footprint tap by tap, 32 bytes)
  L.plib_off = storage == PSFSIM_FUSED ? take(psfsim_pair_library_bytes(n, n_r)) : -1;
  // ... and the generators' column table.
  L.cols_off = storage == PSFSIM_FUSED ? take(psfsim_fused_columns_bytes(K)) : -1;
  L.mtorder_off = storage == PSFSIM_FUSED ? take(psfsim_fused_mtile_order_bytes(n)) : -1;
  L.total = off;
  (void)n_r;
  return L;
}

static bool encode_library_map(psfsim_plan *h, int Wp) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int n = h->n;
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)h->n_r};
  cuuint64_t strides[2] = {(cuuint64_t)n * 4, (cuuint64_t)n * n * 4};
  cuuint32_t box[3] = {(cuuint32_t)Wp, (cuuint32_t)(n + 2), 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(&h->lib_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)h->d_lib, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t psfsim_launch_build(psfsim_plan *h, cudaStream_t st) {
  // Dense storage of an even grid is built from the x > 0, y > 0 quadrant's
  // columns, four quarter-turned copies each, so the geometry tables cover
  // the quadrant only (entry (iy - N/2) (N/2) + ix - N/2).  The split builds
  // take no column order.
  const bool dense_split = h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16;
  const bool sym = !h->quadrant && h->N > 0 && h->N % 2 == 0 &&
                   (dense_split || (h->storage == PSFSIM_FP32 && h->n % kSymBlk == 0));
  const int64_t Kg = sym ? h->K / 4 : h->Kg;
  GeomParams G;
  std::memset(&G, 0, sizeof(G));
  G.n_r = h->n_r;
  G.N = h->N;
  G.interp = h->interp;
  G.K = Kg;
  G.S = h->S;
  G.pts = h->N ? nullptr : reinterpret_cast<const double *>(h->ws + h->pts_off);
  G.quadrant = h->quadrant || sym ? 1 : 0;
  for (int i = 0; i < h->n_r; ++i) G.radii[i] = h->radii[i];
  ColGeom *geom = reinterpret_cast<ColGeom *>(h->ws + h->geom_off);
  int *order = reinterpret_cast<int *>(h->ws + h->order_off);
  int *bstart = reinterpret_cast<int *>(h->ws + h->bstart_off);
  int *status = reinterpret_cast<int *>(h->ws + h->status_off);
  cudaError_t e = cudaMemsetAsync(status, 0, 16, st);
  if (e != cudaSuccess) return e;
  geom_kernel<<<(unsigned)((Kg + 255) / 256), 256, 0, st>>>(G, geom);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!(sym && dense_split)) {
    // chunks of at least 256 columns, and as many as fit in shared memory
    const int nb = psfsim_num_buckets(h->n_r);
    int W = (int)((Kg + 255) / 256);
    const int fit = (int)((200 * 1024) / ((size_t)nb * sizeof(int)));
    W = W < 1 ? 1 : (W > 32 ? 32 : W);
    W = W > fit ? fit : W;
    const size_t smem = (size_t)W * nb * sizeof(int);
    if ((e = cudaFuncSetAttribute(bracket_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    bracket_sort_kernel<<<1, 1024, smem, st>>>(geom, Kg, h->n_r, W, order, bstart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (h->quadrant) {
    // The host needs the number of columns inside the last radius to size launches.
    int kv = 0;
    if ((e = cudaMemcpyAsync(&kv, bstart + psfsim_num_buckets(h->n_r) - 1, sizeof(int), cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return e;
    h->K_valid = kv;
    if (h->storage == PSFSIM_FUSED) {
      angle_sort_kernel<<<h->n_r - 1, 1024, 0, st>>>(geom, h->n_r, order, bstart);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      return psfsim_launch_pair_library(h, st);
    }
    // Compact split-BF16 rows hold just the valid columns (the layout reserved
    // the whole quadrant, an upper bound, before the count was known).
    if (h->storage == PSFSIM_SPLIT_BF16_SYM) h->ld = psfsim_round_up(kv > 0 ? kv : 1, 64);
  }
  if (h->storage == PSFSIM_SPLIT_BF16 || h->storage == PSFSIM_BF16 || h->storage == PSFSIM_SPLIT_BF16_SYM)
    return psfsim_launch_split_build(h, st);
  if (h->storage != PSFSIM_FP32 && h->storage != PSFSIM_FP32_SYM) return cudaErrorNotSupported;
  const bool compact = h->storage == PSFSIM_FP32_SYM;

  const int n = h->n;
  const int Wp = (int)psfsim_round_up(n, 4) + 8;
  const size_t smem = 2ull * (size_t)(n + 2) * Wp * 4;
  const bool vec4 = (n % 4) == 0;
  const bool use_smem = vec4 && smem <= 200 * 1024 && Wp <= 256 && encode_library_map(h, Wp);
  BuildParams P;
  P.n = n;
  P.n_r = h->n_r;
  P.Wp = Wp;
  P.compact = compact ? 1 : 0;
  P.N = h->N;
  P.K = compact ? h->K_valid : h->K;
  P.ld = h->ld;
  P.geom = geom;
  P.order = order;
  P.bstart = bstart;
  P.lib = h->d_lib;
  P.A = reinterpret_cast<float *>(h->ws + h->a_off);
  P.status = status;
  CUtensorMap dummy;
  std::memset(&dummy, 0, sizeof(dummy));
  int threads = 512, per_sm = 1;
  if (sym) {
    // Even grid: the quadrant's columns (the sorted list holds just those),
    // four turned copies each.
    P.K = Kg;
    const size_t blk_bytes = 16ull * kSymBlk * kSymPitch * 4;  // 16 warps
    const bool staged = use_smem && smem + blk_bytes <= 220 * 1024;
    const size_t total = (staged ? smem : 0) + blk_bytes;
    auto kern = staged ? build_fp32_sym_kernel<true> : build_fp32_sym_kernel<false>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, total)) != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    kern<<<h->num_sms * per_sm, 512, total, st>>>(staged ? h->lib_map : dummy, P);
    return cudaGetLastError();
  }
  if (use_smem) {
    threads = smem > 100 * 1024 ? 512 : 256;
    auto kern = build_fp32_kernel<true, true>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess)
      return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    kern<<<h->num_sms * per_sm, threads, smem, st>>>(h->lib_map, P);
  } else {
    threads = 256;
    per_sm = 8;
    if (vec4)
      build_fp32_kernel<false, true><<<h->num_sms * per_sm, threads, 0, st>>>(dummy, P);
    else
      build_fp32_kernel<false, false><<<h->num_sms * per_sm, threads, 0, st>>>(dummy, P);
  }
  return cudaGetLastError();
}
