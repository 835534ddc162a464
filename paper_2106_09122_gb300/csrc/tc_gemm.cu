// Batched S = A Z (Eq. 6) on the 5th-generation tensor cores for split-BF16
// (and BF16) A.
//
// Y[b, i] = sum_j sigma_j (hi_ij + lo_ij) x_bj.  The scene batch is scaled by
// sigma_j and split exactly into three bf16 parts x' = x1 + x2 + x3 (24 bits),
// stacked as the rows of one MMA B operand, so each k-step issues two MMAs:
//   D[:, 0:3Bp] += hi * [x1 x2 x3]^T     D[:, 0:2Bp] += lo * [x1 x2]^T
// and the epilogue sums the three column blocks: (hi + lo)(x1 + x2) + hi x3,
// i.e. only the lo * x3 term (< 2^-24 relative) is dropped; what remains is
// the 2^-17 relative storage error of hi + lo and the FP32 accumulation.
// BF16 storage has no lo: one MMA per k-step over two x parts,
// D[:, 0:2Bp] += hi * [x1 x2]^T, so the result carries the 2^-8 relative
// storage error of hi and the dropped hi * x3 term (< 2^-16 relative).
//
// Persistent warp-specialised kernel, one CTA per SM:
//   warp 0  TMA producer (2D tiled loads, 128-byte swizzle) into a smem ring
//   warp 1  MMA issuer (tcgen05.mma, accumulators in TMEM, double-buffered)
//   warps 2-5 epilogue (tcgen05.ld -> FP32 sums -> partial images)
// Work unit = (128-row m-tile, k-range); k is split KS ways for balance and
// the KS partial images are summed in a fixed order (deterministic).
// Every mbarrier wait is bounded; a timeout sets PSFSIM_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "psfsim_internal.cuh"
#include "ptx_util.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kMaxStages = 8;
constexpr int kThreads = 192;
// TMEM per CTA: two accumulators of up to 256 columns (one CTA per SM), or,
// when every accumulator fits in 128 columns (BF16 storage, 64 scenes or
// fewer), two of 128 so that two CTAs, two load/MMA pipelines, share an SM.
constexpr uint32_t kTmemColsWide = 512, kAccStrideWide = 256;
constexpr uint32_t kTmemColsNarrow = 256, kAccStrideNarrow = 128;
constexpr uint32_t kTileBytes = BM * BK * 2;
constexpr int kMaxBp = 80;       // 3 * Bp <= 256 (MMA N and TMA box limits), Bp % 16 == 0
constexpr int kMaxJobs = 16;
constexpr int kDefaultChunk = 4; // k-tiles (of 64) per TMEM accumulation, split-BF16 storage
constexpr int kDefaultChunkHiMulti = 2;  // BF16 storage (hi alone), several jobs in one launch
constexpr int kMaxMmas = 64;     // accumulating MMAs between drains (bounds the FP32 drift)

// One product S_j = A_j Z_j of a (possibly multi-job) launch.
struct TcJob {
  int64_t rows, M;
  int Bp, KS, m_tiles, k_tiles;
  int has_lo;          // split-BF16 (hi + lo) or BF16 (hi alone)
  int xparts;          // bf16 parts of x in the B operand: 3 (split-BF16) or 2 (BF16)
  int unit_begin;      // first work unit of this job
  int cap;             // scenes in the job's buffers (<= Bp)
  const int *count;    // device int: scenes present (NULL: all cap)
  float *part;         // [KS][cap][rows]
};

// Kernel parameter block: tensor maps (hi, lo, x) and geometry of every job.
struct TcMulti {
  CUtensorMap map[kMaxJobs][3];
  TcJob job[kMaxJobs];
  int njobs, units, stages, chunk;
  uint32_t stage_bytes;
  uint32_t x_off;  // byte offset of the x tile in a stage: after hi and lo, or after hi alone
  int interleave;  // jobs share one A and one unit count: unit u is job u % njobs, unit u / njobs
  uint32_t tmem_cols, acc_stride;
  int *status;
  uint64_t wait_ns;  // limit of every bounded wait
  int64_t stall_it;  // test hook: the producer never issues this load (-1: none)
};

__global__ void xsplit_kernel(const float *__restrict__ x, int B, const int *__restrict__ count, int Bp, int64_t K,
                              int64_t ld, const float *__restrict__ scale, __nv_bfloat16 *__restrict__ xs) {
  const int64_t total = (int64_t)Bp * ld;
  const int nb = count ? min(*count, B) : B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / ld);
    const int64_t j = t % ld;
    const float v = (b < nb && j < K) ? x[(int64_t)b * K + j] * scale[j] : 0.f;
    const __nv_bfloat16 x1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(x1);
    const __nv_bfloat16 x2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(x2);
    xs[t] = x1;
    xs[total + t] = x2;
    xs[2 * total + t] = __float2bfloat16_rn(r2);
  }
}

__device__ __forceinline__ void set_abort(volatile int *abort_flag, int *status) {
  *abort_flag = 1;
  atomicExch(status, PSFSIM_ERR_TIMEOUT);
}

__device__ __forceinline__ int find_job(const TcMulti &P, int u) {
  int j = 0;
  while (j + 1 < P.njobs && u >= P.job[j + 1].unit_begin) ++j;
  return j;
}

// Work unit u -> (job, unit within the job).  Interleaved jobs (several scene
// blocks against one A) put the same (m-tile, k-range) of every job on
// neighbouring units, so CTAs running together read the same A tiles and L2
// serves all but the first read.
__device__ __forceinline__ void unit_of(const TcMulti &P, int u, int &jb, int &lu) {
  if (P.interleave) {
    jb = u % P.njobs;
    lu = u / P.njobs;
  } else {
    jb = find_job(P, u);
    lu = u - P.job[jb].unit_begin;
  }
}

__device__ __forceinline__ int k_begin(const TcJob &J, int ks) { return (int)((int64_t)J.k_tiles * ks / J.KS); }

__global__ void __launch_bounds__(kThreads, 2) tc_gemm_kernel(const __grid_constant__ TcMulti P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tfull_bar[2], tempty_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t lim = P.wait_ns;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      ptx::mbar_init(&full_bar[s], 1);
      ptx::mbar_init(&empty_bar[s], 1);
    }
    ptx::mbar_init(&drain_bar, 1);
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull_bar[a], 1);
      ptx::mbar_init(&tempty_bar[a], 4);
    }
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(&tmem_base_sh, P.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t it = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < P.units && ok && !abort_flag; u += gridDim.x) {
      int jb, lu;
      unit_of(P, u, jb, lu);
      const TcJob &J = P.job[jb];
      const int ks = lu / J.m_tiles, mt = lu % J.m_tiles;
      const uint32_t tx = (J.has_lo ? 2 : 1) * kTileBytes + (uint32_t)(J.xparts * J.Bp) * BK * 2;
      for (int kt = k_begin(J, ks); kt < k_begin(J, ks + 1); ++kt, ++it) {
        const int s = (int)(it % P.stages);
        if (!ptx::mbar_wait_bounded(&empty_bar[s], ((it / P.stages) & 1) ^ 1, lim)) {
          set_abort(&abort_flag, P.status);
          ok = false;
          break;
        }
        if ((int64_t)it == P.stall_it) continue;  // test hook: this stage is never filled
        uint8_t *st = smem + (size_t)s * P.stage_bytes;
        ptx::mbar_arrive_expect_tx(&full_bar[s], tx);
        ptx::tma_load_2d(st, &P.map[jb][0], kt * BK, mt * BM, &full_bar[s]);
        if (J.has_lo) ptx::tma_load_2d(st + kTileBytes, &P.map[jb][1], kt * BK, mt * BM, &full_bar[s]);
        ptx::tma_load_2d(st + P.x_off, &P.map[jb][2], kt * BK, 0, &full_bar[s]);
      }
    }
    // Drain: the last `stages` loads issued may not have been consumed (after
    // a timeout the MMA issuer stops early); wait for each to land so that no
    // copy into this CTA's shared memory is in flight when the CTA exits.
    // Nothing re-armed these stages afterwards, so their phases are final.
    for (uint32_t i = it > (uint32_t)P.stages ? it - (uint32_t)P.stages : 0u; i < it; ++i)
      if ((int64_t)i != P.stall_it && !ptx::mbar_wait_bounded(&full_bar[i % P.stages], (i / P.stages) & 1, lim))
        set_abort(&abort_flag, P.status);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    uint32_t it = 0, c = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < P.units && ok && !abort_flag; u += gridDim.x) {
      int jb, lu;
      unit_of(P, u, jb, lu);
      const TcJob &J = P.job[jb];
      const int ks = lu / J.m_tiles;
      const int k0 = k_begin(J, ks), k1 = k_begin(J, ks + 1);
      const uint32_t idesc3 = ptx::idesc_bf16_f32(BM, J.xparts * J.Bp);
      const uint32_t idesc2 = ptx::idesc_bf16_f32(BM, 2 * J.Bp);
      const bool has_lo = J.has_lo != 0;
      for (int kc = k0; kc < k1 && ok; kc += P.chunk, ++c) {
        const int kc1 = min(kc + P.chunk, k1);
        const uint32_t acc = c & 1;
        if (!ptx::mbar_wait_bounded(&tempty_bar[acc], ((c >> 1) & 1) ^ 1, lim)) {
          set_abort(&abort_flag, P.status);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tbase + acc * P.acc_stride;
        for (int kt = kc; kt < kc1; ++kt, ++it) {
          const int s = (int)(it % P.stages);
          if (!ptx::mbar_wait_bounded(&full_bar[s], (it / P.stages) & 1, lim)) {
            set_abort(&abort_flag, P.status);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint8_t *st = smem + (size_t)s * P.stage_bytes;
          const uint64_t dh = ptx::smem_desc_sw128(st);
          const uint64_t dl = ptx::smem_desc_sw128(st + kTileBytes);
          const uint64_t dx = ptx::smem_desc_sw128(st + P.x_off);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
            ptx::mma_bf16(d_tmem, dh + adv, dx + adv, idesc3, (kt > kc || kk > 0) ? 1u : 0u);
            if (has_lo) ptx::mma_bf16(d_tmem, dl + adv, dx + adv, idesc2, 1u);
          }
          ptx::mma_commit(&empty_bar[s]);
        }
        if (ok) ptx::mma_commit(&tfull_bar[acc]);
      }
    }
    // Drain: wait until every MMA this thread issued has completed, so that
    // none still reads shared memory or writes TMEM when the CTA releases them.
    ptx::mma_commit(&drain_bar);
    if (!ptx::mbar_wait_bounded(&drain_bar, 0, lim)) set_abort(&abort_flag, P.status);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    // The tensor core's FP32 accumulation is not rounded to nearest, so its
    // error grows with the number of accumulating MMAs.  Each accumulator
    // therefore holds at most P.chunk k-tiles; the epilogue drains it into
    // FP32 register sums and hands it back (double-buffered).
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    uint32_t c = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
      int jb, lu;
      unit_of(P, u, jb, lu);
      const TcJob &J = P.job[jb];
      const int ks = lu / J.m_tiles, mt = lu % J.m_tiles;
      const int k0 = k_begin(J, ks), k1 = k_begin(J, ks + 1);
      const int Bp = J.Bp;
      const bool third = J.xparts == 3;
      float sum[kMaxBp];
#pragma unroll
      for (int t = 0; t < kMaxBp; ++t) sum[t] = 0.f;
      for (int kc = k0; kc < k1; kc += P.chunk, ++c) {
        // Lane 0 alone takes the bounded wait and the abort decision, so the
        // warp stays converged for the .sync.aligned TMEM loads below.
        const uint32_t acc = c & 1;
        int good = 0;
        if (lane == 0) {
          good = !abort_flag && ptx::mbar_wait_bounded(&tfull_bar[acc], (c >> 1) & 1, lim);
          if (!good) set_abort(&abort_flag, P.status);
        }
        good = __shfl_sync(0xffffffffu, good, 0);
        if (!good) {
          ok = false;
          break;
        }
        // Already complete (lane 0 saw it): this gives every lane its acquire.
        if (!ptx::mbar_wait_bounded(&tfull_bar[acc], (c >> 1) & 1, lim)) set_abort(&abort_flag, P.status);
        ptx::tc_fence_after();
        const uint32_t tacc = tbase + ((uint32_t)(quarter * 32) << 16) + acc * P.acc_stride;
#pragma unroll
        for (int q = 0; q < kMaxBp / 16; ++q) {
          if (q * 16 < Bp) {
            float v0[16], v1[16], v2[16];
            ptx::tmem_ld16(tacc + q * 16, v0);
            ptx::tmem_ld16(tacc + Bp + q * 16, v1);
            if (third) ptx::tmem_ld16(tacc + 2 * Bp + q * 16, v2);
            ptx::tmem_ld_wait();
            if (third) {
#pragma unroll
              for (int t = 0; t < 16; ++t) sum[q * 16 + t] += (v0[t] + v1[t]) + v2[t];
            } else {
#pragma unroll
              for (int t = 0; t < 16; ++t) sum[q * 16 + t] += v0[t] + v1[t];
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&tempty_bar[acc]);
      }
      if (!ok) break;
      const int nb = J.count ? min(*J.count, J.cap) : J.cap;
      float *out = J.part + (int64_t)ks * J.cap * J.rows + (int64_t)mt * BM + row;
#pragma unroll
      for (int t = 0; t < kMaxBp; ++t)
        if (t < nb) out[(int64_t)t * J.rows] = sum[t];
    }
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tbase, P.tmem_cols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

bool encode_bf16_2d(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                    uint32_t box_outer) {
  auto encode = get_encoder();
  if (!encode) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// Split factor over k: smallest KS whose unit count fills the SMs evenly.
int choose_ks(int m_tiles, int k_tiles, int num_sms) {
  int best = 1;
  double best_eff = 0.0;
  for (int ks = 1; ks <= 64 && ks <= k_tiles; ++ks) {
    const int64_t units = (int64_t)m_tiles * ks;
    const int64_t waves = (units + num_sms - 1) / num_sms;
    const double eff = (double)units / (double)(waves * num_sms);
    const bool enough = units >= 2 * num_sms || ks == k_tiles;
    if (eff > best_eff + 1e-9 && (enough || eff > best_eff + 0.05)) {
      best = ks;
      best_eff = eff;
    }
    if (enough && eff >= 0.97) return ks;
  }
  return best;
}

struct JobSpec {
  const psfsim_plan *h;
  const float *x;
  float *y;
  int cap;
  const int *count;
};

struct JobPlan {
  int Bp, KS, m_tiles, k_tiles;
  int64_t rows;
  size_t xs_off, part_off;
};

struct MultiPlan {
  JobPlan jp[kMaxJobs];
  int njobs, units, stages, chunk, ctas_per_sm;
  uint32_t stage_bytes, x_off, tmem_cols, acc_stride;
  size_t smem, scratch;
};

// Tile/launch shape of a multi-job product.  `tune` fields of 0 take defaults:
// chunk = kDefaultChunk k-tiles per TMEM accumulation; without lo, the most
// that fit for one job and kDefaultChunkHiMulti for several (the fastest
// measured on one 128^2 job and on eight 256^2 jobs); split factors chosen so
// that the whole launch has about units_per_sm work units per SM (or, for a
// single job without tuning, the smallest split that fills the SMs evenly);
// as many smem stages as fit.
MultiPlan plan_multi(const JobSpec *jobs, int nj, const psfsim_tuning_t *tune) {
  MultiPlan mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.njobs = nj;
  const int num_sms = jobs[0].h->num_sms;
  const int ups = tune && tune->units_per_sm > 0 ? tune->units_per_sm : 0;
  int64_t total = 0;
  for (int j = 0; j < nj; ++j) {
    const psfsim_plan *h = jobs[j].h;
    JobPlan &p = mp.jp[j];
    p.Bp = (int)psfsim_round_up(jobs[j].cap, 16);
    p.rows = psfsim_round_up(h->M, BM);
    p.m_tiles = (int)(p.rows / BM);
    p.k_tiles = (int)(h->ld / BK);
    total += (int64_t)p.m_tiles * p.k_tiles;
  }
  const int64_t target_units = (int64_t)(ups ? ups : 4) * num_sms;
  const int64_t per_unit = (total + target_units - 1) / target_units;
  int Bp_max = 16, units = 0;
  size_t off = 0;
  for (int j = 0; j < nj; ++j) {
    JobPlan &p = mp.jp[j];
    if (nj == 1 && !ups) {
      p.KS = choose_ks(p.m_tiles, p.k_tiles, num_sms);
    } else {
      int ks = (int)((p.k_tiles + per_unit - 1) / (per_unit > 0 ? per_unit : 1));
      ks = ks < 1 ? 1 : ks;
      ks = ks > 64 ? 64 : ks;
      p.KS = ks > p.k_tiles ? p.k_tiles : ks;
    }
    units += p.m_tiles * p.KS;
    Bp_max = p.Bp > Bp_max ? p.Bp : Bp_max;
    const psfsim_plan *h = jobs[j].h;
    p.xs_off = off;
    off += (size_t)psfsim_round_up(3ll * p.Bp * h->ld * 2, 256);
    p.part_off = off;
    off += (size_t)psfsim_round_up((int64_t)p.KS * jobs[j].cap * p.rows * 4, 256);
  }
  mp.units = units;
  mp.scratch = off;
  // A stage holds hi, lo (when any job has one) and the x tile; without lo
  // the stage is smaller, so more stages (bytes in flight) fit.
  bool any_lo = false;
  int x_rows = 0;  // largest B operand: x parts x Bp
  for (int j = 0; j < nj; ++j) {
    const bool lo = jobs[j].h->lo_off >= 0;
    any_lo = any_lo || lo;
    const int r = (lo ? 3 : 2) * mp.jp[j].Bp;
    x_rows = r > x_rows ? r : x_rows;
  }
  mp.x_off = (any_lo ? 2 : 1) * kTileBytes;
  mp.stage_bytes = (uint32_t)psfsim_round_up(mp.x_off + (int64_t)x_rows * BK * 2, 1024);
  // Accumulators of at most 128 columns: two CTAs per SM, each with half the
  // shared memory and half the tensor memory.
  const bool narrow = x_rows <= (int)kAccStrideNarrow;
  mp.ctas_per_sm = narrow ? 2 : 1;
  mp.tmem_cols = narrow ? kTmemColsNarrow : kTmemColsWide;
  mp.acc_stride = narrow ? kAccStrideNarrow : kAccStrideWide;
  int fit = (int)(((narrow ? 108 : 220) * 1024) / mp.stage_bytes);
  fit = fit > kMaxStages ? kMaxStages : fit;
  mp.stages = tune && tune->stages >= 2 && tune->stages < fit ? tune->stages : fit;
  // A k-tile is 4 MMAs per accumulator (8 with lo), so at most 16 (8) k-tiles
  // accumulate between drains.
  const int max_chunk = kMaxMmas / ((any_lo ? 2 : 1) * (BK / 16));
  mp.chunk = tune && tune->chunk > 0 ? (tune->chunk > max_chunk ? max_chunk : tune->chunk)
                                     : (any_lo ? kDefaultChunk : (nj > 1 ? kDefaultChunkHiMulti : max_chunk));
  mp.smem = (size_t)mp.stages * mp.stage_bytes + 1024;
  return mp;
}

// Test hook of a launch: a short wait limit, one load the producer never
// issues, and a single CTA (see psfsim_debug_forward_stall).
struct StallHook {
  uint64_t wait_ns;
  int64_t stall_it;
  bool one_cta;
};
constexpr StallHook kNoStall = {2000000000ull, -1, false};

cudaError_t launch_multi(const JobSpec *jobs, int nj, const MultiPlan &mp, void *scratch, cudaStream_t st,
                         const StallHook &hook = kNoStall) {
  char *base = static_cast<char *>(scratch);
  cudaError_t e;
  TcMulti P;  // kernel parameter block, copied at launch
  std::memset(&P, 0, sizeof(P));
  for (int j = 0; j < nj; ++j) {
    const psfsim_plan *h = jobs[j].h;
    const JobPlan &p = mp.jp[j];
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(base + p.xs_off);
    const float *scale = reinterpret_cast<const float *>(h->ws + h->scale_off);
    xsplit_kernel<<<h->num_sms * 4, 256, 0, st>>>(jobs[j].x, jobs[j].cap, jobs[j].count, p.Bp, psfsim_cols(h), h->ld,
                                                  scale,
                                                  xs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool has_lo = h->lo_off >= 0;
    if (!encode_bf16_2d(&P.map[j][0], h->ws + h->a_off, (uint64_t)h->ld, (uint64_t)p.rows, BK, BM) ||
        (has_lo && !encode_bf16_2d(&P.map[j][1], h->ws + h->lo_off, (uint64_t)h->ld, (uint64_t)p.rows, BK, BM)) ||
        !encode_bf16_2d(&P.map[j][2], xs, (uint64_t)h->ld, (uint64_t)(3 * p.Bp), BK,
                        (uint32_t)((has_lo ? 3 : 2) * p.Bp)))
      return cudaErrorInvalidValue;
    TcJob &J = P.job[j];
    J.has_lo = has_lo ? 1 : 0;
    J.xparts = has_lo ? 3 : 2;
    J.rows = p.rows;
    J.M = h->M;
    J.Bp = p.Bp;
    J.KS = p.KS;
    J.m_tiles = p.m_tiles;
    J.k_tiles = p.k_tiles;
    J.unit_begin = j == 0 ? 0 : P.job[j - 1].unit_begin + P.job[j - 1].m_tiles * P.job[j - 1].KS;
    J.cap = jobs[j].cap;
    J.count = jobs[j].count;
    J.part = reinterpret_cast<float *>(base + p.part_off);
  }
  P.njobs = nj;
  P.units = mp.units;
  bool same = nj > 1;
  for (int j = 1; j < nj; ++j)
    same = same && jobs[j].h == jobs[0].h &&
           mp.jp[j].m_tiles * mp.jp[j].KS == mp.jp[0].m_tiles * mp.jp[0].KS;
  P.interleave = same ? 1 : 0;
  P.tmem_cols = mp.tmem_cols;
  P.acc_stride = mp.acc_stride;
  P.stages = mp.stages;
  P.chunk = mp.chunk;
  P.stage_bytes = mp.stage_bytes;
  P.x_off = mp.x_off;
  P.status = reinterpret_cast<int *>(jobs[0].h->ws + jobs[0].h->status_off);
  P.wait_ns = hook.wait_ns;
  P.stall_it = hook.stall_it;
  if ((e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mp.smem)) !=
      cudaSuccess)
    return e;
  const int num_sms = jobs[0].h->num_sms;
  const int slots = hook.one_cta ? 1 : num_sms * mp.ctas_per_sm;
  tc_gemm_kernel<<<mp.units < slots ? mp.units : slots, kThreads, mp.smem, st>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int j = 0; j < nj; ++j) {
    const JobPlan &p = mp.jp[j];
    if ((e = psfsim_launch_reduce_partials(reinterpret_cast<float *>(base + p.part_off), p.KS, jobs[j].cap, p.rows,
                                           jobs[j].h->M, jobs[j].y, jobs[j].count, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace

namespace {

// A batch of B scenes against one plan as jobs of at most kMaxBp scenes (at
// most kMaxJobs of them), run by one interleaved persistent launch.
int tc_jobs(const psfsim_plan *h, const float *x, int B, float *y, JobSpec *js) {
  const int64_t cols = psfsim_cols(h);
  int nj = 0;
  for (int b0 = 0; b0 < B && nj < kMaxJobs; b0 += kMaxBp, ++nj) {
    const int c = (B - b0) < kMaxBp ? (B - b0) : kMaxBp;
    js[nj] = JobSpec{h, x ? x + (int64_t)b0 * cols : nullptr, y ? y + (int64_t)b0 * h->M : nullptr, c, nullptr};
  }
  return nj;
}

constexpr int kMaxLaunchScenes = kMaxJobs * kMaxBp;

}  // namespace

size_t psfsim_forward_tc_scratch(const psfsim_plan *h, int B) {
  JobSpec js[kMaxJobs];
  const int nj = tc_jobs(h, nullptr, B < kMaxLaunchScenes ? B : kMaxLaunchScenes, nullptr, js);
  return plan_multi(js, nj, nullptr).scratch;
}

cudaError_t psfsim_launch_forward_tc(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                     cudaStream_t st) {
  for (int b0 = 0; b0 < B; b0 += kMaxLaunchScenes) {
    const int Bc = (B - b0) < kMaxLaunchScenes ? (B - b0) : kMaxLaunchScenes;
    JobSpec js[kMaxJobs];
    const int nj = tc_jobs(h, x + (int64_t)b0 * psfsim_cols(h), Bc, y + (int64_t)b0 * h->M, js);
    const MultiPlan mp = plan_multi(js, nj, nullptr);
    cudaError_t e = launch_multi(js, nj, mp, scratch, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int psfsim_multi_validate(const psfsim_job_t *jobs, int njobs) {
  if (!jobs || njobs < 1 || njobs > kMaxJobs) return PSFSIM_ERR_ARG;
  for (int j = 0; j < njobs; ++j) {
    const psfsim_plan *h = jobs[j].plan;
    if (!h || !jobs[j].d_x || !jobs[j].d_y || jobs[j].capacity < 1 || jobs[j].capacity > kMaxBp)
      return PSFSIM_ERR_ARG;
    if (h->storage != PSFSIM_SPLIT_BF16 && h->storage != PSFSIM_BF16) return PSFSIM_ERR_UNSUPPORTED;
    if (h->device != jobs[0].plan->device) return PSFSIM_ERR_ARG;
  }
  return PSFSIM_OK;
}

size_t psfsim_forward_multi_scratch(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tune) {
  JobSpec js[kMaxJobs];
  for (int j = 0; j < njobs; ++j) js[j] = JobSpec{jobs[j].plan, jobs[j].d_x, jobs[j].d_y, jobs[j].capacity, jobs[j].d_count};
  return plan_multi(js, njobs, tune).scratch;
}

cudaError_t psfsim_launch_forward_multi(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tune,
                                        void *scratch, cudaStream_t st) {
  JobSpec js[kMaxJobs];
  for (int j = 0; j < njobs; ++j) js[j] = JobSpec{jobs[j].plan, jobs[j].d_x, jobs[j].d_y, jobs[j].capacity, jobs[j].d_count};
  return launch_multi(js, njobs, plan_multi(js, njobs, tune), scratch, st);
}

cudaError_t psfsim_launch_forward_tc_stall(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                           uint64_t wait_ns, int64_t stall_it, cudaStream_t st) {
  JobSpec js[kMaxJobs];
  const int nj = tc_jobs(h, x, B, y, js);
  if (nj != 1) return cudaErrorInvalidValue;
  const StallHook hook = {wait_ns, stall_it, true};
  return launch_multi(js, nj, plan_multi(js, nj, nullptr), scratch, st, hook);
}
