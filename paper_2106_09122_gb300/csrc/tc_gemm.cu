// Batched S = A Z (Eq. 6) on the 5th-generation tensor cores for split-BF16 A.
//
// Y[b, i] = sum_j sigma_j (hi_ij + lo_ij) x_bj.  The scene batch is scaled by
// sigma_j and split exactly into three bf16 parts x' = x1 + x2 + x3 (24 bits),
// stacked as the rows of one MMA B operand, so each k-step issues two MMAs:
//   D[:, 0:3Bp] += hi * [x1 x2 x3]^T     D[:, 0:2Bp] += lo * [x1 x2]^T
// and the epilogue sums the three column blocks: (hi + lo)(x1 + x2) + hi x3,
// i.e. only the lo * x3 term (< 2^-24 relative) is dropped; what remains is
// the 2^-17 relative storage error of hi + lo and the FP32 accumulation.
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
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;  // TMEM column offset of the second accumulator
constexpr uint32_t kTileBytes = BM * BK * 2;
constexpr int kMaxBp = 80;       // 3 * Bp <= 256 (MMA N and TMA box limits), Bp % 16 == 0
constexpr int kChunkTiles = 4;   // k-tiles (of 64) per TMEM accumulation

struct TcParams {
  int64_t rows;  // M rounded up to 128
  int64_t M;
  int B, Bp, KS, m_tiles, k_tiles, stages;
  int chunk;     // k-tiles accumulated in TMEM before the epilogue drains them
  uint32_t stage_bytes;
  float *part;   // [KS][B][rows]
  int *status;
};

__global__ void xsplit_kernel(const float *__restrict__ x, int B, int Bp, int64_t K, int64_t ld,
                              const float *__restrict__ scale, __nv_bfloat16 *__restrict__ xs) {
  const int64_t total = (int64_t)Bp * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / ld);
    const int64_t j = t % ld;
    const float v = (b < B && j < K) ? x[(int64_t)b * K + j] * scale[j] : 0.f;
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

__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                   const __grid_constant__ CUtensorMap map_x, const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      ptx::mbar_init(&full_bar[s], 1);
      ptx::mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull_bar[a], 1);
      ptx::mbar_init(&tempty_bar[a], 4);
    }
    abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&map_hi);
    ptx::prefetch_tensormap(&map_lo);
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

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t it = 0;
    const uint32_t tx = 2 * kTileBytes + (uint32_t)(3 * Bp) * BK * 2;
    for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
      const int ks = u / P.m_tiles, mt = u % P.m_tiles;
      const int k0 = (int)((int64_t)P.k_tiles * ks / P.KS), k1 = (int)((int64_t)P.k_tiles * (ks + 1) / P.KS);
      for (int kt = k0; kt < k1; ++kt, ++it) {
        const int s = (int)(it % P.stages);
        if (!ptx::mbar_wait_bounded(&empty_bar[s], ((it / P.stages) & 1) ^ 1)) {
          set_abort(&abort_flag, P.status);
          break;
        }
        uint8_t *st = smem + (size_t)s * P.stage_bytes;
        ptx::mbar_arrive_expect_tx(&full_bar[s], tx);
        ptx::tma_load_2d(st, &map_hi, kt * BK, mt * BM, &full_bar[s]);
        ptx::tma_load_2d(st + kTileBytes, &map_lo, kt * BK, mt * BM, &full_bar[s]);
        ptx::tma_load_2d(st + 2 * kTileBytes, &map_x, kt * BK, 0, &full_bar[s]);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc3 = ptx::idesc_bf16_f32(BM, 3 * Bp);
    const uint32_t idesc2 = ptx::idesc_bf16_f32(BM, 2 * Bp);
    uint32_t it = 0, c = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < units && ok && !abort_flag; u += gridDim.x) {
      const int ks = u / P.m_tiles;
      const int k0 = (int)((int64_t)P.k_tiles * ks / P.KS), k1 = (int)((int64_t)P.k_tiles * (ks + 1) / P.KS);
      for (int kc = k0; kc < k1 && ok; kc += P.chunk, ++c) {
        const int kc1 = min(kc + P.chunk, k1);
        const uint32_t acc = c & 1;
        if (!ptx::mbar_wait_bounded(&tempty_bar[acc], ((c >> 1) & 1) ^ 1)) {
          set_abort(&abort_flag, P.status);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tbase + acc * kAccStride;
        for (int kt = kc; kt < kc1; ++kt, ++it) {
          const int s = (int)(it % P.stages);
          if (!ptx::mbar_wait_bounded(&full_bar[s], (it / P.stages) & 1)) {
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
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
            ptx::mma_bf16(d_tmem, dh + adv, dx + adv, idesc3, (kt > kc || kk > 0) ? 1u : 0u);
            ptx::mma_bf16(d_tmem, dl + adv, dx + adv, idesc2, 1u);
          }
          ptx::mma_commit(&empty_bar[s]);
        }
        if (ok) ptx::mma_commit(&tfull_bar[acc]);
      }
    }
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
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int ks = u / P.m_tiles, mt = u % P.m_tiles;
      const int k0 = (int)((int64_t)P.k_tiles * ks / P.KS), k1 = (int)((int64_t)P.k_tiles * (ks + 1) / P.KS);
      float sum[kMaxBp];
#pragma unroll
      for (int t = 0; t < kMaxBp; ++t) sum[t] = 0.f;
      for (int kc = k0; kc < k1; kc += P.chunk, ++c) {
        // Lane 0 alone takes the bounded wait and the abort decision, so the
        // warp stays converged for the .sync.aligned TMEM loads below.
        const uint32_t acc = c & 1;
        int good = 0;
        if (lane == 0) {
          good = !abort_flag && ptx::mbar_wait_bounded(&tfull_bar[acc], (c >> 1) & 1);
          if (!good) set_abort(&abort_flag, P.status);
        }
        good = __shfl_sync(0xffffffffu, good, 0);
        if (!good) {
          ok = false;
          break;
        }
        // Already complete (lane 0 saw it): this gives every lane its acquire.
        if (!ptx::mbar_wait_bounded(&tfull_bar[acc], (c >> 1) & 1)) set_abort(&abort_flag, P.status);
        ptx::tc_fence_after();
        const uint32_t tacc = tbase + ((uint32_t)(quarter * 32) << 16) + acc * kAccStride;
#pragma unroll
        for (int q = 0; q < kMaxBp / 16; ++q) {
          if (q * 16 < Bp) {
            float v0[16], v1[16], v2[16];
            ptx::tmem_ld16(tacc + q * 16, v0);
            ptx::tmem_ld16(tacc + Bp + q * 16, v1);
            ptx::tmem_ld16(tacc + 2 * Bp + q * 16, v2);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < 16; ++t) sum[q * 16 + t] += (v0[t] + v1[t]) + v2[t];
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&tempty_bar[acc]);
      }
      if (!ok) break;
      float *out = P.part + (int64_t)ks * P.B * P.rows + (int64_t)mt * BM + row;
#pragma unroll
      for (int t = 0; t < kMaxBp; ++t)
        if (t < P.B) out[(int64_t)t * P.rows] = sum[t];
    }
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tbase, kTmemCols);
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

struct Chunking {
  int Bp, KS, m_tiles, k_tiles, stages;
  uint32_t stage_bytes;
  size_t smem, xs_bytes, part_bytes;
};

Chunking plan_chunk(const psfsim_plan *h, int Bc) {
  Chunking c;
  c.Bp = (int)psfsim_round_up(Bc, 16);
  c.m_tiles = (int)(psfsim_round_up(h->M, BM) / BM);
  c.k_tiles = (int)(h->ld / BK);
  c.KS = choose_ks(c.m_tiles, c.k_tiles, h->num_sms);
  c.stage_bytes = (uint32_t)psfsim_round_up(2 * kTileBytes + 3 * c.Bp * BK * 2, 1024);
  c.stages = (int)((220 * 1024) / c.stage_bytes);
  if (c.stages > kMaxStages) c.stages = kMaxStages;
  c.smem = (size_t)c.stages * c.stage_bytes + 1024;
  c.xs_bytes = (size_t)psfsim_round_up(3ll * c.Bp * h->ld * 2, 256);
  c.part_bytes = (size_t)c.KS * Bc * psfsim_round_up(h->M, BM) * 4;
  return c;
}

}  // namespace

size_t psfsim_forward_tc_scratch(const psfsim_plan *h, int B) {
  const int Bc = B < kMaxBp ? B : kMaxBp;
  const Chunking c = plan_chunk(h, Bc);
  return c.xs_bytes + c.part_bytes;
}

cudaError_t psfsim_launch_forward_tc(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                     cudaStream_t st) {
  const float *scale = reinterpret_cast<const float *>(h->ws + h->scale_off);
  int *status = reinterpret_cast<int *>(h->ws + h->status_off);
  const int64_t rows = psfsim_round_up(h->M, BM);
  for (int b0 = 0; b0 < B; b0 += kMaxBp) {
    const int Bc = (B - b0) < kMaxBp ? (B - b0) : kMaxBp;
    const Chunking c = plan_chunk(h, Bc);
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(scratch);
    float *part = reinterpret_cast<float *>(static_cast<char *>(scratch) + c.xs_bytes);
    xsplit_kernel<<<h->num_sms * 8, 256, 0, st>>>(x + (int64_t)b0 * h->K, Bc, c.Bp, h->K, h->ld, scale, xs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap mhi, mlo, mx;
    if (!encode_bf16_2d(&mhi, h->ws + h->a_off, (uint64_t)h->ld, (uint64_t)rows, BK, BM) ||
        !encode_bf16_2d(&mlo, h->ws + h->lo_off, (uint64_t)h->ld, (uint64_t)rows, BK, BM) ||
        !encode_bf16_2d(&mx, xs, (uint64_t)h->ld, (uint64_t)(3 * c.Bp), BK, (uint32_t)(3 * c.Bp)))
      return cudaErrorInvalidValue;
    TcParams P;
    P.rows = rows;
    P.M = h->M;
    P.B = Bc;
    P.Bp = c.Bp;
    P.KS = c.KS;
    P.m_tiles = c.m_tiles;
    P.k_tiles = c.k_tiles;
    P.stages = c.stages;
    P.chunk = kChunkTiles;
    P.stage_bytes = c.stage_bytes;
    P.part = part;
    P.status = status;
    if ((e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem)) !=
        cudaSuccess)
      return e;
    const int units = c.m_tiles * c.KS;
    const int grid = units < h->num_sms ? units : h->num_sms;
    tc_gemm_kernel<<<grid, kThreads, c.smem, st>>>(mhi, mlo, mx, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = psfsim_launch_reduce_partials(part, c.KS, Bc, rows, h->M, y + (int64_t)b0 * h->M, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}
