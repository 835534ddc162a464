// One fit gradient on an FP32 grid plan in two launches (include/psfsim_fit.h;
// FP32_SYM plans are dispatched to fit_sym.cu):
//
//   fwd_ring_loss_kernel   Z = ring(theta) for each CTA's column range (kept
//                          in shared memory; one tile per column also
//                          stores Z and dZ/dtheta), S = A Z, the residual
//                          r = (S - d)/sigma^2 and FP64 loss partials;
//   adj_chain_kernel       A^T r, its dot with dZ/dtheta, and the final sums
//                          {L, dL/dtheta}.
//
// Both kernels are launched with programmatic stream serialization: the
// forward computes its scene values and streams A before it waits for the
// kernel ahead of it (griddepcontrol.wait), so back-to-back gradients overlap
// one adjoint's tail with the next forward's streaming.
//
// Split-K partial sums are combined inside the kernels: first across a
// 4-CTA cluster through distributed shared memory, then by the last CTA to
// arrive (an arrival counter per slice).  Every sum runs in an order fixed by
// the grid, never by arrival, so results are deterministic.  The counters
// live in the caller's scratch, must be zero before the first call and are
// left at zero by every call.
#include "../../include/psfsim_fit.h"
#include "gemv_device.cuh"
#include "psfsim_internal.cuh"
#include "ptx_util.cuh"
#include "ring_model.cuh"

using namespace psfsim_gemv;

namespace {

constexpr int kFwdCluster = 4;                        // CTAs (consecutive column chunks) per cluster
constexpr int kSliceVec = kFwdThreads / kFwdCluster;  // row quads per slice (64: 256 rows, two warps)
static_assert(kSliceVec % 32 == 0 && kSliceVec <= kFwdThreads, "slices are whole warps");
constexpr int kXCols = 2048;                          // most scene columns one CTA holds

// CTA (tile, ks): rows [1024 tile, 1024 tile + 1024), columns
// [K ks / KS, K (ks + 1) / KS) (at most kXCols).  Cluster rank q reduces
// slice q (256 rows) of the tile over the cluster's kFwdCluster partials in
// rank order and writes the group partial part[grp][rows]; the last of the
// G = KS / kFwdCluster groups to arrive for a slice adds the group partials
// in group order and forms y, r and the slice's loss partial
// sum ((y - d)/sigma)^2.
__global__ void __cluster_dims__(1, kFwdCluster, 1) __launch_bounds__(kFwdThreads, 6)
    fwd_ring_loss_kernel(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K, const RingParams P,
                         float *__restrict__ z, float *__restrict__ jac, float *__restrict__ part,
                         const float *__restrict__ d, double sigma, float inv_s2, float *__restrict__ y,
                         float *__restrict__ res, double *__restrict__ loss_part, unsigned *__restrict__ slice_count,
                         unsigned *__restrict__ adj_count, int n_adj_count) {
  __shared__ float xs[kXCols];
  __shared__ float4 cpart[kFwdThreads];
  const int KS = gridDim.y, ks = blockIdx.y, G = KS / kFwdCluster, grp = ks / kFwdCluster;
  const int64_t j0 = K * ks / KS, j1 = K * (ks + 1) / KS;
  const int64_t tile0 = (int64_t)blockIdx.x * kRowsPerCta;
  ptx::griddep_launch_dependents();
  // Until griddep_wait below, this kernel neither writes global memory nor
  // reads anything an earlier kernel writes: it may overlap the tail of the
  // kernel before it in the stream.
  for (int64_t j = j0 + threadIdx.x; j < j1; j += kFwdThreads) xs[j - j0] = ring_eval<false>(P, j, nullptr);
  __syncthreads();
  {
    const int64_t r = tile0 + 4 * threadIdx.x;
    float acc[1][4] = {{0.f, 0.f, 0.f, 0.f}};
    if (r < ld) fwd_accumulate<1, true>(A, ld, K, xs, 0, r, j0, j1, acc);
    cpart[threadIdx.x] = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
  }
  ptx::griddep_wait();
  if (blockIdx.x == 0 && blockIdx.y == 0)  // the adjoint that follows starts from zeroed counters
    for (int i = threadIdx.x; i < n_adj_count; i += kFwdThreads) adj_count[i] = 0u;
  // Z and dZ/dtheta of column j are stored by the CTA of tile j mod tiles,
  // which spreads that work over the tiles.
  for (int64_t j = j0 + threadIdx.x; j < j1; j += kFwdThreads) {
    if (j % gridDim.x == blockIdx.x) {
      float J[5];
      z[j] = ring_eval<true>(P, j, J);
#pragma unroll
      for (int m = 0; m < 5; ++m) jac[m * K + j] = J[m];
    }
  }
  ptx::cluster_sync();
  const uint32_t q = ptx::cluster_ctarank();
  const int v = (int)q * kSliceVec + (int)threadIdx.x;
  const int64_t rs = tile0 + 4 * (int64_t)v;
  if (threadIdx.x < kSliceVec) {
    float4 t = ptx::ld_dsmem_f4(&cpart[v], 0);
#pragma unroll
    for (uint32_t rk = 1; rk < kFwdCluster; ++rk) {
      const float4 u = ptx::ld_dsmem_f4(&cpart[v], rk);
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    if (rs < ld) *reinterpret_cast<float4 *>(part + (int64_t)grp * ld + rs) = t;
  }
  ptx::cluster_sync();  // every rank has read the others' shared memory
  if (threadIdx.x >= kSliceVec) return;
  // From here only the kSliceVec threads of the slice work (named barrier 1).
  __shared__ unsigned last;
  __shared__ double q2w[kSliceVec / 32];
  __threadfence();
  ptx::named_barrier_sync(1, kSliceVec);
  const unsigned slot = blockIdx.x * kFwdCluster + q;
  if (threadIdx.x == 0) last = atomicAdd(slice_count + slot, 1u) == (unsigned)(G - 1);
  ptx::named_barrier_sync(1, kSliceVec);
  if (!last) return;
  __threadfence();
  double q2 = 0.0;
  if (rs < ld) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(part + rs));
#pragma unroll 8
    for (int g = 1; g < G; ++g) {
      const float4 u = __ldcg(reinterpret_cast<const float4 *>(part + (int64_t)g * ld + rs));
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    const float vals[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (rs + e < M) {
        y[rs + e] = vals[e];
        const float diff = vals[e] - d[rs + e];
        res[rs + e] = diff * inv_s2;
        const double qd = (double)diff / sigma;
        q2 += qd * qd;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
  if ((threadIdx.x & 31) == 0) q2w[threadIdx.x >> 5] = q2;
  ptx::named_barrier_sync(1, kSliceVec);
  if (threadIdx.x == 0) {
    double t = q2w[0];
#pragma unroll
    for (int w = 1; w < kSliceVec / 32; ++w) t += q2w[w];
    loss_part[slot] = t;
    slice_count[slot] = 0u;
  }
}

constexpr int kChainGroup = 32;  // CTAs whose chain partials one group sum covers


// gz[j] = sum_i A[i, j] g[i] for j0 <= j < j1, two columns per pass: one
// block barrier per pair of columns (the barrier after every column left the
// stream with nothing in flight once per column) and each residual load
// serves both.  Per column each thread adds its rows in ascending order
// (strides of the block), then a fixed butterfly and a fixed sum over the
// warps; stash[j - j0] = gz[j] for the first kStashCols columns.
template <bool kVec>
__device__ __forceinline__ void adj_pairs(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K,
                                          const float *__restrict__ g, float *__restrict__ gx, int64_t j0,
                                          int64_t j1, float *stash) {
  __shared__ float red2[2][kAdjThreads / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int parity = 0;
  for (int64_t j = j0; j < j1; j += 2, parity ^= 1) {
    const bool two = j + 1 < j1;
    const float *c0 = A + j * ld;
    const float *c1 = two ? c0 + ld : c0;
    float a0 = 0.f, a1 = 0.f;
    if (kVec) {
      const int64_t M4 = M >> 2;
      constexpr int T = kAdjThreads;
      int64_t i4 = threadIdx.x;
      for (; i4 + T < M4; i4 += 2 * T) {
        const float4 u0 = ld_stream4(c0 + 4 * i4), w0 = ld_stream4(c1 + 4 * i4);
        const float4 u1 = ld_stream4(c0 + 4 * (i4 + T)), w1 = ld_stream4(c1 + 4 * (i4 + T));
        const float4 g0 = __ldg(reinterpret_cast<const float4 *>(g) + i4);
        const float4 g1 = __ldg(reinterpret_cast<const float4 *>(g) + i4 + T);
        a0 = fmaf(u0.x, g0.x, a0); a0 = fmaf(u0.y, g0.y, a0); a0 = fmaf(u0.z, g0.z, a0); a0 = fmaf(u0.w, g0.w, a0);
        a1 = fmaf(w0.x, g0.x, a1); a1 = fmaf(w0.y, g0.y, a1); a1 = fmaf(w0.z, g0.z, a1); a1 = fmaf(w0.w, g0.w, a1);
        a0 = fmaf(u1.x, g1.x, a0); a0 = fmaf(u1.y, g1.y, a0); a0 = fmaf(u1.z, g1.z, a0); a0 = fmaf(u1.w, g1.w, a0);
        a1 = fmaf(w1.x, g1.x, a1); a1 = fmaf(w1.y, g1.y, a1); a1 = fmaf(w1.z, g1.z, a1); a1 = fmaf(w1.w, g1.w, a1);
      }
      for (; i4 < M4; i4 += T) {
        const float4 u0 = ld_stream4(c0 + 4 * i4), w0 = ld_stream4(c1 + 4 * i4);
        const float4 g0 = __ldg(reinterpret_cast<const float4 *>(g) + i4);
        a0 = fmaf(u0.x, g0.x, a0); a0 = fmaf(u0.y, g0.y, a0); a0 = fmaf(u0.z, g0.z, a0); a0 = fmaf(u0.w, g0.w, a0);
        a1 = fmaf(w0.x, g0.x, a1); a1 = fmaf(w0.y, g0.y, a1); a1 = fmaf(w0.z, g0.z, a1); a1 = fmaf(w0.w, g0.w, a1);
      }
    } else {
      for (int64_t i = threadIdx.x; i < M; i += kAdjThreads) {
        const float gi = __ldg(g + i);
        a0 = fmaf(__ldg(c0 + i), gi, a0);
        a1 = fmaf(__ldg(c1 + i), gi, a1);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane == 0) {
      red2[parity][warp][0] = a0;
      red2[parity][warp][1] = a1;
    }
    __syncthreads();
    if (threadIdx.x < (two ? 2 : 1)) {
      float t = red2[parity][0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < kAdjThreads / 32; ++w) t += red2[parity][w][threadIdx.x];
      gx[j + threadIdx.x] = t;
      if (j + threadIdx.x - j0 < kStashCols) stash[j + threadIdx.x - j0] = t;
    }
  }
}

struct ChainArgs {
  const float *jac;         // dZ_j/dtheta_m at jac[m * K + j]
  double *chain_part;       // [gridDim.x][5]
  double *group_part;       // [ceil(gridDim.x / kChainGroup)][5]
  const double *loss_part;  // [n_loss] partials of sum ((y - d)/sigma)^2
  int n_loss;
  unsigned *count;          // [ceil(gridDim.x / kChainGroup) + 1] arrival counters
  double *out;              // {L, dL/dtheta_0..4}
};

// gz = A^T g over the CTA's contiguous column range (adj_pairs: two columns
// per pass, four CTAs of 64 registers per SM so that the stream loop does not
// spill), then warp 0 dots the range's gz with dZ/dtheta (both in shared memory: gz
// stashed as it is produced, the Jacobian copied by cp.async while A
// streams).  Partials are added in two levels, each by the last warp to
// arrive: the 32 CTAs of a group in CTA order, then the groups in group order
// together with the loss partials; the butterfly shuffles are a fixed tree.
template <bool kVec>
__global__ void __launch_bounds__(kAdjThreads, 4)
    adj_chain_kernel(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K, const float *__restrict__ g,
                     float *__restrict__ gz, const ChainArgs c) {
  __shared__ float gzs[kStashCols];
  __shared__ float jacs[5][kStashCols];
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();  // r and dZ/dtheta come from the forward kernel
  {
    const int64_t j0 = K * blockIdx.x / gridDim.x, j1 = K * (blockIdx.x + 1) / gridDim.x;
    for (int t = threadIdx.x; t < 5 * kStashCols; t += kAdjThreads) {
      const int m = t / kStashCols, col = t % kStashCols;
      if (j0 + col < j1)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(ptx::smem_u32(&jacs[m][col])),
                     "l"(c.jac + m * K + j0 + col)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  adj_pairs<kVec>(A, ld, M, K, g, gz, K * blockIdx.x / gridDim.x, K * (blockIdx.x + 1) / gridDim.x, gzs);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();  // gzs (thread 0) and every thread's Jacobian copies are complete
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // The column range again, from fresh special-register reads, so that the
  // streaming loop above keeps no extra registers live for this tail.
  unsigned cta, ncta;
  asm volatile("mov.u32 %0, %%ctaid.x;" : "=r"(cta));
  asm volatile("mov.u32 %0, %%nctaid.x;" : "=r"(ncta));
  const int64_t j0 = K * cta / ncta, j1 = K * (cta + 1) / ncta;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t j = j0 + lane; j < j1; j += 32) {
    const int col = (int)(j - j0);
    const double gj = col < kStashCols ? (double)gzs[col] : (double)gz[j];
#pragma unroll
    for (int m = 0; m < 5; ++m)
      acc[m] += gj * (double)(col < kStashCols ? jacs[m][col] : __ldg(c.jac + m * K + j));
  }
#pragma unroll
  for (int m = 0; m < 5; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  const unsigned grp = cta / kChainGroup, ngrp = (ncta + kChainGroup - 1) / kChainGroup;
  const unsigned gsize = ncta - grp * kChainGroup < kChainGroup ? ncta - grp * kChainGroup : kChainGroup;
  unsigned last = 0;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 5; ++m) c.chain_part[cta * 5 + m] = acc[m];
    __threadfence();
    last = atomicAdd(c.count + grp, 1u) == gsize - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
#pragma unroll
  for (int m = 0; m < 5; ++m)
    acc[m] = (unsigned)lane < gsize ? __ldcg(c.chain_part + (grp * kChainGroup + lane) * 5 + m) : 0.0;
#pragma unroll
  for (int m = 0; m < 5; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  last = 0;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 5; ++m) c.group_part[grp * 5 + m] = acc[m];
    c.count[grp] = 0u;
    __threadfence();
    last = atomicAdd(c.count + ngrp, 1u) == ngrp - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  double t[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
  for (int i = lane; i < c.n_loss; i += 32) t[0] += __ldcg(c.loss_part + i);
  for (int i = lane; i < (int)ngrp; i += 32)
#pragma unroll
    for (int m = 0; m < 5; ++m) t[1 + m] += __ldcg(c.group_part + i * 5 + m);
#pragma unroll
  for (int m = 0; m < 6; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[m] += __shfl_xor_sync(0xffffffffu, t[m], o);
  if (lane == 0) {
    c.out[0] = 0.5 * t[0];
#pragma unroll
    for (int m = 0; m < 5; ++m) c.out[1 + m] = t[1 + m];
    c.count[ngrp] = 0u;
  }
}

// ---------------------------------------------------------------- host side

int forward_tiles(const psfsim_plan *h) { return (int)((h->ld + kRowsPerCta - 1) / kRowsPerCta); }

// Column splits of the forward: a multiple of the cluster size; as many as
// fit one wave of clusters, but never fewer than keep a CTA's columns within
// kXCols, and (where possible) at least 8 columns per CTA.  Fixed in the plan
// at first use, so that the scratch size and every launch agree.
int forward_splits(psfsim_plan *h) {
  if (h->fit_ks > 0) return h->fit_ks;
  const int tiles = forward_tiles(h);
  int clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tiles, kFwdCluster, 1);
  cfg.blockDim = dim3(kFwdThreads, 1, 1);
  if (cudaOccupancyMaxActiveClusters(&clusters, fwd_ring_loss_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    clusters = 0;
  }
  int64_t groups = clusters / tiles;
  const int64_t max_groups = h->K / (8 * kFwdCluster);
  if (groups > max_groups) groups = max_groups;
  const int64_t min_ks = (h->K + kXCols - 1) / kXCols;  // ceil(K / KS) <= kXCols
  const int64_t min_groups = (min_ks + kFwdCluster - 1) / kFwdCluster;
  if (groups < min_groups) groups = min_groups;
  if (groups < 1) groups = 1;
  h->fit_ks = (int)groups * kFwdCluster;
  return h->fit_ks;
}

int adjoint_blocks(const psfsim_plan *h, bool vec) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vec ? adj_chain_kernel<true> : adj_chain_kernel<false>,
                                                    kAdjThreads, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  int64_t grid = (int64_t)h->num_sms * (per_sm < 1 ? 1 : per_sm);
  const int64_t cap = (int64_t)h->num_sms * (2048 / kAdjThreads);
  if (grid > cap) grid = cap;
  if (grid > h->K) grid = h->K;
  return (int)grid;
}

int adjoint_max_blocks(const psfsim_plan *h) {
  const int64_t g = (int64_t)h->num_sms * (2048 / kAdjThreads);
  return (int)(g < h->K ? g : h->K);
}

struct GradScratch {
  size_t part, loss, chain, group, count, jac, total;
  int n_slices, n_groups, n_count;  // counters: slices, then groups + 1
};

GradScratch gradient_scratch(psfsim_plan *h) {
  GradScratch g;
  g.n_slices = forward_tiles(h) * kFwdCluster;
  g.n_groups = (adjoint_max_blocks(h) + kChainGroup - 1) / kChainGroup;
  g.n_count = g.n_slices + g.n_groups + 1;
  const int64_t ks = forward_splits(h);
  g.part = 0;
  g.loss = (size_t)psfsim_round_up((ks / kFwdCluster) * h->ld * 4, 256);
  g.chain = g.loss + (size_t)psfsim_round_up((int64_t)g.n_slices * 8, 256);
  g.group = g.chain + (size_t)psfsim_round_up((int64_t)adjoint_max_blocks(h) * 5 * 8, 256);
  g.count = g.group + (size_t)psfsim_round_up((int64_t)g.n_groups * 5 * 8, 256);
  g.jac = g.count + (size_t)psfsim_round_up((int64_t)g.n_count * 4, 256);
  g.total = g.jac + (size_t)5 * h->K * 4;
  return g;
}

int gradient_args(psfsim_t h, double r_max, const double *h_theta, void *d_scratch, size_t scratch_bytes,
                  RingParams *P, GradScratch *g) {
  if (!h) return PSFSIM_ERR_ARG;
  if (h->storage != PSFSIM_FP32 || h->N < 1) return PSFSIM_ERR_UNSUPPORTED;
  if (!ring_params(h->N, h->S, r_max, h_theta, P)) return PSFSIM_ERR_ARG;
  *g = gradient_scratch(h);
  if (!d_scratch || !aligned256(d_scratch) || scratch_bytes < g->total) return PSFSIM_ERR_WORKSPACE;
  return PSFSIM_OK;
}

// FP32_SYM: an even-N grid plan; the scratch must hold the symmetric layout.
int sym_args(psfsim_t h, double r_max, const double *h_theta, void *d_scratch, size_t scratch_bytes, RingParams *P) {
  if (h->N < 2 || (h->N & 1)) return PSFSIM_ERR_UNSUPPORTED;
  if (!ring_params(h->N, h->S, r_max, h_theta, P)) return PSFSIM_ERR_ARG;
  if (!d_scratch || !aligned256(d_scratch) || scratch_bytes < psfsim_sym_gradient_scratch(h))
    return PSFSIM_ERR_WORKSPACE;
  return PSFSIM_OK;
}

}  // namespace

extern "C" {

int psfsim_ring_gradient_scratch_bytes(psfsim_t h, size_t *bytes) {
  if (!h || !bytes) return PSFSIM_ERR_ARG;
  if (h->N < 1 || (h->storage != PSFSIM_FP32 && h->storage != PSFSIM_FP32_SYM)) return PSFSIM_ERR_UNSUPPORTED;
  *bytes = h->storage == PSFSIM_FP32_SYM ? psfsim_sym_gradient_scratch(h) : gradient_scratch(h).total;
  return PSFSIM_OK;
}

int psfsim_ring_forward_loss(psfsim_t h, double r_max, const double *h_theta, const float *d_target, double sigma,
                             float *d_z, float *d_y, float *d_r, void *d_scratch, size_t scratch_bytes,
                             void *stream) {
  if (!d_target || !d_z || !d_y || !d_r || !(sigma > 0.0) || !std::isfinite(sigma)) return PSFSIM_ERR_ARG;
  RingParams P;
  if (h && h->storage == PSFSIM_FP32_SYM) {
    if (int rc = sym_args(h, r_max, h_theta, d_scratch, scratch_bytes, &P)) return rc;
    return psfsim_sym_forward_loss(h, P, d_target, sigma, d_z, d_y, d_r, d_scratch,
                                   static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? PSFSIM_OK
               : PSFSIM_ERR_CUDA;
  }
  GradScratch g;
  if (int rc = gradient_args(h, r_max, h_theta, d_scratch, scratch_bytes, &P, &g)) return rc;
  char *base = static_cast<char *>(d_scratch);
  unsigned *count = reinterpret_cast<unsigned *>(base + g.count);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = psfsim_pdl_config(dim3((unsigned)forward_tiles(h), (unsigned)forward_splits(h)),
                                            kFwdThreads, static_cast<cudaStream_t>(stream), attr);
  const cudaError_t e = cudaLaunchKernelEx(
      &cfg, fwd_ring_loss_kernel, A, h->ld, h->M, h->K, P, d_z, reinterpret_cast<float *>(base + g.jac),
      reinterpret_cast<float *>(base + g.part), d_target, sigma, (float)(1.0 / (sigma * sigma)), d_y, d_r,
      reinterpret_cast<double *>(base + g.loss), count, count + g.n_slices, g.n_groups + 1);
  return e == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
}

int psfsim_ring_adjoint_chain(psfsim_t h, double r_max, const double *h_theta, const float *d_r, float *d_gz,
                              double *d_out, void *d_scratch, size_t scratch_bytes, void *stream) {
  if (!d_r || !d_gz || !d_out) return PSFSIM_ERR_ARG;
  RingParams P;
  if (h && h->storage == PSFSIM_FP32_SYM) {
    if (int rc = sym_args(h, r_max, h_theta, d_scratch, scratch_bytes, &P)) return rc;
    return psfsim_sym_adjoint_chain(h, d_r, d_gz, d_out, d_scratch, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? PSFSIM_OK
               : PSFSIM_ERR_CUDA;
  }
  GradScratch g;
  if (int rc = gradient_args(h, r_max, h_theta, d_scratch, scratch_bytes, &P, &g)) return rc;
  char *base = static_cast<char *>(d_scratch);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  const bool vec = (h->M % 4 == 0) && ((reinterpret_cast<uintptr_t>(d_r) & 15) == 0);
  const ChainArgs c{reinterpret_cast<const float *>(base + g.jac),
                    reinterpret_cast<double *>(base + g.chain),
                    reinterpret_cast<double *>(base + g.group),
                    reinterpret_cast<const double *>(base + g.loss),
                    g.n_slices,
                    reinterpret_cast<unsigned *>(base + g.count) + g.n_slices,
                    d_out};
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg =
      psfsim_pdl_config(dim3((unsigned)adjoint_blocks(h, vec)), kAdjThreads, static_cast<cudaStream_t>(stream), attr);
  const cudaError_t e = vec ? cudaLaunchKernelEx(&cfg, adj_chain_kernel<true>, A, h->ld, h->M, h->K, d_r, d_gz, c)
                            : cudaLaunchKernelEx(&cfg, adj_chain_kernel<false>, A, h->ld, h->M, h->K, d_r, d_gz, c);
  return e == cudaSuccess ? PSFSIM_OK : PSFSIM_ERR_CUDA;
}

int psfsim_ring_gradient(psfsim_t h, double r_max, const double *h_theta, const float *d_target, double sigma,
                         float *d_z, float *d_y, float *d_r, float *d_gz, double *d_out, void *d_scratch,
                         size_t scratch_bytes, void *stream) {
  int rc = psfsim_ring_forward_loss(h, r_max, h_theta, d_target, sigma, d_z, d_y, d_r, d_scratch, scratch_bytes,
                                    stream);
  if (rc != PSFSIM_OK) return rc;
  return psfsim_ring_adjoint_chain(h, r_max, h_theta, d_r, d_gz, d_out, d_scratch, scratch_bytes, stream);
}

}  // extern "C"
