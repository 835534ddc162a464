// The fit gradient on FP32_SYM storage: A_Q0 holds the columns of the
// x > 0, y > 0 quadrant inside the last radius (column t is scene pixel
// order[t] of the quadrant), the rest of A follows by quarter turns:
//     S = sum_m P^m (A_Q0 X^(m)),     (A^T g)_{R^m(order[t])} = (A_Q0^T (g o P^m))_t,
// with X^(m)_t = x at R^m(order[t]), R the quarter turn of the scene and P
// that of the image.  Three launches (programmatic stream serialization):
//   fwd_sym_kernel       ring scene at the four rotations of the CTA's
//                        columns (shared memory), V_m = A_Q0 X^(m) with the
//                        split-K partials added across a 4-CTA cluster and
//                        then by the last group per slice; Z and dZ/dtheta of
//                        every scene pixel;
//   sym_loss_kernel      S = sum_m P^m V_m, r = (S - d)/sigma^2, FP64 loss
//                        partials, and the four turned copies g o P^m of r;
//   adj_sym_chain_kernel A_Q0^T (g o P^m) per column range, scattered to the
//                        four rotated pixels of gz and dotted with dZ/dtheta;
//                        pixels without a column get zero; two-level sums.
// Deterministic: every sum's order is fixed by the grid.
#include "../../include/psfsim_fit.h"
#include "gemv_device.cuh"
#include "psfsim_internal.cuh"
#include "ptx_util.cuh"
#include "ring_model.cuh"

using namespace psfsim_gemv;

namespace {

constexpr int kCluster = 4;
constexpr int kSliceVec = kFwdThreads / kCluster;  // row quads per 256-row slice
constexpr int kXCols = 1024;                       // most compact columns one CTA holds
constexpr int kGroup = 32;                         // CTAs per first-level chain sum
constexpr int kLossThreads = 256;

// Scene pixel index of the quadrant pixel j0 turned m quarter turns.
__device__ __forceinline__ int64_t turned_pixel(int N, int j0, int m) {
  const int H = N / 2;
  int ix = H + j0 % H, iy = H + j0 / H;
  for (int k = 0; k < m; ++k) {  // R(ix, iy) = (N-1-iy, ix)
    const int nx = N - 1 - iy;
    iy = ix;
    ix = nx;
  }
  return (int64_t)iy * N + ix;
}

// Image pixel i turned m quarter turns by P: (p, q) -> (q, n-1-p).
__device__ __forceinline__ int64_t perm_pixel(int n, int m, int64_t i) {
  int p = (int)(i / n), q = (int)(i % n);
  for (int k = 0; k < m; ++k) {
    const int np = q;
    q = n - 1 - p;
    p = np;
  }
  return (int64_t)p * n + q;
}

// CTA (tile, ks): image rows [1024 tile, +1024), compact columns
// [Kv ks / KS, Kv (ks + 1) / KS).  v[m][row] = (A_Q0 X^(m))_row.
__global__ void __cluster_dims__(1, kCluster, 1) __launch_bounds__(kFwdThreads, 4)
    fwd_sym_kernel(const float *__restrict__ A, int64_t ld, int64_t M, int64_t Kv, const int *__restrict__ order,
                   const RingParams P, float *__restrict__ z, float *__restrict__ jac, float *__restrict__ part,
                   float *__restrict__ v, unsigned *__restrict__ slice_count, unsigned *__restrict__ adj_count,
                   int n_adj_count) {
  __shared__ float xs[4 * kXCols];
  __shared__ float4 cpart[4][kFwdThreads];
  const int KS = gridDim.y, ks = blockIdx.y, G = KS / kCluster, grp = ks / kCluster;
  const int64_t t0 = Kv * ks / KS, t1 = Kv * (ks + 1) / KS;
  const int64_t tile0 = (int64_t)blockIdx.x * kRowsPerCta;
  ptx::griddep_launch_dependents();
  // Until griddep_wait: no global writes, no reads of earlier kernels' results.
  {  // the first columns' rows head for L2 while the scene values are computed
    const int64_t r = tile0 + 4 * threadIdx.x;
    if (r < ld)
      for (int64_t t = t0; t < t0 + 4 && t < t1; ++t)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(A + t * ld + r));
  }
  for (int64_t u = threadIdx.x; u < 4 * (t1 - t0); u += kFwdThreads) {
    const int64_t t = t0 + (u >> 2);
    const int m = (int)(u & 3);
    xs[m * kXCols + (t - t0)] = ring_eval<false>(P, turned_pixel(P.N, __ldg(order + t), m), nullptr);
  }
  __syncthreads();
  {
    const int64_t r = tile0 + 4 * threadIdx.x;
    float acc[4][4] = {};
    if (r < ld) fwd_accumulate<4, true, kXCols>(A, ld, Kv, xs, 0, r, t0, t1, acc);
#pragma unroll
    for (int m = 0; m < 4; ++m) cpart[m][threadIdx.x] = make_float4(acc[m][0], acc[m][1], acc[m][2], acc[m][3]);
  }
  ptx::griddep_wait();
  const int64_t K = (int64_t)P.N * P.N;
  if (blockIdx.x == 0 && blockIdx.y == 0)  // the adjoint that follows starts from zeroed counters
    for (int i = threadIdx.x; i < n_adj_count; i += kFwdThreads) adj_count[i] = 0u;
  {  // Z and dZ/dtheta of every scene pixel, spread over all CTAs
    const int64_t nct = (int64_t)gridDim.x * gridDim.y, lin = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int64_t j = lin * kFwdThreads + threadIdx.x; j < K; j += nct * kFwdThreads) {
      float J[5];
      z[j] = ring_eval<true>(P, j, J);
#pragma unroll
      for (int m = 0; m < 5; ++m) jac[m * K + j] = J[m];
    }
  }
  ptx::cluster_sync();
  const uint32_t q = ptx::cluster_ctarank();
  const int vq = (int)q * kSliceVec + (int)threadIdx.x;
  const int64_t rs = tile0 + 4 * (int64_t)vq;
  if (threadIdx.x < kSliceVec) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float4 t = ptx::ld_dsmem_f4(&cpart[m][vq], 0);
#pragma unroll
      for (uint32_t rk = 1; rk < kCluster; ++rk) {
        const float4 u = ptx::ld_dsmem_f4(&cpart[m][vq], rk);
        t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
      }
      if (rs < ld) *reinterpret_cast<float4 *>(part + ((int64_t)grp * 4 + m) * ld + rs) = t;
    }
  }
  ptx::cluster_sync();  // every rank has read the others' shared memory
  __shared__ unsigned last;
  __threadfence();
  __syncthreads();
  const unsigned slot = blockIdx.x * kCluster + q;
  if (threadIdx.x == 0) last = atomicAdd(slice_count + slot, 1u) == (unsigned)(G - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  {  // the last group of the slice: thread (m, i) sums rotation m of row quad i over the groups
    const int m = (int)threadIdx.x / kSliceVec;
    const int64_t r2 = tile0 + 4 * ((int64_t)q * kSliceVec + (int)threadIdx.x % kSliceVec);
    if (r2 < ld) {
      const float4 *src = reinterpret_cast<const float4 *>(part + (int64_t)m * ld + r2);  // group g at src + g ld
      float4 t = __ldcg(src);
      for (int g0 = 1; g0 < G; g0 += 4) {  // four loads in flight, added in ascending g
        float4 u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (g0 + e < G) u[e] = __ldcg(src + (int64_t)(g0 + e) * ld);
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (g0 + e < G) {
            t.x += u[e].x; t.y += u[e].y; t.z += u[e].z; t.w += u[e].w;
          }
      }
      *reinterpret_cast<float4 *>(v + (int64_t)m * ld + r2) = t;
    }
  }
  if (threadIdx.x == 0) slice_count[slot] = 0u;
}

// S_i = sum_m V_m[P^-m(i)] (m in order), r = (S - d)/sigma^2, loss partial
// per block; gp[m][i] = r[P^m(i)], each recomputed the same way from V.
__global__ void __launch_bounds__(kLossThreads) sym_loss_kernel(const float *__restrict__ v, int64_t ld, int n,
                                                                const float *__restrict__ d, double sigma,
                                                                float inv_s2, float *__restrict__ y,
                                                                float *__restrict__ r, float *__restrict__ gp,
                                                                double *__restrict__ loss_part) {
  __shared__ double red[kLossThreads / 32];
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();
  const int64_t M = (int64_t)n * n;
  const int64_t i = (int64_t)blockIdx.x * kLossThreads + threadIdx.x;
  auto image = [&](int64_t k) -> float {
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) s += __ldcg(v + (int64_t)m * ld + perm_pixel(n, (4 - m) & 3, k));
    return s;
  };
  double q2 = 0.0;
  if (i < M) {
    const float yi = image(i);
    y[i] = yi;
    const float diff = yi - d[i];
    r[i] = diff * inv_s2;
    const double qd = (double)diff / sigma;
    q2 = qd * qd;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int64_t k = perm_pixel(n, m, i);
      gp[(int64_t)m * M + i] = (image(k) - d[k]) * inv_s2;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < kLossThreads / 32; ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

// gc[m][t] = sum_i A_Q0[i, t] gp[m][i] for t0 <= t < t1, kC columns per pass
// so that each load of the four turned residuals (from L2) serves all of
// them (the four rotations would otherwise read four times the bytes of A
// from L2), with 2 kC column loads in flight per thread.  Rows split across
// the CTA (float4 strided), warp sums, then a fixed-order sum over the warps
// through a double-buffered shared array.
template <bool kVec, int kC>
__device__ __forceinline__ void adj_group(const float *__restrict__ A, int64_t ld, int64_t M, int64_t Kv,
                                          const float *__restrict__ gp, float *__restrict__ gc, int64_t t0,
                                          int64_t t1) {
  __shared__ float red[2][kAdjThreads / 32][4 * kC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int parity = 0;
  for (int64_t t = t0; t < t1; t += kC, parity ^= 1) {
    const int nc = (int)(t1 - t < kC ? t1 - t : kC);
    const float *col[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) col[c] = A + (t + (c < nc ? c : 0)) * ld;
    float acc[kC][4] = {};
    if (kVec) {
      const int64_t M4 = M >> 2;
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      auto step = [&](const float4 (&v)[kC], int64_t i4) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float4 gv = __ldg(reinterpret_cast<const float4 *>(gp + (int64_t)b * M) + i4);
#pragma unroll
          for (int c = 0; c < kC; ++c)
            acc[c][b] = fmaf(v[c].x, gv.x, fmaf(v[c].y, gv.y, fmaf(v[c].z, gv.z, fmaf(v[c].w, gv.w, acc[c][b]))));
        }
      };
      int64_t i4 = threadIdx.x;
      for (; i4 + kAdjThreads < M4; i4 += 2 * kAdjThreads) {
        float4 va[kC], vb[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          va[c] = c < nc ? ld_stream4(col[c] + 4 * i4) : zero;
          vb[c] = c < nc ? ld_stream4(col[c] + 4 * (i4 + kAdjThreads)) : zero;
        }
        step(va, i4);
        step(vb, i4 + kAdjThreads);
      }
      for (; i4 < M4; i4 += kAdjThreads) {
        float4 va[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) va[c] = c < nc ? ld_stream4(col[c] + 4 * i4) : zero;
        step(va, i4);
      }
    } else {
      for (int64_t i = threadIdx.x; i < M; i += kAdjThreads) {
        float v[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) v[c] = c < nc ? __ldg(col[c] + i) : 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float g = __ldg(gp + (int64_t)b * M + i);
#pragma unroll
          for (int c = 0; c < kC; ++c) acc[c][b] = fmaf(v[c], g, acc[c][b]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kC; ++c)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float s = acc[c][b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[parity][warp][c * 4 + b] = s;
      }
    __syncthreads();
    if (threadIdx.x < 4 * nc) {
      const int c = threadIdx.x >> 2, b = threadIdx.x & 3;
      float s = red[parity][0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < kAdjThreads / 32; ++w) s += red[parity][w][threadIdx.x];
      gc[(int64_t)b * Kv + t + c] = s;
    }
  }
}

struct SymChainArgs {
  const float *jac;         // dZ_j/dtheta_m at jac[m * K + j]
  double *chain_part;       // [gridDim.x][5]
  double *group_part;       // [ceil(gridDim.x / kGroup)][5]
  const double *loss_part;  // [n_loss]
  int n_loss;
  unsigned *count;          // [ceil(gridDim.x / kGroup) + 1]
  double *out;              // {L, dL/dtheta_0..4}
};

// CTA c: compact columns [Kv c / G, Kv (c+1) / G).  gc[m][t] = (A_Q0^T gp_m)_t
// (adj_group, four columns per pass, eight column loads in flight per thread,
// three CTAs per SM so that nothing spills); pixels whose quadrant column lies
// beyond the last radius get gz = 0 (all threads; disjoint from the pixels
// the columns write); then warp 0 alone writes gz at the four turned pixels
// of each column and forms the FP64 chain partial sum_{t,m} gc[m][t] dZ/dtheta
// at that pixel (lane-strided, fixed butterfly): FP64 runs at a small fraction
// of the FP32 rate, so the other warps take no part in it.
template <bool kVec>
__global__ void __launch_bounds__(kAdjThreads, 3)
    adj_sym_chain_kernel(const float *__restrict__ A, int64_t ld, int64_t M, int64_t Kv, const int *__restrict__ order,
                         const ColGeom *__restrict__ geom, int N, const float *__restrict__ gp,
                         float *__restrict__ gc, float *__restrict__ gz, const SymChainArgs c) {
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();  // gp and dZ/dtheta come from the earlier kernels
  const int64_t t0 = Kv * blockIdx.x / gridDim.x, t1 = Kv * (blockIdx.x + 1) / gridDim.x;
  adj_group<kVec, 4>(A, ld, M, Kv, gp, gc, t0, t1);
  __syncthreads();  // this CTA's gc entries are written
  // The grid shape again, from fresh special-register reads, so that the
  // streaming loop above keeps no extra registers live for this tail.
  unsigned cta, ncta;
  asm volatile("mov.u32 %0, %%ctaid.x;" : "=r"(cta));
  asm volatile("mov.u32 %0, %%nctaid.x;" : "=r"(ncta));
  const int64_t K = (int64_t)N * N;
  {  // pixels without a column
    const int H = N / 2;
    for (int64_t p = (int64_t)cta * kAdjThreads + threadIdx.x; p < K; p += (int64_t)ncta * kAdjThreads) {
      int ix = (int)(p % N), iy = (int)(p / N);
      for (int k = 0; k < 3 && !(ix >= H && iy >= H); ++k) {  // R^-1(ix, iy) = (iy, N-1-ix)
        const int nx = iy;
        iy = N - 1 - ix;
        ix = nx;
      }
      if (geom[(int64_t)(iy - H) * H + (ix - H)].k < 0) gz[p] = 0.f;
    }
  }
  if (threadIdx.x >= 32) return;
  // Warp 0: gz at the four turned pixels of each of the CTA's columns, and the
  // FP64 chain partial (lane-strided entries, then a fixed butterfly).
  const int lane = threadIdx.x;
  const int64_t c0 = Kv * cta / ncta, c1 = Kv * (cta + 1) / ncta;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t u = lane; u < 4 * (c1 - c0); u += 32) {
    const int64_t t = c0 + u / 4;
    const int m = (int)(u % 4);
    const int64_t p = turned_pixel(N, __ldg(order + t), m);
    const float val = gc[(int64_t)m * Kv + t];
    gz[p] = val;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += (double)val * (double)__ldg(c.jac + k * K + p);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  const unsigned grp = cta / kGroup, ngrp = (ncta + kGroup - 1) / kGroup;
  const unsigned gsize = ncta - grp * kGroup < kGroup ? ncta - grp * kGroup : kGroup;
  unsigned last = 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) c.chain_part[cta * 5 + k] = acc[k];
    __threadfence();
    last = atomicAdd(c.count + grp, 1u) == gsize - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < 5; ++k)
    acc[k] = (unsigned)lane < gsize ? __ldcg(c.chain_part + (grp * kGroup + lane) * 5 + k) : 0.0;
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  last = 0;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) c.group_part[grp * 5 + k] = acc[k];
    c.count[grp] = 0u;
    __threadfence();
    last = atomicAdd(c.count + ngrp, 1u) == ngrp - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  double t[6] = {0, 0, 0, 0, 0, 0};
  for (int i = lane; i < c.n_loss; i += 32) t[0] += __ldcg(c.loss_part + i);
  for (int i = lane; i < (int)ngrp; i += 32)
#pragma unroll
    for (int k = 0; k < 5; ++k) t[1 + k] += __ldcg(c.group_part + i * 5 + k);
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
  if (lane == 0) {
    c.out[0] = 0.5 * t[0];
#pragma unroll
    for (int k = 0; k < 5; ++k) c.out[1 + k] = t[1 + k];
    c.count[ngrp] = 0u;
  }
}

// ---------------------------------------------------------------- host side

int sym_tiles(const psfsim_plan *h) { return (int)((h->ld + kRowsPerCta - 1) / kRowsPerCta); }

// Column splits of fwd_sym_kernel: a multiple of the cluster size, one wave
// of clusters where possible, at most kXCols columns per CTA; fixed in the
// plan at first use.
int sym_splits(psfsim_plan *h) {
  if (h->fit_ks > 0) return h->fit_ks;
  const int tiles = sym_tiles(h);
  int clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tiles, kCluster, 1);
  cfg.blockDim = dim3(kFwdThreads, 1, 1);
  if (cudaOccupancyMaxActiveClusters(&clusters, fwd_sym_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    clusters = 0;
  }
  int64_t groups = clusters / tiles;
  const int64_t max_groups = h->K_valid / (8 * kCluster);
  if (groups > max_groups) groups = max_groups;
  const int64_t min_ks = (h->K_valid + kXCols - 1) / kXCols;
  const int64_t min_groups = (min_ks + kCluster - 1) / kCluster;
  if (groups < min_groups) groups = min_groups;
  if (groups < 1) groups = 1;
  h->fit_ks = (int)groups * kCluster;
  return h->fit_ks;
}

int sym_adj_max_blocks(const psfsim_plan *h) {
  int64_t g = (int64_t)h->num_sms * (2048 / kAdjThreads);
  if (g > h->K_valid) g = h->K_valid;
  return (int)(g < 1 ? 1 : g);
}

int sym_adj_blocks(const psfsim_plan *h, bool vec) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, vec ? adj_sym_chain_kernel<true> : adj_sym_chain_kernel<false>, kAdjThreads, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  const int64_t g = (int64_t)h->num_sms * (per_sm < 1 ? 1 : per_sm);
  const int cap = sym_adj_max_blocks(h);
  return (int)(g < cap ? g : cap);
}

int loss_blocks(const psfsim_plan *h) { return (int)((h->M + kLossThreads - 1) / kLossThreads); }

struct SymScratch {
  size_t part, v, gp, gc, loss, chain, group, count, jac, total;
  int n_slices, n_groups, n_count;
};

SymScratch sym_scratch(psfsim_plan *h) {
  SymScratch s;
  s.n_slices = sym_tiles(h) * kCluster;
  s.n_groups = (sym_adj_max_blocks(h) + kGroup - 1) / kGroup;
  s.n_count = s.n_slices + s.n_groups + 1;
  const int64_t K = (int64_t)h->N * h->N;
  auto up = [](int64_t b) { return (size_t)psfsim_round_up(b, 256); };
  s.part = 0;
  s.v = s.part + up((int64_t)(sym_splits(h) / kCluster) * 4 * h->ld * 4);
  s.gp = s.v + up(4 * h->ld * 4);
  s.gc = s.gp + up(4 * h->M * 4);
  s.loss = s.gc + up(4 * (h->K_valid > 0 ? h->K_valid : 1) * 4);
  s.chain = s.loss + up((int64_t)loss_blocks(h) * 8);
  s.group = s.chain + up((int64_t)sym_adj_max_blocks(h) * 5 * 8);
  s.count = s.group + up((int64_t)s.n_groups * 5 * 8);
  s.jac = s.count + up((int64_t)s.n_count * 4);
  s.total = s.jac + (size_t)5 * K * 4;
  return s;
}

}  // namespace

size_t psfsim_sym_gradient_scratch(psfsim_plan *h) { return sym_scratch(h).total; }

cudaError_t psfsim_sym_forward_loss(psfsim_plan *h, const RingParams &P, const float *d, double sigma, float *z,
                                    float *y, float *r, void *scratch, cudaStream_t st) {
  const SymScratch s = sym_scratch(h);
  char *base = static_cast<char *>(scratch);
  unsigned *count = reinterpret_cast<unsigned *>(base + s.count);
  float *v = reinterpret_cast<float *>(base + s.v);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = psfsim_pdl_config(dim3((unsigned)sym_tiles(h), (unsigned)sym_splits(h)), kFwdThreads,
                                             st, attr);
  cudaError_t e = cudaLaunchKernelEx(&cfg, fwd_sym_kernel, A, h->ld, h->M, h->K_valid, order, P, z,
                                     reinterpret_cast<float *>(base + s.jac), reinterpret_cast<float *>(base + s.part),
                                     v, count, count + s.n_slices, s.n_groups + 1);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr2[1];
  cfg = psfsim_pdl_config(dim3((unsigned)loss_blocks(h)), kLossThreads, st, attr2);
  return cudaLaunchKernelEx(&cfg, sym_loss_kernel, (const float *)v, h->ld, h->n, d, sigma,
                            (float)(1.0 / (sigma * sigma)), y, r, reinterpret_cast<float *>(base + s.gp),
                            reinterpret_cast<double *>(base + s.loss));
}

cudaError_t psfsim_sym_adjoint_chain(psfsim_plan *h, const float *r, float *gz, double *out, void *scratch,
                                     cudaStream_t st) {
  (void)r;  // the turned copies of r were written by psfsim_sym_forward_loss
  const SymScratch s = sym_scratch(h);
  char *base = static_cast<char *>(scratch);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  const ColGeom *geom = reinterpret_cast<const ColGeom *>(h->ws + h->geom_off);
  const bool vec = h->M % 4 == 0;
  const SymChainArgs c{reinterpret_cast<const float *>(base + s.jac),
                       reinterpret_cast<double *>(base + s.chain),
                       reinterpret_cast<double *>(base + s.group),
                       reinterpret_cast<const double *>(base + s.loss),
                       loss_blocks(h),
                       reinterpret_cast<unsigned *>(base + s.count) + s.n_slices,
                       out};
  const float *gp = reinterpret_cast<const float *>(base + s.gp);
  float *gc = reinterpret_cast<float *>(base + s.gc);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = psfsim_pdl_config(dim3((unsigned)sym_adj_blocks(h, vec)), kAdjThreads, st, attr);
  return vec ? cudaLaunchKernelEx(&cfg, adj_sym_chain_kernel<true>, A, h->ld, h->M, h->K_valid, order, geom, h->N,
                                  gp, gc, gz, c)
             : cudaLaunchKernelEx(&cfg, adj_sym_chain_kernel<false>, A, h->ld, h->M, h->K_valid, order, geom, h->N,
                                  gp, gc, gz, c);
}
