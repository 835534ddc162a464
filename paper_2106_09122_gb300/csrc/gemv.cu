// Products with a stored FP32 A (column-major, each PSF contiguous):
//   forward  S = A Z   (Eq. 6): row-parallel, split over columns, partials in
//            caller scratch, then a fixed-order reduction (deterministic);
//   adjoint  A^T g:            contiguous column ranges per CTA, rows split
//            across the CTA, fixed-order reduction.
// Both stream A once from HBM with 128-bit loads that bypass L1.
#include "psfsim_internal.cuh"
#include "ptx_util.cuh"

namespace {

__device__ __forceinline__ float4 ld_stream4(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

constexpr int kFwdThreads = 256;
constexpr int kRowsPerCta = kFwdThreads * 4;

// part[(ks*B + b)*ld + r] = sum over the ks-th column chunk of A[r, j] x[b, j].
// acc[b][e] = sum_{j0 <= j < j1} A[r + e, j] x[b0 + b, j] for the thread's 4 rows.
template <int BB>
__device__ __forceinline__ void fwd_accumulate(const float *__restrict__ A, int64_t ld, int64_t K,
                                               const float *__restrict__ x, int b0, int64_t r, int64_t j0,
                                               int64_t j1, float (&acc)[BB][4]) {
#pragma unroll
  for (int b = 0; b < BB; ++b) acc[b][0] = acc[b][1] = acc[b][2] = acc[b][3] = 0.f;
  const float *a = A + j0 * ld + r;
  const float *xb = x + (int64_t)b0 * K;
  int64_t j = j0;
  for (; j + 4 <= j1; j += 4, a += 4 * ld) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ld_stream4(a + u * ld);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int b = 0; b < BB; ++b) {
        const float xv = __ldg(xb + (int64_t)b * K + j + u);
        acc[b][0] = fmaf(v[u].x, xv, acc[b][0]);
        acc[b][1] = fmaf(v[u].y, xv, acc[b][1]);
        acc[b][2] = fmaf(v[u].z, xv, acc[b][2]);
        acc[b][3] = fmaf(v[u].w, xv, acc[b][3]);
      }
    }
  }
  for (; j < j1; ++j, a += ld) {
    const float4 v = ld_stream4(a);
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      const float xv = __ldg(xb + (int64_t)b * K + j);
      acc[b][0] = fmaf(v.x, xv, acc[b][0]);
      acc[b][1] = fmaf(v.y, xv, acc[b][1]);
      acc[b][2] = fmaf(v.z, xv, acc[b][2]);
      acc[b][3] = fmaf(v.w, xv, acc[b][3]);
    }
  }
}

template <int BB>
__global__ void __launch_bounds__(kFwdThreads) fwd_partial_kernel(const float *__restrict__ A, int64_t ld,
                                                                  int64_t K, const float *__restrict__ x,
                                                                  int B, int b0, float *__restrict__ part) {
  const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + 4 * threadIdx.x;
  const int KS = gridDim.y, ks = blockIdx.y;
  if (r >= ld) return;
  float acc[BB][4];
  fwd_accumulate<BB>(A, ld, K, x, b0, r, K * ks / KS, K * (ks + 1) / KS, acc);
#pragma unroll
  for (int b = 0; b < BB; ++b)
    *reinterpret_cast<float4 *>(part + ((int64_t)ks * B + b0 + b) * ld + r) =
        make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
}

// y[b, i] = sum_ks part[ks, b, i] in a fixed order.  A CTA covers 128 rows;
// its 8 warps split the KS partials (ks = warp, warp + 8, ...) and combine
// through shared memory, so every output needs only ~KS/8 loads per thread.
constexpr int kRedRows = 128;
__global__ void __launch_bounds__(256) fwd_reduce_kernel(const float *__restrict__ part, int KS, int B,
                                                         int64_t ld, int64_t M, float *__restrict__ y,
                                                         const int *__restrict__ count) {
  __shared__ float4 red[8][32];
  const int c4 = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t r = ((int64_t)blockIdx.x * 32 + c4) * 4;
  const int b = blockIdx.y;
  if (count && b >= *count) return;  // scene slot not present in this call
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r < ld) {
    const float *p = part + (int64_t)b * ld + r;
    const int64_t step = (int64_t)B * ld;
    int ks = grp;
#pragma unroll 4
    for (; ks < KS; ks += 8) {
      const float4 v = *reinterpret_cast<const float4 *>(p + ks * step);
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
  }
  red[grp][c4] = s;
  __syncthreads();
  if (grp == 0 && r < M) {
    float4 t = red[0][c4];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      const float4 v = red[k][c4];
      t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
    }
    float *out = y + (int64_t)b * M + r;
    out[0] = t.x;
    if (r + 1 < M) out[1] = t.y;
    if (r + 2 < M) out[2] = t.z;
    if (r + 3 < M) out[3] = t.w;
  }
}

// One image, forward fused with the fit's residual and loss.  CTA (tile, ks)
// accumulates its column chunk for the tile's 1024 rows as fwd_partial_kernel
// does.  The kFwdCluster CTAs of a cluster (consecutive ks) then add their
// partials through distributed shared memory: rank q sums rows
// [128 q, 128 q + 128) of the tile over the cluster's ranks in rank order and
// writes that group's partial.  For each 128-row slice, the last group to
// arrive (arrival counter, zeroed before the launch and reset here) adds the
// G = KS / kFwdCluster group partials in group order, writes y and the
// residual r = (y - d)/sigma^2, and stores the slice's FP64 partial of
// sum ((y - d)/sigma)^2.  No sum depends on the arrival order: deterministic.
constexpr int kFwdCluster = 8;
constexpr int kSliceVec = kFwdThreads / kFwdCluster;  // float4 row quads per slice (128 rows)

__global__ void __cluster_dims__(1, kFwdCluster, 1) __launch_bounds__(kFwdThreads, 6)
    fwd_loss_kernel(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K, const float *__restrict__ x,
                    float *__restrict__ part, const float *__restrict__ d, double sigma, float inv_s2,
                    float *__restrict__ y, float *__restrict__ res, double *__restrict__ loss_part,
                    unsigned *__restrict__ slice_count) {
  __shared__ float4 cpart[kFwdThreads];
  const int KS = gridDim.y, ks = blockIdx.y, G = KS / kFwdCluster, grp = ks / kFwdCluster;
  const int64_t tile0 = (int64_t)blockIdx.x * kRowsPerCta;
  {
    const int64_t r = tile0 + 4 * threadIdx.x;
    float acc[1][4] = {{0.f, 0.f, 0.f, 0.f}};
    if (r < ld) fwd_accumulate<1>(A, ld, K, x, 0, r, K * ks / KS, K * (ks + 1) / KS, acc);
    cpart[threadIdx.x] = make_float4(acc[0][0], acc[0][1], acc[0][2], acc[0][3]);
  }
  ptx::cluster_sync();
  const uint32_t q = ptx::cluster_ctarank();
  const int v = (int)q * kSliceVec + (int)threadIdx.x;  // row quad of this thread's slice work
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
  __threadfence();
  __syncwarp();
  const unsigned slot = blockIdx.x * kFwdCluster + q;
  unsigned last = 0;
  if (threadIdx.x == 0) last = atomicAdd(slice_count + slot, 1u) == (unsigned)(G - 1);
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  double q2 = 0.0;
  if (rs < ld) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(part + rs));
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
  if (threadIdx.x == 0) {
    loss_part[slot] = q2;
    slice_count[slot] = 0u;
  }
}

int forward_splits(const psfsim_plan *h) {
  const int64_t row_blocks = (h->ld + kRowsPerCta - 1) / kRowsPerCta;
  int64_t ks = (int64_t)h->num_sms * 8 / row_blocks;
  ks = ks < 1 ? 1 : ks;
  const int64_t max_ks = h->K / 8 > 0 ? h->K / 8 : 1;
  return (int)(ks < max_ks ? ks : max_ks);
}

constexpr int kAdjThreads = 256;

// gx[b, j] = sum_i A[i, j] g[b, i].  CTA c owns the contiguous column range
// [K c / G, K (c+1) / G); for each column its 256 threads split the rows
// (float4 strided), reduce in registers, then across warps through a
// double-buffered shared array.  Fixed assignment and order: deterministic.
template <int BB, bool kVec>
__device__ __forceinline__ void adj_columns(const float *__restrict__ A, int64_t ld, int64_t M, int64_t K,
                                            const float *__restrict__ g, int b0, float *__restrict__ gx, int64_t j0,
                                            int64_t j1) {
  __shared__ float red[2][kAdjThreads / 32][BB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float *gb = g + (int64_t)b0 * M;
  int parity = 0;
  for (int64_t j = j0; j < j1; ++j, parity ^= 1) {
    const float *col = A + j * ld;
    float acc[BB];
#pragma unroll
    for (int b = 0; b < BB; ++b) acc[b] = 0.f;
    if (kVec) {
      const int64_t M4 = M >> 2;
      int64_t i4 = threadIdx.x;
      constexpr int T = kAdjThreads;
      for (; i4 + 3 * T < M4; i4 += 4 * T) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ld_stream4(col + 4 * (i4 + T * u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int b = 0; b < BB; ++b) {
            const float4 gv = __ldg(reinterpret_cast<const float4 *>(gb + (int64_t)b * M) + i4 + T * u);
            acc[b] = fmaf(v[u].x, gv.x, acc[b]);
            acc[b] = fmaf(v[u].y, gv.y, acc[b]);
            acc[b] = fmaf(v[u].z, gv.z, acc[b]);
            acc[b] = fmaf(v[u].w, gv.w, acc[b]);
          }
        }
      }
      for (; i4 < M4; i4 += T) {
        const float4 v = ld_stream4(col + 4 * i4);
#pragma unroll
        for (int b = 0; b < BB; ++b) {
          const float4 gv = __ldg(reinterpret_cast<const float4 *>(gb + (int64_t)b * M) + i4);
          acc[b] = fmaf(v.x, gv.x, acc[b]);
          acc[b] = fmaf(v.y, gv.y, acc[b]);
          acc[b] = fmaf(v.z, gv.z, acc[b]);
          acc[b] = fmaf(v.w, gv.w, acc[b]);
        }
      }
    } else {
      for (int64_t i = threadIdx.x; i < M; i += kAdjThreads) {
        const float v = __ldg(col + i);
#pragma unroll
        for (int b = 0; b < BB; ++b) acc[b] = fmaf(v, __ldg(gb + (int64_t)b * M + i), acc[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < BB; ++b) {
      float s = acc[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[parity][warp][b] = s;
    }
    __syncthreads();
    if (threadIdx.x < BB) {
      float t = red[parity][0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < kAdjThreads / 32; ++w) t += red[parity][w][threadIdx.x];
      gx[(int64_t)(b0 + threadIdx.x) * K + j] = t;
    }
  }
}

template <int BB, bool kVec>
__global__ void __launch_bounds__(kAdjThreads) adj_kernel(const float *__restrict__ A, int64_t ld, int64_t M,
                                                          int64_t K, const float *__restrict__ g, int b0,
                                                          float *__restrict__ gx) {
  adj_columns<BB, kVec>(A, ld, M, K, g, b0, gx, K * blockIdx.x / gridDim.x, K * (blockIdx.x + 1) / gridDim.x);
}

// Where the fit's chain rule and final sums read their partials.
struct ChainArgs {
  const float *jac;         // dZ_j/dtheta_m at jac[m * K + j]
  double *chain_part;       // [gridDim.x][5]
  const double *loss_part;  // [n_loss] partials of sum ((y - d)/sigma)^2
  int n_loss;
  unsigned *count;          // arrival counter, zeroed before the launch and reset here
  double *out;              // {L, dL/dtheta_0..4}
};

// One image: gz = A^T g as adj_kernel<1, kVec>, then warp 0 of each CTA dots
// its columns' gz with the stored Jacobian (FP64, fixed lane order), and the
// last CTA to arrive adds all CTAs' chain partials and the loss partials in
// index order into out.  Deterministic for a fixed grid.
template <bool kVec>
__global__ void __launch_bounds__(kAdjThreads, 6) adj_chain_kernel(const float *__restrict__ A, int64_t ld, int64_t M,
                                                                int64_t K, const float *__restrict__ g,
                                                                float *__restrict__ gz, const ChainArgs c) {
  const int64_t j0 = K * blockIdx.x / gridDim.x, j1 = K * (blockIdx.x + 1) / gridDim.x;
  adj_columns<1, kVec>(A, ld, M, K, g, 0, gz, j0, j1);
  if (threadIdx.x >= 32) return;
  __syncwarp();  // thread 0 wrote every gz[j] of this CTA
  const int lane = threadIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t j = j0 + lane; j < j1; j += 32) {
    const double gj = (double)gz[j];
#pragma unroll
    for (int m = 0; m < 5; ++m) acc[m] += gj * (double)__ldg(c.jac + m * K + j);
  }
#pragma unroll
  for (int m = 0; m < 5; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  unsigned last = 0;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 5; ++m) c.chain_part[blockIdx.x * 5 + m] = acc[m];
    __threadfence();
    last = atomicAdd(c.count, 1u) == gridDim.x - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  double t[6] = {0, 0, 0, 0, 0, 0};
  for (int b = lane; b < c.n_loss; b += 32) t[0] += __ldcg(c.loss_part + b);
  for (int b = lane; b < (int)gridDim.x; b += 32)
#pragma unroll
    for (int m = 0; m < 5; ++m) t[1 + m] += __ldcg(c.chain_part + b * 5 + m);
#pragma unroll
  for (int m = 0; m < 6; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[m] += __shfl_xor_sync(0xffffffffu, t[m], o);
  if (lane == 0) {
    c.out[0] = 0.5 * t[0];
#pragma unroll
    for (int m = 0; m < 5; ++m) c.out[1 + m] = t[1 + m];
    *c.count = 0u;
  }
}

template <int BB>
cudaError_t fwd_group(const psfsim_plan *h, const float *x, int B, int b0, float *part, int KS,
                      cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  dim3 grid((unsigned)((h->ld + kRowsPerCta - 1) / kRowsPerCta), (unsigned)KS);
  fwd_partial_kernel<BB><<<grid, kFwdThreads, 0, st>>>(A, h->ld, h->K, x, B, b0, part);
  return cudaGetLastError();
}

template <int BB>
cudaError_t adj_group(const psfsim_plan *h, const float *g, int b0, float *gx, bool vec, cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  auto kern = vec ? adj_kernel<BB, true> : adj_kernel<BB, false>;
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)h->num_sms * (per_sm < 1 ? 1 : per_sm);
  if (grid > h->K) grid = h->K;
  kern<<<(unsigned)grid, kAdjThreads, 0, st>>>(A, h->ld, h->M, h->K, g, b0, gx);
  return cudaGetLastError();
}

}  // namespace

cudaError_t psfsim_launch_gemv_partials(const float *A, int64_t ld, int64_t K, const float *x, int B, float *part,
                                        int KS, cudaStream_t st) {
  dim3 grid((unsigned)((ld + kRowsPerCta - 1) / kRowsPerCta), (unsigned)KS);
  int b0 = 0;
  while (b0 < B) {
    const int left = B - b0;
    if (left >= 8) { fwd_partial_kernel<8><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 8; }
    else if (left >= 4) { fwd_partial_kernel<4><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 4; }
    else if (left >= 2) { fwd_partial_kernel<2><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 2; }
    else { fwd_partial_kernel<1><<<grid, kFwdThreads, 0, st>>>(A, ld, K, x, B, b0, part); b0 += 1; }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int psfsim_gemv_splits(int64_t ld, int64_t K, int num_sms) {
  const int64_t row_blocks = (ld + kRowsPerCta - 1) / kRowsPerCta;
  int64_t ks = (int64_t)num_sms * 8 / row_blocks;
  ks = ks < 1 ? 1 : ks;
  const int64_t max_ks = K / 8 > 0 ? K / 8 : 1;
  return (int)(ks < max_ks ? ks : max_ks);
}

cudaError_t psfsim_launch_adjoint_cols(const float *A, int64_t ld, int64_t M, int64_t K, const float *g, int B,
                                       float *gx, int num_sms, cudaStream_t st) {
  const bool vec = (M % 4 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
  int b0 = 0;
  while (b0 < B) {
    const int left = B - b0;
    const int bb = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    auto launch = [&](auto kern) -> cudaError_t {
      int per_sm = 1;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, 0);
      if (e != cudaSuccess) return e;
      int64_t grid = (int64_t)num_sms * (per_sm < 1 ? 1 : per_sm);
      if (grid > K) grid = K;
      kern<<<(unsigned)grid, kAdjThreads, 0, st>>>(A, ld, M, K, g, b0, gx);
      return cudaGetLastError();
    };
    cudaError_t e;
    if (bb == 8) e = vec ? launch(adj_kernel<8, true>) : launch(adj_kernel<8, false>);
    else if (bb == 4) e = vec ? launch(adj_kernel<4, true>) : launch(adj_kernel<4, false>);
    else if (bb == 2) e = vec ? launch(adj_kernel<2, true>) : launch(adj_kernel<2, false>);
    else e = vec ? launch(adj_kernel<1, true>) : launch(adj_kernel<1, false>);
    if (e != cudaSuccess) return e;
    b0 += bb;
  }
  return cudaSuccess;
}

static int psfsim_forward_tiles(const psfsim_plan *h) { return (int)((h->ld + kRowsPerCta - 1) / kRowsPerCta); }

int psfsim_forward_loss_slices(const psfsim_plan *h) { return psfsim_forward_tiles(h) * kFwdCluster; }

// Column splits of the fused forward: a multiple of the cluster size, as many
// as fit the GPU in one wave of clusters (at least one cluster per tile).
static int psfsim_forward_loss_splits(const psfsim_plan *h) {
  const int tiles = psfsim_forward_tiles(h);
  int clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tiles, kFwdCluster, 1);
  cfg.blockDim = dim3(kFwdThreads, 1, 1);
  if (cudaOccupancyMaxActiveClusters(&clusters, fwd_loss_kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    clusters = 0;
  }
  int groups = clusters / tiles;
  const int64_t max_groups = h->K / (8 * kFwdCluster);  // at least 8 columns per CTA
  if (groups > max_groups) groups = (int)max_groups;
  return (groups < 1 ? 1 : groups) * kFwdCluster;
}

size_t psfsim_forward_loss_scratch(const psfsim_plan *h) {
  return (size_t)(psfsim_forward_loss_splits(h) / kFwdCluster) * (size_t)h->ld * 4;
}

int psfsim_adjoint_chain_max_blocks(const psfsim_plan *h) {
  const int64_t g = (int64_t)h->num_sms * (2048 / kAdjThreads);
  return (int)(g < h->K ? g : h->K);
}

cudaError_t psfsim_launch_forward_loss(const psfsim_plan *h, const float *x, const float *d, double sigma, float *y,
                                       float *r, void *scratch, double *loss_part, unsigned *slice_count,
                                       cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  dim3 grid((unsigned)psfsim_forward_tiles(h), (unsigned)psfsim_forward_loss_splits(h));
  fwd_loss_kernel<<<grid, kFwdThreads, 0, st>>>(A, h->ld, h->M, h->K, x, static_cast<float *>(scratch), d, sigma,
                                                (float)(1.0 / (sigma * sigma)), y, r, loss_part, slice_count);
  return cudaGetLastError();
}

cudaError_t psfsim_launch_adjoint_chain(const psfsim_plan *h, const float *g, float *gz, const float *jac,
                                        double *chain_part, const double *loss_part, unsigned *count, double *out,
                                        cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  const bool vec = (h->M % 4 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
  auto kern = vec ? adj_chain_kernel<true> : adj_chain_kernel<false>;
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAdjThreads, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)h->num_sms * (per_sm < 1 ? 1 : per_sm);
  const int cap = psfsim_adjoint_chain_max_blocks(h);
  if (grid > cap) grid = cap;
  const ChainArgs c{jac, chain_part, loss_part, psfsim_forward_loss_slices(h), count, out};
  kern<<<(unsigned)grid, kAdjThreads, 0, st>>>(A, h->ld, h->M, h->K, g, gz, c);
  return cudaGetLastError();
}

size_t psfsim_forward_fp32_scratch(const psfsim_plan *h, int B) {
  return (size_t)forward_splits(h) * (size_t)B * (size_t)h->ld * 4;
}

cudaError_t psfsim_launch_forward_fp32(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                       cudaStream_t st) {
  const int KS = forward_splits(h);
  float *part = reinterpret_cast<float *>(scratch);
  cudaError_t e = cudaSuccess;
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 8) { e = fwd_group<8>(h, x, B, b0, part, KS, st); b0 += 8; }
    else if (left >= 4) { e = fwd_group<4>(h, x, B, b0, part, KS, st); b0 += 4; }
    else if (left >= 2) { e = fwd_group<2>(h, x, B, b0, part, KS, st); b0 += 2; }
    else { e = fwd_group<1>(h, x, B, b0, part, KS, st); b0 += 1; }
  }
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((h->ld + kRedRows - 1) / kRedRows), (unsigned)B);
  fwd_reduce_kernel<<<grid, 256, 0, st>>>(part, KS, B, h->ld, h->M, y, nullptr);
  return cudaGetLastError();
}

cudaError_t psfsim_launch_reduce_partials(const float *part, int KS, int B, int64_t ld, int64_t M, float *y,
                                          const int *count, cudaStream_t st) {
  dim3 grid((unsigned)((ld + kRedRows - 1) / kRedRows), (unsigned)B);
  fwd_reduce_kernel<<<grid, 256, 0, st>>>(part, KS, B, ld, M, y, count);
  return cudaGetLastError();
}

cudaError_t psfsim_launch_adjoint_fp32(const psfsim_plan *h, const float *g, int B, float *gx, cudaStream_t st) {
  const bool vec = (h->M % 4 == 0) && ((reinterpret_cast<uintptr_t>(g) & 15) == 0);
  cudaError_t e = cudaSuccess;
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 8) { e = adj_group<8>(h, g, b0, gx, vec, st); b0 += 8; }
    else if (left >= 4) { e = adj_group<4>(h, g, b0, gx, vec, st); b0 += 4; }
    else if (left >= 2) { e = adj_group<2>(h, g, b0, gx, vec, st); b0 += 2; }
    else { e = adj_group<1>(h, g, b0, gx, vec, st); b0 += 1; }
  }
  return e;
}
