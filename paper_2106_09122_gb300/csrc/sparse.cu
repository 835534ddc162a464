// S = A Z over the scene pixels that are not zero (FP32 storage).  A zero
// scene pixel contributes nothing to S = A Z (Eq. 6), so its column need not
// be read: point sources, masked disks and every scene beyond the outer
// working angle leave most of A untouched.  Three steps, all on the device:
//   nz_count_kernel   per 1024-column chunk, how many columns are non-zero in
//                     some scene of the batch;
//   nz_list_kernel    the ascending list of those columns (each chunk's
//                     offset is the sum of the counts before it) and nnz;
//   fwd_sparse_kernel the split-K forward of fwd_partial_kernel over the list
//                     (nnz read on the device), then the fixed-order reduction.
// Same result as psfsim_forward up to the order of the FP32 sums, and
// deterministic: the list order and the split of the list are fixed.
#include "gemv_device.cuh"
#include "psfsim_internal.cuh"

using namespace psfsim_gemv;

namespace {

constexpr int kChunk = 1024;  // columns per listing block (256 threads x 4)

__device__ __forceinline__ bool column_used(const float *__restrict__ x, int B, int64_t K, int64_t j) {
  if (j >= K) return false;
  for (int b = 0; b < B; ++b)
    if (x[(int64_t)b * K + j] != 0.f) return true;
  return false;
}

// counts[c] = used columns in [c kChunk, (c + 1) kChunk).
__global__ void __launch_bounds__(256) nz_count_kernel(const float *__restrict__ x, int B, int64_t K,
                                                       int *__restrict__ counts) {
  __shared__ int warp_sum[8];
  const int64_t base = (int64_t)blockIdx.x * kChunk + 4 * threadIdx.x;
  int n = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) n += column_used(x, B, K, base + e) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += warp_sum[w];
    counts[blockIdx.x] = t;
  }
}

// idx[offset_c + rank] = j for the used columns of chunk c, in ascending j;
// the last chunk also stores nnz.
__global__ void __launch_bounds__(256) nz_list_kernel(const float *__restrict__ x, int B, int64_t K,
                                                      const int *__restrict__ counts, int nchunks,
                                                      int *__restrict__ idx, int *__restrict__ nnz) {
  __shared__ int warp_base[8];
  __shared__ int chunk_base;
  if (threadIdx.x < 32) {  // offset of this chunk: sum of the earlier chunks' counts
    int s = 0;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += 32) s += counts[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) chunk_base = s;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kChunk + 4 * threadIdx.x;
  bool used[4];
  int n = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    used[e] = column_used(x, B, K, base + e);
    n += used[e] ? 1 : 0;
  }
  // inclusive prefix of n over the warp (threads in order, hence columns in order)
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_base[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {  // warp totals -> exclusive warp offsets
    int s = 0;
    for (int w = 0; w < 8; ++w) {
      const int t = warp_base[w];
      warp_base[w] = s;
      s += t;
    }
  }
  __syncthreads();
  int pos = chunk_base + warp_base[warp] + incl - n;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    if (used[e]) idx[pos++] = (int)(base + e);
  if (blockIdx.x == (unsigned)(nchunks - 1) && threadIdx.x == 255) *nnz = pos;
}

// part[(ks B + b) ld + r] = sum over the ks-th share of the listed columns.
template <int BB>
__global__ void __launch_bounds__(kFwdThreads) fwd_sparse_kernel(const float *__restrict__ A, int64_t ld,
                                                                 int64_t K, const float *__restrict__ x, int B,
                                                                 int b0, const int *__restrict__ idx,
                                                                 const int *__restrict__ nnz,
                                                                 float *__restrict__ part) {
  const int64_t r = (int64_t)blockIdx.x * kRowsPerCta + 4 * threadIdx.x;
  const int KS = gridDim.y, ks = blockIdx.y;
  if (r >= ld) return;
  const int64_t n = *nnz;
  float acc[BB][4];
  fwd_accumulate_idx<BB>(A, ld, K, x, b0, r, idx, n * ks / KS, n * (ks + 1) / KS, acc);
#pragma unroll
  for (int b = 0; b < BB; ++b)
    *reinterpret_cast<float4 *>(part + ((int64_t)ks * B + b0 + b) * ld + r) =
        make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
}

struct SparseScratch {
  size_t counts, idx, nnz, part, total;
  int nchunks, KS;
};

SparseScratch sparse_scratch(const psfsim_plan *h, int B) {
  SparseScratch s;
  s.nchunks = (int)((h->K + kChunk - 1) / kChunk);
  s.KS = psfsim_gemv_splits(h->ld, h->K, h->num_sms);
  s.counts = 0;
  s.idx = (size_t)psfsim_round_up((int64_t)s.nchunks * 4, 256);
  s.nnz = s.idx + (size_t)psfsim_round_up(h->K * 4, 256);
  s.part = s.nnz + 256;
  s.total = s.part + (size_t)s.KS * (size_t)B * (size_t)h->ld * 4;
  return s;
}

template <int BB>
cudaError_t sparse_group(const psfsim_plan *h, const float *x, int B, int b0, const int *idx, const int *nnz,
                         float *part, int KS, cudaStream_t st) {
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  const dim3 grid((unsigned)((h->ld + kRowsPerCta - 1) / kRowsPerCta), (unsigned)KS);
  fwd_sparse_kernel<BB><<<grid, kFwdThreads, 0, st>>>(A, h->ld, h->K, x, B, b0, idx, nnz, part);
  return cudaGetLastError();
}

}  // namespace

size_t psfsim_forward_sparse_scratch(const psfsim_plan *h, int B) { return sparse_scratch(h, B).total; }

cudaError_t psfsim_launch_forward_sparse(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                         cudaStream_t st) {
  const SparseScratch s = sparse_scratch(h, B);
  char *base = static_cast<char *>(scratch);
  int *counts = reinterpret_cast<int *>(base + s.counts);
  int *idx = reinterpret_cast<int *>(base + s.idx);
  int *nnz = reinterpret_cast<int *>(base + s.nnz);
  float *part = reinterpret_cast<float *>(base + s.part);
  nz_count_kernel<<<s.nchunks, 256, 0, st>>>(x, B, h->K, counts);
  nz_list_kernel<<<s.nchunks, 256, 0, st>>>(x, B, h->K, counts, s.nchunks, idx, nnz);
  cudaError_t e = cudaGetLastError();
  int b0 = 0;
  while (b0 < B && e == cudaSuccess) {
    const int left = B - b0;
    if (left >= 8) { e = sparse_group<8>(h, x, B, b0, idx, nnz, part, s.KS, st); b0 += 8; }
    else if (left >= 4) { e = sparse_group<4>(h, x, B, b0, idx, nnz, part, s.KS, st); b0 += 4; }
    else if (left >= 2) { e = sparse_group<2>(h, x, B, b0, idx, nnz, part, s.KS, st); b0 += 2; }
    else { e = sparse_group<1>(h, x, B, b0, idx, nnz, part, s.KS, st); b0 += 1; }
  }
  if (e != cudaSuccess) return e;
  return psfsim_launch_reduce_partials(part, s.KS, B, h->ld, h->M, y, nullptr, st);
}
