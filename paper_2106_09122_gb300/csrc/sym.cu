// FP32 storage compacted by two exact structures of A (PSFSIM_FP32_SYM):
//   * columns of scene pixels beyond the last library radius are zero
//     (nothing is stored for them);
//   * quarter-turn symmetry: with fixed-point rotation coordinates the column
//     of scene pixel R(j) = (-y, x) is bit-exactly the column of pixel j with
//     the image turned by a quarter (P), so only the x > 0, y > 0 quadrant
//     Q0 of an even N x N scene is stored.
// Forward:  S = sum_{m=0..3} P^m (A_Q0 X^(m)),  X^(m)_t = x_{R^m(j_t)};
// adjoint:  (A^T g)_{R^m(j_t)} = (A_Q0^T (g o P^m))_t.
// Both reuse the FP32 GEMV kernels on the compact matrix (K_valid columns)
// with the four rotations as a batch of four; gather / permutation kernels
// around them carry the symmetry.  Results equal the dense FP32 path up to
// the order of the FP32 sums.
#include "psfsim_internal.cuh"

namespace {

__device__ __forceinline__ void rotate_pixel(int N, int m, int &ix, int &iy) {
  for (int r = 0; r < m; ++r) {  // R(ix, iy) = (N-1-iy, ix): (x, y) -> (-y, x)
    const int nx = N - 1 - iy;
    iy = ix;
    ix = nx;
  }
}

// P^m of an image pixel: (p, q) -> (q, n-1-p), applied m times.
__device__ __forceinline__ int64_t perm_pixel(int n, int m, int64_t i) {
  int p = (int)(i / n), q = (int)(i % n);
  for (int r = 0; r < m; ++r) {
    const int np = q;
    q = n - 1 - p;
    p = np;
  }
  return (int64_t)p * n + q;
}

// xc[(b*4 + m) * Kv + t] = x[b][R^m(order[t])]
__global__ void sym_gather(const float *__restrict__ x, int B, int N, int64_t Kv, const int *__restrict__ order,
                           float *__restrict__ xc) {
  const int H = N / 2;
  const int64_t total = (int64_t)B * 4 * Kv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int bm = (int)(idx / Kv);
    const int64_t t = idx % Kv;
    const int b = bm >> 2, m = bm & 3;
    const int j0 = order[t];
    int ix = H + j0 % H, iy = H + j0 / H;
    rotate_pixel(N, m, ix, iy);
    xc[idx] = x[(int64_t)b * N * N + (int64_t)iy * N + ix];
  }
}

// y[b][i] = sum_m v[b*4+m][P^-m(i)]  (fixed order; v already reduced over k-splits).
__global__ void sym_permsum(const float *__restrict__ v, int B, int n, float *__restrict__ y) {
  const int64_t M = (int64_t)n * n;
  const int64_t total = (int64_t)B * M;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / M);
    const int64_t i = idx % M;
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) s += v[(int64_t)(b * 4 + m) * M + perm_pixel(n, (4 - m) & 3, i)];  // P^-m = P^(4-m)
    y[idx] = s;
  }
}

// gp[(b*4 + m) * M + i] = g[b][P^m(i)]
__global__ void sym_gperm(const float *__restrict__ g, int B, int n, float *__restrict__ gp) {
  const int64_t M = (int64_t)n * n;
  const int64_t total = (int64_t)B * 4 * M;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int bm = (int)(idx / M);
    const int64_t i = idx % M;
    gp[idx] = g[(int64_t)(bm >> 2) * M + perm_pixel(n, bm & 3, i)];
  }
}

// gx[b][R^m(order[t])] = gc[(b*4 + m) * Kv + t]; every other scene pixel is zero.
__global__ void sym_scatter(const float *__restrict__ gc, int B, int N, int64_t Kv, const int *__restrict__ order,
                            float *__restrict__ gx) {
  const int H = N / 2;
  const int64_t total = (int64_t)B * 4 * Kv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int bm = (int)(idx / Kv);
    const int64_t t = idx % Kv;
    const int j0 = order[t];
    int ix = H + j0 % H, iy = H + j0 / H;
    rotate_pixel(N, bm & 3, ix, iy);
    gx[(int64_t)(bm >> 2) * N * N + (int64_t)iy * N + ix] = gc[idx];
  }
}

unsigned grid_for(int64_t total, int num_sms) {
  const int64_t g = (total + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 16;
  return (unsigned)(g < 1 ? 1 : (g < cap ? g : cap));
}

// K-splits for the compact GEMV: enough CTAs to fill the GPU, but partial sums
// kept well below the bytes of the compact A (at least 64 columns per split).
int sym_splits(const psfsim_plan *h) {
  int ks = psfsim_gemv_splits(h->ld, h->K_valid, h->num_sms);
  const int64_t cap = h->K_valid / 64 > 0 ? h->K_valid / 64 : 1;
  return ks < cap ? ks : (int)cap;
}

}  // namespace

size_t psfsim_forward_sym_scratch(const psfsim_plan *h, int B) {
  const size_t xc = (size_t)psfsim_round_up((int64_t)4 * B * h->K_valid * 4, 256);
  const size_t v = (size_t)psfsim_round_up((int64_t)4 * B * h->M * 4, 256);
  return xc + v + (size_t)sym_splits(h) * 4 * B * h->ld * 4;
}

cudaError_t psfsim_launch_forward_sym(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                      cudaStream_t st) {
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  float *xc = static_cast<float *>(scratch);
  float *v = reinterpret_cast<float *>(static_cast<char *>(scratch) +
                                       psfsim_round_up((int64_t)4 * B * h->K_valid * 4, 256));
  float *part = reinterpret_cast<float *>(reinterpret_cast<char *>(v) + psfsim_round_up((int64_t)4 * B * h->M * 4, 256));
  const int KS = sym_splits(h);
  if (h->K_valid == 0) return cudaMemsetAsync(y, 0, (size_t)B * h->M * 4, st);
  sym_gather<<<grid_for((int64_t)4 * B * h->K_valid, h->num_sms), 256, 0, st>>>(x, B, h->N, h->K_valid, order, xc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = psfsim_launch_gemv_partials(A, h->ld, h->K_valid, xc, 4 * B, part, KS, st)) != cudaSuccess) return e;
  if ((e = psfsim_launch_reduce_partials(part, KS, 4 * B, h->ld, h->M, v, nullptr, st)) != cudaSuccess) return e;
  sym_permsum<<<grid_for((int64_t)B * h->M, h->num_sms), 256, 0, st>>>(v, B, h->n, y);
  return cudaGetLastError();
}

size_t psfsim_adjoint_sym_scratch(const psfsim_plan *h, int B) {
  return (size_t)psfsim_round_up((int64_t)4 * B * h->M * 4, 256) + (size_t)4 * B * h->K_valid * 4;
}

cudaError_t psfsim_launch_adjoint_sym(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                      cudaStream_t st) {
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  const float *A = reinterpret_cast<const float *>(h->ws + h->a_off);
  float *gp = static_cast<float *>(scratch);
  float *gc = reinterpret_cast<float *>(static_cast<char *>(scratch) + psfsim_round_up((int64_t)4 * B * h->M * 4, 256));
  cudaError_t e = cudaMemsetAsync(gx, 0, (size_t)B * h->K * 4, st);
  if (e != cudaSuccess || h->K_valid == 0) return e;
  sym_gperm<<<grid_for((int64_t)4 * B * h->M, h->num_sms), 256, 0, st>>>(g, B, h->n, gp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = psfsim_launch_adjoint_cols(A, h->ld, h->M, h->K_valid, gp, 4 * B, gc, h->num_sms, st)) != cudaSuccess)
    return e;
  sym_scatter<<<grid_for((int64_t)4 * B * h->K_valid, h->num_sms), 256, 0, st>>>(gc, B, h->N, h->K_valid, order, gx);
  return cudaGetLastError();
}

// ---- split-BF16 storage with the same compaction (PSFSIM_SPLIT_BF16_SYM) ----
// Forward: the four rotated scenes of every scene are gathered as a batch of
// 4B for the tcgen05 product over the compact columns, and the 4B partial
// images are summed through the inverse quarter turns.  Adjoint: the residual
// turned four ways, the split adjoint over the compact columns, and a scatter
// to the four rotated scene pixels.

size_t psfsim_forward_split_sym_scratch(const psfsim_plan *h, int B) {
  return (size_t)psfsim_round_up((int64_t)4 * B * h->ld * 4, 256) +
         (size_t)psfsim_round_up((int64_t)4 * B * h->M * 4, 256) + psfsim_forward_tc_scratch(h, 4 * B);
}

cudaError_t psfsim_launch_forward_split_sym(const psfsim_plan *h, const float *x, int B, float *y, void *scratch,
                                            cudaStream_t st) {
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  const int64_t Kv = h->K_valid;
  float *xc = static_cast<float *>(scratch);
  float *v = reinterpret_cast<float *>(static_cast<char *>(scratch) + psfsim_round_up((int64_t)4 * B * h->ld * 4, 256));
  void *tc = reinterpret_cast<char *>(v) + psfsim_round_up((int64_t)4 * B * h->M * 4, 256);
  if (Kv == 0) return cudaMemsetAsync(y, 0, (size_t)B * h->M * 4, st);
  sym_gather<<<grid_for((int64_t)4 * B * Kv, h->num_sms), 256, 0, st>>>(x, B, h->N, Kv, order, xc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = psfsim_launch_forward_tc(h, xc, 4 * B, v, tc, st)) != cudaSuccess) return e;
  sym_permsum<<<grid_for((int64_t)B * h->M, h->num_sms), 256, 0, st>>>(v, B, h->n, y);
  return cudaGetLastError();
}

size_t psfsim_adjoint_split_sym_scratch(const psfsim_plan *h, int B) {
  return (size_t)psfsim_round_up((int64_t)4 * B * h->M * 4, 256) +
         (size_t)psfsim_round_up((int64_t)4 * B * (h->K_valid > 0 ? h->K_valid : 1) * 4, 256) +
         psfsim_adjoint_split_scratch(h, 4 * B);
}

cudaError_t psfsim_launch_adjoint_split_sym(const psfsim_plan *h, const float *g, int B, float *gx, void *scratch,
                                            cudaStream_t st) {
  const int *order = reinterpret_cast<const int *>(h->ws + h->order_off);
  const int64_t Kv = h->K_valid;
  float *gp = static_cast<float *>(scratch);
  float *gc = reinterpret_cast<float *>(static_cast<char *>(scratch) + psfsim_round_up((int64_t)4 * B * h->M * 4, 256));
  void *part = reinterpret_cast<char *>(gc) + psfsim_round_up((int64_t)4 * B * (Kv > 0 ? Kv : 1) * 4, 256);
  cudaError_t e = cudaMemsetAsync(gx, 0, (size_t)B * h->K * 4, st);
  if (e != cudaSuccess || Kv == 0) return e;
  sym_gperm<<<grid_for((int64_t)4 * B * h->M, h->num_sms), 256, 0, st>>>(g, B, h->n, gp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = psfsim_launch_adjoint_split(h, gp, 4 * B, gc, part, st)) != cudaSuccess) return e;
  sym_scatter<<<grid_for((int64_t)4 * B * Kv, h->num_sms), 256, 0, st>>>(gc, B, h->N, Kv, order, gx);
  return cudaGetLastError();
}
