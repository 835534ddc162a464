/*
 * psfsim: field-dependent coronagraphic image simulation on one GPU (sm_103a).
 *
 * The method (Milani & Douglas, "Faster imaging simulation through complex
 * systems: a coronagraphic example", Sec. 2-3): a radial library of off-axis
 * PSFs L[k] (offsets r_k along +x) is linearly interpolated in offset and
 * rotated to the polar angle of every scene pixel; each result, flattened, is
 * one column I_j of the matrix A = [I_1 ... I_K] (Eq. 4-5), and a simulated
 * image is S = A Z for the flattened scene Z (Eq. 6).
 *
 * Conventions (all calls):
 *   - Library d_lib: float32 [n_r][n][n], row p grows with +y, column q with +x,
 *     optical axis at ((n-1)/2, (n-1)/2), PSF k's source at radii[k] along +x.
 *   - Scene: N x N at S lambda/D per pixel, flattened row-major j = iy*N + ix,
 *     pixel centre x_j = (ix - (N-1)/2) S, y_j = (iy - (N-1)/2) S (Eq. 2-3 with
 *     the half-pixel shift).  Image: n x n, flattened i = p*n + q.  M = n*n,
 *     K = N*N (or the number of field points).
 *   - Radial weight: k = max{k : r_k <= r} clamped to [0, n_r-2],
 *     w = (r - r_k)/(r_{k+1} - r_k) (>= 0); r > r_{n_r-1} gives a zero column.
 *     PSFSIM_NEAREST rounds w to 0 or 1, ties to the lower radius.
 *   - Rotation about the centre c = (n-1)/2, bilinear, taps outside the array
 *     read 0: image pixel (p, q) samples column c + cos(q-c) + sin(p-c) and row
 *     c - sin(q-c) + cos(p-c) of the interpolated PSF, cos = x/r, sin = y/r.
 *   - Every device pointer is owned by the caller.  The library allocates no
 *     device memory: A and its build-time tables live in the caller's
 *     workspace, per-call temporaries in the caller's scratch.
 *   - All calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream) unless stated otherwise.
 *   - Errors are returned, never raised: arguments are validated on the host
 *     before anything is enqueued; a failed CUDA call maps to PSFSIM_ERR_CUDA.
 */
#ifndef PSFSIM_H
#define PSFSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psfsim_plan *psfsim_t; /* opaque host handle */

enum psfsim_status {
  PSFSIM_OK = 0,
  PSFSIM_ERR_ARG = -1,         /* null pointer, bad size or enum */
  PSFSIM_ERR_RADII = -2,       /* radii not finite and strictly increasing, or n_r < 2 */
  PSFSIM_ERR_WORKSPACE = -3,   /* workspace / scratch too small or misaligned */
  PSFSIM_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  PSFSIM_ERR_UNSUPPORTED = -5, /* valid request this build does not implement */
  PSFSIM_ERR_TIMEOUT = -6      /* a bounded device-side wait gave up */
};

/* Storage of A.  FP32: column-major float32 (each PSF contiguous, as the
 * paper saves one flattened PSF per iteration, Sec. 2).  SPLIT_BF16: row-major
 * bf16 hi + lo with a power-of-two float32 scale per column, for the
 * tensor-core path.  BF16: the hi part alone (row-major bf16 with the same
 * per-column scale): half the bytes, each element rounded to 8 significant
 * bits, so results carry up to 2^-8 of the error bound (tensor-core forward,
 * CUDA-core adjoint).  FP32_SYM: FP32 columns of the x > 0, y > 0 quadrant only,
 * inside the last radius: the other three quadrants' columns are exact
 * quarter turns of these and the rest are zero (even N, grid builds only;
 * same results as FP32 up to the order of the sums).  SPLIT_BF16_SYM: the
 * same compaction of split-BF16 storage (tensor-core forward on the four
 * rotated scenes at once; same results as SPLIT_BF16 up to the order of the
 * sums).  FUSED: A is never
 * stored; tiles are regenerated from the library on every product (the
 * paper's "standard interpolation method", Table 4, done on chip); a forward
 * runs one launch per 64 scenes, so batches of 33 to 64 scenes cost about the
 * same as 32 (the generation, not the tensor work, sets the time). */
enum psfsim_storage {
  PSFSIM_FP32 = 0,
  PSFSIM_SPLIT_BF16 = 1,
  PSFSIM_BF16 = 2,
  PSFSIM_FUSED = 3,
  PSFSIM_FP32_SYM = 4,
  PSFSIM_SPLIT_BF16_SYM = 5
};

/* Radial interpolation (Sec. 2 compares linear and nearest). */
enum psfsim_interp { PSFSIM_LINEAR = 0, PSFSIM_NEAREST = 1 };

/* Layout of a built plan inside the caller's workspace (byte offsets). */
typedef struct {
  int32_t storage, interp, n, n_r;
  int64_t M, K;
  int64_t ld;           /* FP32, FP32_SYM: column stride in floats; SPLIT_BF16, BF16,
                           SPLIT_BF16_SYM: row stride in elements (K, or K_stored, rounded up to 64) */
  int64_t a_offset;     /* FP32, FP32_SYM: A; SPLIT_BF16, BF16, SPLIT_BF16_SYM: hi */
  int64_t lo_offset;    /* SPLIT_BF16, SPLIT_BF16_SYM: lo (else -1) */
  int64_t scale_offset; /* SPLIT_BF16, BF16, SPLIT_BF16_SYM: float32 per-column scale (else -1) */
  int64_t workspace_bytes;
  int64_t K_stored;     /* columns held (K; FP32_SYM, SPLIT_BF16_SYM, FUSED: quadrant columns inside
                           the last radius, in the order of the sorted geometry) */
} psfsim_info_t;

/* Human-readable name of a status code (static string). */
const char *psfsim_status_string(int status);

/* Bytes of workspace psfsim_build needs for an n x n library of n_r PSFs
 * applied to K columns (K = N*N for a scene grid) with the given storage.
 * Sec. 3: A has n^2 rows and N^2 columns.  Returns PSFSIM_ERR_ARG for bad sizes. */
int psfsim_workspace_bytes(int n, int n_r, int64_t K, int storage, size_t *bytes);

/* Build the interpolated PSF library A for a scene grid (Sec. 2, the loop over
 * all N^2 scene pixels; Eq. 4-5).
 *   d_lib       device float32 [n_r][n][n], 16-byte aligned; read during the
 *               build only (FUSED storage keeps its own copy in the
 *               workspace: for every radial bracket and pixel, the 2 x 2
 *               bilinear footprints of both PSFs of the bracket in one
 *               32-byte entry, and a table of its columns).  FUSED needs an
 *               even N (it uses the exact quarter-turn symmetry of the scene
 *               grid) and synchronizes the stream once.
 *   h_radii     host double [n_r], strictly increasing offsets in lambda/D.
 *   s           PSF pixel scale (lambda/D per pixel).  A depends on s only
 *               through the radii; it is validated (> 0).
 *   N, S        scene size and pixel scale (lambda/D).
 *   d_workspace device buffer of at least psfsim_workspace_bytes bytes,
 *               256-byte aligned; holds A afterwards.
 *   out         receives a host handle; release with psfsim_free.
 * The build is enqueued on `stream`; A is valid once the stream reaches it. */
int psfsim_build(const float *d_lib, const double *h_radii, int n_r, int n, double s,
                 int N, double S, int storage, int interp, void *d_workspace,
                 size_t workspace_bytes, void *stream, psfsim_t *out);

/* Same as psfsim_build for K arbitrary field points h_xy (host double [K][2],
 * (x, y) in lambda/D) instead of a scene grid; column j is the interpolated,
 * rotated PSF of point j (Sec. 2 loop body).  Used for planets at sub-pixel
 * offsets and for the exact invariants.  Copies h_xy synchronously. */
int psfsim_build_points(const float *d_lib, const double *h_radii, int n_r, int n, double s,
                        const double *h_xy, int64_t K, int storage, int interp,
                        void *d_workspace, size_t workspace_bytes, void *stream, psfsim_t *out);

/* Fill *info with the plan's layout. */
int psfsim_info(psfsim_t h, psfsim_info_t *info);

/* Scratch bytes psfsim_forward / psfsim_adjoint need for a batch of B. */
int psfsim_forward_scratch_bytes(psfsim_t h, int B, size_t *bytes);
int psfsim_adjoint_scratch_bytes(psfsim_t h, int B, size_t *bytes);

/* Simulated images S = A Z (Eq. 6) for B scenes.
 *   d_x  device float32 [B][K]; d_y device float32 [B][M] (written);
 *   d_scratch at least psfsim_forward_scratch_bytes(h, B), 256-byte aligned.
 * Deterministic: the same inputs give bitwise the same images. */
int psfsim_forward(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch,
                   size_t scratch_bytes, void *stream);

/* S = A Z (Eq. 6) reading only the columns of scene pixels that are non-zero
 * in some scene of the batch (a zero pixel adds nothing to S): point sources,
 * masked disks and everything beyond the outer working angle leave those
 * columns unread.  FP32 storage only (else PSFSIM_ERR_UNSUPPORTED).  Same
 * arguments and result as psfsim_forward, up to the order of the float32 sums;
 * deterministic.  The list of columns is built on the device, so the call
 * never synchronises. */
int psfsim_forward_sparse_scratch_bytes(psfsim_t h, int B, size_t *bytes);
int psfsim_forward_sparse(psfsim_t h, const float *d_x, int B, float *d_y, void *d_scratch,
                          size_t scratch_bytes, void *stream);

/* One product of a multi-job launch: S = A Z for up to 80 scenes of one
 * SPLIT_BF16 plan.  d_count (device int, may be NULL) holds how many of the
 * `capacity` scene slots are present in this call, so a captured CUDA graph
 * can be replayed for batches of different composition; slots at and beyond
 * *d_count are neither read nor written. */
typedef struct {
  psfsim_t plan;
  const float *d_x;   /* device float32 [capacity][K] */
  float *d_y;         /* device float32 [capacity][M] */
  int capacity;       /* 1..80 */
  const int *d_count; /* device int, or NULL for all `capacity` scenes */
} psfsim_job_t;

/* Launch-shape knobs of the tensor-core forward (0 = default): k-tiles (of 64)
 * accumulated in TMEM between drains (at most 8 with split-BF16 storage, 16
 * with BF16 storage: larger values are clamped), target work units per SM,
 * and shared-memory pipeline stages (2..8; a count outside 2 .. the number
 * that fits takes the default, as many as fit). */
typedef struct {
  int chunk;
  int units_per_sm;
  int stages;
} psfsim_tuning_t;

/* Batched S_j = A_j Z_j (Eq. 6) for several SPLIT_BF16 plans at once — e.g.
 * scenes of different sizes and pixel scales, each with its own A — in one
 * persistent tensor-core launch whose work units interleave all jobs (plus one
 * split and one reduction launch per job).  1 <= njobs <= 16, all plans on
 * the current device.  `tuning` may be NULL.  Deterministic. */
int psfsim_forward_multi_scratch_bytes(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tuning,
                                       size_t *bytes);
int psfsim_forward_multi(const psfsim_job_t *jobs, int njobs, const psfsim_tuning_t *tuning, void *d_scratch,
                         size_t scratch_bytes, void *stream);

/* Capacity of the fixed device array psfsim_forward_static works in. */
#define PSFSIM_STATIC_SCRATCH_BYTES ((size_t)16 * 1024 * 1024)

/* psfsim_forward without caller scratch, for callers that cannot allocate
 * device memory when they simulate an image and have no spare buffer to pass:
 * a plug-in running inside a host application that owns the GPU's allocator,
 * or a fixed-memory loop that may not grow its footprint after start-up.  The
 * paper has no counterpart; this is a deployment convenience.
 *   Same arguments and result as psfsim_forward (FP32 storage only), but the
 *   partial sums live in a PSFSIM_STATIC_SCRATCH_BYTES array compiled into
 *   the library.  The driver reserves that array on a device when it loads
 *   the library's device code there -- with CUDA's default lazy loading, at
 *   the first psfsim_forward_static call on that device, so 16 MiB of device
 *   memory must be free at that moment -- and the device holds it until the
 *   process exits.  The call itself allocates nothing: no cudaMalloc, no
 *   cudaFree, no allocating library call.
 *   Returns PSFSIM_ERR_WORKSPACE when this plan's partial sums for B scenes
 *   (psfsim_forward_scratch_bytes(h, B)) exceed PSFSIM_STATIC_SCRATCH_BYTES,
 *   PSFSIM_ERR_ARG when the current device is not the plan's device.
 *   The first call on a device looks up the array's device address (a
 *   cudaGetSymbolAddress with the device current), and so does the first
 *   call after the device's context was replaced (e.g. by cudaDeviceReset):
 *   the address is cached per context.  Make that first call before any
 *   stream capture.
 *   All calls share the one array: calls whose kernels overlap on the GPU
 *   (other streams, other threads, other plans) race and corrupt each
 *   other's images.  Calls ordered on one stream are safe; leftover contents
 *   from an earlier call are always overwritten before they are read. */
int psfsim_forward_static(psfsim_t h, const float *d_x, int B, float *d_y, void *stream);

/* Transpose product g_x = A^T g for B image-space vectors (the adjoint of
 * psfsim_forward; the paper's S = A Z read backwards, used for gradients).
 *   d_g device float32 [B][M]; d_gx device float32 [B][K] (written). */
int psfsim_adjoint(psfsim_t h, const float *d_g, int B, float *d_gx, void *d_scratch,
                   size_t scratch_bytes, void *stream);

/* Block until `stream` drains, then report a device-side status recorded by
 * this plan's kernels (PSFSIM_ERR_TIMEOUT if a bounded wait gave up). */
int psfsim_sync_status(psfsim_t h, void *stream);

/* Clear the plan's device status word (enqueued on `stream`), so that a
 * later psfsim_sync_status reports only what happens after this call.  The
 * word is sticky otherwise: a timeout stays recorded until it is cleared. */
int psfsim_reset_status(psfsim_t h, void *stream);

/* Release the host handle.  Device buffers stay the caller's. */
void psfsim_free(psfsim_t h);

#ifdef __cplusplus
}
#endif
#endif /* PSFSIM_H */
