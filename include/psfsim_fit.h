/*
 * psfsim fit operators: the exozodiacal ring scene model, the image-space
 * loss and the chain rule into the ring parameters.
 *
 * The paper's flow chart (Fig. 3) ends in retrieving exozodi parameters from
 * simulated images (an MCMC it leaves to future work, Sec. 5); these calls
 * give the pieces a gradient-based retrieval needs around S = A Z (Eq. 6):
 *   Z = ring(theta)  ->  S = A Z (psfsim_forward)  ->  L = 1/2 sum((S-d)/sigma)^2
 *   dL/dZ = A^T (S-d)/sigma^2 (psfsim_adjoint)  ->  dL/dtheta = (dZ/dtheta)^T dL/dZ.
 *
 * Ring model, theta = (R, w, i, g, B) in (lambda/D, lambda/D, rad, -, flux):
 *   yd = y / cos i, rd = sqrt(x^2 + yd^2), mu = sin i * yd / rd (0 at rd = 0)
 *   Z  = B exp(-4 ln2 (rd - R)^2 / w^2) ((1+g^2) / (1+g^2-2 g mu))^(3/2)
 *   for sqrt(x^2 + y^2) <= r_max, else 0 (w is the radial FWHM; the last
 *   factor is the Henyey-Greenstein phase function over its value at mu = 0).
 * Scene pixels as in psfsim.h (x_j = (ix - (N-1)/2) S, row-major j).
 * Per-pixel model values are float32; all reductions are float64 and
 * deterministic (fixed order).  Calls are asynchronous on `stream`; scratch
 * is caller-owned device memory, 256-byte aligned.
 */
#ifndef PSFSIM_FIT_H
#define PSFSIM_FIT_H

#include <stddef.h>
#include <stdint.h>

#include "psfsim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Scratch bytes for psfsim_ring_chain (scene of N*N pixels) and for
 * psfsim_residual_loss (image of M pixels). */
int psfsim_ring_chain_scratch_bytes(int N, size_t *bytes);
int psfsim_loss_scratch_bytes(int64_t M, size_t *bytes);

/* Z(theta) -> d_z (device float32 [N*N]).  h_theta: host double[5]. */
int psfsim_ring_scene(int N, double S, double r_max, const double *h_theta, float *d_z, void *stream);

/* d_dtheta (device double[5]) = sum_j d_gz[j] dZ_j/dtheta. */
int psfsim_ring_chain(int N, double S, double r_max, const double *h_theta, const float *d_gz,
                      double *d_dtheta, void *d_scratch, size_t scratch_bytes, void *stream);

/* d_loss (device double[1]) = 1/2 sum_i ((y_i - d_i)/sigma)^2 and, if d_r is
 * not NULL, d_r[i] = (y_i - d_i)/sigma^2 (float32), the dL/dS the adjoint needs. */
int psfsim_residual_loss(const float *d_y, const float *d_d, int64_t M, double sigma, float *d_r,
                         double *d_loss, void *d_scratch, size_t scratch_bytes, void *stream);

/* One whole fit gradient on an FP32 grid plan, in two launches: the first
 * evaluates the ring scene (d_z) and its parameter Jacobian, S = A Z (d_y),
 * the residual r = (S - d)/sigma^2 (d_r) and FP64 loss partials; the second
 * forms A^T r (d_gz), its dot with the Jacobian and the final sums:
 * d_out (device double[6]) = {L, dL/dR, dL/dw, dL/di, dL/dg, dL/dB}.
 * The scene grid (N, S) is the plan's.  Same quantities as psfsim_ring_scene
 * + psfsim_forward + psfsim_residual_loss + psfsim_adjoint + psfsim_ring_chain,
 * deterministic, with sums in a different (fixed) order.
 * FP32_SYM plans (even N) take three launches: the forward leaves the four
 * quarter-turned partial images, a second kernel sums them into S and forms r
 * and the loss partials, and the adjoint scatters A^T r to the four turned
 * pixels of each stored column.  PSFSIM_ERR_UNSUPPORTED for other storages or
 * point builds.  The two halves
 * are also callable on their own (same scratch, same theta, in this order):
 * the first leaves the loss partials and dZ/dtheta in the scratch for the
 * second.  The scratch holds arrival counters: zero-fill it once before its
 * first use; every call leaves the counters at zero again.  d_target and
 * d_out may also be pinned host memory mapped into the device's address
 * space: the kernels then read the target and write the result across the
 * CPU-GPU link, with no copy between consecutive gradients. */
int psfsim_ring_gradient_scratch_bytes(psfsim_t h, size_t *bytes);
int psfsim_ring_forward_loss(psfsim_t h, double r_max, const double *h_theta, const float *d_target, double sigma,
                             float *d_z, float *d_y, float *d_r, void *d_scratch, size_t scratch_bytes,
                             void *stream);
int psfsim_ring_adjoint_chain(psfsim_t h, double r_max, const double *h_theta, const float *d_r, float *d_gz,
                              double *d_out, void *d_scratch, size_t scratch_bytes, void *stream);
int psfsim_ring_gradient(psfsim_t h, double r_max, const double *h_theta, const float *d_target, double sigma,
                         float *d_z, float *d_y, float *d_r, float *d_gz, double *d_out, void *d_scratch,
                         size_t scratch_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PSFSIM_FIT_H */
