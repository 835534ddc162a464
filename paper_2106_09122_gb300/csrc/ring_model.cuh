// Ring scene model shared by the fit operators (ring.cu) and the fused
// fit-gradient kernels (fit_gradient.cu).  See include/psfsim_fit.h for the model.
#pragma once

#include <stdint.h>

#include <cmath>

struct RingParams {
  int N;
  double S, r_max;
  float r2f;  // r_max^2 rounded to float
  float R, w, inc, g, B;
};

// Z_j and (optionally) dZ_j/d(R, w, i, g, B) for scene pixel j.
template <bool kJac>
__device__ __forceinline__ float ring_eval(const RingParams &P, int64_t j, float *J) {
  const int iy = (int)(j / P.N), ix = (int)(j % P.N);
  const float halff = 0.5f * (float)(P.N - 1);  // exact: a half-integer below 2^15
  const float Sf = (float)P.S;
  const float x = ((float)ix - halff) * Sf, y = ((float)iy - halff) * Sf;
  // Inside the disk of radius r_max: decided in FP32 where x^2 + y^2 is more
  // than a relative 1e-5 away from r_max^2 (the FP32 error is below 1e-6),
  // else by the FP64 test, so the decision equals the FP64 one everywhere.
  const float d2 = x * x + y * y, r2 = P.r2f;
  bool inside;
  if (d2 < r2 * 0.99999f) {
    inside = true;
  } else if (d2 > r2 * 1.00001f) {
    inside = false;
  } else {
    const double half = 0.5 * (double)(P.N - 1);
    const double xs = __dmul_rn((double)ix - half, P.S), ys = __dmul_rn((double)iy - half, P.S);
    inside = __dsqrt_rn(__dadd_rn(__dmul_rn(xs, xs), __dmul_rn(ys, ys))) <= P.r_max;
  }
  if (!inside) {
    if (kJac)
      for (int m = 0; m < 5; ++m) J[m] = 0.f;
    return 0.f;
  }
  float si, ci;
  sincosf(P.inc, &si, &ci);
  const float yd = y / ci;
  const float rd = sqrtf(x * x + yd * yd);
  const bool pos = rd > 0.f;
  const float mu = pos ? si * yd / rd : 0.f;
  const float alpha = 2.7725887222397811f;  // 4 ln 2
  const float dr = rd - P.R;
  const float w2 = P.w * P.w;
  const float G = expf(-alpha * dr * dr / w2);
  const float g2 = 1.f + P.g * P.g;
  const float den = g2 - 2.f * P.g * mu;
  const float ratio = g2 / den;
  const float H = ratio * sqrtf(ratio);
  const float z = P.B * G * H;
  if (kJac) {
    const float dyd_di = yd * si / ci;
    const float drd_di = pos ? yd * dyd_di / rd : 0.f;
    const float dmu_di = pos ? ci * yd / rd + si * (dyd_di * rd - yd * drd_di) / (rd * rd) : 0.f;
    const float dG_dR = G * 2.f * alpha * dr / w2;
    const float dG_dw = G * 2.f * alpha * dr * dr / (w2 * P.w);
    const float dG_di = -dG_dR * drd_di;
    const float dH_dmu = 3.f * P.g * H / den;
    const float dH_dg = H * 1.5f * (2.f * P.g / g2 - (2.f * P.g - 2.f * mu) / den);
    J[0] = P.B * dG_dR * H;
    J[1] = P.B * dG_dw * H;
    J[2] = P.B * (dG_di * H + G * dH_dmu * dmu_di);
    J[3] = P.B * G * dH_dg;
    J[4] = G * H;
  }
  return z;
}

// Host: validate (N, S, r_max, theta) and fill the kernel parameters.
inline bool ring_params(int N, double S, double r_max, const double *th, RingParams *P) {
  if (N < 1 || N > 32768 || !(S > 0.0) || !th || !(r_max >= 0.0)) return false;
  for (int m = 0; m < 5; ++m)
    if (!std::isfinite(th[m])) return false;
  if (!(th[1] > 0.0) || !(std::fabs(std::cos(th[2])) > 1e-6) || !(std::fabs(th[3]) < 1.0)) return false;
  P->N = N;
  P->S = S;
  P->r_max = r_max;
  P->r2f = (float)(r_max * r_max);
  P->R = (float)th[0];
  P->w = (float)th[1];
  P->inc = (float)th[2];
  P->g = (float)th[3];
  P->B = (float)th[4];
  return true;
}

inline bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

