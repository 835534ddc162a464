// Ring scene model shared by the fit operators (ring.cu) and the fused
// adjoint + chain kernel (gemv.cu).  See include/psfsim_fit.h for the model.
#pragma once

#include <stdint.h>

struct RingParams {
  int N;
  double S, r_max;
  float R, w, inc, g, B;
};

// Z_j and (optionally) dZ_j/d(R, w, i, g, B) for scene pixel j.
template <bool kJac>
__device__ __forceinline__ float ring_eval(const RingParams &P, int64_t j, float *J) {
  const int iy = (int)(j / P.N), ix = (int)(j % P.N);
  const double half = 0.5 * (double)(P.N - 1);
  const double xs = __dmul_rn((double)ix - half, P.S), ys = __dmul_rn((double)iy - half, P.S);
  const bool inside = __dsqrt_rn(__dadd_rn(__dmul_rn(xs, xs), __dmul_rn(ys, ys))) <= P.r_max;
  if (!inside) {
    if (kJac)
      for (int m = 0; m < 5; ++m) J[m] = 0.f;
    return 0.f;
  }
  const float x = (float)xs, y = (float)ys;
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

