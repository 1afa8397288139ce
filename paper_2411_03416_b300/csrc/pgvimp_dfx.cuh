// pgvimp_dfx.cuh -- double-float reciprocal and four-term dot product (host
// and device), on top of the df64 arithmetic of pgvimp_device.cuh.
#pragma once
#include "pgvimp_device.cuh"

namespace pgv {

// FP32 reciprocal estimate: the hardware approximation (at most 1 ulp off)
// on the device, IEEE division on the host.
PGV_HD float df_rcp_estimate(float a) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
#else
  return 1.0f / a;
#endif
}

// 1/v by Newton-Raphson steps on the FP32 estimate r of 1/v.hi: one step in
// FP32, r + r (1 - v.hi r), which brings r to within about 2^-24 of 1/v.hi;
// then one double-float step r (1 + e) with the residual e = 1 - v r formed
// by two FMAs, leaving a relative error of about e^2 + 2^-46.  FP32 and FMA
// operations only.
PGV_HD df64 df_rcp(df64 v) {
  float r = df_rcp_estimate(v.hi);
  r = PGV_FFMA(r, PGV_FFMA(-v.hi, r, 1.0f), r);
  const float t = PGV_FFMA(-v.hi, r, 1.0f);
  const float e = PGV_FFMA(-v.lo, r, t);
  return df_fast_two_sum(r, PGV_FMUL(r, e));
}

PGV_HD void df_two_sum(float a, float b, float& s, float& e) {
  s = PGV_FADD(a, b);
  const float z = PGV_FSUB(s, a);
  e = PGV_FADD(PGV_FSUB(a, PGV_FSUB(s, z)), PGV_FSUB(b, z));
}

// sum_{t<4} x_t y_t: the compensated dot product of Ogita, Rump and Oishi
// (2005) on double-float operands -- each product split by the FMA
// two-product (its residual also collecting the cross terms with the low
// parts), the four leading parts summed by a tree of two-sums, every residual
// summed in FP32, one final renormalisation.
PGV_HD df64 df_dot4(const df64* x, const df64* y) {
  float p[4], e[4];
  for (int t = 0; t < 4; ++t) {
    p[t] = PGV_FMUL(x[t].hi, y[t].hi);
    e[t] = PGV_FFMA(x[t].hi, y[t].hi, -p[t]);
    e[t] = PGV_FFMA(x[t].hi, y[t].lo, e[t]);
    e[t] = PGV_FFMA(x[t].lo, y[t].hi, e[t]);
  }
  float s01, r01, s23, r23, s, r;
  df_two_sum(p[0], p[1], s01, r01);
  df_two_sum(p[2], p[3], s23, r23);
  df_two_sum(s01, s23, s, r);
  const float err = PGV_FADD(PGV_FADD(PGV_FADD(e[0], e[1]), PGV_FADD(e[2], e[3])), PGV_FADD(PGV_FADD(r01, r23), r));
  return df_fast_two_sum(s, err);
}

}  // namespace pgv
