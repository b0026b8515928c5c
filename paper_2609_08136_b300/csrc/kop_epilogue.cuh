// Kernel-function epilogue shared by the fused operator kernels.
//
// The kernels see a pre-scaled squared distance u = s * D2, with the scale s
// folded into the row norms and into the MMA result:
//     u = s|q_i|^2 + s|x_j|^2 - 2 s (q_i . x_j)
//   RBF       s = -log2(e) / (2 bw^2):  k = 2^u
//   Laplace   s = (log2(e) / bw)^2:     k = 2^-sqrt(u)
//   Matern52  s = 5 / bw^2:             a = sqrt(u), k = (1 + a + u/3) 2^(-log2(e) a)
// and the bandwidth derivatives dk/dbw:
//   RBF       k D2 / bw^3        = 2^u * u * c2,  c2 = 1 / (s bw^3)
//   Laplace   k r / bw^2         = 2^-sqrt(u) * sqrt(u) * c2,  c2 = 1 / (sqrt(s) bw^2)
//   Matern52  e^-a (a^2/3)(1+a)/bw = 2^(-log2(e) a) (u/3)(1 + a) c2,  c2 = 1 / bw
// and the radial derivatives h(r) = -k'(r) / r of the point gradient:
//   RBF       k / bw^2                = 2^u * c2,                  c2 = 1 / bw^2
//   Laplace   k / (bw r)              = 2^-sqrt(u) / sqrt(u) * c2,  c2 = log2(e) / bw^2
//             (0 at r = 0, where the Laplace kernel has no derivative)
//   Matern52  (5 / 3 bw^2)(1 + a) e^-a = (1 + a) 2^(-log2(e) a) c2,  c2 = 5 / (3 bw^2)
// u can be slightly negative from rounding when D2 ~ 0: the square root takes
// |u|.  It is formed as |u| * rsqrt(max(|u|, 1e-30)) (exactly 0 at u = 0): one
// special-function op, which measured faster than sqrt.approx in the fused
// products.
#pragma once
#include "kop_device.cuh"

namespace kop {

constexpr float kNegLog2e = -1.4426950408889634f;

// sqrt(|u|) and, in rs, 1 / sqrt(max(|u|, 1e-30)).
KOP_DEV float sqrt_rs(float u, float& rs) {
  const float au = fabsf(u);
  rs = rsqrt_approx(fmaxf(au, 1e-30f));
  return au * rs;
}

template <int KF>
KOP_DEV float kval_u(float u, float c2) {
  float rs;
  if constexpr (KF == 0) {
    return ex2_approx(u);
  } else if constexpr (KF == 1) {
    return ex2_approx(-sqrt_rs(u, rs));
  } else if constexpr (KF == 2) {
    const float a = sqrt_rs(u, rs);
    return fmaf(u, 1.0f / 3.0f, 1.0f + a) * ex2_approx(kNegLog2e * a);
  } else if constexpr (KF == 3) {
    return ex2_approx(u) * u * c2;
  } else if constexpr (KF == 4) {
    const float r = sqrt_rs(u, rs);
    return ex2_approx(-r) * r * c2;
  } else if constexpr (KF == 6) {
    return ex2_approx(u) * c2;
  } else if constexpr (KF == 7) {
    const float a = sqrt_rs(u, rs);
    return a > 0.0f ? ex2_approx(-a) * rs * c2 : 0.0f;
  } else if constexpr (KF == 8) {
    const float a = sqrt_rs(u, rs);
    return (1.0f + a) * ex2_approx(kNegLog2e * a) * c2;
  } else {
    const float a = sqrt_rs(u, rs);
    return ex2_approx(kNegLog2e * a) * (u * (1.0f / 3.0f)) * (1.0f + a) * c2;
  }
}

// kval_u on two independent entries; for the Laplace kernel the FP32 product
// sqrt(u) = |u| rsqrt(|u|) is packed two lanes per instruction (each lane's
// value is bit-identical to kval_u).  The other kernels take kval_u per lane:
// packing Matern's arithmetic spilled registers in the symmetric product.
template <int KF>
KOP_DEV float2 kval_u2(float2 u, float c2) {
  if constexpr (KF == 1) {
    const float2 au = make_float2(fabsf(u.x), fabsf(u.y));
    const float2 rs = make_float2(rsqrt_approx(fmaxf(au.x, 1e-30f)), rsqrt_approx(fmaxf(au.y, 1e-30f)));
    const float2 a = mul2(au, rs);
    return make_float2(ex2_approx(-a.x), ex2_approx(-a.y));
  } else {
    return make_float2(kval_u<KF>(u.x, c2), kval_u<KF>(u.y, c2));
  }
}

}  // namespace kop
