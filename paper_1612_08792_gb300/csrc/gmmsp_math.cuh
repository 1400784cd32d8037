// Per-superpixel small-matrix arithmetic of the M-step tail, templated on the
// scalar type: double for the mixed-precision path, float for the all-FP32
// variant.
//
// GB300 runs FP64 at about 1/64 of the FP32 rate and a dependent FP64
// multiply-add takes about 64 clocks, so the FP64 code below avoids FP64
// division, square root and transcendental functions: reciprocals and
// eigenvalues start from an FP32 estimate and are refined by FP64 Newton
// steps, which gives FP64-accurate results with short dependency chains.
//
//  * clamp_sym2 / clamp_sym3: the eigenvalue floor of Eq. (mlams)/(mlamc)
//    followed by the reconstruction of Eq. (eigdecrs)/(eigdecrc).  Writing the
//    covariance as sum_j lambda_j P_j with P_j its spectral projectors, the
//    floored matrix is Sigma + sum_{lambda_j < eps} (eps - lambda_j) P_j.  At
//    most one projector is needed: with one raised eigenvalue it is P_1, with
//    two it is I - P_3 (the floored matrix is then eps I + (lambda_3 - eps) P_3),
//    and each projector is a polynomial in Sigma (Lagrange form over the
//    eigenvalues), so no eigenvectors are formed.  Whether any eigenvalue is
//    below the floor is decided first from the leading principal minors of
//    Sigma - eps I (Sylvester's criterion), which needs no eigenvalues.  The
//    2x2 eigenvalues are in closed form; the 3x3 ones start from the
//    trigonometric solution of the characteristic cubic (O. K. Smith,
//    "Eigenvalues of a symmetric 3x3 matrix", Comm. ACM 4(4), 1961) and are
//    polished by Newton steps on the cubic.
//  * pack_gp: inverse and log-determinant of the floored blocks (adjugate
//    formula) folded into the packed FP32 E-step coefficients.
#pragma once

#include <math.h>

#include "gmmsp_fpconv.cuh"
#include "gmmsp_internal.cuh"

namespace gmmsp {

template <typename T> struct Num;

template <> struct Num<double> {
  static constexpr double kLog2e = 1.4426950408889634074;
  static constexpr double kHalfD_Log2_2Pi = 6.6287403236807968;  // (5/2) log2(2 pi)
  static constexpr double kHalf3_Log2_2Pi = 3.9772441942084784;  // (3/2) log2(2 pi)
  // 1/x: FP32 estimate (MUFU, relative error < 2^-22), two Newton steps.
  static __device__ __forceinline__ double rcp(double x) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(narrow(x)));
    double r = widen(r0);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
  }
  // sqrt(x), x > 0: FP32 estimate of 1/sqrt, two Newton steps, then x * rsqrt.
  static __device__ __forceinline__ double sqrt_(double x) {
    double y = widen(rsqrtf(narrow(x)));
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return x * y;
  }
  // log2(x), x > 0 normal, to FP32 accuracy (the result is stored as FP32):
  // exponent from the bits, mantissa in [1, 2) through the FP32 log2.
  static __device__ __forceinline__ float log2_(double x) {
    const long long b = __double_as_longlong(x);
    const int e = int((b >> 52) & 0x7ff) - 1023;
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    return float(e) + __log2f(narrow(m));
  }
};

template <> struct Num<float> {
  static constexpr float kLog2e = 1.44269504f;
  static constexpr float kHalfD_Log2_2Pi = 6.62874032f;
  static constexpr float kHalf3_Log2_2Pi = 3.97724419f;
  static __device__ __forceinline__ float rcp(float x) { return 1.0f / x; }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float log2_(float x) { return log2f(x); }
};

// Floor the eigenvalues of the symmetric 2x2 A = {xx, xy, yy} at eps.
// Returns the number of raised eigenvalues.
template <typename T>
__device__ int clamp_sym2(T* A, T eps) {
  using M = Num<T>;
  const T a = A[0], b = A[1], c = A[2];
  // Sylvester on A - eps I: both eigenvalues >= eps when both minors are > 0.
  if (a - eps > T(0) && fma(a - eps, c - eps, -b * b) > T(0)) return 0;
  const T m = T(0.5) * (a + c), h = T(0.5) * (a - c);
  const T r2 = fma(h, h, b * b);
  const T r = r2 > T(0) ? M::sqrt_(r2) : T(0);
  const T l1 = m - r, l2 = m + r;  // l1 <= l2
  const int n = (l1 < eps) + (l2 < eps);
  if (n == 0) return 0;
  if (n == 2 || r <= T(1e-12) * (fabs(m) + eps)) {
    const T f = (n == 2) ? eps : (m > eps ? m : eps);
    A[0] = f; A[1] = T(0); A[2] = f;
    return n;
  }
  // One raised: A + (eps - l1) P_1 with P_1 = (l2 I - A) / (l2 - l1).
  const T g = (eps - l1) * M::rcp(T(2) * r);
  A[0] = fma(g, l2 - a, a);
  A[1] = fma(-g, b, b);
  A[2] = fma(g, l2 - c, c);
  return 1;
}

// Eigenvalues of a symmetric 3x3 in FP32 (Smith 1961), ascending.
__device__ __forceinline__ void eig3_seed(float a00, float a01, float a02, float a11, float a12,
                                          float a22, float& l1, float& l2, float& l3) {
  const float q = (a00 + a11 + a22) * (1.f / 3.f);
  const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const float p2 = (b00 * b00 + b11 * b11 + b22 * b22 +
                    2.f * (a01 * a01 + a02 * a02 + a12 * a12)) * (1.f / 6.f);
  if (!(p2 > 0.f)) { l1 = l2 = l3 = q; return; }
  const float p = sqrtf(p2);
  const float detB = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                     a02 * (a01 * a12 - b11 * a02);
  float hr = detB / (2.f * p2 * p);
  hr = fminf(1.f, fmaxf(-1.f, hr));
  const float phi = acosf(hr) * (1.f / 3.f);
  l3 = q + 2.f * p * cosf(phi);
  l1 = q + 2.f * p * cosf(phi + 2.09439510f);
  l2 = 3.f * q - l1 - l3;
}

// Floor the eigenvalues of the symmetric 3x3 A = {LL, La, Lb, aa, ab, bb}.
template <typename T>
__device__ int clamp_sym3(T* A, T eps) {
  using M = Num<T>;
  const T a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
  // Sylvester's criterion on A - eps I: all leading minors > 0 <=> every
  // eigenvalue of A is above the floor.
  {
    const T e00 = a00 - eps, e11 = a11 - eps, e22 = a22 - eps;
    const T m2 = fma(e00, e11, -a01 * a01);
    const T c00 = fma(e11, e22, -a12 * a12);
    const T c01 = fma(a02, a12, -a01 * e22);
    const T c02 = fma(a01, a12, -a02 * e11);
    const T m3 = fma(e00, c00, fma(a01, c01, a02 * c02));
    if (e00 > T(0) && m2 > T(0) && m3 > T(0)) return 0;
  }
  // Characteristic cubic lambda^3 - c2 lambda^2 + c1 lambda - c0.
  const T c2 = a00 + a11 + a22;
  const T c1 = fma(a00, a11, -a01 * a01) + fma(a00, a22, -a02 * a02) + fma(a11, a22, -a12 * a12);
  const T c0 = a00 * fma(a11, a22, -a12 * a12) - a01 * fma(a01, a22, -a12 * a02) +
               a02 * fma(a01, a12, -a11 * a02);
  float f1, f2, f3;
  eig3_seed(to_f32(a00), to_f32(a01), to_f32(a02), to_f32(a11), to_f32(a12), to_f32(a22), f1, f2, f3);
  const T t1 = from_f32<T>(f1), t2 = from_f32<T>(f2), t3 = from_f32<T>(f3);
  const int n = (t1 < eps) + (t2 < eps) + (t3 < eps);
  if (n == 0) return 0;
  const T spread = t3 - t1;
  const T scale = fabs(t3) + eps;
  if (n == 3 || spread <= T(1e-6) * scale) {
    const T f = (n == 3) ? eps : (c2 / T(3) > eps ? c2 / T(3) : eps);
    A[0] = f; A[1] = T(0); A[2] = T(0); A[3] = f; A[4] = T(0); A[5] = f;
    return n;
  }
  // The raised eigenvalue (n = 1) or the one kept (n = 2), polished by two
  // Newton steps on the cubic; the other two enter only through their sum and
  // product, which follow from the cubic's coefficients.
  T lj = (n == 1) ? t1 : t3;
  T dp = T(0);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const T pv = fma(fma(lj - c2, lj, c1), lj, -c0);   // p(lj)
    dp = fma(fma(T(3), lj, -T(2) * c2), lj, c1);        // p'(lj)
    if (fabs(dp) > T(1e-12) * scale * scale) lj -= pv * from_f32<T>(__frcp_rn(to_f32(dp)));
  }
  dp = fma(fma(T(3), lj, -T(2) * c2), lj, c1);  // (lj - la)(lj - lb)
  if (!(fabs(dp) > T(1e-12) * scale * scale)) {
    const T f = c2 / T(3) > eps ? c2 / T(3) : eps;
    A[0] = f; A[1] = T(0); A[2] = T(0); A[3] = f; A[4] = T(0); A[5] = f;
    return n;
  }
  const T sum = c2 - lj;                   // la + lb
  const T prod = fma(-lj, sum, c1);        // la lb
  // S2 = A * A (symmetric, six entries).
  const T s00 = fma(a00, a00, fma(a01, a01, a02 * a02));
  const T s01 = fma(a00, a01, fma(a01, a11, a02 * a12));
  const T s02 = fma(a00, a02, fma(a01, a12, a02 * a22));
  const T s11 = fma(a01, a01, fma(a11, a11, a12 * a12));
  const T s12 = fma(a01, a02, fma(a11, a12, a12 * a22));
  const T s22 = fma(a02, a02, fma(a12, a12, a22 * a22));
  // Projector onto lj: (A^2 - (la + lb) A + la lb I) / ((lj - la)(lj - lb)).
  const T g = ((n == 1) ? (eps - lj) : (lj - eps)) * M::rcp(dp);
  const T P00 = fma(-sum, a00, s00) + prod, P01 = fma(-sum, a01, s01), P02 = fma(-sum, a02, s02);
  const T P11 = fma(-sum, a11, s11) + prod, P12 = fma(-sum, a12, s12), P22 = fma(-sum, a22, s22) + prod;
  if (n == 1) {
    // A + (eps - l1) P_1
    A[0] = fma(g, P00, a00); A[1] = fma(g, P01, a01); A[2] = fma(g, P02, a02);
    A[3] = fma(g, P11, a11); A[4] = fma(g, P12, a12); A[5] = fma(g, P22, a22);
  } else {
    // eps I + (l3 - eps) P_3
    A[0] = fma(g, P00, eps); A[1] = g * P01; A[2] = g * P02;
    A[3] = fma(g, P11, eps); A[4] = g * P12; A[5] = fma(g, P22, eps);
  }
  return n;
}

// Packs mu and the (floored) blocks into the FP32 E-step coefficients.  The
// spatial mean is stored relative to (ox, oy), the first pixel of the
// superpixel's own grid cell (k_x v, k_y v), so that it keeps FP32 precision
// on large images (absolute coordinates near 4000 would round to 2.4e-4 px).
// Returns false when a block is not positive definite (leading minors).
// cm: the colour model.  Split: cc's La, Lb entries are taken as 0.
// Grayscale: only cc[0] and mu[0..2] are read, the a, b coefficients are 0
// and the normaliser is that of a 3-dimensional Gaussian.
template <typename T>
__device__ bool pack_gp(const T* mu, const T* cs, const T* cc_in, T ox, T oy, float* gp, int cm = kColourFull) {
  using M = Num<T>;
  // spatial 2x2
  const T ds = fma(cs[0], cs[2], -cs[1] * cs[1]);
  float4* o = reinterpret_cast<float4*>(gp);
  if (cm == kColourGray) {
    if (!(cs[0] > T(0) && ds > T(0) && cc_in[0] > T(0))) return false;
    const T hs = T(-0.5) * M::kLog2e * M::rcp(ds);
    const T hc = T(-0.5) * M::kLog2e * M::rcp(cc_in[0]);
    o[0] = make_float4(to_f32(mu[0] - ox), to_f32(mu[1] - oy), to_f32(mu[2]), 0.f);
    o[1] = make_float4(0.f, to_f32(hs * cs[2]), to_f32(T(-2) * hs * cs[1]), to_f32(hs * cs[0]));
    o[2] = make_float4(to_f32(hc), 0.f, 0.f, 0.f);
    const float lnorm = -0.5f * (M::log2_(ds) + M::log2_(cc_in[0])) - float(M::kHalf3_Log2_2Pi);
    o[3] = make_float4(0.f, 0.f, lnorm, 0.f);
    return true;
  }
  const bool split = cm == kColourSplit;
  const T cc[6] = {cc_in[0], split ? T(0) : cc_in[1], split ? T(0) : cc_in[2], cc_in[3], cc_in[4], cc_in[5]};
  // colour 3x3 cofactors
  const T c00 = fma(cc[3], cc[5], -cc[4] * cc[4]);
  const T c01 = fma(cc[2], cc[4], -cc[1] * cc[5]);
  const T c02 = fma(cc[1], cc[4], -cc[2] * cc[3]);
  const T c11 = fma(cc[0], cc[5], -cc[2] * cc[2]);
  const T c12 = fma(cc[1], cc[2], -cc[0] * cc[4]);
  const T c22 = fma(cc[0], cc[3], -cc[1] * cc[1]);
  const T dc = fma(cc[0], c00, fma(cc[1], c01, cc[2] * c02));
  if (!(cs[0] > T(0) && ds > T(0) && cc[0] > T(0) && c22 > T(0) && dc > T(0))) return false;
  const T hs = T(-0.5) * M::kLog2e * M::rcp(ds);   // -(1/2) log2(e) / det
  const T hc = T(-0.5) * M::kLog2e * M::rcp(dc);
  o[0] = make_float4(to_f32(mu[0] - ox), to_f32(mu[1] - oy), to_f32(mu[2]), to_f32(mu[3]));
  o[1] = make_float4(to_f32(mu[4]), to_f32(hs * cs[2]), to_f32(T(-2) * hs * cs[1]), to_f32(hs * cs[0]));
  o[2] = make_float4(to_f32(hc * c00), to_f32(hc * c11), to_f32(hc * c22), to_f32(T(2) * hc * c01));
  const float lnorm = -0.5f * (M::log2_(ds) + M::log2_(dc)) - float(M::kHalfD_Log2_2Pi);
  o[3] = make_float4(to_f32(T(2) * hc * c02), to_f32(T(2) * hc * c12), lnorm, 0.f);
  return true;
}

}  // namespace gmmsp
