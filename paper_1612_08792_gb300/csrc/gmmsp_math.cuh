// Per-superpixel small-matrix arithmetic of the M-step tail, templated on the
// scalar type: double for the mixed-precision path, float for the all-FP32
// variant.
//
//  * clamp_sym2 / clamp_sym3: the eigenvalue floor of Eq. (mlams)/(mlamc)
//    followed by the reconstruction of Eq. (eigdecrs)/(eigdecrc).  Writing the
//    covariance as sum_j lambda_j P_j with P_j its spectral projectors, the
//    floored matrix is Sigma + sum_{lambda_j < eps} (eps - lambda_j) P_j.  At
//    most one projector is needed: with one raised eigenvalue it is P_1, with
//    two it is I - P_3 (the floored matrix is then eps I + (lambda_3 - eps) P_3),
//    and each projector is a polynomial in Sigma (Lagrange form over the
//    eigenvalues), so no eigenvectors are formed.  The 2x2 eigenvalues are in
//    closed form; the 3x3 ones use the trigonometric solution of the
//    characteristic cubic (O. K. Smith, "Eigenvalues of a symmetric 3x3
//    matrix", Comm. ACM 4(4), 1961).  A pivot test of Sigma - eps I (its
//    LDL^T inertia) skips the eigenvalues when none is below the floor.
//  * pack_gp: inverse and log-determinant of the floored blocks (adjugate
//    formula) folded into the packed FP32 E-step coefficients.
#pragma once

#include <math.h>

#include "gmmsp_internal.cuh"

namespace gmmsp {

template <typename T> struct MathConst;
template <> struct MathConst<double> {
  static constexpr double kLog2e = 1.4426950408889634074;
  static constexpr double kHalfD_Ln2Pi = 4.5946926660233541;  // (5/2) ln(2 pi)
  static constexpr double kTwoPiOver3 = 2.0943951023931954923;
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double acos_(double x) { return acos(x); }
  static __device__ __forceinline__ double cos_(double x) { return cos(x); }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
};
template <> struct MathConst<float> {
  static constexpr float kLog2e = 1.44269504f;
  static constexpr float kHalfD_Ln2Pi = 4.59469267f;
  static constexpr float kTwoPiOver3 = 2.09439510f;
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float acos_(float x) { return acosf(x); }
  static __device__ __forceinline__ float cos_(float x) { return cosf(x); }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
};

// Floor the eigenvalues of the symmetric 2x2 A = {xx, xy, yy} at eps.
// Returns the number of raised eigenvalues.
template <typename T>
__device__ int clamp_sym2(T* A, T eps) {
  using M = MathConst<T>;
  const T a = A[0], b = A[1], c = A[2];
  const T m = T(0.5) * (a + c), h = T(0.5) * (a - c);
  const T r = M::sqrt_(h * h + b * b);
  const T l1 = m - r, l2 = m + r;           // l1 <= l2
  const int n = (l1 < eps) + (l2 < eps);
  if (n == 0) return 0;
  if (n == 2 || r <= T(1e-12) * (fabs(m) + eps)) {
    const T f = (n == 2) ? eps : (m > eps ? m : eps);
    A[0] = f; A[1] = T(0); A[2] = f;
    return n;
  }
  // One raised: A + (eps - l1) P_1 with P_1 = (l2 I - A) / (l2 - l1).
  const T g = (eps - l1) / (T(2) * r);
  A[0] = a + g * (l2 - a);
  A[1] = b - g * b;
  A[2] = c + g * (l2 - c);
  return 1;
}

// Floor the eigenvalues of the symmetric 3x3 A = {LL, La, Lb, aa, ab, bb}.
template <typename T>
__device__ int clamp_sym3(T* A, T eps) {
  using M = MathConst<T>;
  const T a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
  // Inertia of A - eps I from the pivots of its LDL^T factorisation: all
  // positive means every eigenvalue is above the floor.
  {
    const T d1 = a00 - eps;
    if (d1 > T(0)) {
      const T l10 = a01 / d1, l20 = a02 / d1;
      const T d2 = (a11 - eps) - l10 * a01;
      if (d2 > T(0)) {
        const T e21 = a12 - l20 * a01;
        const T d3 = (a22 - eps) - l20 * a02 - e21 * e21 / d2;
        if (d3 > T(0)) return 0;
      }
    }
  }
  // Eigenvalues (Smith 1961): B = (A - q I) / p, lambda = q + 2 p cos(phi + 2 pi j / 3).
  const T q = (a00 + a11 + a22) / T(3);
  const T b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const T off = a01 * a01 + a02 * a02 + a12 * a12;
  const T p2 = (b00 * b00 + b11 * b11 + b22 * b22 + T(2) * off) / T(6);
  T l1, l2, l3;  // ascending
  if (p2 <= T(0)) {
    l1 = l2 = l3 = q;
  } else {
    const T p = M::sqrt_(p2);
    const T detB = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                   a02 * (a01 * a12 - b11 * a02);
    T hr = detB / (T(2) * p2 * p);
    hr = hr < T(-1) ? T(-1) : (hr > T(1) ? T(1) : hr);
    const T phi = M::acos_(hr) / T(3);
    l3 = q + T(2) * p * M::cos_(phi);
    l1 = q + T(2) * p * M::cos_(phi + M::kTwoPiOver3);
    l2 = T(3) * q - l1 - l3;
  }
  const int n = (l1 < eps) + (l2 < eps) + (l3 < eps);
  if (n == 0) return 0;
  const T spread = l3 - l1;
  if (n == 3 || spread <= T(1e-9) * (fabs(l3) + eps)) {
    const T f = (n == 3) ? eps : (q > eps ? q : eps);
    A[0] = f; A[1] = T(0); A[2] = T(0); A[3] = f; A[4] = T(0); A[5] = f;
    return n;
  }
  // S2 = A * A (symmetric, six entries).
  const T s00 = a00 * a00 + a01 * a01 + a02 * a02;
  const T s01 = a00 * a01 + a01 * a11 + a02 * a12;
  const T s02 = a00 * a02 + a01 * a12 + a02 * a22;
  const T s11 = a01 * a01 + a11 * a11 + a12 * a12;
  const T s12 = a01 * a02 + a11 * a12 + a12 * a22;
  const T s22 = a02 * a02 + a12 * a12 + a22 * a22;
  // Projector onto eigenvalue lj: (A - la I)(A - lb I) / ((lj - la)(lj - lb))
  //   = (A^2 - (la + lb) A + la lb I) / den.
  T lj, la, lb;
  if (n == 1) { lj = l1; la = l2; lb = l3; } else { lj = l3; la = l1; lb = l2; }
  const T sum = la + lb, prod = la * lb;
  const T den = (lj - la) * (lj - lb);
  T P00 = (s00 - sum * a00 + prod) / den, P01 = (s01 - sum * a01) / den;
  T P02 = (s02 - sum * a02) / den, P11 = (s11 - sum * a11 + prod) / den;
  T P12 = (s12 - sum * a12) / den, P22 = (s22 - sum * a22 + prod) / den;
  if (n == 1) {
    const T g = eps - l1;  // A + (eps - l1) P_1
    A[0] = a00 + g * P00; A[1] = a01 + g * P01; A[2] = a02 + g * P02;
    A[3] = a11 + g * P11; A[4] = a12 + g * P12; A[5] = a22 + g * P22;
  } else {
    const T g = l3 - eps;  // eps I + (l3 - eps) P_3
    A[0] = eps + g * P00; A[1] = g * P01; A[2] = g * P02;
    A[3] = eps + g * P11; A[4] = g * P12; A[5] = eps + g * P22;
  }
  return n;
}

// Packs mu and the (floored) blocks into the FP32 E-step coefficients.
// Returns false when a block is not positive definite (leading minors).
template <typename T>
__device__ bool pack_gp(const T* mu, const T* cs, const T* cc, float* gp) {
  using M = MathConst<T>;
  // spatial 2x2
  const T ds = cs[0] * cs[2] - cs[1] * cs[1];
  // colour 3x3 cofactors
  const T c00 = cc[3] * cc[5] - cc[4] * cc[4];
  const T c01 = cc[2] * cc[4] - cc[1] * cc[5];
  const T c02 = cc[1] * cc[4] - cc[2] * cc[3];
  const T c11 = cc[0] * cc[5] - cc[2] * cc[2];
  const T c12 = cc[1] * cc[2] - cc[0] * cc[4];
  const T c22 = cc[0] * cc[3] - cc[1] * cc[1];
  const T dc = cc[0] * c00 + cc[1] * c01 + cc[2] * c02;
  if (!(cs[0] > T(0) && ds > T(0) && cc[0] > T(0) && c22 > T(0) && dc > T(0))) return false;
  const T hs = T(-0.5) * M::kLog2e / ds;   // -(1/2) log2(e) / det
  const T hc = T(-0.5) * M::kLog2e / dc;
  float4* o = reinterpret_cast<float4*>(gp);
  o[0] = make_float4(float(mu[0]), float(mu[1]), float(mu[2]), float(mu[3]));
  o[1] = make_float4(float(mu[4]), float(hs * cs[2]), float(T(-2) * hs * cs[1]), float(hs * cs[0]));
  o[2] = make_float4(float(hc * c00), float(hc * c11), float(hc * c22), float(T(2) * hc * c01));
  const T lnorm = (T(-0.5) * M::log_(ds * dc) - M::kHalfD_Ln2Pi) * M::kLog2e;
  o[3] = make_float4(float(T(2) * hc * c02), float(T(2) * hc * c12), float(lnorm), 0.f);
  return true;
}

}  // namespace gmmsp
