// sRGB (8 bits per channel, D65 white) -> CIE 1976 L*a*b*, per pixel, shared
// by the conversion kernels (gmmsp_prep.cu) and the network's fused
// conversion (gmmsp_cnn.cu), so that both give the same bits.  The sRGB
// transfer curve is a 256-entry table built per block with powf; the RGB ->
// XYZ matrix is derived on the host from the sRGB primaries' chromaticities
// and the white point (rgb2lab_const).
#pragma once

#include <stdint.h>

namespace gmmsp {

struct Rgb2LabConst {
  float m[9];         // linear sRGB -> XYZ, row major
  float inv_white[3]; // 1 / (Xn, Yn, Zn)
};

// The constants of the conversion (computed once on the host).
Rgb2LabConst rgb2lab_const();

__device__ __forceinline__ float cielab_f(float t) {
  // CIE 1976: cube root above (6/29)^3, the linear segment below.  The cube
  // root is taken as 2^(log2(t) / 3) on the special-function unit
  // (lg2.approx, ex2.approx; t is a normal number there): relative error
  // about 3e-7, i.e. under 3e-4 in L*, a*, b*, at two instructions instead
  // of a full-precision cbrtf, three times per pixel.
  const float d3 = 216.f / 24389.f;             // (6/29)^3
  const float slope = 841.f / 108.f;            // 1 / (3 (6/29)^2)
  float lg, cr;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(t));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(cr) : "f"(lg * (1.f / 3.f)));
  return t > d3 ? cr : fmaf(slope, t, 4.f / 29.f);
}

// sRGB decoding of the 256 code values (the transfer curve of IEC 61966-2-1),
// by the threads of the block.
__device__ __forceinline__ void build_srgb_table(float* lin) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const float c = float(i) * (1.f / 255.f);
    lin[i] = c <= 0.04045f ? c * (1.f / 12.92f) : powf((c + 0.055f) * (1.f / 1.055f), 2.4f);
  }
}

// L*, a*, b* of the pixel whose three code values start at p (lin: the table).
__device__ __forceinline__ void srgb8_to_lab(const Rgb2LabConst& k, const float* lin, const uint8_t* p, float& L,
                                             float& A, float& B) {
  const float r = lin[p[0]], g = lin[p[1]], b = lin[p[2]];
  const float* m = k.m;
  const float X = fmaf(m[0], r, fmaf(m[1], g, m[2] * b)) * k.inv_white[0];
  const float Y = fmaf(m[3], r, fmaf(m[4], g, m[5] * b)) * k.inv_white[1];
  const float Z = fmaf(m[6], r, fmaf(m[7], g, m[8] * b)) * k.inv_white[2];
  const float fx = cielab_f(X), fy = cielab_f(Y), fz = cielab_f(Z);
  L = 116.f * fy - 16.f;
  A = 500.f * (fx - fy);
  B = 200.f * (fy - fz);
}

}  // namespace gmmsp
