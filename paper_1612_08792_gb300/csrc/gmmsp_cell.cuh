// Per-cell helpers shared by the EM kernels (gmmsp_em.cu, gmmsp_rows.cu):
// the cell's extent and candidate mask, the special-function approximations
// of the E-step, the log2 density of one candidate, and the image lookup of
// a batch.
#pragma once

#include <math.h>

#include "gmmsp_internal.cuh"

namespace gmmsp {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Cell {
  int cx, cy;      // cell coordinates
  int x0, y0;      // first pixel
  int cw, ch;      // extent (v, or the remainder)
  unsigned mask;   // bit s set when slot s is a seed of the grid
};

__device__ __forceinline__ Cell make_cell(const Geom& g, int cell) {
  Cell c;
  c.cy = cell / g.ncx;
  c.cx = cell - c.cy * g.ncx;
  c.x0 = c.cx * g.v;
  c.y0 = c.cy * g.v;
  c.cw = min(g.v, g.W - c.x0);
  c.ch = min(g.v, g.H - c.y0);
  // slot s = 3 r + q is seed (c_x - 1 + q, c_y - 1 + r): the product of a column
  // mask (q) and a row mask (r) of the seeds on the grid
  const unsigned cols = (c.cx >= 1 && c.cx - 1 < g.nx ? 1u : 0u) | (c.cx < g.nx ? 2u : 0u) |
                        (c.cx + 1 < g.nx ? 4u : 0u);
  const unsigned rows = (c.cy >= 1 && c.cy - 1 < g.ny ? 1u : 0u) | (c.cy < g.ny ? 2u : 0u) |
                        (c.cy + 1 < g.ny ? 4u : 0u);
  c.mask = (rows & 1u ? cols : 0u) | (rows & 2u ? cols << 3 : 0u) | (rows & 4u ? cols << 6 : 0u);
  return c;
}

// The colour of pixel (x, y) of image g, read through GMMSP_IN_BOUNDS (a
// checked build yields 0 outside the image and records the event).
template <int CM, class Src>
__device__ __forceinline__ float4 load_pixel(const Src& s, const Geom& g, int x, int y) {
  if (!(GMMSP_IN_BOUNDS(x, g.W, BND_PIXEL_X) && GMMSP_IN_BOUNDS(y, g.H, BND_PIXEL_Y)))
    return make_float4(0.f, 0.f, 0.f, 0.f);
  return load_z<CM>(s, x, y);
}

// log2 p(z; theta_k) for one candidate: the log normaliser plus the two
// quadratic forms, with -1/2 log2(e) Sigma^{-1} folded into the coefficients.
// fx, fy are the pixel's coordinates relative to the cell origin (the staged
// mean is relative to the same origin).
// DIAG: both blocks diagonal (the Sec. III-C start and the learned start, whose
// packed 2xy, 2La, 2Lb and 2ab coefficients are exactly +-0): the same
// operations without the zero terms, so the same bits, and the normaliser
// read alone instead of the fourth float4.
template <int CM, bool DIAG = false>
__device__ __forceinline__ float log2_density(const float4* P, float fx, float fy, float4 z) {
  if constexpr (DIAG) {
    const float4 p0 = P[0], p1 = P[1], p2 = P[2];
    const float dx = fx - p0.x, dy = fy - p0.y;
    const float dL = z.x - p0.z;
    float q = reinterpret_cast<const float*>(P + 3)[2];
    q = fmaf(p1.y * dx, dx, q);                      // xx dx^2
    q = fmaf(p1.w * dy, dy, q);                      // yy dy^2
    q = fmaf(p2.x * dL, dL, q);                      // LL dL^2
    if constexpr (CM != kColourGray) {
      const float da = z.y - p0.w, db = z.z - p1.x;
      q = fmaf(p2.y * da, da, q);                    // aa da^2
      q = fmaf(p2.z * db, db, q);                    // bb db^2
    }
    return q;
  }
  const float4 p0 = P[0], p1 = P[1], p2 = P[2], p3 = P[3];
  const float dx = fx - p0.x, dy = fy - p0.y;
  const float dL = z.x - p0.z;
  float q = p3.z;
  q = fmaf(fmaf(p1.z, dy, p1.y * dx), dx, q);       // (xx dx + 2xy dy) dx
  q = fmaf(p1.w * dy, dy, q);                        // yy dy^2
  if constexpr (CM == kColourFull) {
    const float da = z.y - p0.w, db = z.z - p1.x;
    q = fmaf(fmaf(p3.x, db, fmaf(p2.w, da, p2.x * dL)), dL, q);  // (LL dL + 2La da + 2Lb db) dL
    q = fmaf(fmaf(p3.y, db, p2.y * da), da, q);      // (aa da + 2ab db) da
    q = fmaf(p2.z * db, db, q);                      // bb db^2
  } else if constexpr (CM == kColourSplit) {
    const float da = z.y - p0.w, db = z.z - p1.x;
    q = fmaf(p2.x * dL, dL, q);                      // LL dL^2
    q = fmaf(fmaf(p3.y, db, p2.y * da), da, q);      // (aa da + 2ab db) da
    q = fmaf(p2.z * db, db, q);                      // bb db^2
  } else {
    q = fmaf(p2.x * dL, dL, q);                      // LL dL^2
  }
  return q;
}

// The batch image owning work item `item` (a cell when which == 0, a
// superpixel when which == 1): binary search over the images' prefix offsets.
__device__ __forceinline__ int find_image(const BatchImage* __restrict__ imgs, int n, int item,
                                          int which /*0 cells, 1 superpixels*/) {
  if (imgs[0].uniform) {  // images of one geometry: a division
    const int i = item / (which == 0 ? imgs[0].g.ncells : imgs[0].g.K);
    return i < n ? i : n - 1;
  }
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    const int off = which == 0 ? imgs[mid].cell_off : imgs[mid].k_off;
    if (off <= item) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace gmmsp
