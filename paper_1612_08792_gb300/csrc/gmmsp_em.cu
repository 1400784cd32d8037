// The EM hot path: fused E-step + M-step partial sums per cell, the FP64
// finalize with the eigenvalue floor, and the label pass.
//
// Work decomposition.  The pixels of one v x v cell share one candidate set
// (see gmmsp_internal.cuh), so one warp (or 2 or 4, the autotuned launch
// shape) takes one cell: it stages the <= 9 candidates' packed parameters in
// shared memory (read back as warp-wide broadcasts) and walks the cell's
// pixels 32 at a time (a cell of 32 b + 1 pixels takes its last pixel first,
// one candidate per lane, instead of ending in a one-pixel batch):
//   E:  each lane evaluates log2 p(z; theta_k) of its pixel for the
//       candidates (Eq. gaussian with the block covariance), forms the
//       posteriors R_ik (Eq. Rik) with the log-sum-exp held in registers, and
//       accumulates ln sum_k p (the log-likelihood L following Eq. ftheta);
//   M:  through shared memory, lane l < 27 adds R_ik, R_ik d and the block
//       entries of R_ik d d^T of slot l mod 9 over a third of the 32 pixels,
//       d = z - mu_k(old) (the data shifted by the previous mean so that the
//       FP32 second moments do not cancel).
// The per-lane sums are added per slot and per cell in shared memory and
// written once per cell: a block-level partial, with no global atomics
// (k_em_pass).  The partials are FP32 sums over one cell's <= v^2 pixels and
// are stored as such.
//
// The finalize adds the <= 9 partials of the cells whose candidate set holds
// k in a fixed order, giving the sums over the pixel set I_k of Eq. (Ik) --
// mixed precision: as an unevaluated FP32 pair (hi, lo) built with the
// error-free TwoSum (Knuth; Moller) and rounded to FP64 once, within about
// 2^-47 of the exact sum, which keeps the FP64 pipe for the update -- and
// turns them into Eq. (UpdateMu), (UpdateSigS) and (UpdateSigC) in FP64:
//   mu = mu_old + S1 / W,   Sigma = S2 / W - (S1 / W)(S1 / W)^T,
// then applies the floor of Eq. (mlams)/(mlamc) and re-packs the E-step
// coefficients (k_finalize_l16: 16 lanes per superpixel for small K;
// k_finalize: one thread per superpixel for large K and the FP32 variant).
// A superpixel with W < 1e-8 keeps its parameters.
//
// Colour models: the E+M and label kernels are compiled per model (template
// CM): the split model of Eq. (BlockSigma1) drops the L-a and L-b terms of
// the quadratic form and of the second moments (4 of 48 FP32 instructions
// per pixel and candidate), grayscale keeps L alone (20 of 48) and reads one
// plane instead of three.  The partial layout is the same for all models;
// the entries a model does not form stay 0.
#include <math.h>

#include <type_traits>

#include "gmmsp_cell.cuh"
#include "gmmsp_internal.cuh"
#include "gmmsp_math.cuh"

namespace gmmsp {

constexpr int kEmWarps = 4;          // cells per 128-thread block

// Copies the packed parameters of the cell's candidate slots into sp[36]
// (float4), with the spatial mean moved from the candidate's cell origin to
// this cell's (mu_x + (s mod 3 - 1) v, mu_y + (s / 3 - 1) v), so that every
// candidate sees the pixel's own coordinates in the cell; slots off the grid
// are zero and never read.
__device__ __forceinline__ float4 staged_param(const Geom& g, const Cell& c, const float* gp, int i) {
  const int s = i >> 2, q = i & 3;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if ((c.mask >> s) & 1u) {
    const int k = (c.cy - 1 + s / 3) * g.nx + (c.cx - 1 + s % 3);
    if (GMMSP_IN_BOUNDS(k, g.K, BND_GP)) v = __ldg(reinterpret_cast<const float4*>(gp) + k * 4 + q);
    if (q == 0) {
      v.x += float((s % 3 - 1) * g.v);
      v.y += float((s / 3 - 1) * g.v);
    }
  }
  return v;
}

__device__ __forceinline__ void stage_params(const Geom& g, const Cell& c, const float* gp,
                                             float4* sp, int lane) {
  for (int i = lane; i < kSlots * 4; i += 32) sp[i] = staged_param(g, c, gp, i);
  __syncwarp();
}

// E part for one pixel: the posteriors of its candidates (Eq. Rik) into
// R[0..8] (zero for slots off the grid) and ln-sum-exp in log2 units into ll.
template <bool FULL, int CM, bool DIAG = false>
__device__ __forceinline__ void e_pixel(const float4* sp, unsigned mask, float fx, float fy, float4 z,
                                        float (&R)[kSlots],
                                        float& ll) {
  float m = -INFINITY;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    R[s] = 0.f;
    if (FULL || ((mask >> s) & 1u)) {
      R[s] = log2_density<CM, DIAG>(sp + 4 * s, fx, fy, z);
      m = fmaxf(m, R[s]);
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (FULL || ((mask >> s) & 1u)) {
      R[s] = ex2_approx(R[s] - m);
      sum += R[s];
    }
  }
  const float inv = rcp_approx(sum);
  ll += m + lg2_approx(sum);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) R[s] *= inv;
}

// Fused E-step + M-step partial sums, stored as PT = float.  SHIFT: mixed
// precision (moments about the previous mean, the per-cell log-likelihood
// stored in log2 units and converted by the FP64 reduction); otherwise the
// all-FP32 variant (raw moments, the log-likelihood in nats).  WPC warps
// share one cell; a 128-thread block holds 4 / WPC cells.
//
// Each warp walks its share of the cell 32 pixels at a time.  Every lane
// takes one pixel through the E part (its <= 9 posteriors and its
// log-likelihood) and leaves the posteriors and the pixel's colour and
// position in shared memory.  Then lane l < 27 accumulates the 15 statistics
// of slot s = l mod 9 over every third pixel of the 32 (pixels l / 9,
// l / 9 + 3, ...), with d = z - mu_s(old): each lane holds 15 accumulators
// instead of 9 x 15, which keeps the register count (and so the occupancy)
// of the kernel independent of the candidate count.  At the end the three
// lanes of each slot, then the WPC warps, are added through shared memory and
// written once per cell as FP32 (no global atomics).
constexpr int kRStride = 12;  // floats per pixel row of posteriors

template <int WPC>
struct EmSmem {
  float4 sp[kEmWarps / WPC][kSlots * 4];            // candidate parameters per cell
  float R[kEmWarps][32 * kRStride];                 // posteriors of the 32 pixels in flight
  float4 Z[kEmWarps][32];                           // (L, a, b, -) of those pixels
  float2 XY[kEmWarps][32];                          // their position in the cell
  float part[kEmWarps][kSlots * kStats + 1 + 3];    // per-warp sums (row 135: log-likelihood)
  float red[kEmWarps][27][kStats + 2];              // per-lane sums before the 3-lane add (odd row
                                                    // stride: the 27 lanes' stores hit 27 banks)
};

template <int WPC>
constexpr int em_smem_bytes() { return int(sizeof(EmSmem<WPC>)); }

template <bool FULL, bool SHIFT, int WPC, class Src, int CM, bool DIAG = false>
__device__ __forceinline__ void em_cell_warp(const Src& lab, const Geom& g, const Cell& c,
                                             EmSmem<WPC>& sm, int slot, int warp, int lane, int wic,
                                             float (&acc)[kStats], float& ll) {
  const int npx = c.cw * c.ch;
  const float inv_cw = 1.f / float(c.cw);
  const float4* sp = sm.sp[slot];
  float* Rw = sm.R[warp];
  float4* Zw = sm.Z[warp];
  float2* XYw = sm.XY[warp];
  // M-part role of this lane: slot ms, pixel phase ph (lanes 27-31 idle there)
  const int ms = lane % 9, ph = lane / 9;
  const bool m_on = lane < 27 && (FULL || ((c.mask >> ms) & 1u));
  float cx = 0.f, cy = 0.f, mL = 0.f, ma = 0.f, mb = 0.f;
  {
    const float4 p0 = sp[4 * ms], p1 = sp[4 * ms + 1];
    // SHIFT: d_x = rx - mu_x (the staged mean, relative to this cell's origin);
    // raw moments: x relative to the candidate's cell origin, rx + (1 - ms % 3) v
    cx = SHIFT ? -p0.x : float((1 - ms % 3) * g.v);
    cy = SHIFT ? -p0.y : float((1 - ms / 3) * g.v);
    if (SHIFT) { mL = p0.z; ma = p0.w; mb = p1.x; }
  }
  auto locate = [&](int p, int& rx, int& ry) {
    ry = __float2int_rz((float(p) + 0.5f) * inv_cw);  // exact floor(p / cw)
    rx = p - ry * c.cw;
  };
  // the statistics of one (pixel, slot ms) pair with posterior r into acc
  auto add_stats = [&](float r, float dx, float dy, float dL, float da, float db) {
    const float rxd = r * dx, ryd = r * dy, rL = r * dL;
    acc[0] += r;
    acc[1] += rxd; acc[2] += ryd; acc[3] += rL;
    acc[6] = fmaf(rxd, dx, acc[6]);
    acc[7] = fmaf(rxd, dy, acc[7]);
    acc[8] = fmaf(ryd, dy, acc[8]);
    acc[9] = fmaf(rL, dL, acc[9]);
    if constexpr (CM != kColourGray) {
      const float ra = r * da, rb = r * db;
      acc[4] += ra; acc[5] += rb;
      if constexpr (CM == kColourFull) {
        acc[10] = fmaf(rL, da, acc[10]);
        acc[11] = fmaf(rL, db, acc[11]);
      }
      acc[12] = fmaf(ra, da, acc[12]);
      acc[13] = fmaf(ra, db, acc[13]);
      acc[14] = fmaf(rb, db, acc[14]);
    }
  };
  // A cell of 32 b + 1 pixels (v = 15: 225) would end in a batch of one
  // pixel that costs a full E part.  That pixel (the last) is taken first,
  // one slot per lane: lane s < 9 evaluates slot s, the log-sum-exp runs
  // over lanes 0-15 by butterflies (lanes 9-15 hold -inf), and lane s adds
  // its pair's statistics to its own accumulators (lane s holds slot s's
  // phase-0 sums).  The batches then cover the other 32 b pixels.
  int npx_b = npx;
  if (WPC == 1 && npx > 32 && (npx & 31) == 1) {
    npx_b = npx - 1;
    int rx, ry;
    locate(npx_b, rx, ry);
    const float4 z = load_pixel<CM>(lab, g, c.x0 + rx, c.y0 + ry);
    const bool on = lane < kSlots && (FULL || ((c.mask >> lane) & 1u));
    const float q = on ? log2_density<CM, DIAG>(sp + 4 * (lane < kSlots ? lane : 0), float(rx), float(ry), z)
                       : -INFINITY;
    float m = q;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float e = on ? ex2_approx(q - m) : 0.f;
    float sum = e;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) ll += m + lg2_approx(sum);
    if (on && m_on) {
      const float r = e * rcp_approx(sum);
      add_stats(r, float(rx) + cx, float(ry) + cy, z.x - mL, z.y - ma, z.z - mb);
    }
  }
  // The colour of this lane's next pixel is loaded one batch ahead.
  float4 zn = make_float4(0.f, 0.f, 0.f, 0.f);
  if (wic * 32 + lane < npx_b) {
    int rx0, ry0;
    locate(wic * 32 + lane, rx0, ry0);
    zn = load_pixel<CM>(lab, g, c.x0 + rx0, c.y0 + ry0);
  }
  for (int base = wic * 32; base < npx_b; base += 32 * WPC) {
    const int p = base + lane;
    float R[kSlots];
    const float4 z = zn;
    if (p + 32 * WPC < npx_b) {
      int rx1, ry1;
      locate(p + 32 * WPC, rx1, ry1);
      zn = load_pixel<CM>(lab, g, c.x0 + rx1, c.y0 + ry1);
    }
    int rx = 0, ry = 0;
    if (p < npx_b) {
      locate(p, rx, ry);
      e_pixel<FULL, CM, DIAG>(sp, c.mask, float(rx), float(ry), z, R, ll);
    } else {
#pragma unroll
      for (int s = 0; s < kSlots; ++s) R[s] = 0.f;
    }
    float4* rrow = reinterpret_cast<float4*>(Rw + lane * kRStride);
    rrow[0] = make_float4(R[0], R[1], R[2], R[3]);
    rrow[1] = make_float4(R[4], R[5], R[6], R[7]);
    Rw[lane * kRStride + 8] = R[8];
    Zw[lane] = z;
    XYw[lane] = make_float2(float(rx), float(ry));
    __syncwarp();
    if (m_on) {
      // statistics of pixel q for this lane's slot
      auto accumulate = [&](int q) {
        const float r = Rw[q * kRStride + ms];
        const float2 xy = XYw[q];
        const float4 zz = Zw[q];
        add_stats(r, xy.x + cx, xy.y + cy, zz.x - mL, zz.y - ma, zz.z - mb);
      };
      const int np = min(32, npx_b - base);
      if (np == 32) {
        // a full batch: pixels ph, ph + 3, ..., fixed offsets, no loop control
#pragma unroll
        for (int i = 0; i < 10; ++i) accumulate(ph + 3 * i);
        if (ph < 2) accumulate(ph + 30);
      } else {
#pragma unroll 4
        for (int q = ph; q < np; q += 3) accumulate(q);
      }
    }
    __syncwarp();
  }
}

// One cell of the fused pass, run by the WPC warps of cell slot `slot` of the
// block (all threads of the block call it together when WPC > 1).
template <typename PT, bool SHIFT, int WPC, class Src, int CM, bool DIAG = false>
__device__ __forceinline__ void em_cell_block(const Src& lab, const Geom& g, const float* __restrict__ gp,
                                              PT* __restrict__ partials, int cell, bool active,
                                              EmSmem<WPC>& sm, int warp, int lane, int slot, int wic,
                                              int t) {
  Cell c = {};
  if (active) c = make_cell(g, cell);
  if (active) {
    for (int i = t; i < kSlots * 4; i += 32 * WPC) sm.sp[slot][i] = staged_param(g, c, gp, i);
  }
  if (WPC == 1) __syncwarp(); else __syncthreads();

  float acc[kStats];
#pragma unroll
  for (int j = 0; j < kStats; ++j) acc[j] = 0.f;
  float ll = 0.f;
  if (active) {
    if (c.mask == 0x1ffu)
      em_cell_warp<true, SHIFT, WPC, Src, CM, DIAG>(lab, g, c, sm, slot, warp, lane, wic, acc, ll);
    else
      em_cell_warp<false, SHIFT, WPC, Src, CM, DIAG>(lab, g, c, sm, slot, warp, lane, wic, acc, ll);
  }
  // Per-warp totals: add the three lanes of each slot, and the lanes' log-likelihoods.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
  if (lane < 27) {
#pragma unroll
    for (int j = 0; j < kStats; ++j) sm.red[warp][lane][j] = acc[j];
  }
  __syncwarp();
  for (int o = lane; o < kSlots * kStats; o += 32) {
    const int s = o / kStats, j = o - s * kStats;
    sm.part[warp][o] = sm.red[warp][s][j] + sm.red[warp][s + 9][j] + sm.red[warp][s + 18][j];
  }
  if (lane == 0) sm.part[warp][kSlots * kStats] = ll;
  if (WPC == 1) __syncwarp(); else __syncthreads();
  // Cell totals (sum over the WPC warps of the cell), written as PT.
  if (active && GMMSP_IN_BOUNDS(cell, g.ncells, BND_PARTIAL_W)) {
    PT* out = partials + (long long)cell * kPartStride;
    const int w0 = slot * WPC;
    for (int o = t; o < kPartStride; o += 32 * WPC) {
      float v = sm.part[w0][o];
#pragma unroll
      for (int w = 1; w < WPC; ++w) v += sm.part[w0 + w][o];
      out[o] = (o < kSlots * kStats || SHIFT) ? PT(v) : PT(v) * PT(0.69314718055994530942);
    }
  }
  if (WPC == 1) __syncwarp(); else __syncthreads();  // the slot's buffers are reused next
}

template <typename PT, bool SHIFT, int WPC, class Src, int CM>
__device__ __forceinline__ void em_pass_body(const Src& lab, const Geom& g, const float* __restrict__ gp,
                                             PT* __restrict__ partials) {
  constexpr int kCellsPerBlock = kEmWarps / WPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EmSmem<WPC>& sm = *reinterpret_cast<EmSmem<WPC>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = warp / WPC;       // cell slot within the block
  const int wic = warp % WPC;        // warp index within the cell
  const int t = wic * 32 + lane;     // thread index within the cell
  const int cell = blockIdx.x * kCellsPerBlock + slot;
  const bool active = cell < g.ncells;  // inactive threads still reach every barrier
  pdl_wait();  // gp and the image are written by the preceding kernels
  pdl_trigger();
  em_cell_block<PT, SHIFT, WPC, Src, CM>(lab, g, gp, partials, cell, active, sm, warp, lane, slot, wic, t);
}

template <typename PT, bool SHIFT, int WPC, class Src, int CM>
__global__ void __launch_bounds__(kEmWarps * 32) k_em_pass(Src lab, Geom g, const float* __restrict__ gp,
                                                           PT* __restrict__ partials) {
  em_pass_body<PT, SHIFT, WPC, Src, CM>(lab, g, gp, partials);
}

// The same, registers capped for 7 blocks per SM (72): the launch for one
// warp per cell in the full colour model, where it raised the occupancy from
// 24% to 40% on large images (the split and grayscale kernels are faster
// uncapped).
template <typename PT, bool SHIFT, int WPC, class Src, int CM>
__global__ void __launch_bounds__(kEmWarps * 32, 7) k_em_pass_capped(Src lab, Geom g, const float* __restrict__ gp,
                                                                     PT* __restrict__ partials) {
  em_pass_body<PT, SHIFT, WPC, Src, CM>(lab, g, gp, partials);
}

// ---------------------------------------------------------------- batches
// Many images in one launch per phase.  Image i owns the cells
// [cell_off, cell_off + ncells), the superpixels [k_off, k_off + K) and the
// pixels [pix_off, pix_off + W H) of the batch (its CIELAB planes start at
// lab + 3 pix_off).  Work items are found by a binary search over these
// prefix offsets; warps (threads for per-superpixel work) loop over the
// batch's items with the grid's stride, so the grid is sized to the machine
// (persistent blocks) rather than to the work.
// MINB caps the registers so that MINB blocks fit on an SM (5: at most 102
// registers, no spills).
template <typename PT, bool SHIFT, int MINB, int CM>
__global__ void __launch_bounds__(kEmWarps * 32, MINB) k_em_pass_batch(const BatchImage* __restrict__ imgs, int n,
                                                                       int total_cells, const float* __restrict__ lab,
                                                                       const float* __restrict__ gp,
                                                                       PT* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EmSmem<1>& sm = *reinterpret_cast<EmSmem<1>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int cell = blockIdx.x * kEmWarps + warp; cell < total_cells; cell += gridDim.x * kEmWarps) {
    const int ii = find_image(imgs, n, cell, 0);
    if (!GMMSP_IN_BOUNDS(ii, n, BND_IMAGE)) continue;
    const BatchImage& im = imgs[ii];
    if (!GMMSP_IN_BOUNDS(cell - im.cell_off, im.g.ncells, BND_ITEM)) continue;
    const LabPlanar src{lab + 3 * im.pix_off, (long long)im.g.W * im.g.H, im.g.W};
    em_cell_block<PT, SHIFT, 1, LabPlanar, CM>(src, im.g, gp + (long long)im.k_off * kGP,
                                               partials + (long long)im.cell_off * kPartStride,
                                               cell - im.cell_off, true, sm, warp, lane, warp, 0, lane);
  }
}

// Non-persistent variant: one cell per warp over a grid sized to the work,
// registers capped so that MINB blocks fit on an SM (6: 80 registers and 8
// bytes of spill; 7: 72 registers and some spill); the autotuner's choice of
// 6 or 7 blocks per SM selects it.  DIAG: every superpixel's blocks are
// diagonal (the first pass after either start).
template <typename PT, bool SHIFT, int MINB, int CM, bool DIAG = false>
__global__ void __launch_bounds__(kEmWarps * 32, MINB) k_em_pass_batch_flat(const BatchImage* __restrict__ imgs, int n,
                                                                      int total_cells,
                                                                      const float* __restrict__ lab,
                                                                      const float* __restrict__ gp,
                                                                      PT* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EmSmem<1>& sm = *reinterpret_cast<EmSmem<1>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kEmWarps + warp;
  if (cell >= total_cells) return;  // whole warps only; a warp works alone on its cell
  const int ii = find_image(imgs, n, cell, 0);
  if (!GMMSP_IN_BOUNDS(ii, n, BND_IMAGE)) return;
  const BatchImage& im = imgs[ii];
  if (!GMMSP_IN_BOUNDS(cell - im.cell_off, im.g.ncells, BND_ITEM)) return;
  const LabPlanar src{lab + 3 * im.pix_off, (long long)im.g.W * im.g.H, im.g.W};
  em_cell_block<PT, SHIFT, 1, LabPlanar, CM, DIAG>(src, im.g, gp + (long long)im.k_off * kGP,
                                                   partials + (long long)im.cell_off * kPartStride,
                                                   cell - im.cell_off, true, sm, warp, lane, warp, 0, lane);
}

// Label pass: argmax posterior per pixel (ties to the smaller k, i.e. the
// smaller slot) and the per-cell log-likelihood.
// Each lane takes kLabelPPL pixels per step (p, p + 32, ...), so that every
// candidate's parameters, read from shared memory once, serve all of them;
// the colours of the next step are loaded one step ahead.
constexpr int kLabelPPL = 2;

// LL = false: argmax only (no log-sum-exp), for callers that want no
// log-likelihood.
template <bool FULL, bool LL, class Src, int CM>
__device__ __forceinline__ void label_cell_pixels(const Src& lab, const Geom& g,
                                                  const Cell& c, const float4* sp, int lane,
                                                  int32_t* __restrict__ labels, float& ll) {
  const int npx_all = c.cw * c.ch;
  const float inv_cw = 1.f / float(c.cw);
  auto locate = [&](int p, int& rx, int& ry) {
    ry = __float2int_rz((float(p) + 0.5f) * inv_cw);  // exact floor(p / cw)
    rx = p - ry * c.cw;
  };
  // start at the cell's first candidate, so that the label is one of the
  // pixel's candidates (Eq. obtLi) even where no density compares (NaN input)
  const int first = __ffs(c.mask) - 1;
  // A cell of 32 b + 1 pixels (v = 15: 225) takes its last pixel first, one
  // candidate per lane (lane s < 9: slot s): the argmax is the smallest slot
  // reaching the maximum (butterflies over lanes 0-15), as in the loop below.
  // The steps then cover 32 b pixels, and a last step of 32 pixels skips its
  // second pixel per lane.
  int npx = npx_all;
  if (npx > 32 && (npx & 31) == 1) {
    npx = npx_all - 1;
    int rx, ry;
    locate(npx, rx, ry);
    const float4 z = load_pixel<CM>(lab, g, c.x0 + rx, c.y0 + ry);
    const bool on = lane < kSlots && (FULL || ((c.mask >> lane) & 1u));
    const float q = on ? log2_density<CM>(sp + 4 * (lane < kSlots ? lane : 0), float(rx), float(ry), z)
                       : -INFINITY;
    float m = q;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int best = on && q == m ? lane : 16;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (best == 16) best = first;
    if (LL) {
      float sum = on ? ex2_approx(q - m) : 0.f;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) ll += m + lg2_approx(sum);
    }
    if (lane == 0) {
      const long long at = (long long)(c.y0 + ry) * g.W + (c.x0 + rx);
      const int kl = (c.cy - 1 + best / 3) * g.nx + (c.cx - 1 + best % 3);
      if (GMMSP_IN_BOUNDS(at, (long long)g.W * g.H, BND_LABEL) && GMMSP_IN_BOUNDS(kl, g.K, BND_LABEL_K)) labels[at] = kl;
    }
  }
  float4 zn[kLabelPPL];
#pragma unroll
  for (int j = 0; j < kLabelPPL; ++j) {
    zn[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int p = lane + 32 * j;
    if (p < npx) {
      int rx, ry;
      locate(p, rx, ry);
      zn[j] = load_pixel<CM>(lab, g, c.x0 + rx, c.y0 + ry);
    }
  }
  // One step: J pixels per lane (p0, p0 + 32, ...), the colours of the next
  // step's pixels loaded ahead into zn.
  auto step = [&](auto jt, int p0) {
    constexpr int J = decltype(jt)::value;
    float4 z[J];
    int rx[J], ry[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      z[j] = zn[j];
      const int pn = p0 + 32 * (j + kLabelPPL);
      if (pn < npx) {
        int x1, y1;
        locate(pn, x1, y1);
        zn[j] = load_pixel<CM>(lab, g, c.x0 + x1, c.y0 + y1);
      }
      locate(p0 + 32 * j, rx[j], ry[j]);
    }
    float e[J][kSlots];
    float m[J];
    int best[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      m[j] = -INFINITY;
      best[j] = first;
    }
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      if (FULL || ((c.mask >> s) & 1u)) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          e[j][s] = log2_density<CM>(sp + 4 * s, float(rx[j]), float(ry[j]), z[j]);
          if (e[j][s] > m[j]) { m[j] = e[j][s]; best[j] = s; }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) e[j][s] = 0.f;
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (p0 + 32 * j >= npx) continue;
      if (LL) {
        float sum = 0.f;
#pragma unroll
        for (int s = 0; s < kSlots; ++s)
          if (FULL || ((c.mask >> s) & 1u)) sum += ex2_approx(e[j][s] - m[j]);
        ll += m[j] + lg2_approx(sum);
      }
      const long long at = (long long)(c.y0 + ry[j]) * g.W + (c.x0 + rx[j]);
      const int kl = (c.cy - 1 + best[j] / 3) * g.nx + (c.cx - 1 + best[j] % 3);
      if (GMMSP_IN_BOUNDS(at, (long long)g.W * g.H, BND_LABEL) && GMMSP_IN_BOUNDS(kl, g.K, BND_LABEL_K)) labels[at] = kl;
    }
  };
  // kLabelPPL pixels per lane while more than 32 remain, then one
  int p0 = lane;
  for (; p0 - lane + 32 < npx; p0 += 32 * kLabelPPL) step(std::integral_constant<int, kLabelPPL>{}, p0);
  if (p0 - lane < npx) step(std::integral_constant<int, 1>{}, p0);
}

// One cell of the label pass, run by one warp.
template <class Src, int CM>
__device__ __forceinline__ void label_cell_warp(const Src& lab, const Geom& g, const float* __restrict__ gp,
                                                int32_t* __restrict__ labels, double* __restrict__ cell_ll,
                                                int cell, float4* sp, int lane) {
  const Cell c = make_cell(g, cell);
  stage_params(g, c, gp, sp, lane);
  float ll = 0.f;
  if (!cell_ll) {  // labels only
    if (c.mask == 0x1ffu)
      label_cell_pixels<true, false, Src, CM>(lab, g, c, sp, lane, labels, ll);
    else
      label_cell_pixels<false, false, Src, CM>(lab, g, c, sp, lane, labels, ll);
    return;
  }
  if (c.mask == 0x1ffu)
    label_cell_pixels<true, true, Src, CM>(lab, g, c, sp, lane, labels, ll);
  else
    label_cell_pixels<false, true, Src, CM>(lab, g, c, sp, lane, labels, ll);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
  if (lane == 0 && GMMSP_IN_BOUNDS(cell, g.ncells, BND_CELL_LL)) cell_ll[cell] = double(ll) * 0.69314718055994530942;
}

template <class Src, int CM>
__global__ void __launch_bounds__(kEmWarps * 32) k_label_pass(Src lab, Geom g, const float* __restrict__ gp,
                                                              int32_t* __restrict__ labels,
                                                              double* __restrict__ cell_ll) {
  __shared__ float4 sp_all[kEmWarps][kSlots * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kEmWarps + warp;
  pdl_wait();
  pdl_trigger();
  if (cell >= g.ncells) return;
  label_cell_warp<Src, CM>(lab, g, gp, labels, cell_ll, cell, sp_all[warp], lane);
}

template <int CM>
__global__ void __launch_bounds__(kEmWarps * 32, 5) k_label_pass_batch(const BatchImage* __restrict__ imgs, int n,
                                                                    int total_cells,
                                                                    const float* __restrict__ lab,
                                                                    const float* __restrict__ gp,
                                                                    double* __restrict__ cell_ll) {
  __shared__ float4 sp_all[kEmWarps][kSlots * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int cell = blockIdx.x * kEmWarps + warp; cell < total_cells; cell += gridDim.x * kEmWarps) {
    const int ii = find_image(imgs, n, cell, 0);
    if (!GMMSP_IN_BOUNDS(ii, n, BND_IMAGE)) continue;
    const BatchImage& im = imgs[ii];
    if (!GMMSP_IN_BOUNDS(cell - im.cell_off, im.g.ncells, BND_ITEM)) continue;
    const LabPlanar src{lab + 3 * im.pix_off, (long long)im.g.W * im.g.H, im.g.W};
    label_cell_warp<LabPlanar, CM>(src, im.g, gp + (long long)im.k_off * kGP, im.labels,
                                   cell_ll ? cell_ll + im.cell_off : nullptr, cell - im.cell_off, sp_all[warp],
                                   lane);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- finalize
constexpr int kFinThreads = 32;  // one warp per block: spreads small K over more SMs

// Deterministic sum of the per-cell log-likelihoods: each block adds a fixed
// strided subset and a tree, the last block to finish adds the block sums in
// block order (one atomic ticket; no thread waits on another).  LOG2: the
// values are in log2 units and are turned into nats (in FP64) as they are read.
template <typename PT, int NT, bool LOG2>
__device__ void block_ll_sum(const PT* vals, long long stride, int n, double* blk, unsigned* ticket,
                             double* out) {
  __shared__ double red[NT];
  __shared__ bool last;
  double s = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT)
    s += LOG2 ? double(vals[(long long)i * stride]) * 0.69314718055994530942 : double(vals[(long long)i * stride]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  // The last block adds the block sums: thread t takes blocks t, t + NT, ...,
  // then a tree (FP64 adds are slow on this part: keep the chain short).
  if (last) {
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) t += *((volatile double*)&blk[b]);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      *out = red[0];
      *ticket = 0u;
    }
  }
}

// s + b as the unevaluated pair (hi, lo): TwoSum's exact error of the FP32
// addition goes into lo (no contraction or reassociation: _rn intrinsics).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// Update of superpixel k from the partial sums of its <= 9 cells (see the
// header comment).  Adds to the caller's tallies: dead (no weight), rs and rc
// (eigenvalues raised to the floor, spatial and colour), which a thread that
// updates several superpixels sums over them.  SHIFT: the
// mixed-precision path (pair sums rounded to FP64, FP64 arithmetic, moments
// about the previous mean); otherwise the FP32 variant.
template <typename PT, bool SHIFT>
__device__ __forceinline__ void finalize_k(const Geom& g, const PT* __restrict__ partials,
                                           double* __restrict__ theta, float* __restrict__ gp,
                                           double eps_s, double eps_c, int k, unsigned& dead,
                                           unsigned& rs, unsigned& rc) {
  using T = typename std::conditional<SHIFT, double, float>::type;  // arithmetic type of the update
  constexpr bool kShifted = SHIFT;
  if (!GMMSP_IN_BOUNDS(k, g.K, BND_THETA)) return;
  const int kx = k % g.nx, ky = k / g.nx;
  T S[kStats];
  float hi[kStats], lo[kStats];
#pragma unroll
  for (int j = 0; j < kStats; ++j) {
    S[j] = T(0);
    hi[j] = 0.f;
    lo[j] = 0.f;
  }
  // The cells (kx+dx, ky+dy) hold k in slot (1-dy)*3 + (1-dx); fixed order.
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int cy = ky + dy;
    if (cy < 0 || cy >= g.ncy) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int cx = kx + dx;
      if (cx < 0 || cx >= g.ncx) continue;
      if (!GMMSP_IN_BOUNDS(cy * g.ncx + cx, g.ncells, BND_PARTIAL_R)) continue;
      const PT* P = partials + (long long)(cy * g.ncx + cx) * kPartStride + ((1 - dy) * 3 + (1 - dx)) * kStats;
#pragma unroll
      for (int j = 0; j < kStats; ++j) {
        if (SHIFT) two_sum_acc(hi[j], lo[j], P[j]);
        else S[j] += T(P[j]);
      }
    }
  }
  if (SHIFT) {
#pragma unroll
    for (int j = 0; j < kStats; ++j) S[j] = T(widen(hi[j]) + widen(lo[j]));
  }
  const T Wk = S[ST_W];
  if (!(Wk >= T(1e-8))) {
    dead += 1;  // reading: a superpixel with no weight keeps theta_k
  } else {
    float* G = gp + (long long)k * kGP;
    const T iw = Num<T>::rcp(Wk);
    T mu[5], cs[3], cc[6];
    // origin of k's cell (through FP32, exact below 2^24)
    const int ix = kx * g.v, iy = ky * g.v;
    const T ox = ix < (1 << 24) ? from_f32<T>(float(ix)) : T(ix);
    const T oy = iy < (1 << 24) ? from_f32<T>(float(iy)) : T(iy);
    // Moments about r: Sigma = S2 / W - d d^T with d = S1 / W.  The shifted
    // path has r = mu_ref, the FP32 mean the E-step subtracted (spatial part
    // relative to the cell origin); the raw path has r = 0.
    T dl[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) dl[j] = S[ST_S1 + j] * iw;
    cs[0] = fma(-dl[0], dl[0], S[ST_S2S + 0] * iw);
    cs[1] = fma(-dl[0], dl[1], S[ST_S2S + 1] * iw);
    cs[2] = fma(-dl[1], dl[1], S[ST_S2S + 2] * iw);
    cc[0] = fma(-dl[2], dl[2], S[ST_S2C + 0] * iw);
    cc[1] = fma(-dl[2], dl[3], S[ST_S2C + 1] * iw);
    cc[2] = fma(-dl[2], dl[4], S[ST_S2C + 2] * iw);
    cc[3] = fma(-dl[3], dl[3], S[ST_S2C + 3] * iw);
    cc[4] = fma(-dl[3], dl[4], S[ST_S2C + 4] * iw);
    cc[5] = fma(-dl[4], dl[4], S[ST_S2C + 5] * iw);
    if (kShifted) {
      mu[0] = ox + (from_f32<T>(G[0]) + dl[0]);
      mu[1] = oy + (from_f32<T>(G[1]) + dl[1]);
#pragma unroll
      for (int j = 2; j < 5; ++j) mu[j] = from_f32<T>(G[j]) + dl[j];
    } else {
      mu[0] = ox + dl[0];
      mu[1] = oy + dl[1];
#pragma unroll
      for (int j = 2; j < 5; ++j) mu[j] = dl[j];
    }
    rs += clamp_sym2<T>(cs, T(eps_s));
    if (g.cm == kColourFull) {
      rc += clamp_sym3<T>(cc, T(eps_c));
    } else {
      // Eq. (BlockSigma1) / grayscale: no L-(a, b) entries; each block floored on its own
      cc[1] = cc[2] = T(0);
      if (!(cc[0] >= T(eps_c))) {
        cc[0] = T(eps_c);
        rc += 1;
      }
      if (g.cm == kColourSplit) {
        T ab[3] = {cc[3], cc[4], cc[5]};
        rc += clamp_sym2<T>(ab, T(eps_c));
        cc[3] = ab[0]; cc[4] = ab[1]; cc[5] = ab[2];
      } else {
        cc[3] = cc[4] = cc[5] = T(0);
        mu[3] = mu[4] = T(0);
      }
    }
    double* th = theta + (long long)k * kTheta;
#pragma unroll
    for (int j = 0; j < 5; ++j) th[j] = double(mu[j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) th[5 + j] = double(cs[j]);
#pragma unroll
    for (int j = 0; j < 6; ++j) th[8 + j] = double(cc[j]);
    pack_gp<T>(mu, cs, cc, ox, oy, G, g.cm);
  }
}

template <typename PT, bool SHIFT>
__global__ void __launch_bounds__(kFinThreads) k_finalize(Geom g, const PT* __restrict__ partials,
                                                          double* __restrict__ theta,
                                                          float* __restrict__ gp, double eps_s,
                                                          double eps_c, double* llk_out,
                                                          double* blk, unsigned* ticket,
                                                          unsigned long long* counters) {
  pdl_wait();
  pdl_trigger();
  if (llk_out)
    block_ll_sum<PT, kFinThreads, SHIFT>(partials + kSlots * kStats, kPartStride, g.ncells, blk, ticket, llk_out);

  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned dead = 0, rs = 0, rc = 0;
  if (k < g.K) finalize_k<PT, SHIFT>(g, partials, theta, gp, eps_s, eps_c, k, dead, rs, rc);
  dead = __reduce_add_sync(0xffffffffu, dead);
  rs = __reduce_add_sync(0xffffffffu, rs);
  rc = __reduce_add_sync(0xffffffffu, rc);
  if ((threadIdx.x & 31) == 0) {
    if (dead) atomicAdd(&counters[CNT_DEAD], (unsigned long long)dead);
    if (rs) atomicAdd(&counters[CNT_RAISED_S], (unsigned long long)rs);
    if (rc) atomicAdd(&counters[CNT_RAISED_C], (unsigned long long)rc);
  }
}

template <typename PT, bool SHIFT>
__global__ void __launch_bounds__(kFinThreads) k_finalize_batch(const BatchImage* __restrict__ imgs, int n,
                                                                int total_k, const PT* __restrict__ partials,
                                                                double* __restrict__ theta,
                                                                float* __restrict__ gp, double eps_s,
                                                                double eps_c,
                                                                unsigned long long* counters) {
  unsigned dead = 0, rs = 0, rc = 0;
  const int stride = gridDim.x * kFinThreads;
  for (int base = blockIdx.x * kFinThreads; base < total_k; base += stride) {
    const int k = base + threadIdx.x;
    if (k < total_k) {
      const int ii = find_image(imgs, n, k, 1);
      if (!GMMSP_IN_BOUNDS(ii, n, BND_IMAGE)) continue;
      const BatchImage& im = imgs[ii];
      if (!GMMSP_IN_BOUNDS(k - im.k_off, im.g.K, BND_ITEM)) continue;
      finalize_k<PT, SHIFT>(im.g, partials + (long long)im.cell_off * kPartStride, theta + (long long)im.k_off * kTheta,
                     gp + (long long)im.k_off * kGP, eps_s, eps_c, k - im.k_off, dead, rs, rc);
    }
  }
  dead = __reduce_add_sync(0xffffffffu, dead);
  rs = __reduce_add_sync(0xffffffffu, rs);
  rc = __reduce_add_sync(0xffffffffu, rc);
  if ((threadIdx.x & 31) == 0) {
    if (dead) atomicAdd(&counters[CNT_DEAD], (unsigned long long)dead);
    if (rs) atomicAdd(&counters[CNT_RAISED_S], (unsigned long long)rs);
    if (rc) atomicAdd(&counters[CNT_RAISED_C], (unsigned long long)rc);
  }
}

// Finalize for small K (mixed precision): 16 lanes per superpixel.  On
// GB300 an FP64 warp instruction occupies its SM sub-partition for ~64
// clocks whatever the number of active lanes, so the latency of a small
// finalize is the count of FP64 instructions on one warp's path.  Here the
// lanes of a half-warp share one superpixel and evaluate the independent
// pieces side by side with one instruction, reading their operands through a
// per-superpixel shared-memory array and small index tables:
//   lane j < 15 adds statistic j over the <= 9 cells holding k;
//   lanes 0-8 form the moment entries M (Sigma_s: xx xy yy, Sigma_c: LL La Lb
//   aa ab bb); lanes 0-6 form the 2x2 products-minus-products that the floor
//   test, the characteristic cubic, the projector and the adjugate need;
//   lanes 5-13 scale the packed coefficients.
// The floor itself (Eq. mlams/mlamc) is decided by Sylvester's criterion on
// Sigma - eps I; a raised colour eigenvalue starts from the FP32 Smith
// solution and takes one FP64 Newton step on the cubic, and the floored block
// is Sigma + (eps - l1) P1 or eps I + (l3 - eps) P3 with the projector a
// polynomial in Sigma (see gmmsp_math.cuh).
constexpr int kFin16Threads = 64;  // 4 superpixels per block

__device__ __forceinline__ int nib(unsigned long long table, int i) {
  return int((table >> (4 * i)) & 0xFull);
}

// FP64 1/x from the MUFU FP32 estimate (relative error < 2^-22) and one
// FP64 Newton step (relative error < 2^-44).
__device__ __forceinline__ double rcp64(double x) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(float(x)));
  const double r = double(r0);
  return fma(r, fma(-x, r, 1.0), r);
}

// x > 0 for a finite double, tested on its bits (integer pipe, not FP64).
__device__ __forceinline__ bool dpos(double x) { return __double_as_longlong(x) > 0; }

// One superpixel per half-warp (lane l = threadIdx.x & 15): superpixel k of
// the image with geometry g, partials, theta and gp; all 32 lanes of the warp
// call it together (valid = false for a half-warp without a superpixel).
// X (48 doubles) and F (8 floats) are the half-warp's shared scratch.
__device__ __forceinline__ void finalize_l16_body(const Geom& g, const float* __restrict__ partials,
                                                  double* __restrict__ theta, float* __restrict__ gp,
                                                  double eps_s, double eps_c, int k, bool valid, double* X,
                                                  float* F, unsigned long long* counters) {
  constexpr unsigned kFull = 0xffffffffu;
  const int l = threadIdx.x & 15;
  // X: [0..14] sums, [16..20] d, [21..29] M, [30..36] products, [37..45] scratch
  valid = valid && GMMSP_IN_BOUNDS(k, g.K, BND_THETA);
  const int kk = valid ? k : 0;
  const int kx = kk % g.nx, ky = kk / g.nx;

  // 1. Sums over the pixel set I_k: lane l < 15 adds statistic l of the <= 9
  //    cells holding k (cell (kx+dx, ky+dy) holds k in slot (1-dy)*3+(1-dx)).
  {
    float v[9];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int cy = ky + dy, cx = kx + dx;
        const bool in = valid && l < kStats && cy >= 0 && cy < g.ncy && cx >= 0 && cx < g.ncx &&
                        GMMSP_IN_BOUNDS(cy * g.ncx + cx, g.ncells, BND_PARTIAL_R);
        v[(dy + 1) * 3 + (dx + 1)] =
            in ? __ldg(partials + (long long)(cy * g.ncx + cx) * kPartStride +
                       ((1 - dy) * 3 + (1 - dx)) * kStats + l)
               : 0.f;
      }
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int j = 0; j < 9; ++j) two_sum_acc(hi, lo, v[j]);
    if (l < kStats) X[l] = double(hi) + double(lo);
  }
  __syncwarp();
  const double Wk = X[ST_W];
  // reading: no weight -> theta_k kept (positive doubles order like their bits)
  const bool live = valid && __double_as_longlong(Wk) >= __double_as_longlong(1e-8);
  const double iw = rcp64(live ? Wk : 1.0);
  if (l < 5) X[16 + l] = X[ST_S1 + l] * iw;  // d = S1 / W
  __syncwarp();
  // 2. Moments about the new mean: M_e = S2_e / W - d_a d_b.
  if (l < 9)
    X[21 + l] = fma(-X[16 + nib(0x433222100ull, l)], X[16 + nib(0x443432110ull, l)], X[ST_S2S + l] * iw);
  // new mean (lanes 0-4): mu_ref + d, mu_ref being the FP32 mean the E-step used
  float* G = gp + (long long)kk * kGP;
  const double org = (l == 0) ? double(kx * g.v) : (l == 1 ? double(ky * g.v) : 0.0);
  const double mu_l = org + (double(G[l < 5 ? l : 0]) + X[16 + (l < 5 ? l : 0)]);
  __syncwarp();

  // 3. Floor test (Sylvester on M - eps I).  E = M with shifted diagonals in
  //    X[37..45]; products (lane j): 0 c00' 1 unused 2 m2 3 c01' 4 c02' 5 det2 spatial.
  if (l < 9) {
    const double sft = (l == 0 || l == 2) ? eps_s : ((l == 3 || l == 6 || l == 8) ? eps_c : 0.0);
    X[37 + l] = X[21 + l] - sft;
  }
  __syncwarp();
  //            lane:  6 5 4 3 2 1 0
  // p (E index)        . 0 4 5 3 3 6      q: . 2 7 7 6 8 8
  // r                  . 1 5 4 4 5 7      t: . 1 6 8 4 5 7
  if (l < 6) {
    const double* E = X + 37;
    X[30 + l] = fma(E[nib(0x045336ull, l)], E[nib(0x277688ull, l)],
                    -E[nib(0x154457ull, l)] * E[nib(0x168457ull, l)]);
  }
  __syncwarp();
  bool need_s, need_c;
  {
    const double* E = X + 37;
    const double m3 = fma(E[3], X[30], fma(E[4], X[33], E[5] * X[34]));
    need_c = live && !(dpos(E[3]) && dpos(X[32]) && dpos(m3));
    need_s = live && !(dpos(E[0]) && dpos(X[35]));
  }
  int rc = 0, rs = 0;
  __syncwarp();
  if (__any_sync(kFull, need_c)) {
    // Characteristic cubic lambda^3 - c2 lambda^2 + c1 lambda - c0 of the colour
    // block: products (lane j < 5) M00 M11 M22 c01 c02 of M.
    if (l < 5) {
      const double* A = X + 21;
      X[30 + l] = fma(A[nib(0x45336ull, l)], A[nib(0x77688ull, l)], -A[nib(0x54457ull, l)] * A[nib(0x68457ull, l)]);
    }
    if (l < 6) F[l] = float(X[24 + l]);
    __syncwarp();
    const double a00 = X[24], a01 = X[25], a02 = X[26], a11 = X[27], a22 = X[29];
    const double c2 = a00 + a11 + a22;
    const double c1 = X[30] + X[31] + X[32];
    const double c0 = fma(a00, X[30], fma(a01, X[33], a02 * X[34]));
    float f1, f2, f3;
    eig3_seed(F[0], F[1], F[2], F[3], F[4], F[5], f1, f2, f3);
    const float fe = float(eps_c);
    const int n = (f1 < fe) + (f2 < fe) + (f3 < fe);
    const double scale = fabs(double(f3)) + eps_c;
    const bool degenerate = n == 3 || double(f3) - double(f1) <= 1e-6 * scale;
    double lj = double(n == 1 ? f1 : f3);
    {
      const double pv = fma(fma(lj - c2, lj, c1), lj, -c0);
      const double dp0 = fma(fma(3.0, lj, -2.0 * c2), lj, c1);
      float r;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(float(dp0)));
      if (fabs(dp0) > 1e-12 * scale * scale) lj = fma(-pv, double(r), lj);
    }
    const double dp = fma(fma(3.0, lj, -2.0 * c2), lj, c1);  // (lj - la)(lj - lb)
    const double sum = c2 - lj, prod = fma(-lj, sum, c1);
    const bool flat = degenerate || !(fabs(dp) > 1e-12 * scale * scale);
    const double gnum = (n == 1) ? eps_c - lj : lj - eps_c;
    const double gk = gnum * rcp64(flat ? 1.0 : dp);
    // Projector entry j (lanes 0-5, order LL La Lb aa ab bb):
    //   (A^2)_j - sum A_j + prod [j diagonal]; A^2_j = row_r . col_c (3 terms).
    double newA = 0.0;
    if (l < 6) {
      const double* A = X + 24;
      // (A^2)_j = sum_m A[r][m] A[m][c] with (r, c) of entry j
      const int rr = nib(0x211000ull, l), cc_ = nib(0x221210ull, l);
      auto idx = [](int a, int b) {  // packed index of A[a][b]
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
      };
      double a2 = 0.0;
#pragma unroll
      for (int m = 0; m < 3; ++m) a2 = fma(A[idx(rr, m)], A[idx(m, cc_)], a2);
      const bool diag = (l == 0 || l == 3 || l == 5);
      const double P = fma(-sum, A[l], a2) + (diag ? prod : 0.0);
      const double base = (n == 1) ? A[l] : (diag ? eps_c : 0.0);
      newA = flat ? (diag ? (n == 3 ? eps_c : fmax(c2 / 3.0, eps_c)) : 0.0) : fma(gk, P, base);
    }
    __syncwarp();
    if (need_c && l < 6) X[24 + l] = newA;
    rc = need_c ? n : 0;
  }
  __syncwarp();
  if (need_s) {  // spatial floor: rare (eigenvalues ~ v^2 / 12 against eps_s = 2)
    double cs[3] = {X[21], X[22], X[23]};
    rs = clamp_sym2<double>(cs, eps_s);
    __syncwarp(__activemask());
    if (l < 3) X[21 + l] = cs[l];
  }
  __syncwarp();

  // 4. Pack: colour cofactors and the spatial determinant (lanes 0-6):
  //    0 c00 1 c01 2 c02 3 c11 4 c12 5 c22 6 ds (indices into M = X[21..29]).
  if (l < 7) {
    const double* M = X + 21;
    X[30 + l] = fma(M[nib(0x0343456ull, l)], M[nib(0x2658778ull, l)],
                    -M[nib(0x1435547ull, l)] * M[nib(0x1475687ull, l)]);
  }
  __syncwarp();
  const double dc = fma(X[24], X[30], fma(X[25], X[31], X[26] * X[32]));
  const double ds = X[36];
  const bool pd = dpos(X[21]) && dpos(ds) && dpos(X[24]) && dpos(X[35]) && dpos(dc);
  const double idet = rcp64((l & 1) ? (dpos(dc) ? dc : 1.0) : (dpos(ds) ? ds : 1.0));
  const double ids = __shfl_sync(kFull, idet, 0, 16), idc = __shfl_sync(kFull, idet, 1, 16);
  // Coefficient lane l in 5..13: factor * numerator, numerators
  //   5 yy 6 xy 7 xx (from M) | 8 c00 9 c11 10 c22 11 c01 12 c02 13 c12 (from X[30..])
  float out = 0.f;
  {
    const int li = l < 5 ? 5 : (l > 13 ? 13 : l);
    const int j = li - 5;
    const bool spatial = j < 3;
    const double num = spatial ? X[21 + nib(0x012ull, j)] : X[30 + nib(0x421530ull, j - 3 < 0 ? 0 : j - 3)];
    const double mult = spatial ? (j == 1 ? -2.0 : 1.0) : (j >= 6 ? 2.0 : 1.0);
    const double coef = (-0.5 * Num<double>::kLog2e * mult) * (spatial ? ids : idc) * num;
    if (l >= 5 && l <= 13) out = float(coef);
  }
  if (l < 5) out = float(mu_l - org);
  if (l == 14)
    out = -0.5f * (Num<double>::log2_(dpos(ds) ? ds : 1.0) + Num<double>::log2_(dpos(dc) ? dc : 1.0)) -
          float(Num<double>::kHalfD_Log2_2Pi);
  if (live && pd) {
    G[l] = out;
    // theta: [0..4] mu, [5..7] Sigma_s, [8..13] Sigma_c (= M in order)
    if (l < 14) theta[(long long)kk * kTheta + l] = (l < 5) ? mu_l : X[21 + (l - 5)];
  }
  unsigned dead = (valid && !live && l == 0) ? 1u : 0u;
  unsigned urs = (live && l == 0) ? unsigned(rs) : 0u, urc = (live && l == 0) ? unsigned(rc) : 0u;
  dead = __reduce_add_sync(kFull, dead);
  urs = __reduce_add_sync(kFull, urs);
  urc = __reduce_add_sync(kFull, urc);
  if ((threadIdx.x & 31) == 0) {
    if (dead) atomicAdd(&counters[CNT_DEAD], (unsigned long long)dead);
    if (urs) atomicAdd(&counters[CNT_RAISED_S], (unsigned long long)urs);
    if (urc) atomicAdd(&counters[CNT_RAISED_C], (unsigned long long)urc);
  }
}

__global__ void __launch_bounds__(kFin16Threads) k_finalize_l16(Geom g, const float* __restrict__ partials,
                                                              double* __restrict__ theta,
                                                              float* __restrict__ gp, double eps_s,
                                                              double eps_c, double* llk_out, double* blk,
                                                              unsigned* ticket,
                                                              unsigned long long* counters) {
  __shared__ double sh[kFin16Threads / 16][48];
  __shared__ float shf[kFin16Threads / 16][8];
  pdl_wait();
  pdl_trigger();
  if (llk_out)
    block_ll_sum<float, kFin16Threads, true>(partials + kSlots * kStats, kPartStride, g.ncells, blk, ticket,
                                        llk_out);
  const int q = threadIdx.x >> 4;
  const int k = blockIdx.x * (kFin16Threads / 16) + q;
  finalize_l16_body(g, partials, theta, gp, eps_s, eps_c, k, k < g.K, sh[q], shf[q], counters);
}

// The same over a batch: half-warp q of block b takes superpixel 4 b + q of
// the batch, found in its image by a binary search over the offsets.
__global__ void __launch_bounds__(kFin16Threads) k_finalize_l16_batch(const BatchImage* __restrict__ imgs, int n,
                                                                    int total_k, const float* __restrict__ partials,
                                                                    double* __restrict__ theta,
                                                                    float* __restrict__ gp, double eps_s,
                                                                    double eps_c, unsigned long long* counters) {
  __shared__ double sh[kFin16Threads / 16][48];
  __shared__ float shf[kFin16Threads / 16][8];
  const int q = threadIdx.x >> 4;
  const int kg = blockIdx.x * (kFin16Threads / 16) + q;
  const int ii = find_image(imgs, n, kg < total_k ? kg : 0, 1);
  const bool img_ok = GMMSP_IN_BOUNDS(ii, n, BND_IMAGE);
  const BatchImage& im = imgs[img_ok ? ii : 0];
  const bool valid = kg < total_k && img_ok && GMMSP_IN_BOUNDS(kg - im.k_off, im.g.K, BND_ITEM);
  finalize_l16_body(im.g, partials + (long long)im.cell_off * kPartStride, theta + (long long)im.k_off * kTheta,
                    gp + (long long)im.k_off * kGP, eps_s, eps_c, valid ? kg - im.k_off : 0, valid, sh[q], shf[q],
                    counters);
}

__global__ void __launch_bounds__(kFinThreads) k_ll_reduce(const double* __restrict__ cell_ll, int n,
                                                           double* blk, unsigned* ticket, double* out) {
  pdl_wait();
  pdl_trigger();
  block_ll_sum<double, kFinThreads, false>(cell_ll, 1, n, blk, ticket, out);
}

// ---------------------------------------------------------------- bounds status
cudaError_t bounds_take_em(unsigned long long* word) {
  *word = 0ull;
#ifdef GMMSP_CHECK_BOUNDS
  cudaError_t e = cudaMemcpyFromSymbol(word, g_bounds_word, sizeof(*word));
  if (e != cudaSuccess) return e;
  const unsigned long long zero = 0ull;
  return cudaMemcpyToSymbol(g_bounds_word, &zero, sizeof(zero));
#else
  return cudaSuccess;
#endif
}

// ---------------------------------------------------------------- launchers
static int ll_blocks(const Geom& g) { return (g.K + kFinThreads - 1) / kFinThreads; }

// Superpixel count up to which the 16-lane finalize is used.
constexpr int kFin16MaxK = 4096;

size_t finalize_workspace_doubles(const Geom& g) {
  const size_t b16 = size_t((g.K + kFin16Threads / 16 - 1) / (kFin16Threads / 16));
  return (b16 > size_t(ll_blocks(g)) ? b16 : size_t(ll_blocks(g))) + 1;
}

template <typename PT, bool SHIFT, int WPC, class Src, int CM>
static cudaError_t em_pass_impl(Src lab, const Geom& g, const float* gp, PT* partials,
                                cudaStream_t s) {
  constexpr int smem = em_smem_bytes<WPC>();
  static_assert(smem <= 227 * 1024, "shared memory");
  const auto kernel = [] {
    if constexpr (WPC == 1 && CM == kColourFull) return k_em_pass_capped<PT, SHIFT, WPC, Src, CM>;
    else return k_em_pass<PT, SHIFT, WPC, Src, CM>;
  }();
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set && smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  constexpr int cpb = kEmWarps / WPC;
  const int blocks = (g.ncells + cpb - 1) / cpb;
  return launch_pdl(kernel, dim3(blocks), dim3(kEmWarps * 32), smem, s, lab, g, gp, partials);
}

template <typename PT, bool SHIFT, class Src, int CM>
static cudaError_t em_pass_wpc(Src lab, const Geom& g, const float* gp, PT* partials, int wpc,
                               cudaStream_t s) {
  switch (wpc) {
    case 2: return em_pass_impl<PT, SHIFT, 2, Src, CM>(lab, g, gp, partials, s);
    case 4: return em_pass_impl<PT, SHIFT, 4, Src, CM>(lab, g, gp, partials, s);
    default: return em_pass_impl<PT, SHIFT, 1, Src, CM>(lab, g, gp, partials, s);
  }
}

// The FP32 variant and the caller-pitched source take the full colour model
// only (the entry points check it).
template <class Src>
cudaError_t launch_em_pass(Src lab, const Geom& g, const float* gp, void* partials, int precision,
                           int wpc, cudaStream_t s) {
  float* part = static_cast<float*>(partials);
  if (precision == 1) return em_pass_wpc<float, false, Src, kColourFull>(lab, g, gp, part, wpc, s);
  if constexpr (std::is_same<Src, LabPlanar>::value) {
    if (g.cm == kColourSplit) return em_pass_wpc<float, true, Src, kColourSplit>(lab, g, gp, part, wpc, s);
    if (g.cm == kColourGray) return em_pass_wpc<float, true, Src, kColourGray>(lab, g, gp, part, wpc, s);
  }
  if (g.cm != kColourFull) return cudaErrorInvalidValue;
  return em_pass_wpc<float, true, Src, kColourFull>(lab, g, gp, part, wpc, s);
}

template <class Src>
cudaError_t launch_label_pass(Src lab, const Geom& g, const float* gp, int32_t* labels,
                              double* cell_ll, cudaStream_t s) {
  const int blocks = (g.ncells + kEmWarps - 1) / kEmWarps;
  if constexpr (std::is_same<Src, LabPlanar>::value) {
    if (g.cm == kColourSplit)
      return launch_pdl(k_label_pass<Src, kColourSplit>, dim3(blocks), dim3(kEmWarps * 32), 0, s, lab, g, gp,
                        labels, cell_ll);
    if (g.cm == kColourGray)
      return launch_pdl(k_label_pass<Src, kColourGray>, dim3(blocks), dim3(kEmWarps * 32), 0, s, lab, g, gp,
                        labels, cell_ll);
  }
  if (g.cm != kColourFull) return cudaErrorInvalidValue;
  return launch_pdl(k_label_pass<Src, kColourFull>, dim3(blocks), dim3(kEmWarps * 32), 0, s, lab, g, gp, labels,
                    cell_ll);
}

template cudaError_t launch_em_pass<LabPlanar>(LabPlanar, const Geom&, const float*, void*, int, int,
                                               cudaStream_t);
template cudaError_t launch_em_pass<LabPitched>(LabPitched, const Geom&, const float*, void*, int, int,
                                                cudaStream_t);
template cudaError_t launch_label_pass<LabPlanar>(LabPlanar, const Geom&, const float*, int32_t*, double*,
                                                  cudaStream_t);
template cudaError_t launch_label_pass<LabPitched>(LabPitched, const Geom&, const float*, int32_t*,
                                                   double*, cudaStream_t);

cudaError_t launch_finalize(const Geom& g, const void* partials, double* theta, float* gp,
                            double eps_s, double eps_c, double* llk_out, double* ws,
                            unsigned* ticket, unsigned long long* counters, int precision,
                            cudaStream_t s) {
  if (precision != 1 && g.K <= kFin16MaxK && g.cm == kColourFull) {
    const int blocks16 = (g.K + kFin16Threads / 16 - 1) / (kFin16Threads / 16);
    return launch_pdl(k_finalize_l16, dim3(blocks16), dim3(kFin16Threads), 0, s, g,
                      static_cast<const float*>(partials), theta, gp, eps_s, eps_c, llk_out, ws, ticket,
                      counters);
  }
  const int blocks = ll_blocks(g);
  if (precision == 1)
    return launch_pdl(k_finalize<float, false>, dim3(blocks), dim3(kFinThreads), 0, s, g,
                      static_cast<const float*>(partials), theta, gp, eps_s, eps_c, llk_out, ws, ticket,
                      counters);
  return launch_pdl(k_finalize<float, true>, dim3(blocks), dim3(kFinThreads), 0, s, g,
                    static_cast<const float*>(partials), theta, gp, eps_s, eps_c, llk_out, ws, ticket,
                    counters);
}

cudaError_t launch_ll_reduce(const double* cell_ll, int n, double* out, double* ws, unsigned* ticket,
                             const Geom& g, cudaStream_t s) {
  return launch_pdl(k_ll_reduce, dim3(ll_blocks(g)), dim3(kFinThreads), 0, s, cell_ll, n, ws, ticket, out);
}

}  // namespace gmmsp

// ---------------------------------------------------------------- batch launchers
namespace gmmsp {

template <int CM>
static void em_pass_batch_mixed(const BatchImage* imgs, int n, int total_cells, const float* lab, const float* gp,
                                float* partials, int blocks, int minb, bool diag, cudaStream_t s) {
  constexpr int smem = em_smem_bytes<1>();
  if (minb >= 6) {  // one cell per warp over a grid sized to the work
    const int nb = (total_cells + kEmWarps - 1) / kEmWarps;
    auto kernel = minb >= 7 ? (diag ? k_em_pass_batch_flat<float, true, 7, CM, true>
                                    : k_em_pass_batch_flat<float, true, 7, CM, false>)
                            : (diag ? k_em_pass_batch_flat<float, true, 6, CM, true>
                                    : k_em_pass_batch_flat<float, true, 6, CM, false>);
    kernel<<<nb, kEmWarps * 32, smem, s>>>(imgs, n, total_cells, lab, gp, partials);
  } else {
    k_em_pass_batch<float, true, 5, CM><<<blocks, kEmWarps * 32, smem, s>>>(imgs, n, total_cells, lab, gp,
                                                                          partials);
  }
}

cudaError_t launch_em_pass_batch(const BatchImage* imgs, int n, int total_cells, const float* lab,
                                 const float* gp, void* partials, int precision, int blocks, int minb,
                                 int cm, cudaStream_t s, bool diag) {
  constexpr int smem = em_smem_bytes<1>();
  if (precision == 1) {  // full colour model only
    if (cm != kColourFull) return cudaErrorInvalidValue;
    if (minb >= 6) {
      const int nb = (total_cells + kEmWarps - 1) / kEmWarps;
      k_em_pass_batch_flat<float, false, 6, kColourFull><<<nb, kEmWarps * 32, smem, s>>>(
          imgs, n, total_cells, lab, gp, static_cast<float*>(partials));
    } else {
      k_em_pass_batch<float, false, 5, kColourFull><<<blocks, kEmWarps * 32, smem, s>>>(
          imgs, n, total_cells, lab, gp, static_cast<float*>(partials));
    }
    return cudaGetLastError();
  }
  float* part = static_cast<float*>(partials);
  switch (cm) {
    case kColourFull: em_pass_batch_mixed<kColourFull>(imgs, n, total_cells, lab, gp, part, blocks, minb, diag, s); break;
    case kColourSplit: em_pass_batch_mixed<kColourSplit>(imgs, n, total_cells, lab, gp, part, blocks, minb, diag, s); break;
    case kColourGray: em_pass_batch_mixed<kColourGray>(imgs, n, total_cells, lab, gp, part, blocks, minb, diag, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const BatchImage* imgs, int n, int total_k, const void* partials,
                                  double* theta, float* gp, double eps_s, double eps_c,
                                  unsigned long long* counters, int precision, int blocks,
                                  cudaStream_t s) {
  if (precision != 1 && blocks == 0) {  // 16 lanes per superpixel
    const int nb = (total_k + kFin16Threads / 16 - 1) / (kFin16Threads / 16);
    k_finalize_l16_batch<<<nb, kFin16Threads, 0, s>>>(imgs, n, total_k, static_cast<const float*>(partials), theta,
                                                     gp, eps_s, eps_c, counters);
    return cudaGetLastError();
  }
  if (precision == 1)
    k_finalize_batch<float, false><<<blocks, kFinThreads, 0, s>>>(imgs, n, total_k,
                                                                  static_cast<const float*>(partials), theta, gp,
                                                                  eps_s, eps_c, counters);
  else
    k_finalize_batch<float, true><<<blocks, kFinThreads, 0, s>>>(imgs, n, total_k,
                                                                 static_cast<const float*>(partials), theta, gp,
                                                                 eps_s, eps_c, counters);
  return cudaGetLastError();
}

int label_pass_batch_occupancy() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_label_pass_batch<kColourFull>, kEmWarps * 32, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 4;
  }
  return nb;
}

cudaError_t launch_label_pass_batch(const BatchImage* imgs, int n, int total_cells, const float* lab,
                                    const float* gp, double* cell_ll, int blocks, int cm, cudaStream_t s) {
  switch (cm) {
    case kColourFull:
      k_label_pass_batch<kColourFull><<<blocks, kEmWarps * 32, 0, s>>>(imgs, n, total_cells, lab, gp, cell_ll);
      break;
    case kColourSplit:
      k_label_pass_batch<kColourSplit><<<blocks, kEmWarps * 32, 0, s>>>(imgs, n, total_cells, lab, gp, cell_ll);
      break;
    case kColourGray:
      k_label_pass_batch<kColourGray><<<blocks, kEmWarps * 32, 0, s>>>(imgs, n, total_cells, lab, gp, cell_ll);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gmmsp
