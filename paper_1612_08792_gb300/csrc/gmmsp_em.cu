// The EM hot path: fused E-step + M-step partial sums per cell, the FP64
// finalize with the eigenvalue floor, and the label pass.
//
// Work decomposition.  The pixels of one v x v cell share one candidate set
// (see gmmsp_internal.cuh), so one warp takes one cell: it stages the <= 9
// candidates' packed parameters in shared memory (read back as warp-wide
// broadcasts), walks the cell's pixels 32 at a time with one 16-byte load per
// pixel, and per pixel
//   E:  evaluates log2 p(z; theta_k) for its candidates (Eq. gaussian with the
//       block covariance), forms the posteriors R_ik (Eq. Rik) with the
//       log-sum-exp held in registers, and accumulates ln sum_k p (the
//       log-likelihood L following Eq. ftheta);
//   M:  adds R_ik and R_ik d, R_ik d d^T (block-diagonal entries only) into
//       per-lane FP32 accumulators, d = z - mu_k(old) (the data shifted by
//       the previous mean so the second moments do not cancel).
// The 32 lanes' 9 x 15 accumulators are then summed through shared memory
// (a transpose, so every lane adds up whole rows) and written once per cell
// as FP64: a block-level partial, with no global atomics.
//
// The finalize (one thread per superpixel k, FP64) adds the <= 9 partials of
// the cells whose candidate set holds k in a fixed order, giving the sums
// over the pixel set I_k of Eq. (Ik), and turns them into Eq. (UpdateMu),
// (UpdateSigS) and (UpdateSigC):
//   mu = mu_old + S1 / W,   Sigma = S2 / W - (S1 / W)(S1 / W)^T,
// then applies the floor of Eq. (mlams)/(mlamc) and re-packs the E-step
// coefficients.  A superpixel with W < 1e-8 keeps its parameters.
#include <math.h>

#include "gmmsp_internal.cuh"
#include "gmmsp_math.cuh"

namespace gmmsp {

constexpr int kEmWarps = 4;          // cells per 128-thread block
constexpr int kRedRows = 68;         // rows of the reduction buffer (2 halves of 136)

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
  unsigned m = 0;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int kx = c.cx - 1 + s % 3, ky = c.cy - 1 + s / 3;
    if (kx >= 0 && kx < g.nx && ky >= 0 && ky < g.ny) m |= 1u << s;
  }
  c.mask = m;
  return c;
}

// Copies the packed parameters of the cell's candidate slots into sp[36]
// (float4); slots off the grid are zero and never read.
__device__ __forceinline__ void stage_params(const Geom& g, const Cell& c, const float* gp,
                                             float4* sp, int lane) {
  for (int i = lane; i < kSlots * 4; i += 32) {
    const int s = i >> 2, q = i & 3;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((c.mask >> s) & 1u) {
      const int k = (c.cy - 1 + s / 3) * g.nx + (c.cx - 1 + s % 3);
      v = __ldg(reinterpret_cast<const float4*>(gp) + k * 4 + q);
    }
    sp[i] = v;
  }
  __syncwarp();
}

// log2 p(z; theta_k) for one candidate: the log normaliser plus the two
// quadratic forms, with -1/2 log2(e) Sigma^{-1} folded into the coefficients.
// fx, fy are the pixel's coordinates relative to the candidate's cell origin.
__device__ __forceinline__ float log2_density(const float4* P, float fx, float fy, float4 z) {
  const float4 p0 = P[0], p1 = P[1], p2 = P[2], p3 = P[3];
  const float dx = fx - p0.x, dy = fy - p0.y;
  const float dL = z.x - p0.z, da = z.y - p0.w, db = z.z - p1.x;
  float q = p3.z;
  q = fmaf(fmaf(p1.z, dy, p1.y * dx), dx, q);       // (xx dx + 2xy dy) dx
  q = fmaf(p1.w * dy, dy, q);                        // yy dy^2
  q = fmaf(fmaf(p3.x, db, fmaf(p2.w, da, p2.x * dL)), dL, q);  // (LL dL + 2La da + 2Lb db) dL
  q = fmaf(fmaf(p3.y, db, p2.y * da), da, q);        // (aa da + 2ab db) da
  q = fmaf(p2.z * db, db, q);                        // bb db^2
  return q;
}

// One pixel of the fused E + M-partial pass.  fxs[j] / fys[j] are the
// pixel's coordinates relative to the origin of the candidate cells of
// column / row j (exact small integers), see rel_coords().
template <bool FULL, bool SHIFT>
__device__ __forceinline__ void em_pixel(const float4* sp, unsigned mask, const float (&fxs)[3],
                                         const float (&fys)[3], float4 z,
                                         float (&acc)[kSlots * kStats], float& ll) {
  float e[kSlots];
  float m = -INFINITY;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    e[s] = 0.f;
    if (FULL || ((mask >> s) & 1u)) {
      e[s] = log2_density(sp + 4 * s, fxs[s % 3], fys[s / 3], z);
      m = fmaxf(m, e[s]);
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (FULL || ((mask >> s) & 1u)) {
      e[s] = ex2_approx(e[s] - m);
      sum += e[s];
    }
  }
  const float inv = rcp_approx(sum);
  ll += m + lg2_approx(sum);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (FULL || ((mask >> s) & 1u)) {
      const float r = e[s] * inv;
      float dx = fxs[s % 3], dy = fys[s / 3], dL = z.x, da = z.y, db = z.z;
      if (SHIFT) {
        const float4 p0 = sp[4 * s], p1 = sp[4 * s + 1];
        dx -= p0.x; dy -= p0.y; dL -= p0.z; da -= p0.w; db -= p1.x;
      }
      float* A = acc + s * kStats;
      const float rx = r * dx, ry = r * dy, rL = r * dL, ra = r * da, rb = r * db;
      A[0] += r;
      A[1] += rx; A[2] += ry; A[3] += rL; A[4] += ra; A[5] += rb;
      A[6] = fmaf(rx, dx, A[6]);
      A[7] = fmaf(rx, dy, A[7]);
      A[8] = fmaf(ry, dy, A[8]);
      A[9] = fmaf(rL, dL, A[9]);
      A[10] = fmaf(rL, da, A[10]);
      A[11] = fmaf(rL, db, A[11]);
      A[12] = fmaf(ra, da, A[12]);
      A[13] = fmaf(ra, db, A[13]);
      A[14] = fmaf(rb, db, A[14]);
    }
  }
}

// Coordinates of pixel (rx, ry) of a cell relative to the cell origins of
// the candidate columns/rows cx-1, cx, cx+1: rx + v, rx, rx - v.
__device__ __forceinline__ void rel_coords(int rx, int ry, int v, float (&fxs)[3], float (&fys)[3]) {
  fxs[0] = float(rx + v); fxs[1] = float(rx); fxs[2] = float(rx - v);
  fys[0] = float(ry + v); fys[1] = float(ry); fys[2] = float(ry - v);
}

template <bool FULL, bool SHIFT, int LANES, class Src>
__device__ __forceinline__ void em_cell_pixels(const Src& lab, const Geom& g,
                                               const Cell& c, const float4* sp, int t,
                                               float (&acc)[kSlots * kStats], float& ll) {
  const int npx = c.cw * c.ch;
  const float inv_cw = 1.f / float(c.cw);
  // Pixel p of the cell: row floor(p / cw) (exact: (p + 1/2) / cw is at least
  // 1/(2 cw) away from an integer), column p - row * cw.  The next pixel's
  // colour is loaded before the current one is processed.
  auto locate = [&](int p, int& rx, int& ry) {
    ry = __float2int_rz((float(p) + 0.5f) * inv_cw);
    rx = p - ry * c.cw;
  };
  int p = t, rx = 0, ry = 0;
  float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p < npx) {
    locate(p, rx, ry);
    z = lab.load(c.x0 + rx, c.y0 + ry);
  }
  while (p < npx) {
    const int pn = p + LANES;
    int rxn = 0, ryn = 0;
    float4 zn = z;
    if (pn < npx) {
      locate(pn, rxn, ryn);
      zn = lab.load(c.x0 + rxn, c.y0 + ryn);
    }
    float fxs[3], fys[3];
    rel_coords(rx, ry, g.v, fxs, fys);
    em_pixel<FULL, SHIFT>(sp, c.mask, fxs, fys, z, acc, ll);
    p = pn; rx = rxn; ry = ryn; z = zn;
  }
}

// Fused E-step + M-step partial sums.  PT = double (mixed precision, shifted
// moments) or float (all-FP32 variant, raw moments).  WPC warps share one
// cell (more parallelism for small images); a 128-thread block holds
// 4 / WPC cells.  The WPC x 32 per-thread accumulator sets of a cell are
// summed through shared memory: every thread writes its column of a
// 68-row tile (two tiles for the 136 sums), then each thread adds up whole rows.
template <typename PT, bool SHIFT, int WPC, class Src>
__global__ void __launch_bounds__(kEmWarps * 32) k_em_pass(Src lab, Geom g,
                                                           const float* __restrict__ gp,
                                                           PT* __restrict__ partials) {
  constexpr int kLanes = 32 * WPC;             // threads per cell
  constexpr int kCellsPerBlock = kEmWarps / WPC;
  constexpr int kLd = kLanes + 1;              // padded row: conflict-free transposes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = warp / WPC;                 // cell slot within the block
  const int t = (warp % WPC) * 32 + lane;      // thread index within the cell
  float4* sp = reinterpret_cast<float4*>(smem_raw) + slot * (kSlots * 4);
  float* red = reinterpret_cast<float*>(smem_raw + kCellsPerBlock * kSlots * 4 * 16) +
               slot * (kRedRows * kLd);
  const int cell = blockIdx.x * kCellsPerBlock + slot;
  const bool active = cell < g.ncells;         // inactive threads still reach every barrier
  Cell c = {};
  if (active) {
    c = make_cell(g, cell);
    for (int i = t; i < kSlots * 4; i += kLanes) {
      const int s = i >> 2, q = i & 3;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((c.mask >> s) & 1u) {
        const int k = (c.cy - 1 + s / 3) * g.nx + (c.cx - 1 + s % 3);
        v = __ldg(reinterpret_cast<const float4*>(gp) + k * 4 + q);
      }
      sp[i] = v;
    }
  }
  if (WPC == 1) __syncwarp(); else __syncthreads();

  float acc[kSlots * kStats];
#pragma unroll
  for (int j = 0; j < kSlots * kStats; ++j) acc[j] = 0.f;
  float ll = 0.f;
  if (active) {
    if (c.mask == 0x1ffu)
      em_cell_pixels<true, SHIFT, kLanes, Src>(lab, g, c, sp, t, acc, ll);
    else
      em_cell_pixels<false, SHIFT, kLanes, Src>(lab, g, c, sp, t, acc, ll);
  }

  // Row 135 carries the log-likelihood (log2 units until written).
  PT* out = partials + (long long)cell * kPartStride;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int j = 0; j < kRedRows; ++j) {
      const int row = h * kRedRows + j;
      red[j * kLd + t] = (row < kSlots * kStats) ? acc[row] : ll;
    }
    if (WPC == 1) __syncwarp(); else __syncthreads();
    if (active) {
      for (int j = t; j < kRedRows; j += kLanes) {
        float s = 0.f;
#pragma unroll 8
        for (int q = 0; q < kLanes; ++q) s += red[j * kLd + q];
        const int row = h * kRedRows + j;
        out[row] = (row < kSlots * kStats) ? PT(s) : PT(s) * PT(0.69314718055994530942);
      }
    }
    if (WPC == 1) __syncwarp(); else __syncthreads();
  }
}

template <int WPC>
constexpr int em_smem_bytes() {
  return (kEmWarps / WPC) * (kSlots * 4 * 16 + kRedRows * (32 * WPC + 1) * 4);
}

// Label pass: argmax posterior per pixel (ties to the smaller k, i.e. the
// smaller slot) and the per-cell log-likelihood.
template <bool FULL, class Src>
__device__ __forceinline__ void label_cell_pixels(const Src& lab, const Geom& g,
                                                  const Cell& c, const float4* sp, int lane,
                                                  int32_t* __restrict__ labels, float& ll) {
  const int npx = c.cw * c.ch;
  const float inv_cw = 1.f / float(c.cw);
  for (int p = lane; p < npx; p += 32) {
    const int ry = __float2int_rz((float(p) + 0.5f) * inv_cw);
    const int rx = p - ry * c.cw;
    const int x = c.x0 + rx, y = c.y0 + ry;
    const float4 z = lab.load(x, y);
    float fxs[3], fys[3];
    rel_coords(rx, ry, g.v, fxs, fys);
    float e[kSlots];
    float m = -INFINITY;
    int best = 0;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      e[s] = 0.f;
      if (FULL || ((c.mask >> s) & 1u)) {
        e[s] = log2_density(sp + 4 * s, fxs[s % 3], fys[s / 3], z);
        if (e[s] > m) { m = e[s]; best = s; }
      }
    }
    float sum = 0.f;
#pragma unroll
    for (int s = 0; s < kSlots; ++s)
      if (FULL || ((c.mask >> s) & 1u)) sum += ex2_approx(e[s] - m);
    ll += m + lg2_approx(sum);
    labels[(long long)y * g.W + x] = (c.cy - 1 + best / 3) * g.nx + (c.cx - 1 + best % 3);
  }
}

template <class Src>
__global__ void __launch_bounds__(kEmWarps * 32) k_label_pass(Src lab, Geom g, const float* __restrict__ gp,
                                                              int32_t* __restrict__ labels,
                                                              double* __restrict__ cell_ll) {
  __shared__ float4 sp_all[kEmWarps][kSlots * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kEmWarps + warp;
  if (cell >= g.ncells) return;
  const Cell c = make_cell(g, cell);
  float4* sp = sp_all[warp];
  stage_params(g, c, gp, sp, lane);
  float ll = 0.f;
  if (c.mask == 0x1ffu)
    label_cell_pixels<true, Src>(lab, g, c, sp, lane, labels, ll);
  else
    label_cell_pixels<false, Src>(lab, g, c, sp, lane, labels, ll);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
  if (lane == 0) cell_ll[cell] = double(ll) * 0.69314718055994530942;
}

// ---------------------------------------------------------------- finalize
constexpr int kFinThreads = 32;  // one warp per block: spreads small K over more SMs

// Deterministic sum of the per-cell log-likelihoods: each block adds a fixed
// strided subset and a tree, the last block to finish adds the block sums in
// block order (one atomic ticket; no thread waits on another).
template <typename PT>
__device__ void block_ll_sum(const PT* vals, long long stride, int n, double* blk, unsigned* ticket,
                             double* out) {
  __shared__ double red[kFinThreads];
  __shared__ bool last;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += double(vals[(long long)i * stride]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += *((volatile double*)&blk[b]);
    *out = t;
    *ticket = 0u;
  }
}

template <typename PT>
__global__ void __launch_bounds__(kFinThreads) k_finalize(Geom g, const PT* __restrict__ partials,
                                                          double* __restrict__ theta,
                                                          float* __restrict__ gp, double eps_s,
                                                          double eps_c, double* llk_out,
                                                          double* blk, unsigned* ticket,
                                                          unsigned long long* counters) {
  using T = PT;  // arithmetic type of the update: double, or float for the FP32 variant
  constexpr bool kShifted = sizeof(PT) == 8;
  if (llk_out) block_ll_sum<PT>(partials + kSlots * kStats, kPartStride, g.ncells, blk, ticket, llk_out);

  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned dead = 0, rs = 0, rc = 0;
  if (k < g.K) {
    const int kx = k % g.nx, ky = k / g.nx;
    T S[kStats];
#pragma unroll
    for (int j = 0; j < kStats; ++j) S[j] = T(0);
    // The cells (kx+dx, ky+dy) hold k in slot (1-dy)*3 + (1-dx); fixed order.
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = ky + dy;
      if (cy < 0 || cy >= g.ncy) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int cx = kx + dx;
        if (cx < 0 || cx >= g.ncx) continue;
        const PT* P = partials + (long long)(cy * g.ncx + cx) * kPartStride + ((1 - dy) * 3 + (1 - dx)) * kStats;
#pragma unroll
        for (int j = 0; j < kStats; ++j) S[j] += P[j];
      }
    }
    const T Wk = S[ST_W];
    if (!(Wk >= T(1e-8))) {
      dead = 1;  // reading: a superpixel with no weight keeps theta_k
    } else {
      float* G = gp + (long long)k * kGP;
      const T iw = Num<T>::rcp(Wk);
      T mu[5], cs[3], cc[6];
      const T ox = T(kx * g.v), oy = T(ky * g.v);  // origin of k's cell
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
        mu[0] = ox + (T(G[0]) + dl[0]);
        mu[1] = oy + (T(G[1]) + dl[1]);
#pragma unroll
        for (int j = 2; j < 5; ++j) mu[j] = T(G[j]) + dl[j];
      } else {
        mu[0] = ox + dl[0];
        mu[1] = oy + dl[1];
#pragma unroll
        for (int j = 2; j < 5; ++j) mu[j] = dl[j];
      }
      rs = clamp_sym2<T>(cs, T(eps_s));
      rc = clamp_sym3<T>(cc, T(eps_c));
      double* th = theta + (long long)k * kTheta;
#pragma unroll
      for (int j = 0; j < 5; ++j) th[j] = double(mu[j]);
#pragma unroll
      for (int j = 0; j < 3; ++j) th[5 + j] = double(cs[j]);
#pragma unroll
      for (int j = 0; j < 6; ++j) th[8 + j] = double(cc[j]);
      pack_gp<T>(mu, cs, cc, ox, oy, G);
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

__global__ void __launch_bounds__(kFinThreads) k_ll_reduce(const double* __restrict__ cell_ll, int n,
                                                           double* blk, unsigned* ticket, double* out) {
  block_ll_sum<double>(cell_ll, 1, n, blk, ticket, out);
}

// ---------------------------------------------------------------- launchers
static int ll_blocks(const Geom& g) { return (g.K + kFinThreads - 1) / kFinThreads; }

size_t finalize_workspace_doubles(const Geom& g) { return size_t(ll_blocks(g)) + 1; }

template <typename PT, bool SHIFT, int WPC, class Src>
static cudaError_t em_pass_impl(Src lab, const Geom& g, const float* gp, PT* partials,
                                cudaStream_t s) {
  constexpr int smem = em_smem_bytes<WPC>();
  static_assert(smem <= 227 * 1024, "shared memory");
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set && smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_em_pass<PT, SHIFT, WPC, Src>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  constexpr int cpb = kEmWarps / WPC;
  const int blocks = (g.ncells + cpb - 1) / cpb;
  k_em_pass<PT, SHIFT, WPC, Src><<<blocks, kEmWarps * 32, smem, s>>>(lab, g, gp, partials);
  return cudaGetLastError();
}

template <typename PT, bool SHIFT, class Src>
static cudaError_t em_pass_wpc(Src lab, const Geom& g, const float* gp, PT* partials, int wpc,
                               cudaStream_t s) {
  switch (wpc) {
    case 2: return em_pass_impl<PT, SHIFT, 2, Src>(lab, g, gp, partials, s);
    case 4: return em_pass_impl<PT, SHIFT, 4, Src>(lab, g, gp, partials, s);
    default: return em_pass_impl<PT, SHIFT, 1, Src>(lab, g, gp, partials, s);
  }
}

template <class Src>
cudaError_t launch_em_pass(Src lab, const Geom& g, const float* gp, void* partials, int precision,
                           int wpc, cudaStream_t s) {
  if (precision == 1)
    return em_pass_wpc<float, false, Src>(lab, g, gp, static_cast<float*>(partials), wpc, s);
  return em_pass_wpc<double, true, Src>(lab, g, gp, static_cast<double*>(partials), wpc, s);
}

template <class Src>
cudaError_t launch_label_pass(Src lab, const Geom& g, const float* gp, int32_t* labels,
                              double* cell_ll, cudaStream_t s) {
  const int blocks = (g.ncells + kEmWarps - 1) / kEmWarps;
  k_label_pass<Src><<<blocks, kEmWarps * 32, 0, s>>>(lab, g, gp, labels, cell_ll);
  return cudaGetLastError();
}

template cudaError_t launch_em_pass<LabPacked>(LabPacked, const Geom&, const float*, void*, int, int,
                                               cudaStream_t);
template cudaError_t launch_em_pass<LabPitched>(LabPitched, const Geom&, const float*, void*, int, int,
                                                cudaStream_t);
template cudaError_t launch_label_pass<LabPacked>(LabPacked, const Geom&, const float*, int32_t*, double*,
                                                  cudaStream_t);
template cudaError_t launch_label_pass<LabPitched>(LabPitched, const Geom&, const float*, int32_t*,
                                                   double*, cudaStream_t);

cudaError_t launch_finalize(const Geom& g, const void* partials, double* theta, float* gp,
                            double eps_s, double eps_c, double* llk_out, double* ws,
                            unsigned* ticket, unsigned long long* counters, int precision,
                            cudaStream_t s) {
  const int blocks = ll_blocks(g);
  if (precision == 1)
    k_finalize<float><<<blocks, kFinThreads, 0, s>>>(g, static_cast<const float*>(partials), theta, gp,
                                                     eps_s, eps_c, llk_out, ws, ticket, counters);
  else
    k_finalize<double><<<blocks, kFinThreads, 0, s>>>(g, static_cast<const double*>(partials), theta,
                                                      gp, eps_s, eps_c, llk_out, ws, ticket, counters);
  return cudaGetLastError();
}

cudaError_t launch_ll_reduce(const double* cell_ll, int n, double* out, double* ws, unsigned* ticket,
                             const Geom& g, cudaStream_t s) {
  k_ll_reduce<<<ll_blocks(g), kFinThreads, 0, s>>>(cell_ll, n, ws, ticket, out);
  return cudaGetLastError();
}

}  // namespace gmmsp
