// The learned initialiser (include/gmmsp_cnn.h): a small convolutional
// network that predicts, for every superpixel of a CIELAB image, the offset
// of its fitted mean from the Sec. III-C start and the logarithms of its
// fitted covariance diagonal.  It stands in for Algorithm 1, step 1, so that
// fewer EM iterations reach the same likelihood; the EM steps themselves are
// unchanged.  The paper has no such network.
//
// Kernels (activations and weights BF16, accumulation FP32 in tensor memory,
// every product on the tcgen05 tensor cores):
//   k_pix   x0 -> h1 -> h2 -> c0 fused: one block per group of cells (128
//           rows = 3 x 3 pixel patches), both 1 x 1 layers as 128 x 32 x 32
//           MMAs with the accumulators in TMEM, the average pooling in shared
//           memory.  Reads the CIELAB planes once and writes c0 (and, when
//           training, x0, h1 and h2 for the backward pass).
//   k_gemm  implicit-GEMM convolution in three modes: forward (rows =
//           positions, columns = output channels, K = taps x 32), data
//           gradient (rows = positions, columns = input channels, K = taps x
//           output channels, the ReLU mask of the layer input applied in the
//           epilogue) and weight gradient (rows = taps x 32 + 1, the extra
//           row of ones giving the bias gradient; columns = output channels;
//           K = positions, split over blocks and reduced in a fixed order).
//   k_pool_bwd, k_loss, k_wgrad_reduce, k_adam, k_targets, k_init_from_net.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_cnn.h"
#include "gmmsp_cnn_internal.cuh"
#include "gmmsp_internal.cuh"
#include "gmmsp_lab.cuh"
#include "gmmsp_math.cuh"
#include "gmmsp_tc.cuh"

namespace gmmsp {
namespace cnn {

constexpr int kC = 32;                     // channels of every hidden layer
constexpr int kOut = GMMSP_NET_CHANNELS;   // output channels of the last layer (16)
constexpr int kUsed = GMMSP_NET_OUTPUTS;   // outputs used per superpixel (10)
constexpr int kStageK = 32;                // K per shared-memory stage (two K = 16 MMAs)
constexpr uint32_t kWaitTries = 1u << 22;  // bound on every mbarrier wait
constexpr int kChunk = 2048;               // positions per weight-gradient block
constexpr int kLossBlocks = 128;

constexpr float kInScale = 0.02f;    // L, a, b -> about [-1, 1] (L shifted by 50)
constexpr int kStartCh = 29;         // c0 channels 29-31: the start pixel's scaled colour (not pooled)
constexpr float kColourUnit = 10.f;  // colour mean offsets in units of 10

// Flat parameter vector W1, b1, ..., W6, b6 with W[cout][taps * 32 + cin].
struct ParamLayout {
  int w[6], b[6], taps[6], cout[6];
  int total;
};
inline ParamLayout param_layout() {
  ParamLayout p{};
  const int taps[6] = {1, 1, 9, 9, 9, 9};
  const int cout[6] = {kC, kC, kC, kC, kC, kOut};
  int off = 0;
  for (int l = 0; l < 6; ++l) {
    p.taps[l] = taps[l];
    p.cout[l] = cout[l];
    p.w[l] = off;
    off += cout[l] * taps[l] * kC;
    p.b[l] = off;
    off += cout[l];
  }
  p.total = off;
  return p;
}

enum Mode : int { FWD = 0, DGRAD = 1, WGRAD = 2 };

// One convolution over a batch of B images of H x W positions (NHWC).
struct Layer {
  int B, H, W;
  int taps;                   // 1 or 9 (3 x 3, padding 1)
  int cout;                   // 32 or 16
  int relu;                   // forward: ReLU after the bias
  const __nv_bfloat16* x;     // layer input [B H W][32]
  const __nv_bfloat16* w;     // weights [cout][taps 32]
  const float* bias;          // [cout]
  __nv_bfloat16* y;           // forward output, BF16 [B H W][cout] ...
  float* y32;                 // ... or FP32 (the last layer)
  const __nv_bfloat16* gy;    // gradient of the layer output (pre-activation) [B H W][cout]
  const __nv_bfloat16* mask;  // data gradient: zero where mask <= 0 (or null)
  __nv_bfloat16* gx;          // data gradient output [B H W][32]
  float* wpart;               // weight-gradient partials [splits][taps 32 + 1][cout]
};

__device__ __forceinline__ int tap_dy(int t, int taps) { return taps == 1 ? 0 : t / 3 - 1; }
__device__ __forceinline__ int tap_dx(int t, int taps) { return taps == 1 ? 0 : t % 3 - 1; }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// 8 consecutive K-elements (k a multiple of 8) of the A row of position
// (img, y, x), forward and data-gradient modes.
template <int MODE>
__device__ __forceinline__ uint4 a_vec8(const Layer& L, bool row_ok, int img, int y, int x, int k, int kdim) {
  const uint4 z = make_uint4(0, 0, 0, 0);
  if (!row_ok || k >= kdim) return z;
  if (MODE == FWD) {
    const int t = k >> 5, c = k & 31;
    const int yy = y + tap_dy(t, L.taps), xx = x + tap_dx(t, L.taps);
    if (yy < 0 || yy >= L.H || xx < 0 || xx >= L.W) return z;
    return __ldg(reinterpret_cast<const uint4*>(L.x + (((long long)img * L.H + yy) * L.W + xx) * kC + c));
  } else {
    // gx[p] = sum_t W_t^T gy[p - d_t]
    const int t = k / L.cout, co = k - t * L.cout;
    const int yy = y - tap_dy(t, L.taps), xx = x - tap_dx(t, L.taps);
    if (yy < 0 || yy >= L.H || xx < 0 || xx >= L.W) return z;
    return __ldg(reinterpret_cast<const uint4*>(L.gy + (((long long)img * L.H + yy) * L.W + xx) * L.cout + co));
  }
}

// Implicit GEMM D[rows x N] = A[rows x K] B[N x K]^T: one 128-row tile per
// block of 128 threads, FP32 accumulator in TMEM (32 columns), K in stages of
// 32 gathered into shared memory (K-major, no swizzle).  Weight-gradient
// blocks (blockIdx.y) cover the positions [y chunk, (y + 1) chunk).
template <int MODE, int N>
__global__ void __launch_bounds__(128) k_gemm(Layer L, int rows, int kdim, int chunk, int* err) {
  __shared__ __align__(1024) unsigned char sA[128 * kStageK * 2];
  __shared__ __align__(1024) unsigned char sB[N * kStageK * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = blockIdx.x * 128 + tid;  // this thread's A row
  int k_begin = 0, k_end = kdim;
  if (MODE == WGRAD) {
    k_begin = blockIdx.y * chunk;
    k_end = min(k_begin + chunk, kdim);
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_sh, 32);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  // forward / data gradient: the row is a position
  int img = 0, y = 0, x = 0;
  const bool row_ok = r < rows;
  if (MODE != WGRAD && row_ok) {
    const int hw = L.H * L.W;
    img = r / hw;
    const int rem = r - img * hw;
    y = rem / L.W;
    x = rem - y * L.W;
  }
  // weight gradient: the row is (tap, input channel) or the bias row; the
  // stage's positions are walked incrementally from k_begin
  const int wt = r / kC, wc = r - (r / kC) * kC;
  int pimg = 0, py = 0, px = 0;
  if (MODE == WGRAD && k_begin < k_end) {
    const int hw = L.H * L.W;
    pimg = k_begin / hw;
    const int rem = k_begin - pimg * hw;
    py = rem / L.W;
    px = rem - py * L.W;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N);
  bool ok = true;
  uint32_t phase = 0;
  for (int k0 = k_begin; k0 < k_end && ok; k0 += kStageK) {
    if (MODE != WGRAD) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 v = a_vec8<MODE>(L, row_ok, img, y, x, k0 + 8 * j, k_end);
        *reinterpret_cast<uint4*>(sA + tc::tile_offset(tid, 8 * j, kStageK)) = v;
      }
      if (tid < N) {
        if (MODE == FWD) {
          // B row = output channel tid: 32 contiguous weights (K is a multiple of 32)
          const uint4* src = reinterpret_cast<const uint4*>(L.w + (long long)tid * L.taps * kC + k0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint4 v = tid < L.cout ? __ldg(src + j) : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4*>(sB + tc::tile_offset(tid, 8 * j, kStageK)) = v;
          }
        } else {
          // B row = input channel tid; column k = (tap, output channel)
          uint32_t u[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float e[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int k = k0 + 2 * j + h;
              e[h] = 0.f;
              if (k < k_end) {
                const int t = k / L.cout, co = k - t * L.cout;
                e[h] = __bfloat162float(L.w[(long long)co * L.taps * kC + t * kC + tid]);
              }
            }
            u[j] = pack2(e[0], e[1]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint4*>(sB + tc::tile_offset(tid, 8 * j, kStageK)) =
                make_uint4(u[4 * j], u[4 * j + 1], u[4 * j + 2], u[4 * j + 3]);
        }
      }
    } else {
      const int dy = tap_dy(wt, L.taps), dx = tap_dx(wt, L.taps);
      const bool is_w = wt < L.taps, is_b = r == L.taps * kC;
      const bool has_b = tid < N && tid < L.cout;
      float ea[32], eb[32];
      int qi = pimg, qy = py, qx = px;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        ea[j] = 0.f;
        eb[j] = 0.f;
        if (k0 + j < k_end) {
          if (is_b) {
            ea[j] = 1.f;
          } else if (is_w) {
            const int yy = qy + dy, xx = qx + dx;
            if (yy >= 0 && yy < L.H && xx >= 0 && xx < L.W)
              ea[j] = __bfloat162float(L.x[(((long long)qi * L.H + yy) * L.W + xx) * kC + wc]);
          }
          if (has_b) eb[j] = __bfloat162float(L.gy[(long long)(k0 + j) * L.cout + tid]);
        }
        if (++qx == L.W) {
          qx = 0;
          if (++qy == L.H) {
            qy = 0;
            ++qi;
          }
        }
      }
      pimg = qi;
      py = qy;
      px = qx;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        *reinterpret_cast<uint4*>(sA + tc::tile_offset(tid, 8 * j, kStageK)) =
            make_uint4(pack2(ea[8 * j], ea[8 * j + 1]), pack2(ea[8 * j + 2], ea[8 * j + 3]),
                       pack2(ea[8 * j + 4], ea[8 * j + 5]), pack2(ea[8 * j + 6], ea[8 * j + 7]));
        if (tid < N)
          *reinterpret_cast<uint4*>(sB + tc::tile_offset(tid, 8 * j, kStageK)) =
              make_uint4(pack2(eb[8 * j], eb[8 * j + 1]), pack2(eb[8 * j + 2], eb[8 * j + 3]),
                         pack2(eb[8 * j + 4], eb[8 * j + 5]), pack2(eb[8 * j + 6], eb[8 * j + 7]));
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kStageK / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, (kStageK / 8) * 128);
        const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, (kStageK / 8) * 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (k0 > k_begin || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&mbar);
    }
    // The stage buffers are refilled next: wait until the MMAs have read them.
    const bool w = tc::mbar_wait(&mbar, phase & 1u, kWaitTries);
    ok = __syncthreads_and(w) != 0;
    if (ok) ++phase;
  }
  tc::fence_after_sync();
  const int row = blockIdx.x * 128 + warp * 32 + lane;
  if (!ok) {
    // give the MMAs in flight one more bounded chance to land before TMEM is freed
    tc::mbar_wait(&mbar, phase & 1u, kWaitTries);
    if (tid == 0) atomicExch(err, 1);
  } else if (k_begin < k_end) {
    // Epilogue: warp w holds TMEM lanes (rows) 32 w .. 32 w + 31.
    float acc[N];
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[c0 + i] = v[i];
    }
    if (row < rows) {
      if (MODE == FWD) {
        if (L.y32) {
#pragma unroll
          for (int c = 0; c < N; ++c) L.y32[(long long)row * N + c] = acc[c] + __ldg(L.bias + c);
        } else {
          uint32_t u[N / 2];
#pragma unroll
          for (int c = 0; c < N; c += 2) {
            float a = acc[c] + __ldg(L.bias + c), b = acc[c + 1] + __ldg(L.bias + c + 1);
            if (L.relu) {
              a = fmaxf(a, 0.f);
              b = fmaxf(b, 0.f);
            }
            u[c / 2] = pack2(a, b);
          }
          uint4* dst = reinterpret_cast<uint4*>(L.y + (long long)row * N);
#pragma unroll
          for (int j = 0; j < N / 8; ++j) dst[j] = make_uint4(u[4 * j], u[4 * j + 1], u[4 * j + 2], u[4 * j + 3]);
        }
      } else if (MODE == DGRAD) {
        uint4 m[4] = {};
        if (L.mask) {
          const uint4* ms = reinterpret_cast<const uint4*>(L.mask + (long long)row * kC);
#pragma unroll
          for (int j = 0; j < 4; ++j) m[j] = ms[j];
        }
        const uint32_t* mw = reinterpret_cast<const uint32_t*>(m);
        uint32_t u[16];
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
          float a = acc[c], b = acc[c + 1];
          if (L.mask) {
            if (!(bf_lo(mw[c / 2]) > 0.f)) a = 0.f;
            if (!(bf_hi(mw[c / 2]) > 0.f)) b = 0.f;
          }
          u[c / 2] = pack2(a, b);
        }
        uint4* dst = reinterpret_cast<uint4*>(L.gx + (long long)row * kC);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_uint4(u[4 * j], u[4 * j + 1], u[4 * j + 2], u[4 * j + 3]);
      } else {
        float* out = L.wpart + ((long long)blockIdx.y * rows + row) * N;
#pragma unroll
        for (int c = 0; c < N; ++c) out[c] = acc[c];
      }
    }
  } else if (MODE == WGRAD && row < rows) {
    float* out = L.wpart + ((long long)blockIdx.y * rows + row) * N;
    for (int c = 0; c < N; ++c) out[c] = 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------------ k_pix
struct PixArgs {
  const float* lab;  // B images, each three planes of W H floats (L, a, b), consecutive
  // Converting mode (rgb non-null): the cells' pixels are read as sRGB from
  // the batch table's RGB8 rows and their CIELAB values written to lab_out
  // (planes as `lab`) on the way; `lab` is then unused.
  const BatchImage* rgb;
  float* lab_out;
  const float* srgb;  // 256 decoded sRGB code values (k_srgb_table)
  Rgb2LabConst k;
  int W, H, v, f, nx, ny;
  int cells;         // B n_x n_y
  int cpb;           // cells per block: floor(128 / f^2)
  const __nv_bfloat16* w1;
  const float* b1;
  const __nv_bfloat16* w2;
  const float* b2;
  __nv_bfloat16* c0;            // [cells][32]
  __nv_bfloat16 *x0, *h1, *h2;  // training: [blocks 128][32], or null
  int* err;
};

// Row r of block b is patch q = r mod f^2 of cell b cpb + r / f^2; the patch
// covers the pixels (k_x v + 3 (q mod f) + dx, k_y v + 3 (q / f) + dy),
// dx, dy in {0, 1, 2}; input channel (3 dy + dx) 3 + colour.  The inputs are
// gathered by patch rows: thread t takes patch (q mod f = t mod f, q / f =
// t / (cpb f)) of the block's cell (t mod (cpb f)) / f, so that a warp's
// loads run along image rows across the block's cells; the thread writes the
// patch's row of the A tile.  After the MMAs thread t owns row t.
//
// Shared memory: the A tile (8 KB) and both weight tiles (4 KB) while the
// MMAs run; the pooling buffer (128 rows of 16 BF16 pairs, 17 words apart)
// reuses the same bytes once the second MMA has completed.  Both layers
// accumulate into the same 32 TMEM columns (the second MMA is issued after
// every thread has read the first result).  In the converting mode each
// thread converts its patch's 9 pixels in registers (its inputs) and stores
// their CIELAB values to the planes.
constexpr int kPixMinBlocks = 8;
constexpr int kPixSmem = 128 * kC * 2 + 2 * kC * kC * 2;  // A + weight tiles (12 KB)
constexpr int kPoolLd = kC / 2 + 1;                       // words per pooling row
static_assert(128 * kPoolLd * 4 <= kPixSmem, "pooling buffer");

// The sRGB decoding table of the converting mode, once per network (the
// conversion kernels' own table code, so that both give the same bits).
__global__ void k_srgb_table(float* lin) { build_srgb_table(lin); }

__global__ void __launch_bounds__(128, kPixMinBlocks) k_pix(PixArgs a) {
  __shared__ __align__(1024) unsigned char smem[kPixSmem];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  unsigned char* sA = smem;
  unsigned char (*sW)[kC * kC * 2] = reinterpret_cast<unsigned char (*)[kC * kC * 2]>(smem + 128 * kC * 2);
  uint32_t (*sH)[kPoolLd] = reinterpret_cast<uint32_t (*)[kPoolLd]>(smem);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_sh, 32);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  const int ff = a.f * a.f;
  // row tid (after the MMAs)
  const int lc = tid / ff;
  const bool valid = lc < a.cpb && (long long)blockIdx.x * a.cpb + lc < a.cells;
  // the patch this thread gathers (patch-row order) and its row of the A tile
  const int prow = a.cpb * a.f;                  // patches per patch row of the block
  const int qy = tid / prow, qr = tid - qy * prow;
  const int lci = qr / a.f, qx = qr - lci * a.f;
  const bool pad = qy >= a.f;                    // tid >= cpb f^2: a zero row
  const int row_in = pad ? tid : lci * ff + qy * a.f + qx;
  const int cell = blockIdx.x * a.cpb + lci;  // < cells + cpb, an int
  const bool valid_in = !pad && cell < a.cells;
  uint32_t u[16];
  // the Sec. III-C start pixel (k_x v + v/2, k_y v + v/2) lies in patch (qs, qs) at (ds, ds)
  const int qs = (a.v / 2) / 3, ds = (a.v / 2) % 3;
  const bool start_row = valid_in && qy == qs && qx == qs;
  float zs[3] = {0.f, 0.f, 0.f};
  __shared__ float lin[256];  // converting mode: the sRGB table
  if (a.rgb) {
    lin[tid] = __ldg(a.srgb + tid);
    lin[tid + 128] = __ldg(a.srgb + tid + 128);
  }
  {
    float in[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) in[i] = 0.f;
    const int K = a.nx * a.ny;
    const int img = valid_in ? int(cell / K) : 0, k = valid_in ? int(cell - (long long)img * K) : 0;
    const int ky = k / a.nx, kx = k - ky * a.nx;
    const int px0 = kx * a.v + 3 * qx, py0 = ky * a.v + 3 * qy;
    if (a.rgb) {
      // all 27 code values first (independent loads), then the table, then
      // the conversion; each pixel's CIELAB values are stored from registers
      // A patch row is 9 consecutive bytes; they are read as the three aligned
      // 32-bit words that hold them.  The first word holds the row's first
      // byte and the last word its last, so no word reaches past the page of
      // a byte of the image (the bytes after the 9th are not used).
      uint8_t code[27];
      const BatchImage* im = a.rgb + img;
      if (valid_in) {
        const long long pitch = im->pitch;
        const uint8_t* S = static_cast<const uint8_t*>(im->image) + (long long)py0 * pitch + 3LL * px0;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const uintptr_t at = reinterpret_cast<uintptr_t>(S + dy * pitch);
          const uint32_t* w = reinterpret_cast<const uint32_t*>(at & ~uintptr_t(3));
          const uint32_t sh = uint32_t(at & 3) * 8;
          const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
          const uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            code[dy * 9 + j] = uint8_t(lo >> (8 * j));
            code[dy * 9 + 4 + j] = uint8_t(hi >> (8 * j));
          }
          code[dy * 9 + 8] = uint8_t(w2 >> sh);
        }
      }
      __syncthreads();  // the table
      const long long N = (long long)a.W * a.H;
      const long long p0 = (long long)py0 * a.W + px0;
      float* T = a.lab_out + 3 * (valid_in ? im->pix_off : 0) + p0;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          if (!valid_in) continue;
          const int c = (dy * 3 + dx) * 3;
          float L, A, B;
          srgb8_to_lab(a.k, lin, code + c, L, A, B);
          float* t = T + (long long)dy * a.W + dx;
          if (GMMSP_IN_BOUNDS((t - a.lab_out) + 2 * N, (long long)(a.cells / K) * 3 * N, BND_PIXEL_Y)) {
            t[0] = L;
            t[N] = A;
            t[2 * N] = B;
          }
          in[c + 0] = fmaf(L, kInScale, -1.f);
          in[c + 1] = A * kInScale;
          in[c + 2] = B * kInScale;
          if (start_row && dy == ds && dx == ds) {
            zs[0] = in[c + 0];
            zs[1] = in[c + 1];
            zs[2] = in[c + 2];
          }
        }
    } else if (valid_in) {
      const long long N = (long long)a.W * a.H;
      const float* P = a.lab + (long long)img * 3 * N;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const long long i = (long long)(py0 + dy) * a.W + (px0 + dx);
          const int c = (dy * 3 + dx) * 3;
          in[c + 0] = fmaf(__ldg(P + i), kInScale, -1.f);
          in[c + 1] = __ldg(P + N + i) * kInScale;
          in[c + 2] = __ldg(P + 2 * N + i) * kInScale;
          if (start_row && dy == ds && dx == ds) {
            zs[0] = in[c + 0];
            zs[1] = in[c + 1];
            zs[2] = in[c + 2];
          }
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) u[i] = pack2(in[2 * i], in[2 * i + 1]);
  }
  if (tid < 64) {
    const uint4* src = reinterpret_cast<const uint4*>((tid < 32 ? a.w1 : a.w2) + (tid & 31) * kC);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<uint4*>(sW[tid >> 5] + tc::tile_offset(tid & 31, 8 * j, kC)) = __ldg(src + j);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint4 v4 = make_uint4(u[4 * j], u[4 * j + 1], u[4 * j + 2], u[4 * j + 3]);
    *reinterpret_cast<uint4*>(sA + tc::tile_offset(row_in, 8 * j, kC)) = v4;
    if (a.x0) reinterpret_cast<uint4*>(a.x0 + ((long long)blockIdx.x * 128 + row_in) * kC)[j] = v4;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kC);
  const uint32_t a0 = tc::smem_u32(sA);
  bool ok = true;
  int layer = 0;
  for (; layer < 2; ++layer) {
    if (tid == 0) {
      const uint32_t b0 = tc::smem_u32(sW[layer]);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc(a0 + kk * 256, 128, 512),
                     tc::smem_desc(b0 + kk * 256, 128, 512), idesc, kk > 0 ? 1u : 0u);
      tc::mma_commit(&mbar);
    }
    const bool w = tc::mbar_wait(&mbar, uint32_t(layer), kWaitTries);
    ok = __syncthreads_and(w) != 0;
    tc::fence_after_sync();
    if (!ok) break;
    float acc[32];
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[c0 + i] = v[i];
    }
    const float* bias = layer == 0 ? a.b1 : a.b2;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float e0 = valid ? fmaxf(acc[2 * i] + __ldg(bias + 2 * i), 0.f) : 0.f;
      const float e1 = valid ? fmaxf(acc[2 * i + 1] + __ldg(bias + 2 * i + 1), 0.f) : 0.f;
      u[i] = pack2(e0, e1);
    }
    __nv_bfloat16* store = layer == 0 ? a.h1 : a.h2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 v4 = make_uint4(u[4 * j], u[4 * j + 1], u[4 * j + 2], u[4 * j + 3]);
      if (layer == 0) *reinterpret_cast<uint4*>(sA + tc::tile_offset(tid, 8 * j, kC)) = v4;
      if (store) reinterpret_cast<uint4*>(store + ((long long)blockIdx.x * 128 + tid) * kC)[j] = v4;
    }
    if (layer == 0) {
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    } else {
      __syncthreads();  // every thread is past the tiles before they are overwritten
#pragma unroll
      for (int i = 0; i < 16; ++i) sH[tid][i] = u[i];
      __syncthreads();
      // pooling: channel pair (2 cp, 2 cp + 1) of cell l, summed over its f^2 rows in order
      for (int idx = tid; idx < a.cpb * (kC / 2); idx += 128) {
        const int l = idx >> 4, cp = idx & 15;
        const long long cl = (long long)blockIdx.x * a.cpb + l;
        if (cl >= a.cells || 2 * cp >= kStartCh) continue;
        float s0 = 0.f, s1 = 0.f;
        for (int p = 0; p < ff; ++p) {
          const uint32_t w = sH[l * ff + p][cp];
          s0 += bf_lo(w);
          s1 += bf_hi(w);
        }
        a.c0[cl * kC + 2 * cp] = __float2bfloat16(s0 / float(ff));
        if (2 * cp + 1 < kStartCh) a.c0[cl * kC + 2 * cp + 1] = __float2bfloat16(s1 / float(ff));
      }
      if (start_row) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.c0[(long long)cell * kC + kStartCh + c] = __float2bfloat16(zs[c]);
      }
    }
  }
  if (!ok) {
    tc::mbar_wait(&mbar, uint32_t(layer & 1), kWaitTries);
    if (tid == 0) atomicExch(a.err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------ elementwise
// Gradient of the pre-activation of h2 from the gradient of c0 (average
// pooling, then the ReLU of h2): g[row] = g_c0[cell(row)] / f^2 where h2 > 0,
// for the pooled channels (channels kStartCh.. are the start pixel's inputs).
__global__ void k_pool_bwd(const __nv_bfloat16* __restrict__ gc0, const __nv_bfloat16* __restrict__ h2,
                           long long nrows, int cpb, int ff, long long cells, __nv_bfloat16* __restrict__ g) {
  const float inv = 1.f / float(ff);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrows * kC;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i >> 5;
    const int ch = int(i & 31);
    const long long blk = row >> 7;
    const int lc = int(row & 127) / ff;
    const long long cell = blk * cpb + lc;
    float v = 0.f;
    if (lc < cpb && cell < cells && ch < kStartCh && __bfloat162float(h2[i]) > 0.f)
      v = __bfloat162float(gc0[cell * kC + ch]) * inv;
    g[i] = __float2bfloat16(v);
  }
}

// Mean squared error over the used outputs: gradient (BF16) into g, per-block
// sums of squares (FP64) into lpart.
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ out, const float* __restrict__ target,
                                              long long cells, __nv_bfloat16* __restrict__ g,
                                              double* __restrict__ lpart) {
  __shared__ double red[256];
  double s = 0.0;
  const float scale = float(2.0 / double(cells * kUsed));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells * kOut;
       i += (long long)gridDim.x * blockDim.x) {
    const long long cell = i / kOut;
    const int j = int(i - cell * kOut);
    float gv = 0.f;
    if (j < kUsed) {
      const float d = out[i] - target[cell * kUsed + j];
      s += double(d) * double(d);
      gv = scale * d;
    }
    g[i] = __float2bfloat16(gv);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// Sum of the weight-gradient partials over the splits (fixed order): row
// t 32 + c -> gw[cout][t 32 + c], the last row -> gb[cout].
__global__ void k_wgrad_reduce(const float* __restrict__ part, int splits, int rows, int cout,
                               float* __restrict__ gw, float* __restrict__ gb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cout; i += gridDim.x * blockDim.x) {
    const int r = i / cout, c = i - r * cout;
    float s = 0.f;
    for (int sp = 0; sp < splits; ++sp) s += part[((long long)sp * rows + r) * cout + c];
    if (r == rows - 1) gb[c] = s;
    else gw[(long long)c * (rows - 1) + r] = s;
  }
}

// Adam (Kingma and Ba, 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// Targets from fitted parameters of B images of geometry g (theta and the
// CIELAB planes laid out image after image); units as the network outputs.
__global__ void k_targets(const double* __restrict__ theta, const float* __restrict__ lab, int B, Geom g,
                          double lambda_c, float* __restrict__ t) {
  const long long total = (long long)B * g.K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int img = int(i / g.K), k = int(i - (long long)img * g.K);
    const int kx = k % g.nx, ky = k / g.nx;
    const int x = kx * g.v + g.v / 2, y = ky * g.v + g.v / 2;
    const long long N = (long long)g.W * g.H, j = (long long)y * g.W + x;
    const float* P = lab + (long long)img * 3 * N;
    const double* th = theta + i * kTheta;
    float* o = t + i * kUsed;
    const double v = g.v, l2 = lambda_c * lambda_c;
    o[0] = float((th[0] - x) / v);
    o[1] = float((th[1] - y) / v);
    o[2] = float((th[2] - double(P[j])) / kColourUnit);
    o[3] = float((th[3] - double(P[N + j])) / kColourUnit);
    o[4] = float((th[4] - double(P[2 * N + j])) / kColourUnit);
    o[5] = float(log(th[5] / (v * v)));
    o[6] = float(log(th[7] / (v * v)));
    o[7] = float(log(th[8] / l2));
    o[8] = float(log(th[11] / l2));
    o[9] = float(log(th[13] / l2));
  }
}

// theta_0 from the network outputs (the inverse of the target map): spatial
// mean clipped to the three cells around the seed's own, [(k_x - 1) v,
// (k_x + 2) v] x [(k_y - 1) v, (k_y + 2) v] (the span of Eq. Ik's window
// without its clamp to the image), axis-aligned covariances with
// the diagonal (their eigenvalues) floored at eps (Eq. mlams, mlamc); then
// the packed E-step coefficients.  Superpixel i reads its 5 mean offsets at
// dmu + i ds and its 5 log-eigenvalues at logeig + i ls (the network's output
// rows: ds = ls = 16; a caller's arrays: 5).
__global__ void k_init_from_net(const float* __restrict__ dmu, int ds, const float* __restrict__ logeig, int ls,
                                const float* __restrict__ lab, int B, Geom g, double lambda_c, double eps_s,
                                double eps_c, double* __restrict__ theta, float* __restrict__ gp,
                                unsigned long long* __restrict__ counters) {
  const long long total = (long long)B * g.K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int img = int(i / g.K), k = int(i - (long long)img * g.K);
    const int kx = k % g.nx, ky = k / g.nx;
    const int x = kx * g.v + g.v / 2, y = ky * g.v + g.v / 2;
    const long long N = (long long)g.W * g.H, j = (long long)y * g.W + x;
    const float* P = lab + (long long)img * 3 * N;
    float o[10];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      o[q] = dmu[i * ds + q];
      o[5 + q] = logeig[i * ls + q];
    }
    const double v = g.v, l2 = lambda_c * lambda_c;
    double mu[5] = {x + v * widen(o[0]), y + v * widen(o[1]), widen(P[j]) + kColourUnit * widen(o[2]),
                    widen(P[N + j]) + kColourUnit * widen(o[3]),
                    widen(P[2 * N + j]) + kColourUnit * widen(o[4])};
    mu[0] = fmin(fmax(mu[0], double(kx - 1) * v), double(kx + 2) * v);
    mu[1] = fmin(fmax(mu[1], double(ky - 1) * v), double(ky + 2) * v);
    const float lo = -10.f, hi = 10.f;
    const double cs[3] = {fmax(v * v * exp(widen(fminf(fmaxf(o[5], lo), hi))), eps_s), 0.0,
                          fmax(v * v * exp(widen(fminf(fmaxf(o[6], lo), hi))), eps_s)};
    const double cc[6] = {fmax(l2 * exp(widen(fminf(fmaxf(o[7], lo), hi))), eps_c), 0.0, 0.0,
                          fmax(l2 * exp(widen(fminf(fmaxf(o[8], lo), hi))), eps_c), 0.0,
                          fmax(l2 * exp(widen(fminf(fmaxf(o[9], lo), hi))), eps_c)};
    double* th = theta + i * kTheta;
    bool fin = true;
    for (int q = 0; q < 5; ++q) {
      th[q] = mu[q];
      fin = fin && isfinite(mu[q]);
    }
    for (int q = 0; q < 3; ++q) th[5 + q] = cs[q];
    for (int q = 0; q < 6; ++q) th[8 + q] = cc[q];
    th[14] = th[15] = 0.0;
    fin = pack_gp<double>(mu, cs, cc, double(kx * g.v), double(ky * g.v), gp + i * kGP) && fin;
    if (!fin) atomicAdd(counters + CNT_NONFINITE, 1ull);
  }
}

// Self-test of the bounded waits: allocates TMEM like the network kernels,
// waits on an mbarrier that nothing arrives on for max_tries polls, waits
// once more (bounded), frees the TMEM and records that it gave up.
__global__ void __launch_bounds__(128) k_wait_selftest(uint32_t max_tries, int* gave_up) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_sh, 32);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, max_tries)) != 0;
  if (!ok) {
    tc::mbar_wait(&mbar, 0, max_tries);
    if (tid == 0) atomicExch(gave_up, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  b = std::min<long long>(b, 152LL * 16);
  return int(std::max<long long>(b, 1));
}

}  // namespace cnn

cudaError_t bounds_take_cnn(unsigned long long* word) {
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

}  // namespace gmmsp

using gmmsp::BatchImage;
using gmmsp::Geom;
using gmmsp::rgb2lab_const;
using namespace gmmsp::cnn;

// --------------------------------------------------------------- the object
struct gmmsp_net_s {
  int v = 0, f = 0, cpb = 0;
  cudaStream_t stream = nullptr;
  ParamLayout pl{};
  void* pslab = nullptr;  // parameters, Adam state, gradients, error word
  float *w32 = nullptr, *m = nullptr, *vv = nullptr, *grad = nullptr;
  __nv_bfloat16* wbf = nullptr;
  int* err = nullptr;
  float* srgb = nullptr;  // the converting mode's sRGB table
  long long adam_t = 0;
  // workspace (grown on demand, never during stream capture)
  void* wslab = nullptr;
  long long cap_cells = 0;
  bool cap_train = false;
  long long generation = 0;
  __nv_bfloat16* c[4] = {};
  __nv_bfloat16 *x0 = nullptr, *h1 = nullptr, *h2 = nullptr, *gp0 = nullptr, *gp1 = nullptr, *gout = nullptr;
  __nv_bfloat16* gc[2] = {};
  float *out = nullptr, *wpart = nullptr;
  double* lpart = nullptr;
  long long last_cells = 0;  // superpixels of the last forward pass
  std::string msg;
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

gmmsp_status nfail(gmmsp_net n, gmmsp_status s, const std::string& m) {
  if (n) n->msg = m;
  return s;
}

#define GN_CHECK(n, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return nfail((n), e_ == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA, \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

long long nblocks_of(gmmsp_net n, long long cells) { return (cells + n->cpb - 1) / n->cpb; }

// The EM seed grid of a W x H image at the network's spacing (Eq. nxyK).
bool net_geom(gmmsp_net n, int W, int H, Geom* g) {
  if (W < n->v || H < n->v) return false;
  g->W = W; g->H = H; g->v = n->v;
  g->nx = W / n->v; g->ny = H / n->v;
  g->K = g->nx * g->ny;
  g->ncx = (W + n->v - 1) / n->v;
  g->ncy = (H + n->v - 1) / n->v;
  g->ncells = g->ncx * g->ncy;
  return true;
}

// Largest batch (in superpixels) the kernels index with 32-bit rows.
bool cells_fit(gmmsp_net n, long long cells) { return nblocks_of(n, cells) * 128 <= (1LL << 30); }

gmmsp_status reserve(gmmsp_net n, long long cells, bool train) {
  if (cells <= n->cap_cells && (!train || n->cap_train)) return GMMSP_OK;
  cells = std::max(cells, n->cap_cells);
  train = train || n->cap_train;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(n->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return nfail(n, GMMSP_E_STATE, "network workspace must be reserved before stream capture");
  const long long nrows = nblocks_of(n, cells) * 128;
  const long long splits_pix = (nrows + kChunk - 1) / kChunk;
  const long long splits_cell = (cells + kChunk - 1) / kChunk;
  const size_t wpart = size_t(std::max(splits_pix * (kC + 1), splits_cell * (9 * kC + 1))) * kC * sizeof(float);
  const size_t act = up256(size_t(cells) * kC * 2);
  const size_t pix = up256(size_t(nrows) * kC * 2);
  size_t off = 0;
  const size_t o_c = off;   off += 4 * act;
  const size_t o_out = off; off += up256(size_t(cells) * kOut * sizeof(float));
  size_t o_x0 = 0, o_gp0 = 0, o_gout = 0, o_gc = 0, o_wp = 0, o_lp = 0;
  if (train) {
    o_x0 = off;   off += 3 * pix;  // x0, h1, h2
    o_gp0 = off;  off += 2 * pix;  // gp0, gp1
    o_gout = off; off += up256(size_t(cells) * kOut * 2);
    o_gc = off;   off += 2 * act;
    o_wp = off;   off += up256(wpart);
    o_lp = off;   off += up256(kLossBlocks * sizeof(double));
  }
  if (n->wslab) {
    GN_CHECK(n, cudaStreamSynchronize(n->stream));
    cudaFree(n->wslab);
    n->wslab = nullptr;
    n->cap_cells = 0;
    n->cap_train = false;
  }
  void* slab = nullptr;
  GN_CHECK(n, cudaMalloc(&slab, off));
  ++n->generation;
  char* b = static_cast<char*>(slab);
  n->wslab = slab;
  for (int i = 0; i < 4; ++i) n->c[i] = reinterpret_cast<__nv_bfloat16*>(b + o_c + i * act);
  n->out = reinterpret_cast<float*>(b + o_out);
  if (train) {
    n->x0 = reinterpret_cast<__nv_bfloat16*>(b + o_x0);
    n->h1 = reinterpret_cast<__nv_bfloat16*>(b + o_x0 + pix);
    n->h2 = reinterpret_cast<__nv_bfloat16*>(b + o_x0 + 2 * pix);
    n->gp0 = reinterpret_cast<__nv_bfloat16*>(b + o_gp0);
    n->gp1 = reinterpret_cast<__nv_bfloat16*>(b + o_gp0 + pix);
    n->gout = reinterpret_cast<__nv_bfloat16*>(b + o_gout);
    n->gc[0] = reinterpret_cast<__nv_bfloat16*>(b + o_gc);
    n->gc[1] = reinterpret_cast<__nv_bfloat16*>(b + o_gc + act);
    n->wpart = reinterpret_cast<float*>(b + o_wp);
    n->lpart = reinterpret_cast<double*>(b + o_lp);
  } else {
    n->x0 = n->h1 = n->h2 = n->gp0 = n->gp1 = n->gout = n->gc[0] = n->gc[1] = nullptr;
    n->wpart = nullptr;
    n->lpart = nullptr;
  }
  n->cap_cells = cells;
  n->cap_train = train;
  return GMMSP_OK;
}

Layer cell_layer(gmmsp_net n, int B, const Geom& g, int l) {
  Layer L{};
  L.B = B;
  L.H = g.ny;
  L.W = g.nx;
  L.taps = n->pl.taps[l];
  L.cout = n->pl.cout[l];
  L.relu = l < 5;
  L.w = n->wbf + n->pl.w[l];
  L.bias = n->w32 + n->pl.b[l];
  return L;
}

// Forward pass; out receives [B K][16] FP32.  Training also stores x0, h1, h2.
// With rgb non-null the first kernel reads the cells' pixels as RGB8 through
// the batch table and writes their CIELAB values to lab_out.
gmmsp_status enqueue_forward(gmmsp_net n, const float* lab, int B, const Geom& g, float* out, bool train,
                             cudaStream_t s, const BatchImage* rgb = nullptr, float* lab_out = nullptr) {
  const long long cells = (long long)B * g.K;
  n->last_cells = cells;
  PixArgs a{};
  a.lab = lab;
  a.rgb = rgb;
  a.lab_out = lab_out;
  a.srgb = n->srgb;
  if (rgb) a.k = rgb2lab_const();
  a.W = g.W; a.H = g.H; a.v = g.v; a.f = n->f; a.nx = g.nx; a.ny = g.ny;
  a.cells = int(cells);
  a.cpb = n->cpb;
  a.w1 = n->wbf + n->pl.w[0];
  a.b1 = n->w32 + n->pl.b[0];
  a.w2 = n->wbf + n->pl.w[1];
  a.b2 = n->w32 + n->pl.b[1];
  a.c0 = n->c[0];
  a.x0 = train ? n->x0 : nullptr;
  a.h1 = train ? n->h1 : nullptr;
  a.h2 = train ? n->h2 : nullptr;
  a.err = n->err;
  k_pix<<<unsigned(nblocks_of(n, cells)), 128, 0, s>>>(a);
  GN_CHECK(n, cudaGetLastError());
  const int rows = int(cells);
  const unsigned tiles = unsigned((rows + 127) / 128);
  for (int l = 2; l < 6; ++l) {
    Layer L = cell_layer(n, B, g, l);
    L.x = n->c[l - 2];
    const int kdim = L.taps * kC;
    if (l < 5) {
      L.y = n->c[l - 1];
      k_gemm<FWD, 32><<<tiles, 128, 0, s>>>(L, rows, kdim, 0, n->err);
    } else {
      L.y32 = out;
      k_gemm<FWD, 16><<<tiles, 128, 0, s>>>(L, rows, kdim, 0, n->err);
    }
    GN_CHECK(n, cudaGetLastError());
  }
  return GMMSP_OK;
}

// Weight and bias gradient of layer l from its input L.x and the gradient
// L.gy of its pre-activation output, over `positions` positions.
gmmsp_status enqueue_wgrad(gmmsp_net n, Layer L, int l, int positions, cudaStream_t s) {
  const int rows = L.taps * kC + 1;
  const unsigned tiles = unsigned((rows + 127) / 128);
  const unsigned splits = unsigned((positions + kChunk - 1) / kChunk);
  L.wpart = n->wpart;
  if (L.cout == kC)
    k_gemm<WGRAD, 32><<<dim3(tiles, splits), 128, 0, s>>>(L, rows, positions, kChunk, n->err);
  else
    k_gemm<WGRAD, 16><<<dim3(tiles, splits), 128, 0, s>>>(L, rows, positions, kChunk, n->err);
  GN_CHECK(n, cudaGetLastError());
  k_wgrad_reduce<<<grid_for(rows * L.cout, 256), 256, 0, s>>>(n->wpart, int(splits), rows, L.cout,
                                                               n->grad + n->pl.w[l], n->grad + n->pl.b[l]);
  GN_CHECK(n, cudaGetLastError());
  return GMMSP_OK;
}

// Forward, loss, and the gradient of every parameter into n->grad.
gmmsp_status enqueue_grad(gmmsp_net n, const float* lab, int B, const Geom& g, const float* target,
                          cudaStream_t s) {
  gmmsp_status st = enqueue_forward(n, lab, B, g, n->out, true, s);
  if (st != GMMSP_OK) return st;
  const long long cells = (long long)B * g.K;
  const int rows = int(cells);
  const unsigned tiles = unsigned((rows + 127) / 128);
  k_loss<<<kLossBlocks, 256, 0, s>>>(n->out, target, cells, n->gout, n->lpart);
  GN_CHECK(n, cudaGetLastError());
  // the 3 x 3 layers, last to first
  const __nv_bfloat16* gy = n->gout;
  for (int l = 5; l >= 2; --l) {
    Layer L = cell_layer(n, B, g, l);
    L.x = n->c[l - 2];
    L.gy = gy;
    st = enqueue_wgrad(n, L, l, rows, s);
    if (st != GMMSP_OK) return st;
    L.gx = n->gc[l & 1];
    L.mask = l > 2 ? n->c[l - 2] : nullptr;  // c0 is a pooled value with no ReLU of its own
    k_gemm<DGRAD, 32><<<tiles, 128, 0, s>>>(L, rows, L.taps * L.cout, 0, n->err);
    GN_CHECK(n, cudaGetLastError());
    gy = L.gx;
  }
  // pooling and the ReLU of h2, then the two 1 x 1 layers over the patch rows
  const long long nrows = nblocks_of(n, cells) * 128;
  k_pool_bwd<<<grid_for(nrows * kC, 256), 256, 0, s>>>(gy, n->h2, nrows, n->cpb, n->f * n->f, cells, n->gp0);
  GN_CHECK(n, cudaGetLastError());
  Layer L2{};
  L2.B = 1; L2.H = 1; L2.W = int(nrows);
  L2.taps = 1; L2.cout = kC;
  L2.w = n->wbf + n->pl.w[1];
  L2.x = n->h1;
  L2.gy = n->gp0;
  st = enqueue_wgrad(n, L2, 1, int(nrows), s);
  if (st != GMMSP_OK) return st;
  L2.gx = n->gp1;
  L2.mask = n->h1;
  k_gemm<DGRAD, 32><<<unsigned(nrows / 128), 128, 0, s>>>(L2, int(nrows), kC, 0, n->err);
  GN_CHECK(n, cudaGetLastError());
  Layer L1 = L2;
  L1.w = n->wbf + n->pl.w[0];
  L1.x = n->x0;
  L1.gy = n->gp1;
  L1.gx = nullptr;
  L1.mask = nullptr;
  return enqueue_wgrad(n, L1, 0, int(nrows), s);
}

gmmsp_status check_err(gmmsp_net n) {
  int e = 0;
  GN_CHECK(n, cudaMemcpyAsync(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  GN_CHECK(n, cudaStreamSynchronize(n->stream));
  if (e) return nfail(n, GMMSP_E_TIMEOUT, "a tensor-core kernel gave up waiting on its MMA barrier");
  return GMMSP_OK;
}

gmmsp_status loss_to_host(gmmsp_net n, long long cells, double* loss_host) {
  double lp[kLossBlocks];
  GN_CHECK(n, cudaMemcpyAsync(lp, n->lpart, sizeof(lp), cudaMemcpyDeviceToHost, n->stream));
  const gmmsp_status st = check_err(n);
  if (st != GMMSP_OK) return st;
  double s = 0.0;
  for (int i = 0; i < kLossBlocks; ++i) s += lp[i];
  *loss_host = s / double(cells * kUsed);
  return GMMSP_OK;
}

}  // namespace

// ------------------------------------------------ library-internal entry points
namespace gmmsp {

gmmsp_status net_reserve(gmmsp_net n, int B, const Geom& g, std::string* why) {
  if (!n) return GMMSP_E_INVALID;
  if (g.v != n->v) {
    if (why) *why = "the network's spacing differs from the context's";
    return GMMSP_E_INVALID;
  }
  if (!cells_fit(n, (long long)B * g.K)) {
    if (why) *why = "batch too large for the network";
    return GMMSP_E_INVALID;
  }
  const gmmsp_status st = reserve(n, (long long)B * g.K, false);
  if (st != GMMSP_OK && why) *why = n->msg;
  return st;
}

long long net_generation(gmmsp_net n) { return n ? n->generation : -1; }

cudaError_t net_enqueue_init(gmmsp_net n, float* lab, const BatchImage* rgb, int B, const Geom& g,
                             double lambda_c, double eps_s, double eps_c, double* theta, float* gp,
                             unsigned long long* counters, cudaStream_t s) {
  if ((long long)B * g.K > n->cap_cells) return cudaErrorInvalidValue;
  if (enqueue_forward(n, lab, B, g, n->out, false, s, rgb, rgb ? lab : nullptr) != GMMSP_OK)
    return cudaErrorLaunchFailure;
  return launch_init_from_outputs(n->out, kOut, n->out + 5, kOut, lab, B, g, lambda_c, eps_s, eps_c, theta, gp,
                                  counters, s);
}

cudaError_t launch_init_from_outputs(const float* dmu, int ds, const float* logeig, int ls, const float* lab, int B,
                                     const Geom& g, double lambda_c, double eps_s, double eps_c, double* theta,
                                     float* gp, unsigned long long* counters, cudaStream_t s) {
  const long long total = (long long)B * g.K;
  k_init_from_net<<<grid_for(total, 128), 128, 0, s>>>(dmu, ds, logeig, ls, lab, B, g, lambda_c, eps_s, eps_c,
                                                       theta, gp, counters);
  return cudaGetLastError();
}

cudaError_t launch_targets(const double* theta, const float* lab, int B, const Geom& g, double lambda_c,
                           float* target, cudaStream_t s) {
  const long long total = (long long)B * g.K;
  k_targets<<<grid_for(total, 128), 128, 0, s>>>(theta, lab, B, g, lambda_c, target);
  return cudaGetLastError();
}

}  // namespace gmmsp

// --------------------------------------------------------------------- C ABI
extern "C" {

long long gmmsp_net_param_count(void) { return param_layout().total; }

gmmsp_status gmmsp_net_create(gmmsp_net* out, int spacing, void* stream) {
  if (!out) return GMMSP_E_INVALID;
  *out = nullptr;
  if (spacing < 3 || spacing > 33 || spacing % 3 != 0) return GMMSP_E_INVALID;
  gmmsp_net n = new (std::nothrow) gmmsp_net_s();
  if (!n) return GMMSP_E_NOMEM;
  n->v = spacing;
  n->f = spacing / 3;
  n->cpb = 128 / (n->f * n->f);
  n->stream = static_cast<cudaStream_t>(stream);
  n->pl = param_layout();
  const size_t np = size_t(n->pl.total);
  size_t off = 0;
  const size_t o_w = off; off += up256(np * 4);
  const size_t o_m = off; off += up256(np * 4);
  const size_t o_v = off; off += up256(np * 4);
  const size_t o_g = off; off += up256(np * 4);
  const size_t o_b = off; off += up256(np * 2);
  const size_t o_e = off; off += 256;
  const size_t o_t = off; off += 256 * 4;
  const char* inj = getenv("GMMSP_FAIL_ALLOC");
  cudaError_t e = (inj && inj[0] == '1') ? cudaErrorMemoryAllocation : cudaMalloc(&n->pslab, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(n->pslab);
  n->w32 = reinterpret_cast<float*>(b + o_w);
  n->m = reinterpret_cast<float*>(b + o_m);
  n->vv = reinterpret_cast<float*>(b + o_v);
  n->grad = reinterpret_cast<float*>(b + o_g);
  n->wbf = reinterpret_cast<__nv_bfloat16*>(b + o_b);
  n->err = reinterpret_cast<int*>(b + o_e);
  n->srgb = reinterpret_cast<float*>(b + o_t);
  e = cudaMemsetAsync(n->pslab, 0, off, n->stream);
  if (e == cudaSuccess) {
    k_srgb_table<<<1, 256, 0, n->stream>>>(n->srgb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    cudaFree(n->pslab);
    delete n;
    return GMMSP_E_CUDA;
  }
  *out = n;
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_set_weights(gmmsp_net n, const float* host, long long count) {
  if (!n) return GMMSP_E_INVALID;
  if (!host || count != n->pl.total) return nfail(n, GMMSP_E_INVALID, "weight count mismatch");
  for (long long i = 0; i < count; ++i)
    if (!isfinite(host[i])) return nfail(n, GMMSP_E_INVALID, "non-finite weight");
  const size_t bytes = size_t(count) * 4;
  GN_CHECK(n, cudaMemcpyAsync(n->w32, host, bytes, cudaMemcpyHostToDevice, n->stream));
  GN_CHECK(n, cudaMemsetAsync(n->m, 0, bytes, n->stream));
  GN_CHECK(n, cudaMemsetAsync(n->vv, 0, bytes, n->stream));
  k_to_bf16<<<grid_for(count, 256), 256, 0, n->stream>>>(n->w32, n->wbf, int(count));
  GN_CHECK(n, cudaGetLastError());
  GN_CHECK(n, cudaStreamSynchronize(n->stream));
  n->adam_t = 0;
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_get_weights(gmmsp_net n, float* host, long long count) {
  if (!n) return GMMSP_E_INVALID;
  if (!host || count != n->pl.total) return nfail(n, GMMSP_E_INVALID, "weight count mismatch");
  GN_CHECK(n, cudaMemcpyAsync(host, n->w32, size_t(count) * 4, cudaMemcpyDeviceToHost, n->stream));
  GN_CHECK(n, cudaStreamSynchronize(n->stream));
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_get_adam(gmmsp_net n, float* m_host, float* v_host, long long count, long long* step) {
  if (!n) return GMMSP_E_INVALID;
  if (!m_host || !v_host || !step || count != n->pl.total) return nfail(n, GMMSP_E_INVALID, "bad arguments");
  GN_CHECK(n, cudaMemcpyAsync(m_host, n->m, size_t(count) * 4, cudaMemcpyDeviceToHost, n->stream));
  GN_CHECK(n, cudaMemcpyAsync(v_host, n->vv, size_t(count) * 4, cudaMemcpyDeviceToHost, n->stream));
  GN_CHECK(n, cudaStreamSynchronize(n->stream));
  *step = n->adam_t;
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_set_adam(gmmsp_net n, const float* m_host, const float* v_host, long long count,
                                long long step) {
  if (!n) return GMMSP_E_INVALID;
  if (!m_host || !v_host || count != n->pl.total || step < 0) return nfail(n, GMMSP_E_INVALID, "bad arguments");
  for (long long i = 0; i < count; ++i)
    if (!isfinite(m_host[i]) || !(v_host[i] >= 0.f) || !isfinite(v_host[i]))
      return nfail(n, GMMSP_E_INVALID, "non-finite or negative optimiser state");
  GN_CHECK(n, cudaMemcpyAsync(n->m, m_host, size_t(count) * 4, cudaMemcpyHostToDevice, n->stream));
  GN_CHECK(n, cudaMemcpyAsync(n->vv, v_host, size_t(count) * 4, cudaMemcpyHostToDevice, n->stream));
  GN_CHECK(n, cudaStreamSynchronize(n->stream));
  n->adam_t = step;
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_forward(gmmsp_net n, const float* lab_dev, int B, int W, int H, float* out_dev) {
  GMMSP_NVTX("gmmsp_net_forward");
  if (!n) return GMMSP_E_INVALID;
  Geom g;
  if (!lab_dev || !out_dev || B < 1 || !net_geom(n, W, H, &g)) return nfail(n, GMMSP_E_INVALID, "bad arguments");
  if (!cells_fit(n, (long long)B * g.K)) return nfail(n, GMMSP_E_INVALID, "batch too large");
  const gmmsp_status st = reserve(n, (long long)B * g.K, false);
  if (st != GMMSP_OK) return st;
  return enqueue_forward(n, lab_dev, B, g, out_dev, false, n->stream);
}

gmmsp_status gmmsp_net_grad(gmmsp_net n, const float* lab_dev, int B, int W, int H, const float* target_dev,
                            float* grad_host, double* loss_host) {
  GMMSP_NVTX("gmmsp_net_grad");
  if (!n) return GMMSP_E_INVALID;
  Geom g;
  if (!lab_dev || !target_dev || B < 1 || !net_geom(n, W, H, &g))
    return nfail(n, GMMSP_E_INVALID, "bad arguments");
  const long long cells = (long long)B * g.K;
  if (!cells_fit(n, cells)) return nfail(n, GMMSP_E_INVALID, "batch too large");
  gmmsp_status st = reserve(n, cells, true);
  if (st != GMMSP_OK) return st;
  st = enqueue_grad(n, lab_dev, B, g, target_dev, n->stream);
  if (st != GMMSP_OK) return st;
  if (grad_host)
    GN_CHECK(n, cudaMemcpyAsync(grad_host, n->grad, size_t(n->pl.total) * 4, cudaMemcpyDeviceToHost, n->stream));
  if (loss_host) return loss_to_host(n, cells, loss_host);
  if (grad_host) return check_err(n);
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_adam(gmmsp_net n, float lr, float beta1, float beta2, float eps) {
  if (!n) return GMMSP_E_INVALID;
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return nfail(n, GMMSP_E_INVALID, "bad Adam hyper-parameters");
  ++n->adam_t;
  const float c1 = float(1.0 / (1.0 - pow(double(beta1), double(n->adam_t))));
  const float c2 = float(1.0 / (1.0 - pow(double(beta2), double(n->adam_t))));
  const int np = n->pl.total;
  k_adam<<<grid_for(np, 256), 256, 0, n->stream>>>(n->w32, n->m, n->vv, n->grad, n->wbf, np, lr, beta1, beta2,
                                                   eps, c1, c2);
  GN_CHECK(n, cudaGetLastError());
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_train_step(gmmsp_net n, const float* lab_dev, int B, int W, int H,
                                  const float* target_dev, float lr, double* loss_host) {
  GMMSP_NVTX("gmmsp_net_train_step");
  gmmsp_status st = gmmsp_net_grad(n, lab_dev, B, W, H, target_dev, nullptr, nullptr);
  if (st != GMMSP_OK) return st;
  st = gmmsp_net_adam(n, lr, 0.9f, 0.999f, 1e-8f);
  if (st != GMMSP_OK || !loss_host) return st;
  Geom g;
  net_geom(n, W, H, &g);
  return loss_to_host(n, (long long)B * g.K, loss_host);
}

gmmsp_status gmmsp_net_get_activation(gmmsp_net n, int layer, float* host, long long count) {
  if (!n) return GMMSP_E_INVALID;
  if (layer < 0 || layer > 3 || !host || count != n->last_cells * kC || n->last_cells == 0)
    return nfail(n, GMMSP_E_INVALID, "bad activation request");
  std::vector<uint16_t> tmp(static_cast<size_t>(count));
  GN_CHECK(n, cudaMemcpyAsync(tmp.data(), n->c[layer], size_t(count) * 2, cudaMemcpyDeviceToHost, n->stream));
  const gmmsp_status st = check_err(n);
  if (st != GMMSP_OK) return st;
  for (long long i = 0; i < count; ++i) {  // a bfloat16 is the top half of a float32
    const uint32_t u = uint32_t(tmp[size_t(i)]) << 16;
    memcpy(host + i, &u, 4);
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_net_check(gmmsp_net n) {
  if (!n) return GMMSP_E_INVALID;
  return check_err(n);
}

gmmsp_status gmmsp_tc_wait_selftest(int max_tries, void* stream) {
  if (max_tries < 1 || max_tries > (1 << 20)) return GMMSP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return GMMSP_E_NOMEM;
  }
  int host = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 128, 0, s>>>(uint32_t(max_tries), flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  if (e != cudaSuccess) return GMMSP_E_CUDA;
  return host ? GMMSP_E_TIMEOUT : GMMSP_OK;
}

const char* gmmsp_net_last_error(gmmsp_net n) { return n ? n->msg.c_str() : "null network"; }

void gmmsp_net_destroy(gmmsp_net n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  if (n->wslab) cudaFree(n->wslab);
  if (n->pslab) cudaFree(n->pslab);
  delete n;
}

}  // extern "C"
