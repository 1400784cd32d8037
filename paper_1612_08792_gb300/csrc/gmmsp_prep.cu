// Input preparation and initial parameters.
//
//  * k_rgb2lab: sRGB uint8 -> CIELAB as three float32 planes (L, a, b).  The
//    paper runs in CIELAB (Sec. IV, first paragraph) without fixing the RGB
//    space or the white; this library reads the input as sRGB with the D65
//    white.  The RGB -> XYZ matrix is not a literal table: the host derives
//    it from the sRGB primaries and the white point (see api), and the
//    kernel applies the sRGB transfer curve (through a 256-entry table built
//    per block with powf) and the CIE 1976 L*a*b* formulas.
//  * k_lab32: repacks a caller's float32 L,a,b image into planes and counts
//    non-finite values.
//  * k_gray2l: grey levels -> CIE L*.  A grey pixel drives the three
//    primaries equally, so its luminance relative to the white is the decoded
//    grey level itself: L* = 116 f(decode(g / 255)) - 16.
//  Under the grayscale colour model every conversion writes plane L only;
//  the context keeps the a, b planes at zero.
//  * k_init_theta: Sec. III-C initialisation: mu_k = z of the centre pixel of
//    cell k, Sigma_s = diag(v^2, v^2), Sigma_c = lambda_c^2 I.
//  * k_pack_theta: re-derives the packed E-step coefficients from FP64
//    parameters supplied by the caller (resume / external initialisation).
#include <math.h>

#include <algorithm>

#include "gmmsp_internal.cuh"
#include "gmmsp_lab.cuh"
#include "gmmsp_math.cuh"

namespace gmmsp {

__global__ void __launch_bounds__(256) k_rgb2lab(const uint8_t* __restrict__ img, long long pitch,
                                                 int W, int H, float* __restrict__ lab,
                                                 Rgb2LabConst k, bool l_only) {
  __shared__ float lin[256];
  build_srgb_table(lin);
  pdl_wait();  // the CIELAB buffer may still be read by the previous pipeline run
  pdl_trigger();
  __syncthreads();
  const long long N = (long long)W * H;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = int(idx / W), x = int(idx - (long long)y * W);
    float L, A, B;
    srgb8_to_lab(k, lin, img + (long long)y * pitch + 3LL * x, L, A, B);
    lab[idx] = L;
    if (!l_only) {
      lab[N + idx] = A;
      lab[2 * N + idx] = B;
    }
  }
}

__global__ void __launch_bounds__(256) k_gray2l(const uint8_t* __restrict__ img, long long pitch, int W, int H,
                                                float* __restrict__ lab) {
  __shared__ float lin[256];
  build_srgb_table(lin);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const long long N = (long long)W * H;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = int(idx / W), x = int(idx - (long long)y * W);
    lab[idx] = 116.f * cielab_f(lin[img[(long long)y * pitch + x]]) - 16.f;
  }
}

__global__ void __launch_bounds__(256) k_lab32(const float* __restrict__ img, long long pitch, int W,
                                               int H, float* __restrict__ lab,
                                               unsigned long long* __restrict__ counters, bool l_only) {
  const long long N = (long long)W * H;
  unsigned bad = 0;
  pdl_wait();
  pdl_trigger();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = int(idx / W), x = int(idx - (long long)y * W);
    const float* p = reinterpret_cast<const float*>(reinterpret_cast<const char*>(img) +
                                                    (long long)y * pitch) + 3LL * x;
    const float L = p[0];
    lab[idx] = L;
    if (l_only) {
      bad += !isfinite(L);
    } else {
      const float a = p[1], b = p[2];
      bad += !(isfinite(L) && isfinite(a) && isfinite(b));
      lab[N + idx] = a;
      lab[2 * N + idx] = b;
    }
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&counters[CNT_NONFINITE], (unsigned long long)bad);
}

// Sec. III-C initialisation of superpixel k.
template <class Src>
__device__ __forceinline__ void init_k(const Src& lab, const Geom& g, double lambda_c,
                                       double* __restrict__ theta, float* __restrict__ gp, int k) {
  if (!GMMSP_IN_BOUNDS(k, g.K, BND_THETA)) return;
  const int kx = k % g.nx, ky = k / g.nx;
  const int x = kx * g.v + g.v / 2, y = ky * g.v + g.v / 2;
  float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
  if (GMMSP_IN_BOUNDS(x, g.W, BND_PIXEL_X) && GMMSP_IN_BOUNDS(y, g.H, BND_PIXEL_Y)) c = lab.load(x, y);
  const bool gray = g.cm == kColourGray;
  const double mu[5] = {double(x), double(y), double(c.x), gray ? 0.0 : double(c.y), gray ? 0.0 : double(c.z)};
  const double vv = double(g.v) * double(g.v), ll = lambda_c * lambda_c;
  const double cs[3] = {vv, 0.0, vv};
  const double cc[6] = {ll, 0.0, 0.0, gray ? 0.0 : ll, 0.0, gray ? 0.0 : ll};
  double* th = theta + (long long)k * kTheta;
  for (int i = 0; i < 5; ++i) th[i] = mu[i];
  for (int i = 0; i < 3; ++i) th[5 + i] = cs[i];
  for (int i = 0; i < 6; ++i) th[8 + i] = cc[i];
  th[14] = th[15] = 0.0;
  pack_gp<double>(mu, cs, cc, double(kx * g.v), double(ky * g.v), gp + (long long)k * kGP, g.cm);
}

template <class Src>
__global__ void k_init_theta(Src lab, Geom g, double lambda_c, double* __restrict__ theta,
                             float* __restrict__ gp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (k >= g.K) return;
  init_k<Src>(lab, g, lambda_c, theta, gp, k);
}

__global__ void k_pack_theta(Geom g, const double* __restrict__ theta, float* __restrict__ gp,
                             int* __restrict__ bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.K) return;
  const double* th = theta + (long long)k * kTheta;
  bool ok = true;
  for (int i = 0; i < 14; ++i) ok = ok && isfinite(th[i]);
  const int kx = k % g.nx, ky = k / g.nx;
  ok = ok && pack_gp<double>(th, th + 5, th + 8, double(kx * g.v), double(ky * g.v),
                             gp + (long long)k * kGP, g.cm);
  if (!ok) atomicAdd(bad, 1);
}

static int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 16) b = 152LL * 16;
  return int(b < 1 ? 1 : b);
}

// Host-side construction of the sRGB -> XYZ matrix from the primaries'
// chromaticities and the white point (standard RGB colourimetry: each
// column is a primary's XYZ scaled so that RGB = (1, 1, 1) maps to white).
static Rgb2LabConst make_rgb2lab_const() {
  const double prim[3][2] = {{0.64, 0.33}, {0.30, 0.60}, {0.15, 0.06}};  // R, G, B (x, y)
  const double white[3] = {0.95047, 1.0, 1.08883};                        // D65 XYZ, Y = 1
  double P[3][3];
  for (int j = 0; j < 3; ++j) {
    const double x = prim[j][0], y = prim[j][1];
    P[0][j] = x / y;
    P[1][j] = 1.0;
    P[2][j] = (1.0 - x - y) / y;
  }
  // Solve P s = white by Cramer's rule.
  auto det3 = [](const double A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
           A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  };
  const double D = det3(P);
  double s[3];
  for (int j = 0; j < 3; ++j) {
    double Q[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Q[r][c] = (c == j) ? white[r] : P[r][c];
    s[j] = det3(Q) / D;
  }
  Rgb2LabConst k;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) k.m[3 * r + c] = float(P[r][c] * s[c]);
  for (int r = 0; r < 3; ++r) k.inv_white[r] = float(1.0 / white[r]);
  return k;
}

Rgb2LabConst rgb2lab_const() {
  static const Rgb2LabConst k = make_rgb2lab_const();
  return k;
}

cudaError_t launch_rgb2lab(const uint8_t* img, long long pitch, const Geom& g, float* lab,
                           unsigned long long* counters, cudaStream_t s) {
  (void)counters;
  static const Rgb2LabConst k = make_rgb2lab_const();
  const long long N = (long long)g.W * g.H;
  return launch_pdl(k_rgb2lab, dim3(grid_for(N, 256)), dim3(256), 0, s, img, pitch, g.W, g.H, lab, k,
                    g.cm == kColourGray);
}

cudaError_t launch_gray2l(const uint8_t* img, long long pitch, const Geom& g, float* lab, cudaStream_t s) {
  const long long N = (long long)g.W * g.H;
  return launch_pdl(k_gray2l, dim3(grid_for(N, 256)), dim3(256), 0, s, img, pitch, g.W, g.H, lab);
}

cudaError_t launch_lab32(const float* img, long long pitch, const Geom& g, float* lab,
                         unsigned long long* counters, cudaStream_t s) {
  const long long N = (long long)g.W * g.H;
  return launch_pdl(k_lab32, dim3(grid_for(N, 256)), dim3(256), 0, s, img, pitch, g.W, g.H, lab, counters,
                    g.cm == kColourGray);
}

template <class Src>
cudaError_t launch_init_theta(Src lab, const Geom& g, double lambda_c, double* theta, float* gp,
                              cudaStream_t s) {
  return launch_pdl(k_init_theta<Src>, dim3((g.K + 63) / 64), dim3(64), 0, s, lab, g, lambda_c, theta, gp);
}

template cudaError_t launch_init_theta<LabPlanar>(LabPlanar, const Geom&, double, double*, float*,
                                                  cudaStream_t);
template cudaError_t launch_init_theta<LabPitched>(LabPitched, const Geom&, double, double*, float*,
                                                   cudaStream_t);

cudaError_t launch_pack_theta(const Geom& g, double* theta, float* gp, int* bad, cudaStream_t s) {
  k_pack_theta<<<(g.K + 63) / 64, 64, 0, s>>>(g, theta, gp, bad);
  return cudaGetLastError();
}

}  // namespace gmmsp

// ---------------------------------------------------------------- batches
namespace gmmsp {

// Image of batch row `row` (binary search over the images' first rows).
__device__ __forceinline__ int find_row_image(const BatchImage* __restrict__ imgs, int n, int row) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (imgs[mid].row_off <= row) lo = mid; else hi = mid;
  }
  return lo;
}

cudaError_t bounds_take_prep(unsigned long long* word) {
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

// CIELAB conversion of every image of a batch: one warp per image row, rows
// of all images taken in turn by the persistent warps.
__global__ void __launch_bounds__(256) k_prepare_batch(const BatchImage* __restrict__ imgs, int n,
                                                       int total_rows, int input_format,
                                                       float* __restrict__ lab, Rgb2LabConst k,
                                                       unsigned long long* __restrict__ counters) {
  __shared__ float lin[256];
  build_srgb_table(lin);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  unsigned bad = 0;
  for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < total_rows; row += warps) {
    const BatchImage& im = imgs[find_row_image(imgs, n, row)];
    const int W = im.g.W, y = row - im.row_off;
    const long long N = (long long)W * im.g.H;
    float* P = lab + 3 * im.pix_off;
    const char* src = static_cast<const char*>(im.image) + (long long)y * im.pitch;
    const bool l_only = im.g.cm == kColourGray;
    for (int x = lane; x < W; x += 32) {
      float L, a = 0.f, b = 0.f;
      if (input_format == 2) {  // grey levels
        L = 116.f * cielab_f(lin[reinterpret_cast<const uint8_t*>(src)[x]]) - 16.f;
      } else if (input_format == 0) {
        srgb8_to_lab(k, lin, reinterpret_cast<const uint8_t*>(src) + 3LL * x, L, a, b);
      } else {
        const float* p = reinterpret_cast<const float*>(src) + 3LL * x;
        L = p[0];
        if (!l_only) { a = p[1]; b = p[2]; }
        bad += !(isfinite(L) && isfinite(a) && isfinite(b));
      }
      const long long q = (long long)y * W + x;
      if (!GMMSP_IN_BOUNDS(q, N, BND_PIXEL_Y)) continue;
      P[q] = L;
      if (!l_only) { P[N + q] = a; P[2 * N + q] = b; }
    }
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if (lane == 0 && bad) atomicAdd(&counters[CNT_NONFINITE], (unsigned long long)bad);
}

// sRGB -> CIELAB of the pixels outside the n_x v x n_y v cell region of n
// images of one geometry g (the right strip x >= n_x v, y < n_y v, then the
// bottom strip y >= n_y v), each thread taking pixels in turn.
__global__ void __launch_bounds__(256) k_prepare_rest(const BatchImage* __restrict__ imgs, int n, Geom g,
                                                      float* __restrict__ lab, Rgb2LabConst k) {
  __shared__ float lin[256];
  build_srgb_table(lin);
  __syncthreads();
  const int cx = g.nx * g.v, cy = g.ny * g.v;
  const long long right = (long long)(g.W - cx) * cy;
  const long long per = right + (long long)g.W * (g.H - cy);
  const long long N = (long long)g.W * g.H;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < per * n;
       r += (long long)gridDim.x * blockDim.x) {
    const int img = int(r / per);
    const long long q = r - (long long)img * per;
    int x, y;
    if (q < right) {
      y = int(q / (g.W - cx));
      x = cx + int(q - (long long)y * (g.W - cx));
    } else {
      const long long t = q - right;
      y = cy + int(t / g.W);
      x = int(t - (long long)(y - cy) * g.W);
    }
    const BatchImage& im = imgs[img];
    const long long i = (long long)y * g.W + x;
    if (!GMMSP_IN_BOUNDS(i, N, BND_PIXEL_Y)) continue;
    float L, A, B;
    srgb8_to_lab(k, lin, static_cast<const uint8_t*>(im.image) + (long long)y * im.pitch + 3LL * x, L, A, B);
    float* P = lab + 3 * im.pix_off;
    P[i] = L;
    P[N + i] = A;
    P[2 * N + i] = B;
  }
}

__global__ void __launch_bounds__(128) k_init_batch(const BatchImage* __restrict__ imgs, int n, int total_k,
                                                    const float* __restrict__ lab, double lambda_c,
                                                    double* __restrict__ theta, float* __restrict__ gp) {
  for (int kg = blockIdx.x * blockDim.x + threadIdx.x; kg < total_k; kg += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (imgs[mid].k_off <= kg) lo = mid; else hi = mid;
    }
    const BatchImage& im = imgs[lo];
    if (!GMMSP_IN_BOUNDS(kg - im.k_off, im.g.K, BND_ITEM)) continue;
    const LabPlanar src{lab + 3 * im.pix_off, (long long)im.g.W * im.g.H, im.g.W};
    init_k<LabPlanar>(src, im.g, lambda_c, theta + (long long)im.k_off * kTheta,
                      gp + (long long)im.k_off * kGP, kg - im.k_off);
  }
}

__global__ void __launch_bounds__(128) k_ll_per_image(const BatchImage* __restrict__ imgs,
                                                      const double* __restrict__ cell_ll,
                                                      double* __restrict__ out) {
  __shared__ double red[128];
  const BatchImage& im = imgs[blockIdx.x];
  double s = 0.0;
  for (int c = threadIdx.x; c < im.g.ncells; c += 128) s += cell_ll[im.cell_off + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

cudaError_t launch_prepare_batch(const BatchImage* imgs, int n, long long total_rows, int input_format,
                                 float* lab, unsigned long long* counters, int blocks, cudaStream_t s) {
  static const Rgb2LabConst k = make_rgb2lab_const();
  k_prepare_batch<<<blocks, 256, 0, s>>>(imgs, n, int(total_rows), input_format, lab, k, counters);
  return cudaGetLastError();
}

cudaError_t launch_prepare_rest(const BatchImage* imgs, int n, const Geom& g, float* lab, int sm_count,
                                cudaStream_t s) {
  static const Rgb2LabConst k = make_rgb2lab_const();
  const long long per =
      (long long)(g.W - g.nx * g.v) * (g.ny * g.v) + (long long)g.W * (g.H - g.ny * g.v);
  if (per * n == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((per * n + 255) / 256, (long long)sm_count * 4);
  k_prepare_rest<<<unsigned(blocks), 256, 0, s>>>(imgs, n, g, lab, k);
  return cudaGetLastError();
}

cudaError_t launch_init_batch(const BatchImage* imgs, int n, int total_k, const float* lab,
                              double lambda_c, double* theta, float* gp, int blocks, cudaStream_t s) {
  k_init_batch<<<blocks, 128, 0, s>>>(imgs, n, total_k, lab, lambda_c, theta, gp);
  return cudaGetLastError();
}

cudaError_t launch_ll_per_image(const BatchImage* imgs, int n, const double* cell_ll, double* ll_out,
                                cudaStream_t s) {
  k_ll_per_image<<<n, 128, 0, s>>>(imgs, cell_ll, ll_out);
  return cudaGetLastError();
}

}  // namespace gmmsp
