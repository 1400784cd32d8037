// Internal declarations shared by the translation units of libgmmsp.
//
// Geometry (Eq. vxy, nxyK, Ik, kxy).  The image is covered by cells of
// v x v pixels; cell (cx, cy) spans x in [cx v, min((cx+1) v, W)).  When
// W mod v != 0 the last cell column cx = n_x is a narrower remainder strip
// (likewise for rows).  Every pixel of a cell has the same candidate set:
// k_x in {cx-1, cx, cx+1} and k_y in {cy-1, cy, cy+1}, clipped to the seed
// grid [0, n_x) x [0, n_y).  This is Eq. (Ik) evaluated per cell: pixel x
// lies in the x-window [max(0, v(k_x-1)), min(W, v(k_x+2))) exactly when
// |floor(x/v) - k_x| <= 1 (the min(W, .) bound only matters for k_x = n_x-1,
// whose window then reaches W and so covers the remainder strip).
//
// A candidate is addressed by its slot s = (k_y - cy + 1) * 3 + (k_x - cx + 1),
// so increasing s is increasing k.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gmmsp.h"

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GMMSP_HAVE_NVTX 1
#endif

namespace gmmsp {

// An NVTX range around a C entry point (named in profiler timelines; free
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) {
#ifdef GMMSP_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~NvtxRange() {
#ifdef GMMSP_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GMMSP_NVTX(name) ::gmmsp::NvtxRange gmmsp_nvtx_range_(name)

constexpr int kSlots = 9;          // |K_i| <= 9
constexpr int kStats = 15;         // W, S1[5], S2s[3], S2c[6]
constexpr int kPartStride = kSlots * kStats + 1;  // + per-cell log-likelihood = 136
constexpr int kGP = 16;            // floats of packed E-step parameters per superpixel
constexpr int kTheta = 16;         // doubles of master parameters per superpixel

// Statistic index inside a slot.
enum : int { ST_W = 0, ST_S1 = 1, ST_S2S = 6, ST_S2C = 9 };

// Packed FP32 E-step parameters of superpixel k (64 bytes, 16-byte aligned):
//   [0..4]   mu (x - k_x v, y - k_y v, L, a, b): the spatial mean relative
//            to the first pixel of the superpixel's own cell
//   [5..7]   spatial quadratic form coefficients (xx, 2xy, yy) of
//            -(1/2) log2(e) Sigma_s^{-1}
//   [8..13]  colour coefficients (LL, aa, bb, 2La, 2Lb, 2ab) of
//            -(1/2) log2(e) Sigma_c^{-1}
//   [14]     log2 of the Gaussian normaliser (2 pi)^{-5/2} det(Sigma)^{-1/2}
//   [15]     unused
// so log2 p(z; theta_k) = gp[14] + the two quadratic forms in d = z - mu.
//
// Master FP64 parameters (128 bytes): [0..4] mu, [5..7] Sigma_s (xx, xy, yy),
// [8..13] Sigma_c (LL, La, Lb, aa, ab, bb), [14..15] unused.
//
// Colour models (Sec. III-A, III-C; gmmsp_params.colour_model): the full
// 3x3 Sigma_c of Eq. (BlockSigma); the split diag(sigma_l^2, Sigma_(a,b)) of
// Eq. (BlockSigma1), whose La, Lb entries and coefficients are 0; grayscale,
// a scalar colour L with mu's a, b and every Sigma_c entry but LL at 0, the
// a, b coefficients 0 and the normaliser of a 3-dimensional Gaussian.  The
// layouts above are shared by all three; the E-step and M-step kernels are
// compiled per model and skip the terms a model does not have.
enum : int { kColourFull = 0, kColourSplit = 1, kColourGray = 2 };

struct Geom {
  int W, H;      // image size
  int v;         // spacing v_x = v_y
  int nx, ny;    // seed grid, K = nx * ny
  int K;
  int ncx, ncy;  // cell grid incl. remainder strips: ceil(W / v), ceil(H / v)
  int ncells;
  int cm = kColourFull;  // colour model
};

// Where the kernels read the CIELAB colour of pixel (x, y) from.
struct LabPlanar {  // the context's image: three float32 planes L, a, b of W H pixels
  const float* p;     // plane L; plane a at p + plane, plane b at p + 2 plane
  long long plane;
  int W;
  __device__ __forceinline__ float4 load(int x, int y) const {
    const long long i = (long long)y * W + x;
    return make_float4(__ldg(p + i), __ldg(p + plane + i), __ldg(p + 2 * plane + i), 0.f);
  }
  __device__ __forceinline__ float load_l(int x, int y) const { return __ldg(p + (long long)y * W + x); }
};
struct LabPitched {  // a caller's image: rows of (L, a, b) float32, row pitch in bytes
  const char* p;
  long long pitch;
  __device__ __forceinline__ float4 load(int x, int y) const {
    const float* q = reinterpret_cast<const float*>(p + (long long)y * pitch) + 3LL * x;
    return make_float4(__ldg(q), __ldg(q + 1), __ldg(q + 2), 0.f);
  }
  __device__ __forceinline__ float load_l(int x, int y) const {
    return __ldg(reinterpret_cast<const float*>(p + (long long)y * pitch) + 3LL * x);
  }
};

// The colour of pixel (x, y) under colour model CM: grayscale reads L only.
template <int CM, class Src>
__device__ __forceinline__ float4 load_z(const Src& s, int x, int y) {
  if constexpr (CM == kColourGray) return make_float4(s.load_l(x, y), 0.f, 0.f, 0.f);
  else return s.load(x, y);
}

// Bounds checking (compile flag GMMSP_CHECK_BOUNDS; a stand-in for a memory
// checker).  A checked build tests the index of every global access at the
// sites below against the extent of its buffer.  An index outside [0, n) is
// not used (the load yields 0, the store is skipped) and the first such event
// of a translation unit is kept in its status word as
//   (1 << 63) | site << 40 | (index mod 2^40),
// which gmmsp_bounds_status reads.  Without the flag GMMSP_IN_BOUNDS is the
// constant true and the checks compile away.
enum : unsigned {  // the sites, as numbered in include/gmmsp.h
  BND_GP = GMMSP_BND_GP,
  BND_PIXEL_X = GMMSP_BND_PIXEL_X,
  BND_PIXEL_Y = GMMSP_BND_PIXEL_Y,
  BND_PARTIAL_W = GMMSP_BND_PARTIAL_W,
  BND_PARTIAL_R = GMMSP_BND_PARTIAL_R,
  BND_THETA = GMMSP_BND_THETA,
  BND_LABEL = GMMSP_BND_LABEL,
  BND_LABEL_K = GMMSP_BND_LABEL_K,
  BND_CELL_LL = GMMSP_BND_CELL_LL,
  BND_IMAGE = GMMSP_BND_IMAGE,
  BND_ITEM = GMMSP_BND_ITEM,
};
__host__ __device__ constexpr unsigned long long bounds_code(unsigned site, long long i) {
  return (1ull << 63) | (static_cast<unsigned long long>(site) << 40) |
         (static_cast<unsigned long long>(i) & ((1ull << 40) - 1));
}
#ifdef GMMSP_CHECK_BOUNDS
static __device__ unsigned long long g_bounds_word = 0ull;  // one per translation unit
__device__ __forceinline__ bool bounds_ok(long long i, long long n, unsigned site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_bounds_word, 0ull, bounds_code(site, i));
  return false;
}
#define GMMSP_IN_BOUNDS(i, n, site) ::gmmsp::bounds_ok((long long)(i), (long long)(n), (site))
#else
#define GMMSP_IN_BOUNDS(i, n, site) true
#endif
// Reads and clears the status words of the translation units with checked
// kernels (0 when nothing was recorded or the build is unchecked).
cudaError_t bounds_take_em(unsigned long long* word);
cudaError_t bounds_take_prep(unsigned long long* word);
cudaError_t bounds_take_cnn(unsigned long long* word);

// Programmatic dependent launch (off unless GMMSP_PDL=1: measured slower on
// this pipeline of short dependent kernels).  When on, the single-image
// kernels are launched with cudaLaunchAttributeProgrammaticStreamSerialization;
// each waits for its predecessor's completion and memory (pdl_wait,
// griddepcontrol.wait, a hardware wait) and then lets its successor start
// launching (pdl_trigger).  Without a programmatic predecessor pdl_wait
// returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

bool pdl_enabled();  // true only when GMMSP_PDL=1 is set in the environment

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// One image of a batch (device-side table, one entry per image, ordered).
struct BatchImage {
  Geom g;
  const void* image;   // this call's input rows (RGB8 or LAB32)
  long long pitch;     // its row pitch in bytes
  int32_t* labels;     // output labels, W H int32
  long long pix_off;   // first pixel of the image in the batch (CIELAB planes at lab + 3 pix_off)
  int row_off;         // first row of the image in the batch's list of rows
  int cell_off;        // first cell of the image in the batch
  int k_off;           // first superpixel of the image in the batch
  int uniform;         // 1 when every image of the table has this geometry
};

// Device counters (unsigned long long): dead, raised_s, raised_c, nonfinite input.
enum : int { CNT_DEAD = 0, CNT_RAISED_S = 1, CNT_RAISED_C = 2, CNT_NONFINITE = 3, CNT_N = 4 };

// ---- launchers (each returns the launch's cudaError_t) ----
// lab: three planes of W H floats (L, a, b), plane stride W H.
// Under the grayscale model only plane L is written (the a, b planes are
// left as they are: zero, set once by the context).
cudaError_t launch_rgb2lab(const uint8_t* img, long long pitch, const Geom& g, float* lab,
                           unsigned long long* counters, cudaStream_t s);
cudaError_t launch_lab32(const float* img, long long pitch, const Geom& g, float* lab,
                         unsigned long long* counters, cudaStream_t s);
cudaError_t launch_gray2l(const uint8_t* img, long long pitch, const Geom& g, float* lab, cudaStream_t s);
template <class Src>
cudaError_t launch_init_theta(Src lab, const Geom& g, double lambda_c, double* theta, float* gp,
                              cudaStream_t s);
// wpc: warps per cell (1, 2 or 4); the colour model is g.cm.
template <class Src>
cudaError_t launch_em_pass(Src lab, const Geom& g, const float* gp, void* partials, int precision,
                           int wpc, cudaStream_t s);
// cell_ll == nullptr: labels only, no log-likelihood.
template <class Src>
cudaError_t launch_label_pass(Src lab, const Geom& g, const float* gp, int32_t* labels,
                              double* cell_ll, cudaStream_t s);
// Finalize: ws holds finalize_workspace_doubles(g) doubles, ticket one zeroed
// unsigned that the kernel leaves at zero.  llk_out (device) receives the
// log-likelihood of the E-step that produced the partials.
cudaError_t launch_finalize(const Geom& g, const void* partials, double* theta, float* gp,
                            double eps_s, double eps_c, double* llk_out, double* ws,
                            unsigned* ticket, unsigned long long* counters, int precision,
                            cudaStream_t s);
cudaError_t launch_ll_reduce(const double* cell_ll, int n, double* out, double* ws, unsigned* ticket,
                             const Geom& g, cudaStream_t s);
size_t finalize_workspace_doubles(const Geom& g);
cudaError_t launch_pack_theta(const Geom& g, double* theta, float* gp, int* bad, cudaStream_t s);

// Batches: the same steps over all images of a BatchImage table in one launch
// each; `blocks` is the persistent grid size.
// Grayscale model (the images' g.cm): plane L only, as launch_rgb2lab.
cudaError_t launch_prepare_batch(const BatchImage* imgs, int n, long long total_rows, int input_format,
                                 float* lab, unsigned long long* counters, int blocks, cudaStream_t s);
// RGB8 input, full colour model, n images of geometry g: the pixels outside
// the n_x v x n_y v cell region only (the network's converting first kernel
// writes the others).
cudaError_t launch_prepare_rest(const BatchImage* imgs, int n, const Geom& g, float* lab, int sm_count,
                                cudaStream_t s);
cudaError_t launch_init_batch(const BatchImage* imgs, int n, int total_k, const float* lab,
                              double lambda_c, double* theta, float* gp, int blocks, cudaStream_t s);
// minb >= 6: the non-persistent variant (one cell per warp, registers capped
// for 6 blocks per SM; `blocks` is then ignored); otherwise the persistent
// kernel on `blocks` blocks.  diag: every superpixel's covariance blocks are
// diagonal (true after either start, until the first finalize); the mixed-
// precision one-cell-per-warp kernels then skip the zero terms (same bits).
cudaError_t launch_em_pass_batch(const BatchImage* imgs, int n, int total_cells, const float* lab,
                                 const float* gp, void* partials, int precision, int blocks, int minb,
                                 int cm, cudaStream_t s, bool diag = false);
// blocks == 0 (mixed precision and the full colour model only): 16 lanes per
// superpixel, one block per 4 superpixels; otherwise one thread per
// superpixel on `blocks` blocks.
cudaError_t launch_finalize_batch(const BatchImage* imgs, int n, int total_k, const void* partials,
                                  double* theta, float* gp, double eps_s, double eps_c,
                                  unsigned long long* counters, int precision, int blocks,
                                  cudaStream_t s);
cudaError_t launch_label_pass_batch(const BatchImage* imgs, int n, int total_cells, const float* lab,
                                    const float* gp, double* cell_ll, int blocks, int cm, cudaStream_t s);
// Resident 128-thread blocks per SM of the batch label pass.
int label_pass_batch_occupancy();
// ll_out[i] = sum of image i's per-cell log-likelihoods (fixed order).
cudaError_t launch_ll_per_image(const BatchImage* imgs, int n, const double* cell_ll, double* ll_out,
                                cudaStream_t s);

}  // namespace gmmsp

#include "../../include/gmmsp_conn.h"
namespace gmmsp {
// Device scratch a context keeps between post-processing calls (grown on demand).
struct ConnScratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
// Connectivity post-processing of one image (labels in place; lab: three
// FP32 planes of W H values); synchronises `s`.  cache: kept scratch, or
// nullptr to allocate and free within the call.
gmmsp_status enforce_connectivity(int32_t* labels_dev, const float* lab, int W, int H, int K,
                                  gmmsp_conn_stats* stats, cudaStream_t s, ConnScratch* cache);
// The same on n images in one set of launches (totals in stats).
gmmsp_status enforce_connectivity_many(int n, const int* W, const int* H, const int* K, int32_t* const* labels,
                                       const float* const* lab, gmmsp_conn_stats* stats, cudaStream_t s,
                                       ConnScratch* cache);
}  // namespace gmmsp
