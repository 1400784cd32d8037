// Batched segmentation (declared in include/gmmsp.h, gmmsp_batch_*): many
// images of uneven sizes through Algorithm 1, steps 1-7, with one launch per
// step for the whole batch, the step sequence captured once into a CUDA
// graph, and a persistent grid whose size the autotuner picks.
//
// Device memory of a batch context is one allocation: the CIELAB planes of
// all images, theta / packed coefficients of all superpixels, the per-cell
// partial sums and log-likelihoods of all cells, the image table and the
// per-image log-likelihoods.  Images, cells and superpixels are numbered
// consecutively over the batch (offsets in the table).
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

using gmmsp::BatchImage;
using gmmsp::Geom;

struct gmmsp_batch_s {
  int n = 0;
  gmmsp_params p{};
  cudaStream_t stream = nullptr;
  int sm_count = 152;
  int blocks_per_sm = 4;           // persistent grid of the E + M pass (autotuned)
  int first_bps = 0;               // the first E + M pass (diagonal blocks); 0: as blocks_per_sm
  double first_ms[2] = {0.0, 0.0}; // autotuned first-pass times at 6 and 7 blocks per SM
  int label_blocks_per_sm = 4;     // persistent grid of the label pass (its occupancy)
  bool fin16 = false;              // finalize with 16 lanes per superpixel (autotuned)
  double fin_ms[2] = {0.0, 0.0};   // autotuned finalize times: 16 lanes, one thread per superpixel
  std::vector<BatchImage> host;    // the table as last uploaded
  long long total_pix = 0;
  int total_rows = 0, total_cells = 0, total_k = 0;
  void* slab = nullptr;
  float* lab = nullptr;
  double* theta = nullptr;
  float* gp = nullptr;
  void* partials = nullptr;
  double* cell_ll = nullptr;
  double* img_ll = nullptr;
  BatchImage* table = nullptr;
  unsigned long long* counters = nullptr;
  gmmsp_net net = nullptr;         // learned initialiser (null: Sec. III-C start)
  bool uniform = true;             // all images of one size
  cudaGraphExec_t exec = nullptr;
  int g_iters = -1;
  bool g_ll = false;
  int g_bps = -1;
  int g_fbps = -1;
  gmmsp_net g_net = nullptr;
  long long g_gen = -1;
  gmmsp::ConnScratch conn;         // post-processing scratch, kept between calls
  std::string err;
  gmmsp_status state = GMMSP_OK;
};

namespace {

gmmsp_status bfail(gmmsp_batch b, gmmsp_status s, const std::string& m) {
  if (b) {
    if (s != GMMSP_E_INVALID) b->state = s;
    b->err = m;
  }
  return s;
}

#define GB_CHECK(b, call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA,      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// Eq. (vxy), (nxyK) as for a single context.
bool geom_of(int W, int H, int K_req, int spacing, Geom* g) {
  long long v;
  if (spacing > 0) {
    v = spacing;
  } else {
    if (K_req < 1) return false;
    const long long N = (long long)W * H;
    long long lo = 0, hi = 1;
    while (hi * hi * (long long)K_req <= N) hi *= 2;
    while (hi - lo > 1) {
      const long long mid = (lo + hi) / 2;
      if (mid * mid * (long long)K_req <= N) lo = mid; else hi = mid;
    }
    v = lo;
  }
  if (v < 1 || v > W || v > H) return false;
  if ((long long)W * H > 2147483647LL) return false;  // pixel offsets are 32-bit in the kernels
  g->W = W; g->H = H; g->v = int(v);
  g->nx = int(W / v); g->ny = int(H / v);
  g->K = g->nx * g->ny;
  g->ncx = int((W + v - 1) / v);
  g->ncy = int((H + v - 1) / v);
  g->ncells = g->ncx * g->ncy;
  return g->nx >= 1 && g->ny >= 1;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// The 16-lane finalize exists for the mixed-precision full colour model only.
bool use_fin16(gmmsp_batch b) {
  return b->fin16 && b->p.precision != GMMSP_PREC_FP32 && b->p.colour_model == GMMSP_COLOUR_FULL;
}

int em_blocks(gmmsp_batch b, int bps) {
  const long long need = (b->total_cells + 3) / 4;
  const long long cap = (long long)b->sm_count * bps;
  return int(need < cap ? need : cap);
}

int first_bps(gmmsp_batch b) { return b->first_bps > 0 ? b->first_bps : b->blocks_per_sm; }

// The start of a segment: the CIELAB conversion and theta_0 (Sec. III-C or
// the network), whose covariance blocks are diagonal.
gmmsp_status enqueue_start(gmmsp_batch b) {
  cudaStream_t s = b->stream;
  const int n = b->n;
  GB_CHECK(b, cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long) * gmmsp::CNT_N, s));
  const int prep_blocks = int(std::min<long long>((b->total_rows + 7) / 8, (long long)b->sm_count * 8));
  // With the network on RGB8 input, its first kernel converts the cells'
  // pixels (it reads them anyway) and the conversion pass only the rest.
  const bool fused = b->net && b->p.input_format == GMMSP_RGB8 && b->p.colour_model == GMMSP_COLOUR_FULL;
  if (fused)
    GB_CHECK(b, gmmsp::launch_prepare_rest(b->table, n, b->host[0].g, b->lab, b->sm_count, s));
  else
    GB_CHECK(b, gmmsp::launch_prepare_batch(b->table, n, b->total_rows, b->p.input_format, b->lab,
                                            b->counters, prep_blocks, s));
  if (b->net) {
    GB_CHECK(b, gmmsp::net_enqueue_init(b->net, b->lab, fused ? b->table : nullptr, n, b->host[0].g,
                                        b->p.lambda_c, b->p.eps_s, b->p.eps_c, b->theta, b->gp, b->counters, s));
  } else {
    const int kblocks = int(std::min<long long>((b->total_k + 127) / 128, (long long)b->sm_count * 8));
    GB_CHECK(b, gmmsp::launch_init_batch(b->table, n, b->total_k, b->lab, b->p.lambda_c, b->theta, b->gp,
                                         kblocks, s));
  }
  return GMMSP_OK;
}

gmmsp_status enqueue_batch(gmmsp_batch b, int iters, bool want_ll) {
  cudaStream_t s = b->stream;
  const int n = b->n;
  const gmmsp_status st = enqueue_start(b);
  if (st != GMMSP_OK) return st;
  const int fblocks = int(std::min<long long>((b->total_k + 31) / 32, (long long)b->sm_count * 16));
  for (int t = 0; t < iters; ++t) {
    // the first pass follows the start (Sec. III-C or learned): diagonal blocks,
    // with a launch choice of its own
    const int bps = t == 0 ? first_bps(b) : b->blocks_per_sm;
    GB_CHECK(b, gmmsp::launch_em_pass_batch(b->table, n, b->total_cells, b->lab, b->gp, b->partials,
                                            b->p.precision, em_blocks(b, bps), bps, b->p.colour_model, s,
                                            t == 0));
    GB_CHECK(b, gmmsp::launch_finalize_batch(b->table, n, b->total_k, b->partials, b->theta, b->gp,
                                             b->p.eps_s, b->p.eps_c, b->counters, b->p.precision,
                                             use_fin16(b) ? 0 : fblocks, s));
  }
  const long long lneed = (b->total_cells + 3) / 4;
  const int lb = int(std::min<long long>(lneed, (long long)b->sm_count * b->label_blocks_per_sm));
  GB_CHECK(b, gmmsp::launch_label_pass_batch(b->table, n, b->total_cells, b->lab, b->gp,
                                              want_ll ? b->cell_ll : nullptr, lb, b->p.colour_model, s));
  if (want_ll) GB_CHECK(b, gmmsp::launch_ll_per_image(b->table, n, b->cell_ll, b->img_ll, s));
  return GMMSP_OK;
}

gmmsp_status upload_table(gmmsp_batch b, const void* const* images, const int* pitches,
                          int32_t* const* labels) {
  const long long mult = b->p.input_format == GMMSP_RGB8 ? 3 : (b->p.input_format == GMMSP_GRAY8 ? 1 : 12);
  for (int i = 0; i < b->n; ++i) {
    if (!images[i] || !labels[i]) return bfail(b, GMMSP_E_INVALID, "null image or label pointer");
    if (pitches[i] < mult * b->host[i].g.W) return bfail(b, GMMSP_E_INVALID, "pitch too small");
    b->host[i].image = images[i];
    b->host[i].pitch = pitches[i];
    b->host[i].labels = labels[i];
  }
  // Pageable source: the copy is staged by the driver before the call returns,
  // so the host table may be reused at once.
  GB_CHECK(b, cudaMemcpyAsync(b->table, b->host.data(), sizeof(BatchImage) * b->n, cudaMemcpyHostToDevice,
                              b->stream));
  return GMMSP_OK;
}

void drop_graph(gmmsp_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->g_iters = -1;
}

}  // namespace

extern "C" {

gmmsp_status gmmsp_batch_create(gmmsp_batch* out, int n, const int* widths, const int* heights,
                                const gmmsp_params* p, void* stream) {
  if (!out) return GMMSP_E_INVALID;
  *out = nullptr;
  if (n < 1 || !widths || !heights || !p) return GMMSP_E_INVALID;
  if (p->input_format != GMMSP_RGB8 && p->input_format != GMMSP_LAB32 && p->input_format != GMMSP_GRAY8)
    return GMMSP_E_INVALID;
  if (p->precision != GMMSP_PREC_MIXED && p->precision != GMMSP_PREC_FP32) return GMMSP_E_INVALID;
  if (p->colour_model < GMMSP_COLOUR_FULL || p->colour_model > GMMSP_COLOUR_GRAY) return GMMSP_E_INVALID;
  if (p->colour_model != GMMSP_COLOUR_FULL && p->precision != GMMSP_PREC_MIXED) return GMMSP_E_INVALID;
  if (p->input_format == GMMSP_GRAY8 && p->colour_model != GMMSP_COLOUR_GRAY) return GMMSP_E_INVALID;
  if (!(p->eps_s > 0.f) || !(p->eps_c > 0.f) || !(p->lambda_c > 0.f) || !isfinite(p->eps_s) ||
      !isfinite(p->eps_c) || !isfinite(p->lambda_c))
    return GMMSP_E_INVALID;
  if (p->spacing <= 0 && p->K <= 0) return GMMSP_E_INVALID;
  gmmsp_batch b = new (std::nothrow) gmmsp_batch_s();
  if (!b) return GMMSP_E_NOMEM;
  b->n = n;
  b->p = *p;
  b->stream = static_cast<cudaStream_t>(stream);
  b->host.resize(n);
  long long pix = 0, rows = 0, cells = 0, ks = 0;
  for (int i = 0; i < n; ++i) {
    Geom g;
    if (widths[i] < 1 || heights[i] < 1 || !geom_of(widths[i], heights[i], p->K, p->spacing, &g)) {
      delete b;
      return GMMSP_E_INVALID;
    }
    BatchImage& im = b->host[i];
    memset(&im, 0, sizeof(im));
    g.cm = p->colour_model;
    im.g = g;
    im.pix_off = pix;
    im.row_off = int(rows);
    im.cell_off = int(cells);
    im.k_off = int(ks);
    if (g.W != b->host[0].g.W || g.H != b->host[0].g.H) b->uniform = false;
    pix += (long long)g.W * g.H;
    rows += g.H;
    cells += g.ncells;
    ks += g.K;
    if (rows > INT32_MAX || cells > INT32_MAX || ks > INT32_MAX) {
      delete b;
      return GMMSP_E_INVALID;
    }
  }
  for (BatchImage& im : b->host) im.uniform = b->uniform ? 1 : 0;
  b->total_pix = pix;
  b->total_rows = int(rows);
  b->total_cells = int(cells);
  b->total_k = int(ks);
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    delete b;
    return GMMSP_E_CUDA;
  }
  b->sm_count = prop.multiProcessorCount;
  b->label_blocks_per_sm = std::max(1, gmmsp::label_pass_batch_occupancy());
  const size_t pbytes = size_t(cells) * gmmsp::kPartStride * sizeof(float);
  size_t off = 0;
  const size_t o_lab = off;   off += up256(3 * size_t(pix) * sizeof(float));
  const size_t o_theta = off; off += up256(size_t(ks) * gmmsp::kTheta * sizeof(double));
  const size_t o_gp = off;    off += up256(size_t(ks) * gmmsp::kGP * sizeof(float));
  const size_t o_part = off;  off += up256(pbytes);
  const size_t o_cll = off;   off += up256(size_t(cells) * sizeof(double));
  const size_t o_ill = off;   off += up256(size_t(n) * sizeof(double));
  const size_t o_tab = off;   off += up256(size_t(n) * sizeof(BatchImage));
  const size_t o_cnt = off;   off += up256(sizeof(unsigned long long) * gmmsp::CNT_N);
  const char* inj = getenv("GMMSP_FAIL_ALLOC");
  cudaError_t e = (inj && inj[0] == '1') ? cudaErrorMemoryAllocation : cudaMalloc(&b->slab, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* base = static_cast<char*>(b->slab);
  b->lab = reinterpret_cast<float*>(base + o_lab);
  b->theta = reinterpret_cast<double*>(base + o_theta);
  b->gp = reinterpret_cast<float*>(base + o_gp);
  b->partials = base + o_part;
  b->cell_ll = reinterpret_cast<double*>(base + o_cll);
  b->img_ll = reinterpret_cast<double*>(base + o_ill);
  b->table = reinterpret_cast<BatchImage*>(base + o_tab);
  b->counters = reinterpret_cast<unsigned long long*>(base + o_cnt);
  if (p->colour_model == GMMSP_COLOUR_GRAY) {
    // the a, b planes stay zero: the conversion writes plane L only
    e = cudaMemsetAsync(b->lab, 0, 3 * size_t(pix) * sizeof(float), b->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b->slab);
      delete b;
      return GMMSP_E_CUDA;
    }
  }
  *out = b;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_get_tuning(gmmsp_batch b, int* blocks_per_sm, int* finalize16, double* finalize_ms) {
  if (!b) return GMMSP_E_INVALID;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (finalize16) *finalize16 = use_fin16(b) ? 1 : 0;
  if (finalize_ms) {
    finalize_ms[0] = b->fin_ms[0];
    finalize_ms[1] = b->fin_ms[1];
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_info(gmmsp_batch b, long long* total_pixels, int* total_k, int* total_cells) {
  if (!b) return GMMSP_E_INVALID;
  if (total_pixels) *total_pixels = b->total_pix;
  if (total_k) *total_k = b->total_k;
  if (total_cells) *total_cells = b->total_cells;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_segment(gmmsp_batch b, const void* const* images_dev, const int* pitches, int iters,
                                 int32_t* const* labels_dev, double* loglik_host) {
  GMMSP_NVTX("gmmsp_batch_segment");
  if (!b) return GMMSP_E_INVALID;
  if (!images_dev || !pitches || !labels_dev || iters < 0) return bfail(b, GMMSP_E_INVALID, "bad arguments");
  if (b->state == GMMSP_E_CUDA || b->state == GMMSP_E_NOMEM) return GMMSP_E_STATE;
  b->state = GMMSP_OK;
  gmmsp_status st = upload_table(b, images_dev, pitches, labels_dev);
  if (st != GMMSP_OK) return st;
  const bool want_ll = loglik_host != nullptr;
  if (b->stream == nullptr) {
    st = enqueue_batch(b, iters, want_ll);
    if (st != GMMSP_OK) return st;
  } else {
    const long long gen = gmmsp::net_generation(b->net);
    if (!(b->exec && b->g_iters == iters && b->g_ll == want_ll && b->g_bps == b->blocks_per_sm &&
          b->g_fbps == first_bps(b) && b->g_net == b->net && b->g_gen == gen)) {
      drop_graph(b);
      GB_CHECK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_batch(b, iters, want_ll);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
      if (st != GMMSP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return bfail(b, GMMSP_E_CUDA, cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, GMMSP_E_CUDA, cudaGetErrorString(e));
      }
      b->g_iters = iters;
      b->g_ll = want_ll;
      b->g_bps = b->blocks_per_sm;
      b->g_fbps = first_bps(b);
      b->g_net = b->net;
      b->g_gen = gen;
    }
    GB_CHECK(b, cudaGraphLaunch(b->exec, b->stream));
  }
  if (want_ll) {
    GB_CHECK(b, cudaMemcpyAsync(loglik_host, b->img_ll, sizeof(double) * b->n, cudaMemcpyDeviceToHost,
                                b->stream));
    GB_CHECK(b, cudaStreamSynchronize(b->stream));
    unsigned long long cnt[gmmsp::CNT_N];
    GB_CHECK(b, cudaMemcpy(cnt, b->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (cnt[gmmsp::CNT_NONFINITE]) return bfail(b, GMMSP_E_NUMERIC, "non-finite input values");
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_get_params(gmmsp_batch b, int i, double* mu_host, double* cov_s_host,
                                    double* cov_c_host) {
  if (!b || i < 0 || i >= b->n) return GMMSP_E_INVALID;
  const BatchImage& im = b->host[i];
  std::vector<double> th(size_t(im.g.K) * gmmsp::kTheta);
  GB_CHECK(b, cudaMemcpyAsync(th.data(), b->theta + size_t(im.k_off) * gmmsp::kTheta, th.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, b->stream));
  GB_CHECK(b, cudaStreamSynchronize(b->stream));
  for (int k = 0; k < im.g.K; ++k) {
    const double* t = th.data() + size_t(k) * gmmsp::kTheta;
    if (mu_host) memcpy(mu_host + 5 * size_t(k), t, 5 * sizeof(double));
    if (cov_s_host) memcpy(cov_s_host + 3 * size_t(k), t + 5, 3 * sizeof(double));
    if (cov_c_host) memcpy(cov_c_host + 6 * size_t(k), t + 8, 6 * sizeof(double));
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_get_lab(gmmsp_batch b, int i, float* lab_host) {
  if (!b || !lab_host || i < 0 || i >= b->n) return GMMSP_E_INVALID;
  const BatchImage& im = b->host[i];
  const size_t N = size_t(im.g.W) * im.g.H;
  std::vector<float> tmp(3 * N);
  GB_CHECK(b, cudaMemcpyAsync(tmp.data(), b->lab + 3 * size_t(im.pix_off), 3 * N * sizeof(float),
                              cudaMemcpyDeviceToHost, b->stream));
  GB_CHECK(b, cudaStreamSynchronize(b->stream));
  for (size_t q = 0; q < N; ++q) {
    lab_host[3 * q + 0] = tmp[q];
    lab_host[3 * q + 1] = tmp[N + q];
    lab_host[3 * q + 2] = tmp[2 * N + q];
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_set_tuning(gmmsp_batch b, int blocks_per_sm, int finalize16) {
  if (!b || blocks_per_sm < 1 || blocks_per_sm > 16 || finalize16 < 0 || finalize16 > 1) return GMMSP_E_INVALID;
  b->blocks_per_sm = blocks_per_sm;
  b->first_bps = 0;
  b->fin16 = finalize16 != 0;
  drop_graph(b);
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_set_launch(gmmsp_batch b, int blocks_per_sm) {
  if (!b || blocks_per_sm < 1 || blocks_per_sm > 16) return GMMSP_E_INVALID;
  b->blocks_per_sm = blocks_per_sm;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_set_first_pass(gmmsp_batch b, int blocks_per_sm) {
  if (!b || blocks_per_sm < 0 || blocks_per_sm > 16) return GMMSP_E_INVALID;
  b->first_bps = blocks_per_sm;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_get_first_pass(gmmsp_batch b, int* blocks_per_sm, double* times_ms) {
  if (!b) return GMMSP_E_INVALID;
  if (blocks_per_sm) *blocks_per_sm = first_bps(b);
  if (times_ms) {
    times_ms[0] = b->first_ms[0];
    times_ms[1] = b->first_ms[1];
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_first_pass_partials(gmmsp_batch b, const void* const* images_dev, const int* pitches,
                                             int32_t* const* labels_dev, int blocks_per_sm, int diagonal,
                                             float* partials_host, long long* n_floats) {
  if (!b || (!partials_host && !n_floats) || blocks_per_sm < 1 || blocks_per_sm > 16 || diagonal < 0 ||
      diagonal > 1)
    return GMMSP_E_INVALID;
  const long long nf = (long long)b->total_cells * gmmsp::kPartStride;
  if (n_floats) *n_floats = nf;
  if (!partials_host) return GMMSP_OK;
  if (b->state == GMMSP_E_CUDA || b->state == GMMSP_E_NOMEM) return GMMSP_E_STATE;
  b->state = GMMSP_OK;
  gmmsp_status st = upload_table(b, images_dev, pitches, labels_dev);
  if (st != GMMSP_OK) return st;
  st = enqueue_start(b);
  if (st != GMMSP_OK) return st;
  GB_CHECK(b, gmmsp::launch_em_pass_batch(b->table, b->n, b->total_cells, b->lab, b->gp, b->partials,
                                          b->p.precision, em_blocks(b, blocks_per_sm), blocks_per_sm,
                                          b->p.colour_model, b->stream, diagonal != 0));
  GB_CHECK(b, cudaMemcpyAsync(partials_host, b->partials, size_t(nf) * sizeof(float), cudaMemcpyDeviceToHost,
                              b->stream));
  GB_CHECK(b, cudaStreamSynchronize(b->stream));
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_autotune(gmmsp_batch b, const void* const* images_dev, const int* pitches,
                                  int32_t* const* labels_dev, int reps, int* best, double* times_ms) {
  GMMSP_NVTX("gmmsp_batch_autotune");
  if (!b || reps < 1) return GMMSP_E_INVALID;
  gmmsp_status st = upload_table(b, images_dev, pitches, labels_dev);
  if (st != GMMSP_OK) return st;
  const int prep_blocks = int(std::min<long long>((b->total_rows + 7) / 8, (long long)b->sm_count * 8));
  GB_CHECK(b, gmmsp::launch_prepare_batch(b->table, b->n, b->total_rows, b->p.input_format, b->lab, b->counters,
                                          prep_blocks, b->stream));
  const int kblocks = int(std::min<long long>((b->total_k + 127) / 128, (long long)b->sm_count * 8));
  GB_CHECK(b, gmmsp::launch_init_batch(b->table, b->n, b->total_k, b->lab, b->p.lambda_c, b->theta, b->gp,
                                       kblocks, b->stream));
  const int cand[5] = {3, 4, 5, 6, 7};
  cudaEvent_t e0, e1;
  GB_CHECK(b, cudaEventCreate(&e0));
  GB_CHECK(b, cudaEventCreate(&e1));
  // mean time of one E + M pass at `bps` blocks per SM, after a warm-up launch;
  // theta stays the start's, so its covariance blocks are diagonal throughout
  auto time_pass = [&](int bps, bool diag, double* per) -> gmmsp_status {
    const int eb = em_blocks(b, bps);
    GB_CHECK(b, gmmsp::launch_em_pass_batch(b->table, b->n, b->total_cells, b->lab, b->gp, b->partials,
                                            b->p.precision, eb, bps, b->p.colour_model, b->stream, diag));
    GB_CHECK(b, cudaEventRecord(e0, b->stream));
    for (int r = 0; r < reps; ++r)
      GB_CHECK(b, gmmsp::launch_em_pass_batch(b->table, b->n, b->total_cells, b->lab, b->gp, b->partials,
                                              b->p.precision, eb, bps, b->p.colour_model, b->stream, diag));
    GB_CHECK(b, cudaEventRecord(e1, b->stream));
    GB_CHECK(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    GB_CHECK(b, cudaEventElapsedTime(&ms, e0, e1));
    *per = double(ms) / reps;
    return GMMSP_OK;
  };
  double best_ms = 1e30, first_best = 1e30;
  int best_c = b->blocks_per_sm, first_c = 0;
  for (int i = 0; i < 5; ++i) {
    double per = 0.0;
    st = time_pass(cand[i], false, &per);
    if (st != GMMSP_OK) return st;
    if (times_ms) times_ms[i] = per;
    if (per < best_ms) { best_ms = per; best_c = cand[i]; }
    if (cand[i] < 6 && per < first_best) { first_best = per; first_c = cand[i]; }  // no diagonal variant
  }
  // the first pass: the diagonal kernels of the one-cell-per-warp launch
  for (int i = 0; i < 2; ++i) {
    st = time_pass(6 + i, true, &b->first_ms[i]);
    if (st != GMMSP_OK) return st;
    if (b->first_ms[i] < first_best) { first_best = b->first_ms[i]; first_c = 6 + i; }
  }
  b->blocks_per_sm = best_c;
  b->first_bps = first_c;
  if (b->p.precision != GMMSP_PREC_FP32 && b->p.colour_model == GMMSP_COLOUR_FULL) {
    // finalize: 16 lanes per superpixel against one thread per superpixel
    // (theta changes here; every segment starts again from theta_0)
    const int fblocks = int(std::min<long long>((b->total_k + 31) / 32, (long long)b->sm_count * 16));
    double fin_ms[2] = {0.0, 0.0};
    for (int variant = 0; variant < 2; ++variant) {
      const int blocks = variant == 0 ? 0 : fblocks;
      GB_CHECK(b, gmmsp::launch_finalize_batch(b->table, b->n, b->total_k, b->partials, b->theta, b->gp,
                                               b->p.eps_s, b->p.eps_c, b->counters, b->p.precision, blocks,
                                               b->stream));
      GB_CHECK(b, cudaEventRecord(e0, b->stream));
      for (int r = 0; r < reps; ++r)
        GB_CHECK(b, gmmsp::launch_finalize_batch(b->table, b->n, b->total_k, b->partials, b->theta, b->gp,
                                                 b->p.eps_s, b->p.eps_c, b->counters, b->p.precision, blocks,
                                                 b->stream));
      GB_CHECK(b, cudaEventRecord(e1, b->stream));
      GB_CHECK(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      GB_CHECK(b, cudaEventElapsedTime(&ms, e0, e1));
      fin_ms[variant] = double(ms) / reps;
    }
    b->fin16 = fin_ms[0] <= fin_ms[1];
    b->fin_ms[0] = fin_ms[0];
    b->fin_ms[1] = fin_ms[1];
    GB_CHECK(b, cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long) * gmmsp::CNT_N, b->stream));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(b);
  if (best) *best = best_c;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_set_init_net(gmmsp_batch b, gmmsp_net net) {
  if (!b) return GMMSP_E_INVALID;
  if (net) {
    if (!b->uniform) return bfail(b, GMMSP_E_INVALID, "a learned start needs images of one size");
    if (b->p.colour_model != GMMSP_COLOUR_FULL)
      return bfail(b, GMMSP_E_INVALID, "a learned start needs the full colour model");
    std::string why;
    const gmmsp_status st = gmmsp::net_reserve(net, b->n, b->host[0].g, &why);
    if (st != GMMSP_OK) return bfail(b, st == GMMSP_E_INVALID ? GMMSP_E_INVALID : st, why);
  }
  b->net = net;
  drop_graph(b);
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_connectivity(gmmsp_batch b, int32_t* const* labels_dev, gmmsp_conn_stats* stats_host) {
  GMMSP_NVTX("gmmsp_batch_connectivity");
  if (!b || !labels_dev) return GMMSP_E_INVALID;
  std::vector<int> W(b->n), H(b->n), K(b->n);
  std::vector<const float*> lab(b->n);
  for (int i = 0; i < b->n; ++i) {
    if (!labels_dev[i]) return bfail(b, GMMSP_E_INVALID, "null labels");
    const BatchImage& im = b->host[i];
    W[i] = im.g.W;
    H[i] = im.g.H;
    K[i] = im.g.K;
    lab[i] = b->lab + 3 * im.pix_off;
  }
  const gmmsp_status r = gmmsp::enforce_connectivity_many(b->n, W.data(), H.data(), K.data(), labels_dev, lab.data(),
                                                          stats_host, b->stream, &b->conn);
  if (r != GMMSP_OK) return bfail(b, r, "connectivity post-processing failed");
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_lab(gmmsp_batch b, const float** lab_dev) {
  if (!b || !lab_dev) return GMMSP_E_INVALID;
  *lab_dev = b->lab;
  return GMMSP_OK;
}

gmmsp_status gmmsp_batch_targets(gmmsp_batch b, float* target_dev) {
  GMMSP_NVTX("gmmsp_batch_targets");
  if (!b || !target_dev) return GMMSP_E_INVALID;
  if (!b->uniform) return bfail(b, GMMSP_E_INVALID, "targets need images of one size");
  if (b->p.colour_model != GMMSP_COLOUR_FULL) return bfail(b, GMMSP_E_INVALID, "targets need the full colour model");
  GB_CHECK(b, gmmsp::launch_targets(b->theta, b->lab, b->n, b->host[0].g, b->p.lambda_c, target_dev, b->stream));
  return GMMSP_OK;
}

const char* gmmsp_batch_last_error(gmmsp_batch b) { return b ? b->err.c_str() : "null batch"; }

void gmmsp_batch_destroy(gmmsp_batch b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->slab) cudaFree(b->slab);
  if (b->conn.ptr) cudaFree(b->conn.ptr);
  delete b;
}

}  // extern "C"
