// C ABI of libgmmsp (declared in include/gmmsp.h): context life cycle,
// argument checks, device buffers and the launch sequence of Algorithm 1.
//
// Device memory of a context is one allocation carved into:
//   lab       3 W H float         CIELAB image as planes L, a, b
//   theta     K x 16 double       master parameters (mu, Sigma_s, Sigma_c)
//   gp        K x 16 float        packed E-step coefficients
//   partials  ncells x 136        per-cell FP32 partial sums
//   cell_ll   ncells double       per-cell log-likelihood of the label pass
//   llk       kLlkCap double      L(theta_t) per E-step
//   ws        finalize workspace; ticket; counters; bad flag
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_cnn.h"
#include "gmmsp_cnn_internal.cuh"
#include "gmmsp_internal.cuh"

using gmmsp::Geom;

namespace gmmsp {
// Programmatic dependent launch measured slower than plain stream order for
// this pipeline on GB300 (about 2x per EM iteration on 481x321), so it is off
// unless GMMSP_PDL=1 is set.
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("GMMSP_PDL");
    return e && e[0] == '1';
  }();
  return on;
}
}  // namespace gmmsp

namespace {

constexpr int kLlkCap = 1024;

struct Graph {
  cudaGraphExec_t exec = nullptr;
  int iters = -1;
  const void* image = nullptr;
  int pitch = 0;
  int32_t* labels = nullptr;
  bool want_ll = false;
};

}  // namespace

struct gmmsp_ctx_s {
  Geom g{};
  gmmsp_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  void* slab = nullptr;
  float* lab = nullptr;           // CIELAB planes L, a, b (W H floats each)
  double* theta = nullptr;
  float* gp = nullptr;
  void* partials = nullptr;
  double* cell_ll = nullptr;
  double* llk = nullptr;
  double* ws = nullptr;
  unsigned* ticket = nullptr;
  unsigned long long* counters = nullptr;
  int* bad = nullptr;
  int wpc = 1;                    // warps per cell of the E+M pass (launch shape)
  gmmsp::ConnScratch conn;        // post-processing scratch, kept between calls
  bool timing = false;            // record events between the kernels (gmmsp_set_timing)
  std::vector<cudaEvent_t> tev;   // timing events, created on demand
  int tev_used = 0;               // events recorded by the last enqueued sequence
  gmmsp_status state = GMMSP_OK;  // sticky error
  std::string err;
  Graph graph;
};

namespace {

// Records an error on c.  Invalid arguments leave the context usable; every
// other error makes it sticky until gmmsp_reinit.
gmmsp_status fail(gmmsp_ctx c, gmmsp_status s, const std::string& msg) {
  if (c) {
    if (s != GMMSP_E_INVALID) c->state = s;
    c->err = msg;
  }
  return s;
}

gmmsp_status cuda_fail(gmmsp_ctx c, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return fail(c, GMMSP_E_NOMEM, msg);
  return fail(c, GMMSP_E_CUDA, msg);
}

#define GM_CHECK(c, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

// Eq. (vxy), (nxyK): v = floor(sqrt(W H / K)) in exact integer arithmetic
// (the largest v with v^2 K <= W H), n_x = floor(W / v), n_y = floor(H / v).
bool make_geom(int W, int H, int K_req, int spacing, Geom* g) {
  long long v;
  if (spacing > 0) {
    v = spacing;
  } else {
    if (K_req < 1) return false;
    const long long N = (long long)W * H;
    long long lo = 0, hi = 1;
    while (hi * hi * (long long)K_req <= N) hi *= 2;
    while (hi - lo > 1) {  // invariant: lo^2 K <= N < hi^2 K
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

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Launch shape of the E+M pass before any autotuning: enough warps to give
// every SM about 16 of them (152 SMs on GB300), at most 4 warps per cell.
int default_wpc(const Geom& g) {
  const long long target = 152LL * 16;
  if ((long long)g.ncells >= target) return 1;
  if ((long long)g.ncells * 2 >= target) return 2;
  return 4;
}

bool inject_alloc_failure() {
  const char* s = getenv("GMMSP_FAIL_ALLOC");
  return s && s[0] == '1';
}

size_t partial_bytes(const Geom& g, int precision) {
  (void)precision;
  return size_t(g.ncells) * gmmsp::kPartStride * sizeof(float);
}

gmmsp_status check_ready(gmmsp_ctx c) {
  if (!c) return GMMSP_E_INVALID;
  if (c->state != GMMSP_OK) return GMMSP_E_STATE;
  return GMMSP_OK;
}

// With timing on, records an event on the context's stream (as an event
// node when the stream is being captured into a graph).
gmmsp_status mark(gmmsp_ctx c) {
  if (!c->timing) return GMMSP_OK;
  if (c->tev_used == int(c->tev.size())) {
    cudaEvent_t e = nullptr;
    GM_CHECK(c, cudaEventCreate(&e));
    c->tev.push_back(e);
  }
  GM_CHECK(c, cudaEventRecordWithFlags(c->tev[c->tev_used], c->stream, cudaEventRecordExternal));
  ++c->tev_used;
  return GMMSP_OK;
}

#define GM_MARK(c)                          \
  do {                                      \
    gmmsp_status s_ = mark(c);              \
    if (s_ != GMMSP_OK) return s_;          \
  } while (0)

// Smallest row pitch of a W-pixel row of the input format.
long long row_bytes(int format, int W) {
  return (long long)W * (format == GMMSP_RGB8 ? 3 : (format == GMMSP_GRAY8 ? 1 : 12));
}

// Enqueues step 1 of Algorithm 1: image -> CIELAB, theta_0; clears counters.
gmmsp_status enqueue_prepare(gmmsp_ctx c, const void* image, int pitch) {
  const Geom& g = c->g;
  GM_MARK(c);
  GM_CHECK(c, cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * gmmsp::CNT_N, c->stream));
  if (c->p.input_format == GMMSP_RGB8)
    GM_CHECK(c, gmmsp::launch_rgb2lab(static_cast<const uint8_t*>(image), pitch, g, c->lab, c->counters,
                                      c->stream));
  else if (c->p.input_format == GMMSP_GRAY8)
    GM_CHECK(c, gmmsp::launch_gray2l(static_cast<const uint8_t*>(image), pitch, g, c->lab, c->stream));
  else
    GM_CHECK(c, gmmsp::launch_lab32(static_cast<const float*>(image), pitch, g, c->lab, c->counters,
                                    c->stream));
  GM_CHECK(c, gmmsp::launch_init_theta(gmmsp::LabPlanar{c->lab, (long long)g.W * g.H, g.W}, g, c->p.lambda_c, c->theta, c->gp, c->stream));
  GM_MARK(c);
  return GMMSP_OK;
}

// Enqueues `iters` EM rounds; with want_ll, llk[t0 + t] receives L(theta_t).
gmmsp_status enqueue_em(gmmsp_ctx c, int iters, int t0, bool want_ll) {
  for (int t = 0; t < iters; ++t) {
    GM_CHECK(c, gmmsp::launch_em_pass(gmmsp::LabPlanar{c->lab, (long long)c->g.W * c->g.H, c->g.W}, c->g, c->gp, c->partials, c->p.precision, c->wpc,
                                      c->stream));
    double* llk_out = want_ll ? c->llk + ((t0 + t) % kLlkCap) : nullptr;
    GM_MARK(c);
    GM_CHECK(c, gmmsp::launch_finalize(c->g, c->partials, c->theta, c->gp, c->p.eps_s, c->p.eps_c,
                                       llk_out, c->ws, c->ticket, c->counters, c->p.precision,
                                       c->stream));
    GM_MARK(c);
  }
  return GMMSP_OK;
}

gmmsp_status enqueue_labels(gmmsp_ctx c, int32_t* labels, double* llk_out) {
  GM_CHECK(c, gmmsp::launch_label_pass(gmmsp::LabPlanar{c->lab, (long long)c->g.W * c->g.H, c->g.W}, c->g, c->gp,
                                       labels, llk_out ? c->cell_ll : nullptr, c->stream));
  if (llk_out)
    GM_CHECK(c, gmmsp::launch_ll_reduce(c->cell_ll, c->g.ncells, llk_out, c->ws, c->ticket, c->g,
                                        c->stream));
  GM_MARK(c);
  return GMMSP_OK;
}

// Synchronises and turns device-side findings into a status.
gmmsp_status sync_and_check(gmmsp_ctx c) {
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  unsigned long long cnt[gmmsp::CNT_N];
  GM_CHECK(c, cudaMemcpy(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  if (cnt[gmmsp::CNT_NONFINITE])
    return fail(c, GMMSP_E_NUMERIC, std::to_string(cnt[gmmsp::CNT_NONFINITE]) +
                                        " non-finite input values");
  return GMMSP_OK;
}

void free_graph(gmmsp_ctx c) {
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  c->graph = Graph();
}

void free_timing(gmmsp_ctx c) {
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  c->tev.clear();
  c->tev_used = 0;
}

}  // namespace

extern "C" {

void gmmsp_default_params(gmmsp_params* p) {
  if (!p) return;
  p->spacing = 0;
  p->K = 0;
  p->eps_s = 2.0f;
  p->eps_c = 8.0f;
  p->lambda_c = 8.0f;
  p->input_format = GMMSP_RGB8;
  p->precision = GMMSP_PREC_MIXED;
  p->colour_model = GMMSP_COLOUR_FULL;
}

const char* gmmsp_status_string(gmmsp_status s) {
  switch (s) {
    case GMMSP_OK: return "GMMSP_OK";
    case GMMSP_E_INVALID: return "GMMSP_E_INVALID";
    case GMMSP_E_CUDA: return "GMMSP_E_CUDA";
    case GMMSP_E_NOMEM: return "GMMSP_E_NOMEM";
    case GMMSP_E_NUMERIC: return "GMMSP_E_NUMERIC";
    case GMMSP_E_TIMEOUT: return "GMMSP_E_TIMEOUT";
    case GMMSP_E_STATE: return "GMMSP_E_STATE";
  }
  return "GMMSP_E_UNKNOWN";
}

const char* gmmsp_last_error(gmmsp_ctx c) { return c ? c->err.c_str() : "null context"; }

gmmsp_status gmmsp_init(gmmsp_ctx* out, const void* image_dev, int width, int height,
                        int pitch_bytes, const gmmsp_params* p, void* stream) {
  GMMSP_NVTX("gmmsp_init");
  if (!out) return GMMSP_E_INVALID;
  *out = nullptr;
  if (!p || !image_dev || width < 1 || height < 1) return GMMSP_E_INVALID;
  if (p->input_format != GMMSP_RGB8 && p->input_format != GMMSP_LAB32 && p->input_format != GMMSP_GRAY8)
    return GMMSP_E_INVALID;
  if (p->precision != GMMSP_PREC_MIXED && p->precision != GMMSP_PREC_FP32) return GMMSP_E_INVALID;
  if (p->colour_model < GMMSP_COLOUR_FULL || p->colour_model > GMMSP_COLOUR_GRAY) return GMMSP_E_INVALID;
  if (p->colour_model != GMMSP_COLOUR_FULL && p->precision != GMMSP_PREC_MIXED) return GMMSP_E_INVALID;
  if (p->input_format == GMMSP_GRAY8 && p->colour_model != GMMSP_COLOUR_GRAY) return GMMSP_E_INVALID;
  if (pitch_bytes < row_bytes(p->input_format, width)) return GMMSP_E_INVALID;
  if (p->input_format == GMMSP_LAB32 && (pitch_bytes % 4 != 0 || (uintptr_t)image_dev % 4 != 0))
    return GMMSP_E_INVALID;
  if (!(p->eps_s > 0.f) || !(p->eps_c > 0.f) || !(p->lambda_c > 0.f) || !isfinite(p->eps_s) ||
      !isfinite(p->eps_c) || !isfinite(p->lambda_c))
    return GMMSP_E_INVALID;
  if (p->spacing <= 0 && p->K <= 0) return GMMSP_E_INVALID;
  Geom g;
  if (!make_geom(width, height, p->K, p->spacing, &g)) return GMMSP_E_INVALID;
  g.cm = p->colour_model;

  gmmsp_ctx c = new (std::nothrow) gmmsp_ctx_s();
  if (!c) return GMMSP_E_NOMEM;
  c->g = g;
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return GMMSP_E_CUDA; }
  c->wpc = default_wpc(g);

  const size_t N = size_t(width) * height;
  size_t off = 0;
  const size_t o_lab = off;      off += align_up(3 * N * sizeof(float));
  const size_t o_theta = off;    off += align_up(size_t(g.K) * gmmsp::kTheta * sizeof(double));
  const size_t o_gp = off;       off += align_up(size_t(g.K) * gmmsp::kGP * sizeof(float));
  const size_t o_part = off;     off += align_up(partial_bytes(g, p->precision));
  const size_t o_cll = off;      off += align_up(size_t(g.ncells) * sizeof(double));
  const size_t o_llk = off;      off += align_up(kLlkCap * sizeof(double));
  const size_t o_ws = off;       off += align_up(gmmsp::finalize_workspace_doubles(g) * sizeof(double));
  const size_t o_ticket = off;   off += align_up(sizeof(unsigned));
  const size_t o_cnt = off;      off += align_up(sizeof(unsigned long long) * gmmsp::CNT_N);
  const size_t o_bad = off;      off += align_up(sizeof(int));
  cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&c->slab, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(c->slab);
  c->lab = reinterpret_cast<float*>(b + o_lab);
  c->theta = reinterpret_cast<double*>(b + o_theta);
  c->gp = reinterpret_cast<float*>(b + o_gp);
  c->partials = b + o_part;
  c->cell_ll = reinterpret_cast<double*>(b + o_cll);
  c->llk = reinterpret_cast<double*>(b + o_llk);
  c->ws = reinterpret_cast<double*>(b + o_ws);
  c->ticket = reinterpret_cast<unsigned*>(b + o_ticket);
  c->counters = reinterpret_cast<unsigned long long*>(b + o_cnt);
  c->bad = reinterpret_cast<int*>(b + o_bad);
  e = cudaMemsetAsync(c->slab, 0, off, c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->slab);
    delete c;
    return GMMSP_E_CUDA;
  }
  gmmsp_status st = enqueue_prepare(c, image_dev, pitch_bytes);
  if (st != GMMSP_OK) {
    cudaFree(c->slab);
    delete c;
    return st;
  }
  *out = c;
  return GMMSP_OK;
}

gmmsp_status gmmsp_reinit(gmmsp_ctx c, const void* image_dev, int pitch_bytes) {
  GMMSP_NVTX("gmmsp_reinit");
  if (!c) return GMMSP_E_INVALID;
  if (!image_dev) return fail(c, GMMSP_E_INVALID, "null image");
  if (pitch_bytes < row_bytes(c->p.input_format, c->g.W)) return fail(c, GMMSP_E_INVALID, "pitch too small");
  if (c->state == GMMSP_E_CUDA || c->state == GMMSP_E_NOMEM) return GMMSP_E_STATE;
  c->state = GMMSP_OK;
  c->err.clear();
  return enqueue_prepare(c, image_dev, pitch_bytes);
}

gmmsp_status gmmsp_em_iters(gmmsp_ctx c, int iters, double* loglik_host) {
  GMMSP_NVTX("gmmsp_em_iters");
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (iters < 0) return fail(c, GMMSP_E_INVALID, "iters < 0");
  c->tev_used = 0;
  GM_MARK(c);
  for (int done = 0; done < iters; done += kLlkCap) {
    const int n = iters - done < kLlkCap ? iters - done : kLlkCap;
    st = enqueue_em(c, n, 0, loglik_host != nullptr);
    if (st != GMMSP_OK) return st;
    if (loglik_host) {
      GM_CHECK(c, cudaMemcpyAsync(loglik_host + done, c->llk, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                  c->stream));
      st = sync_and_check(c);
      if (st != GMMSP_OK) return st;
    }
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_labels(gmmsp_ctx c, int32_t* labels_dev, double* loglik_host) {
  GMMSP_NVTX("gmmsp_labels");
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!labels_dev) return fail(c, GMMSP_E_INVALID, "null labels");
  c->tev_used = 0;
  GM_MARK(c);
  st = enqueue_labels(c, labels_dev, loglik_host ? c->llk : nullptr);
  if (st != GMMSP_OK) return st;
  if (loglik_host) {
    GM_CHECK(c, cudaMemcpyAsync(loglik_host, c->llk, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sync_and_check(c);
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_segment(gmmsp_ctx c, const void* image_dev, int pitch_bytes, int iters,
                           int32_t* labels_dev, double* loglik_host) {
  GMMSP_NVTX("gmmsp_segment");
  if (!c) return GMMSP_E_INVALID;
  if (!image_dev || !labels_dev) return fail(c, GMMSP_E_INVALID, "null image or labels");
  if (iters < 0 || iters + 1 > kLlkCap) return fail(c, GMMSP_E_INVALID, "iters out of range");
  if (pitch_bytes < row_bytes(c->p.input_format, c->g.W)) return fail(c, GMMSP_E_INVALID, "pitch too small");
  if (c->state == GMMSP_E_CUDA || c->state == GMMSP_E_NOMEM) return GMMSP_E_STATE;
  c->state = GMMSP_OK;
  c->err.clear();
  gmmsp_status st;
  const bool want_ll = loglik_host != nullptr;
  if (c->stream == nullptr) {
    // The legacy default stream cannot be captured: plain launches.
    c->tev_used = 0;
    st = enqueue_prepare(c, image_dev, pitch_bytes);
    if (st == GMMSP_OK) st = enqueue_em(c, iters, 0, want_ll);
    if (st == GMMSP_OK) st = enqueue_labels(c, labels_dev, want_ll ? c->llk + iters : nullptr);
    if (st != GMMSP_OK) return st;
  } else {
    Graph& gr = c->graph;
    if (!(gr.exec && gr.iters == iters && gr.image == image_dev && gr.pitch == pitch_bytes &&
          gr.labels == labels_dev && gr.want_ll == want_ll)) {
      free_graph(c);
      c->tev_used = 0;
      GM_CHECK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_prepare(c, image_dev, pitch_bytes);
      if (st == GMMSP_OK) st = enqueue_em(c, iters, 0, want_ll);
      if (st == GMMSP_OK) st = enqueue_labels(c, labels_dev, want_ll ? c->llk + iters : nullptr);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (st != GMMSP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&gr.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        gr.exec = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
      }
      gr.iters = iters;
      gr.image = image_dev;
      gr.pitch = pitch_bytes;
      gr.labels = labels_dev;
      gr.want_ll = want_ll;
    }
    GM_CHECK(c, cudaGraphLaunch(gr.exec, c->stream));
  }
  if (loglik_host) {
    GM_CHECK(c, cudaMemcpyAsync(loglik_host, c->llk, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost,
                                c->stream));
    return sync_and_check(c);
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_lab(gmmsp_ctx c, float* lab_host) {
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!lab_host) return fail(c, GMMSP_E_INVALID, "null output");
  const size_t N = size_t(c->g.W) * c->g.H;
  std::vector<float> tmp(3 * N);
  GM_CHECK(c, cudaMemcpyAsync(tmp.data(), c->lab, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < N; ++i) {
    lab_host[3 * i + 0] = tmp[i];
    lab_host[3 * i + 1] = tmp[N + i];
    lab_host[3 * i + 2] = tmp[2 * N + i];
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_grid(gmmsp_ctx c, int* v, int* nx, int* ny, int* K) {
  if (!c) return GMMSP_E_INVALID;
  if (v) *v = c->g.v;
  if (nx) *nx = c->g.nx;
  if (ny) *ny = c->g.ny;
  if (K) *K = c->g.K;
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_params(gmmsp_ctx c, double* mu_host, double* cov_s_host, double* cov_c_host) {
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  const int K = c->g.K;
  std::vector<double> th(size_t(K) * gmmsp::kTheta);
  GM_CHECK(c, cudaMemcpyAsync(th.data(), c->theta, th.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < K; ++k) {
    const double* t = th.data() + size_t(k) * gmmsp::kTheta;
    if (mu_host) memcpy(mu_host + 5 * size_t(k), t, 5 * sizeof(double));
    if (cov_s_host) memcpy(cov_s_host + 3 * size_t(k), t + 5, 3 * sizeof(double));
    if (cov_c_host) memcpy(cov_c_host + 6 * size_t(k), t + 8, 6 * sizeof(double));
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_set_params(gmmsp_ctx c, const double* mu_host, const double* cov_s_host,
                              const double* cov_c_host) {
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!mu_host || !cov_s_host || !cov_c_host) return fail(c, GMMSP_E_INVALID, "null parameter array");
  const int K = c->g.K;
  std::vector<double> th(size_t(K) * gmmsp::kTheta, 0.0);
  for (int k = 0; k < K; ++k) {
    double* t = th.data() + size_t(k) * gmmsp::kTheta;
    memcpy(t, mu_host + 5 * size_t(k), 5 * sizeof(double));
    memcpy(t + 5, cov_s_host + 3 * size_t(k), 3 * sizeof(double));
    memcpy(t + 8, cov_c_host + 6 * size_t(k), 6 * sizeof(double));
  }
  GM_CHECK(c, cudaMemsetAsync(c->bad, 0, sizeof(int), c->stream));
  GM_CHECK(c, cudaMemcpyAsync(c->theta, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  GM_CHECK(c, gmmsp::launch_pack_theta(c->g, c->theta, c->gp, c->bad, c->stream));
  int bad = 0;
  GM_CHECK(c, cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  if (bad) {
    c->err = std::to_string(bad) + " superpixels with non-finite or non-SPD parameters";
    return GMMSP_E_NUMERIC;  // theta is left as given; the caller should set valid parameters
  }
  return GMMSP_OK;
}

gmmsp_status gmmsp_connectivity(gmmsp_ctx c, int32_t* labels_dev, gmmsp_conn_stats* stats_host) {
  GMMSP_NVTX("gmmsp_connectivity");
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!labels_dev) return fail(c, GMMSP_E_INVALID, "null labels");
  st = gmmsp::enforce_connectivity(labels_dev, c->lab, c->g.W, c->g.H, c->g.K, stats_host, c->stream, &c->conn);
  if (st == GMMSP_E_CUDA || st == GMMSP_E_NOMEM) return fail(c, st, "connectivity post-processing failed");
  if (st != GMMSP_OK) c->err = "connectivity post-processing: a bounded device loop ran out";
  return st;
}

gmmsp_status gmmsp_set_init(gmmsp_ctx c, const float* dmu_dev, const float* logeig_dev) {
  GMMSP_NVTX("gmmsp_set_init");
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!dmu_dev || !logeig_dev) return fail(c, GMMSP_E_INVALID, "null array");
  if (c->g.cm == gmmsp::kColourGray) return fail(c, GMMSP_E_INVALID, "theta_0 arrays need a colour model with a, b");
  GM_CHECK(c, gmmsp::launch_init_from_outputs(dmu_dev, 5, logeig_dev, 5, c->lab, 1, c->g, c->p.lambda_c, c->p.eps_s,
                                              c->p.eps_c, c->theta, c->gp, c->counters, c->stream));
  return GMMSP_OK;
}

gmmsp_status gmmsp_init_from_net(gmmsp_ctx c, gmmsp_net n) {
  GMMSP_NVTX("gmmsp_init_from_net");
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (!n) return fail(c, GMMSP_E_INVALID, "null network");
  if (c->g.cm != gmmsp::kColourFull) {
    c->err = "a learned start needs the full colour model";  // the context stays usable
    return GMMSP_E_INVALID;
  }
  std::string why;
  st = gmmsp::net_reserve(n, 1, c->g, &why);
  if (st != GMMSP_OK) {
    c->err = why;  // the network's failure: the context stays usable
    return st;
  }
  GM_CHECK(c, gmmsp::net_enqueue_init(n, c->lab, nullptr, 1, c->g, c->p.lambda_c, c->p.eps_s, c->p.eps_c, c->theta, c->gp,
                                      c->counters, c->stream));
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_stats(gmmsp_ctx c, long long* dead, long long* raised_s, long long* raised_c) {
  if (!c) return GMMSP_E_INVALID;
  unsigned long long cnt[gmmsp::CNT_N];
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  GM_CHECK(c, cudaMemcpy(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  if (dead) *dead = (long long)cnt[gmmsp::CNT_DEAD];
  if (raised_s) *raised_s = (long long)cnt[gmmsp::CNT_RAISED_S];
  if (raised_c) *raised_c = (long long)cnt[gmmsp::CNT_RAISED_C];
  return GMMSP_OK;
}

gmmsp_status gmmsp_profile_kernel(gmmsp_ctx c, int which, int reps, int32_t* labels_dev,
                                  void* flush_dev, unsigned long long flush_bytes, double* avg_ms) {
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (reps < 1 || !avg_ms ||
      (which != GMMSP_KERNEL_EM_PASS && which != GMMSP_KERNEL_LABELS && which != GMMSP_KERNEL_FINALIZE) ||
      (which == GMMSP_KERNEL_LABELS && !labels_dev))
    return fail(c, GMMSP_E_INVALID, "bad profile arguments");
  const size_t th_bytes = size_t(c->g.K) * gmmsp::kTheta * sizeof(double);
  const size_t gp_bytes = size_t(c->g.K) * gmmsp::kGP * sizeof(float);
  void* save = nullptr;
  if (which == GMMSP_KERNEL_FINALIZE) {
    // The finalize rewrites theta from the partial sums; keep a copy of theta
    // and the packed coefficients and put them back before every launch.
    GM_CHECK(c, cudaMalloc(&save, th_bytes + gp_bytes));
    GM_CHECK(c, cudaMemcpyAsync(save, c->theta, th_bytes, cudaMemcpyDeviceToDevice, c->stream));
    GM_CHECK(c, cudaMemcpyAsync(static_cast<char*>(save) + th_bytes, c->gp, gp_bytes,
                                cudaMemcpyDeviceToDevice, c->stream));
  }
  std::vector<cudaEvent_t> ev(2 * size_t(reps), nullptr);
  gmmsp_status out = GMMSP_OK;
  for (auto& e : ev)
    if (out == GMMSP_OK && cudaEventCreate(&e) != cudaSuccess) out = fail(c, GMMSP_E_CUDA, "cudaEventCreate");
  for (int r = 0; r < reps && out == GMMSP_OK; ++r) {
    cudaError_t e = cudaSuccess;
    if (save) {
      e = cudaMemcpyAsync(c->theta, save, th_bytes, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->gp, static_cast<char*>(save) + th_bytes, gp_bytes, cudaMemcpyDeviceToDevice,
                            c->stream);
    }
    if (e == cudaSuccess && flush_dev && flush_bytes) e = cudaMemsetAsync(flush_dev, r & 0xff, flush_bytes, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * r], c->stream);
    if (e == cudaSuccess) {
      if (which == GMMSP_KERNEL_EM_PASS)
        e = gmmsp::launch_em_pass(gmmsp::LabPlanar{c->lab, (long long)c->g.W * c->g.H, c->g.W}, c->g, c->gp, c->partials, c->p.precision, c->wpc, c->stream);
      else if (which == GMMSP_KERNEL_LABELS)
        e = gmmsp::launch_label_pass(gmmsp::LabPlanar{c->lab, (long long)c->g.W * c->g.H, c->g.W}, c->g, c->gp, labels_dev, c->cell_ll, c->stream);
      else
        e = gmmsp::launch_finalize(c->g, c->partials, c->theta, c->gp, c->p.eps_s, c->p.eps_c, nullptr,
                                   c->ws, c->ticket, c->counters, c->p.precision, c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 * r + 1], c->stream);
    if (e != cudaSuccess) out = cuda_fail(c, e, "profile launch");
  }
  if (out == GMMSP_OK) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    double sum = 0.0;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
      sum += ms;
    }
    if (e != cudaSuccess) out = cuda_fail(c, e, "profile timing");
    else *avg_ms = sum / reps;
  }
  if (save) {
    cudaMemcpyAsync(c->theta, save, th_bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->gp, static_cast<char*>(save) + th_bytes, gp_bytes, cudaMemcpyDeviceToDevice,
                    c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(save);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return out;
}

gmmsp_status gmmsp_bounds_status(int* checked, unsigned long long* first_violation) {
#ifdef GMMSP_CHECK_BOUNDS
  if (checked) *checked = 1;
  if (cudaDeviceSynchronize() != cudaSuccess) return GMMSP_E_CUDA;
  unsigned long long w[3] = {0ull, 0ull, 0ull};
  if (gmmsp::bounds_take_em(&w[0]) != cudaSuccess || gmmsp::bounds_take_prep(&w[1]) != cudaSuccess ||
      gmmsp::bounds_take_cnn(&w[2]) != cudaSuccess)
    return GMMSP_E_CUDA;
  if (first_violation) *first_violation = w[0] ? w[0] : (w[1] ? w[1] : w[2]);
#else
  if (checked) *checked = 0;
  if (first_violation) *first_violation = 0ull;
#endif
  return GMMSP_OK;
}

gmmsp_status gmmsp_set_launch(gmmsp_ctx c, int warps_per_cell) {
  if (!c) return GMMSP_E_INVALID;
  if (warps_per_cell != 1 && warps_per_cell != 2 && warps_per_cell != 4)
    return fail(c, GMMSP_E_INVALID, "warps_per_cell must be 1, 2 or 4");
  if (warps_per_cell != c->wpc) free_graph(c);
  c->wpc = warps_per_cell;
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_launch(gmmsp_ctx c, int* warps_per_cell) {
  if (!c || !warps_per_cell) return GMMSP_E_INVALID;
  *warps_per_cell = c->wpc;
  return GMMSP_OK;
}

gmmsp_status gmmsp_autotune(gmmsp_ctx c, int reps, int* best, double* times_ms) {
  gmmsp_status st = check_ready(c);
  if (st != GMMSP_OK) return st;
  if (reps < 1) return fail(c, GMMSP_E_INVALID, "reps < 1");
  const int cand[3] = {1, 2, 4};
  const int keep = c->wpc;
  double best_ms = 1e30;
  int best_w = keep;
  for (int i = 0; i < 3; ++i) {
    c->wpc = cand[i];
    double ms = 0.0;
    st = gmmsp_profile_kernel(c, GMMSP_KERNEL_EM_PASS, reps + 1, nullptr, nullptr, 0, &ms);
    if (st != GMMSP_OK) { c->wpc = keep; return st; }
    if (times_ms) times_ms[i] = ms;
    if (ms < best_ms) { best_ms = ms; best_w = cand[i]; }
  }
  c->wpc = keep;
  st = gmmsp_set_launch(c, best_w);
  if (best) *best = best_w;
  return st;
}

gmmsp_status gmmsp_set_timing(gmmsp_ctx c, int enable) {
  if (!c) return GMMSP_E_INVALID;
  if (bool(enable) != c->timing) free_graph(c);
  c->timing = enable != 0;
  c->tev_used = 0;
  return GMMSP_OK;
}

gmmsp_status gmmsp_get_timing(gmmsp_ctx c, double* ms, int cap, int* n) {
  if (!c || !n || (cap > 0 && !ms)) return GMMSP_E_INVALID;
  GM_CHECK(c, cudaStreamSynchronize(c->stream));
  const int m = c->tev_used > 0 ? c->tev_used - 1 : 0;
  *n = m;
  for (int i = 0; i < m && i < cap; ++i) {
    float t = 0.f;
    GM_CHECK(c, cudaEventElapsedTime(&t, c->tev[i], c->tev[i + 1]));
    ms[i] = t;
  }
  return GMMSP_OK;
}

void gmmsp_destroy(gmmsp_ctx c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_graph(c);
  free_timing(c);
  if (c->slab) cudaFree(c->slab);
  if (c->conn.ptr) cudaFree(c->conn.ptr);
  delete c;
}

}  // extern "C"
