// gmmsp_segment_lab_noalloc: the whole EM pipeline on a caller's CIELAB image
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want
// superpixels: code running inside a memory pool that owns all device memory
// (a framework's caching allocator, a fixed real-time budget), code that
// must not synchronise the device (cudaMalloc/cudaFree can), or plug-ins that
// are only handed input and output buffers.  For them this entry point keeps
// its working memory (theta, the packed E-step coefficients, the per-cell
// partial sums and a few counters) in one file-scope __device__ array of fixed
// size, GMMSP_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library
// holds until the process exits.  The caller passes the image and the label
// output; nothing is allocated or freed.
//
// The kernels are the ones gmmsp_segment runs, instantiated to read the
// caller's (L, a, b) float32 rows directly instead of the context's planar
// copy of the image, so the results are those of gmmsp_init with
// GMMSP_LAB32 input followed by gmmsp_em_iters and gmmsp_labels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "../../include/gmmsp.h"
#include "gmmsp_internal.cuh"

namespace {

using gmmsp::Geom;

constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array (byte offsets).
constexpr size_t kOffTheta = 0;
constexpr size_t kOffGp = kOffTheta + up(size_t(GMMSP_NOALLOC_MAX_CELLS) * gmmsp::kTheta * sizeof(double));
constexpr size_t kOffPart = kOffGp + up(size_t(GMMSP_NOALLOC_MAX_CELLS) * gmmsp::kGP * sizeof(float));
constexpr size_t kOffCellLl = kOffPart + up(size_t(GMMSP_NOALLOC_MAX_CELLS) * gmmsp::kPartStride * sizeof(float));
constexpr size_t kOffLlk = kOffCellLl + up(size_t(GMMSP_NOALLOC_MAX_CELLS) * sizeof(double));
constexpr size_t kOffWs = kOffLlk + up(sizeof(double));
constexpr size_t kOffTicket = kOffWs + up((GMMSP_NOALLOC_MAX_CELLS / 4 + 2) * sizeof(double));
constexpr size_t kOffCounters = kOffTicket + up(sizeof(unsigned));
constexpr size_t kScratchBytes = kOffCounters + up(sizeof(unsigned long long) * gmmsp::CNT_N);
static_assert(kScratchBytes <= GMMSP_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented size");

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol: its device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GMMSP_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

void set_err(char* err, int err_len, const char* msg) {
  if (err && err_len > 0) snprintf(err, size_t(err_len), "%s", msg);
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Eq. (vxy)/(nxyK) on the host, as for a context.
bool grid_of(int W, int H, int K_req, int spacing, Geom* g) {
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
  g->W = W; g->H = H; g->v = int(v);
  g->nx = int(W / v); g->ny = int(H / v);
  g->K = g->nx * g->ny;
  g->ncx = int((W + v - 1) / v);
  g->ncy = int((H + v - 1) / v);
  g->ncells = g->ncx * g->ncy;
  return g->nx >= 1 && g->ny >= 1;
}

}  // namespace

extern "C" gmmsp_status gmmsp_segment_lab_noalloc(const float* lab_dev, int width, int height,
                                                  int pitch_bytes, const gmmsp_params* p, int iters,
                                                  int32_t* labels_dev, void* stream, char* err,
                                                  int err_len) {
  set_err(err, err_len, "");
  if (!p || !lab_dev || !labels_dev || width < 1 || height < 1) {
    set_err(err, err_len, "null pointer or empty image");
    return GMMSP_E_INVALID;
  }
  if (pitch_bytes < 12LL * width || pitch_bytes % 4 != 0 || (uintptr_t)lab_dev % 4 != 0) {
    set_err(err, err_len, "pitch must be >= 12 * width bytes and 4-byte aligned");
    return GMMSP_E_INVALID;
  }
  if (p->precision != GMMSP_PREC_MIXED || p->colour_model != GMMSP_COLOUR_FULL || !(p->eps_s > 0.f) ||
      !(p->eps_c > 0.f) || !(p->lambda_c > 0.f) || !isfinite(p->eps_s) || !isfinite(p->eps_c) ||
      !isfinite(p->lambda_c) || iters < 0 || (p->spacing <= 0 && p->K <= 0)) {
    set_err(err, err_len,
            "invalid parameters (mixed precision and the full colour model only; eps, lambda_c finite and > 0; "
            "iters >= 0)");
    return GMMSP_E_INVALID;
  }
  Geom g;
  if (!grid_of(width, height, p->K, p->spacing, &g)) {
    set_err(err, err_len, "empty seed grid for this size and spacing/K");
    return GMMSP_E_INVALID;
  }
  if (g.ncells > GMMSP_NOALLOC_MAX_CELLS) {
    char msg[160];
    snprintf(msg, sizeof(msg), "grid has %d cells; the allocation-free path holds at most %d "
             "(ceil(W/v) * ceil(H/v))", g.ncells, GMMSP_NOALLOC_MAX_CELLS);
    set_err(err, err_len, msg);
    return GMMSP_E_INVALID;
  }
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(base);
  double* theta = reinterpret_cast<double*>(b + kOffTheta);
  float* gp = reinterpret_cast<float*>(b + kOffGp);
  float* partials = reinterpret_cast<float*>(b + kOffPart);
  double* ws = reinterpret_cast<double*>(b + kOffWs);
  unsigned* ticket = reinterpret_cast<unsigned*>(b + kOffTicket);
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(b + kOffCounters);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const gmmsp::LabPitched src{reinterpret_cast<const char*>(lab_dev), pitch_bytes};
  const int wpc = g.ncells >= 152 * 16 ? 1 : (2 * g.ncells >= 152 * 16 ? 2 : 4);

  // The previous call's contents stay in the array: reset what must start at zero.
  e = cudaMemsetAsync(b + kOffTicket, 0, kScratchBytes - kOffTicket, s);
  if (e == cudaSuccess) e = gmmsp::launch_init_theta(src, g, p->lambda_c, theta, gp, s);
  for (int t = 0; t < iters && e == cudaSuccess; ++t) {
    e = gmmsp::launch_em_pass(src, g, gp, partials, GMMSP_PREC_MIXED, wpc, s);
    if (e == cudaSuccess)
      e = gmmsp::launch_finalize(g, partials, theta, gp, p->eps_s, p->eps_c, nullptr, ws, ticket, counters,
                                 GMMSP_PREC_MIXED, s);
  }
  if (e == cudaSuccess) e = gmmsp::launch_label_pass(src, g, gp, labels_dev, nullptr, s);
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return GMMSP_E_CUDA;
  }
  return GMMSP_OK;
}
