// Accuracy metrics of Sec. IV against a ground-truth segmentation
// (declared in include/gmmsp_metrics.h): boundary recall, the
// under-segmentation error of Eq. (ue) and the achievable segmentation
// accuracy of Eq. (asa).  Everything is integer counting, so the results are
// exact and independent of the order of the atomics:
//   k_overlap     the overlap table |s_k & s_g| (dense K x G, integer atomics)
//   k_sp_boundary superpixel boundary pixels (a 4-neighbour with another label)
//   k_recall      ground-truth boundary pixels, and those with a superpixel
//                 boundary pixel within the Chebyshev radius
//   k_table       per superpixel |s_k|, max_g |s_k & s_g| and the Eq. (ue)
//                 terms, summed per block and added with 64-bit atomics
// Every kernel takes a table of images and blockIdx.y as the image, so a
// batch of images is four launches, one allocation and one synchronisation.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_metrics.h"
#include "gmmsp_internal.cuh"

namespace gmmsp {
namespace metrics {

enum : int { C_BAD = 0, C_BR_REC = 1, C_BR_TOT = 2, C_UE = 3, C_ASA = 4, C_N = 5 };

// One image of a call and its scratch.
struct MImg {
  const int32_t* labels;     // W H superpixel labels in [0, K)
  const int32_t* gt;         // W H ground-truth ids in [0, G)
  int W, H, K, G;
  unsigned* table;           // K x G overlap counts
  uint8_t* sb;               // W H superpixel boundary flags
  unsigned long long* cnt;   // C_N counters
};

#define FOR_IMAGE_PIXELS(im, i)                                                                    \
  const MImg im = imgs[blockIdx.y];                                                                \
  const long long im##_N = (long long)im.W * im.H;                                                 \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < im##_N;                 \
       i += (long long)gridDim.x * blockDim.x)

__global__ void k_overlap(const MImg* __restrict__ imgs) {
  unsigned bad = 0;
  const MImg* me = imgs + blockIdx.y;
  FOR_IMAGE_PIXELS(im, i) {
    const int k = im.labels[i], g = im.gt[i];
    if (k >= 0 && k < im.K && g >= 0 && g < im.G) atomicAdd(im.table + (long long)k * im.G + g, 1u);
    else ++bad;
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(me->cnt + C_BAD, (unsigned long long)bad);
}

__device__ __forceinline__ bool is_boundary(const int32_t* __restrict__ m, int W, int H, int x, int y) {
  const int32_t v = m[(long long)y * W + x];
  return (x > 0 && m[(long long)y * W + x - 1] != v) || (x + 1 < W && m[(long long)y * W + x + 1] != v) ||
         (y > 0 && m[(long long)(y - 1) * W + x] != v) || (y + 1 < H && m[(long long)(y + 1) * W + x] != v);
}

__global__ void k_sp_boundary(const MImg* __restrict__ imgs) {
  FOR_IMAGE_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    im.sb[i] = is_boundary(im.labels, im.W, im.H, x, y) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) k_recall(const MImg* __restrict__ imgs, int radius) {
  unsigned rec = 0, tot = 0;
  const MImg* me = imgs + blockIdx.y;
  FOR_IMAGE_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    if (!is_boundary(im.gt, im.W, im.H, x, y)) continue;
    ++tot;
    bool hit = false;
    for (int yy = max(0, y - radius); yy <= min(im.H - 1, y + radius) && !hit; ++yy)
      for (int xx = max(0, x - radius); xx <= min(im.W - 1, x + radius); ++xx)
        if (im.sb[(long long)yy * im.W + xx]) {
          hit = true;
          break;
        }
    rec += hit;
  }
  rec = __reduce_add_sync(0xffffffffu, rec);
  tot = __reduce_add_sync(0xffffffffu, tot);
  if ((threadIdx.x & 31) == 0) {
    if (rec) atomicAdd(me->cnt + C_BR_REC, (unsigned long long)rec);
    if (tot) atomicAdd(me->cnt + C_BR_TOT, (unsigned long long)tot);
  }
}

__global__ void __launch_bounds__(256) k_table(const MImg* __restrict__ imgs, double eps) {
  const MImg im = imgs[blockIdx.y];
  unsigned long long ue = 0, asa = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < im.K; k += gridDim.x * blockDim.x) {
    const unsigned* row = im.table + (long long)k * im.G;
    unsigned long long size = 0;
    unsigned best = 0;
    for (int g = 0; g < im.G; ++g) {
      size += row[g];
      best = max(best, row[g]);
    }
    asa += best;
    const double lim = eps * double(size);
    for (int g = 0; g < im.G; ++g)
      if (double(row[g]) > lim) ue += size;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ue += __shfl_xor_sync(0xffffffffu, ue, o);
    asa += __shfl_xor_sync(0xffffffffu, asa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ue) atomicAdd(im.cnt + C_UE, ue);
    if (asa) atomicAdd(im.cnt + C_ASA, asa);
  }
}

}  // namespace metrics
}  // namespace gmmsp

using namespace gmmsp::metrics;

extern "C" gmmsp_status gmmsp_segmentation_metrics_many(int n, const int32_t* const* labels_dev,
                                                        const int32_t* const* gt_dev, const int* W, const int* H,
                                                        const int* K, const int* G, int radius, double eps,
                                                        gmmsp_seg_metrics* out, void* stream) {
  GMMSP_NVTX("gmmsp_segmentation_metrics_many");
  if (n < 1 || n > 65535 || !labels_dev || !gt_dev || !W || !H || !K || !G || !out || radius < 0 || radius > 64 ||
      !(eps >= 0.0 && eps < 1.0))
    return GMMSP_E_INVALID;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  std::vector<MImg> host(n);
  std::vector<size_t> o_table(n), o_sb(n);
  size_t off = up(sizeof(MImg) * n);                      // image table first
  const size_t o_cnt = off;
  off += up(sizeof(unsigned long long) * C_N * n);
  long long maxN = 0, maxK = 0;
  for (int i = 0; i < n; ++i) {
    if (!labels_dev[i] || !gt_dev[i] || W[i] < 1 || H[i] < 1 || K[i] < 1 || G[i] < 1) return GMMSP_E_INVALID;
    const long long N = (long long)W[i] * H[i], cells = (long long)K[i] * G[i];
    if (cells > (1LL << 31)) return GMMSP_E_INVALID;
    o_table[i] = off;
    off += up(size_t(cells) * 4);
    o_sb[i] = off;
    off += up(size_t(N));
    maxN = std::max(maxN, N);
    maxK = std::max<long long>(maxK, K[i]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* slab = nullptr;
  cudaError_t e = cudaMalloc(&slab, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(slab);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b + o_cnt);
  for (int i = 0; i < n; ++i)
    host[i] = MImg{labels_dev[i], gt_dev[i], W[i], H[i], K[i], G[i], reinterpret_cast<unsigned*>(b + o_table[i]),
                   reinterpret_cast<uint8_t*>(b + o_sb[i]), cnt + size_t(C_N) * i};
  MImg* table = reinterpret_cast<MImg*>(b);
  std::vector<unsigned long long> hc(size_t(C_N) * n, 0ull);
  // pixel kernels: enough blocks per image to fill the machine across the images
  const unsigned per = unsigned(std::max<long long>(1, std::min<long long>((maxN + 255) / 256, (152LL * 16 + n - 1) / n)));
  const unsigned perk = unsigned(std::max<long long>(1, std::min<long long>((maxK + 255) / 256, (152LL * 16 + n - 1) / n)));
  do {
    if ((e = cudaMemcpyAsync(table, host.data(), sizeof(MImg) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b + o_cnt, 0, off - o_cnt, s)) != cudaSuccess) break;  // counters and tables
    k_overlap<<<dim3(per, n), 256, 0, s>>>(table);
    k_sp_boundary<<<dim3(per, n), 256, 0, s>>>(table);
    k_recall<<<dim3(per, n), 256, 0, s>>>(table, radius);
    k_table<<<dim3(perk, n), 256, 0, s>>>(table, eps);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long) * C_N * n, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      break;
    e = cudaStreamSynchronize(s);
  } while (false);
  cudaFree(slab);
  if (e != cudaSuccess) return GMMSP_E_CUDA;
  gmmsp_status st = GMMSP_OK;
  for (int i = 0; i < n; ++i) {
    const unsigned long long* h = hc.data() + size_t(C_N) * i;
    const double N = double((long long)W[i] * H[i]);
    gmmsp_seg_metrics& o = out[i];
    if (h[C_BAD]) st = GMMSP_E_INVALID;
    o.br_recovered = (long long)h[C_BR_REC];
    o.br_total = (long long)h[C_BR_TOT];
    o.ue_sum = (long long)h[C_UE];
    o.asa_sum = (long long)h[C_ASA];
    o.br = o.br_total ? double(o.br_recovered) / double(o.br_total) : 1.0;
    o.ue = double(o.ue_sum) / N - 1.0;
    o.asa = double(o.asa_sum) / N;
  }
  return st;
}

extern "C" gmmsp_status gmmsp_segmentation_metrics(const int32_t* labels_dev, const int32_t* gt_dev, int W, int H,
                                                   int K, int G, int radius, double eps,
                                                   gmmsp_seg_metrics* out, void* stream) {
  if (!labels_dev || !gt_dev || !out) return GMMSP_E_INVALID;
  return gmmsp_segmentation_metrics_many(1, &labels_dev, &gt_dev, &W, &H, &K, &G, radius, eps, out, stream);
}
