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
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_metrics.h"

namespace gmmsp {
namespace metrics {

enum : int { C_BAD = 0, C_BR_REC = 1, C_BR_TOT = 2, C_UE = 3, C_ASA = 4, C_N = 5 };

__global__ void k_overlap(const int32_t* __restrict__ labels, const int32_t* __restrict__ gt, long long N, int K,
                          int G, unsigned* __restrict__ table, unsigned long long* __restrict__ cnt) {
  unsigned bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int k = labels[i], g = gt[i];
    if (k >= 0 && k < K && g >= 0 && g < G) atomicAdd(table + (long long)k * G + g, 1u);
    else ++bad;
  }
  bad = __reduce_add_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(cnt + C_BAD, (unsigned long long)bad);
}

__device__ __forceinline__ bool is_boundary(const int32_t* __restrict__ m, int W, int H, int x, int y) {
  const int32_t v = m[(long long)y * W + x];
  return (x > 0 && m[(long long)y * W + x - 1] != v) || (x + 1 < W && m[(long long)y * W + x + 1] != v) ||
         (y > 0 && m[(long long)(y - 1) * W + x] != v) || (y + 1 < H && m[(long long)(y + 1) * W + x] != v);
}

__global__ void k_sp_boundary(const int32_t* __restrict__ labels, int W, int H, uint8_t* __restrict__ sb) {
  const long long N = (long long)W * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int y = int(i / W), x = int(i - (long long)y * W);
    sb[i] = is_boundary(labels, W, H, x, y) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) k_recall(const int32_t* __restrict__ gt, const uint8_t* __restrict__ sb,
                                                int W, int H, int radius, unsigned long long* __restrict__ cnt) {
  const long long N = (long long)W * H;
  unsigned rec = 0, tot = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int y = int(i / W), x = int(i - (long long)y * W);
    if (!is_boundary(gt, W, H, x, y)) continue;
    ++tot;
    bool hit = false;
    for (int yy = max(0, y - radius); yy <= min(H - 1, y + radius) && !hit; ++yy)
      for (int xx = max(0, x - radius); xx <= min(W - 1, x + radius); ++xx)
        if (sb[(long long)yy * W + xx]) {
          hit = true;
          break;
        }
    rec += hit;
  }
  rec = __reduce_add_sync(0xffffffffu, rec);
  tot = __reduce_add_sync(0xffffffffu, tot);
  if ((threadIdx.x & 31) == 0) {
    if (rec) atomicAdd(cnt + C_BR_REC, (unsigned long long)rec);
    if (tot) atomicAdd(cnt + C_BR_TOT, (unsigned long long)tot);
  }
}

__global__ void __launch_bounds__(256) k_table(const unsigned* __restrict__ table, int K, int G, double eps,
                                               unsigned long long* __restrict__ cnt) {
  unsigned long long ue = 0, asa = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const unsigned* row = table + (long long)k * G;
    unsigned long long size = 0;
    unsigned best = 0;
    for (int g = 0; g < G; ++g) {
      size += row[g];
      best = max(best, row[g]);
    }
    asa += best;
    const double lim = eps * double(size);
    for (int g = 0; g < G; ++g)
      if (double(row[g]) > lim) ue += size;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ue += __shfl_xor_sync(0xffffffffu, ue, o);
    asa += __shfl_xor_sync(0xffffffffu, asa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ue) atomicAdd(cnt + C_UE, ue);
    if (asa) atomicAdd(cnt + C_ASA, asa);
  }
}

int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  return int(std::max<long long>(1, std::min<long long>(b, 152LL * 16)));
}

}  // namespace metrics
}  // namespace gmmsp

using namespace gmmsp::metrics;

extern "C" gmmsp_status gmmsp_segmentation_metrics(const int32_t* labels_dev, const int32_t* gt_dev, int W, int H,
                                                   int K, int G, int radius, double eps,
                                                   gmmsp_seg_metrics* out, void* stream) {
  if (!labels_dev || !gt_dev || !out || W < 1 || H < 1 || K < 1 || G < 1 || radius < 0 || radius > 64 ||
      !(eps >= 0.0 && eps < 1.0))
    return GMMSP_E_INVALID;
  const long long N = (long long)W * H;
  const long long cells = (long long)K * G;
  if (cells > (1LL << 31)) return GMMSP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t o_table = 0;
  const size_t o_sb = (size_t(cells) * 4 + 255) & ~size_t(255);
  const size_t o_cnt = (o_sb + size_t(N) + 255) & ~size_t(255);
  const size_t bytes = o_cnt + sizeof(unsigned long long) * C_N;
  void* slab = nullptr;
  cudaError_t e = cudaMalloc(&slab, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(slab);
  unsigned* table = reinterpret_cast<unsigned*>(b + o_table);
  uint8_t* sb = reinterpret_cast<uint8_t*>(b + o_sb);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b + o_cnt);
  unsigned long long host[C_N] = {};
  e = cudaMemsetAsync(table, 0, size_t(cells) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(host), s);
  if (e == cudaSuccess) {
    k_overlap<<<grid_for(N, 256), 256, 0, s>>>(labels_dev, gt_dev, N, K, G, table, cnt);
    k_sp_boundary<<<grid_for(N, 256), 256, 0, s>>>(labels_dev, W, H, sb);
    k_recall<<<grid_for(N, 256), 256, 0, s>>>(gt_dev, sb, W, H, radius, cnt);
    k_table<<<grid_for(K, 256), 256, 0, s>>>(table, K, G, eps, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, cnt, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(slab);
  if (e != cudaSuccess) return GMMSP_E_CUDA;
  if (host[C_BAD]) return GMMSP_E_INVALID;
  out->br_recovered = (long long)host[C_BR_REC];
  out->br_total = (long long)host[C_BR_TOT];
  out->ue_sum = (long long)host[C_UE];
  out->asa_sum = (long long)host[C_ASA];
  out->br = out->br_total ? double(out->br_recovered) / double(out->br_total) : 1.0;
  out->ue = double(out->ue_sum) / double(N) - 1.0;
  out->asa = double(out->asa_sum) / double(N);
  return GMMSP_OK;
}
