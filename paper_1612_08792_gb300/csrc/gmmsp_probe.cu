// Arithmetic-rate probes (declared in include/gmmsp_probe.h).  Each kernel
// runs a fixed number of independent dependency chains per thread so that
// the pipe, not latency, limits it; a single-thread kernel measures the
// latency of a dependent chain with clock64().
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include "../../include/gmmsp_probe.h"

namespace {

constexpr int kChains = 8;

__global__ void k_ffma(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 1e-3f + j;
  const float b = 0.9999f, c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same chains as k_ffma, two per packed fma.rn.f32x2 (sm_100 and later):
// half the instructions for the same number of FMAs.
__global__ void k_ffma2(float* out, int iters) {
  float2 a[kChains / 2];
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) a[j] = make_float2(threadIdx.x * 1e-3f + 2 * j, threadIdx.x * 1e-3f + 2 * j + 1);
  const float2 b = make_float2(0.9999f, 0.9999f), c = make_float2(1e-4f, 1e-4f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains / 2; ++j) a[j] = __ffma2_rn(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) s += a[j].x + a[j].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, int iters, int active_lanes) {
  if ((threadIdx.x & 31) >= active_lanes) return;
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 1e-3 + j;
  const double b = 0.9999, c = 1e-4;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = -0.001f * (threadIdx.x & 63) - 0.1f * j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[j]));
      a[j] = -y;  // stays in (-1, 0)
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_latency(double* out, long long* clk, int iters) {
  float f = out[0] > 1e300 ? 2.f : 1.0001f;
  double d = out[1] > 1e300 ? 2.0 : 1.0000001;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) f = fmaf(f, 0.99999f, 1e-6f);
  const long long t1 = clock64();
  for (int i = 0; i < iters; ++i) d = fma(d, 0.9999999, 1e-9);
  const long long t2 = clock64();
  out[2] = f;
  out[3] = d;
  clk[0] = t1 - t0;
  clk[1] = t2 - t1;
}

// Shared-memory load patterns of the EM kernels, one kernel per pattern so
// that a profiler attributes the l1tex shared-memory wavefronts of each
// (wavefronts per instruction = l1tex__data_pipe_lsu_wavefronts_mem_shared_op_ld
// / smsp__inst_executed_op_shared_ld).  Lanes 27-31 repeat lane 0, as the M
// part's idle lanes would.  Every index stays inside the 4096-float buffer:
// w = warp * 1024 with warp < 4, and each pattern adds at most 555.
//   0  16-byte load, one address for the warp (a candidate's coefficients)
//   1  8-byte load, one address
//   2  4-byte load, one address
//   3  16-byte load, three addresses 16 bytes apart
//   4  4-byte load, rows of 12 floats: pixel l / 9, slot l % 9 (the posteriors)
//   5  the same with rows of 11 floats
//   6  8-byte load, three addresses in rows of 12 floats
//   7  16-byte load, eight consecutive addresses
//   8  16-byte load, 32 consecutive addresses
//   9  16-byte load, three addresses in rows of 12 floats (a pixel's colour)
constexpr int kSmemIters = 1024;
template <int MODE>
__global__ void __launch_bounds__(128) k_lds_pattern(float* out) {
  __shared__ __align__(16) float buf[4096];
  for (int i = threadIdx.x; i < 4096; i += 128) buf[i] = float(i) * 1e-3f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ms = lane < 27 ? lane % 9 : 0, ph = lane < 27 ? lane / 9 : 0;
  const float* w = buf + warp * 1024;
  float acc = 0.f;
#pragma unroll 4
  for (int i = 0; i < kSmemIters; ++i) {
    const int o = (i * 20) & 511;  // a multiple of 4 floats, varying
    if (MODE == 0) { const float4 v = *reinterpret_cast<const float4*>(w + o); acc += v.x + v.y + v.z + v.w; }
    if (MODE == 1) { const float2 v = *reinterpret_cast<const float2*>(w + o); acc += v.x + v.y; }
    if (MODE == 2) acc += w[o];
    if (MODE == 3) { const float4 v = *reinterpret_cast<const float4*>(w + o + 4 * ph); acc += v.x + v.y + v.z + v.w; }
    if (MODE == 4) acc += w[(o & 255) + 12 * ph + ms];
    if (MODE == 5) acc += w[(o & 255) + 11 * ph + ms];
    if (MODE == 6) { const float2 v = *reinterpret_cast<const float2*>(w + o + 12 * ph + 10); acc += v.x + v.y; }
    if (MODE == 7) { const float4 v = *reinterpret_cast<const float4*>(w + o + 4 * (lane & 7)); acc += v.x + v.y + v.z + v.w; }
    if (MODE == 8) { const float4 v = *reinterpret_cast<const float4*>(w + ((o + 4 * lane) & 1023)); acc += v.x + v.y + v.z + v.w; }
    if (MODE == 9) { const float4 v = *reinterpret_cast<const float4*>(w + (o & 255) + 12 * ph); acc += v.x + v.y + v.z + v.w; }
  }
  out[blockIdx.x * 128 + threadIdx.x] = acc;
}

template <typename F>
float time_ms(F launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();  // warm-up
  cudaEventRecord(a);
  launch();
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace

extern "C" int gmmsp_probe_peaks(gmmsp_peaks* out, char* err, int err_len) {
  if (!out) return 1;
  memset(out, 0, sizeof(*out));
  int dev = 0;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
  int clk_khz = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) {
    if (err && err_len > 0) snprintf(err, err_len, "%s", cudaGetErrorString(e));
    return 2;
  }
  out->sm_count = prop.multiProcessorCount;
  out->clock_mhz = clk_khz / 1000;
  const int blocks = prop.multiProcessorCount * 8, threads = 256;
  void* buf = nullptr;
  e = cudaMalloc(&buf, size_t(blocks) * threads * sizeof(double) + 64);
  if (e != cudaSuccess) {
    if (err && err_len > 0) snprintf(err, err_len, "%s", cudaGetErrorString(e));
    return 2;
  }
  const int it32 = 256, it64 = 1024, itx = 4096;
  float ms = time_ms([&] { k_ffma<<<blocks, threads>>>((float*)buf, it32); });
  out->fp32_fma_tflops = double(blocks) * threads * it32 * 4 * kChains * 2 / (ms * 1e-3) / 1e12;
  ms = time_ms([&] { k_ffma2<<<blocks, threads>>>((float*)buf, it32); });
  out->fp32x2_fma_tflops = double(blocks) * threads * it32 * 4 * kChains * 2 / (ms * 1e-3) / 1e12;
  ms = time_ms([&] { k_dfma<<<blocks, threads>>>((double*)buf, it64, 32); });
  out->fp64_fma_tflops = double(blocks) * threads * it64 * kChains * 2 / (ms * 1e-3) / 1e12;
  ms = time_ms([&] { k_dfma<<<blocks, threads>>>((double*)buf, it64, 1); });
  out->fp64_fma_tflops_lane1 = double(blocks) * (threads / 32) * it64 * kChains * 2 / (ms * 1e-3) / 1e12;
  ms = time_ms([&] { k_ex2<<<blocks, threads>>>((float*)buf, itx); });
  out->mufu_ex2_tops = double(blocks) * threads * itx * kChains / (ms * 1e-3) / 1e12;
  e = cudaMemset(buf, 0, 64);
  long long* clk = reinterpret_cast<long long*>(static_cast<char*>(buf) + 32);
  const int itl = 1 << 16;
  if (e == cudaSuccess) {
    k_latency<<<1, 1>>>((double*)buf, clk, itl);
    e = cudaDeviceSynchronize();
  }
  long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
  out->fp32_fma_latency_clk = double(h[0]) / itl;
  out->fp64_fma_latency_clk = double(h[1]) / itl;
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(buf);
  if (e != cudaSuccess) {
    if (err && err_len > 0) snprintf(err, err_len, "%s", cudaGetErrorString(e));
    return 2;
  }
  return 0;
}

extern "C" int gmmsp_probe_smem_patterns(char* err, int err_len) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* out = nullptr;
  const int blocks = sms * 4;
  if (e == cudaSuccess) e = cudaMalloc(&out, size_t(blocks) * 128 * sizeof(float));
  if (e == cudaSuccess) {
    k_lds_pattern<0><<<blocks, 128>>>(out);
    k_lds_pattern<1><<<blocks, 128>>>(out);
    k_lds_pattern<2><<<blocks, 128>>>(out);
    k_lds_pattern<3><<<blocks, 128>>>(out);
    k_lds_pattern<4><<<blocks, 128>>>(out);
    k_lds_pattern<5><<<blocks, 128>>>(out);
    k_lds_pattern<6><<<blocks, 128>>>(out);
    k_lds_pattern<7><<<blocks, 128>>>(out);
    k_lds_pattern<8><<<blocks, 128>>>(out);
    k_lds_pattern<9><<<blocks, 128>>>(out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(out);
  }
  if (e != cudaSuccess) {
    if (err && err_len > 0) snprintf(err, err_len, "%s", cudaGetErrorString(e));
    return 2;
  }
  return 0;
}
