// Connectivity post-processing (Algorithm 1, step 8; Sec. III-D), declared in
// include/gmmsp_conn.h.  The paper sorts the isolated superpixels by size
// and merges, one after the other, those smaller than a quarter of the
// desired size into the neighbouring superpixel nearest in colour, adding
// the source's size to the destination's.  Readings (the same as the
// oracle's): an isolated superpixel is a 4-connected component of one label;
// small means 4 K |c| < N; order (size, smallest pixel index); a group keeps
// the colour of the component that founded it (mean of its fixed-point
// colour sum); nearest = smallest squared CIELAB distance, ties to the
// smaller index; pixels take the label of their group's founder.
//
// Parallel form with the same result.  A large component is never a source,
// so its group and colour never change; two small components therefore only
// influence each other through a chain of adjacent small components.  The
// small components split into clusters (connected sets of the small-small
// adjacency), and the sequential rule restricted to one cluster, in the
// cluster's own (size, index) order, gives exactly what the sequential pass
// over the whole image gives there.  One thread runs each cluster.
//
// Kernels: union-find component labelling (k_cc_*), component sizes and
// colour sums (k_comp_stats), small-component indices (k_small_index), one
// edge walk (k_edges) three times -- small-small clusters, then the
// adjacency lists of the small components -- a block scan for the offsets,
// the cluster member lists (k_cluster_count / _fill), the per-cluster merge
// (k_cluster_merge) and the relabelling (k_relabel).
// Every loop over a parent chain or a retry is bounded; running out sets the
// error word (reported as GMMSP_E_TIMEOUT).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_conn.h"
#include "gmmsp_internal.cuh"

namespace gmmsp {
namespace conn {

constexpr int kMaxHops = 1 << 24;      // bound on any parent-chain walk or union retry
constexpr int kFixedShift = 20;        // colour sums in units of 2^-20
constexpr int kMaxCluster = 1 << 16;   // bound on the members one cluster thread sorts

struct Scratch {
  int* parent;                // per pixel: component union-find, then the component root
  int* size;                  // per root: component size
  long long* csum;            // per root: 3 fixed-point colour sums
  int* cpar;                  // per small root: cluster union-find over roots
  int* sid;                   // per root: index of the small component, or -1
  int* sroot;                 // per small index: its root
  int* deg;                   // per small index: adjacency count, then fill cursor
  int* aoff;                  // per small index + 1: adjacency offsets
  int* adj;                   // adjacency lists (roots of neighbouring components)
  int* cl_count;              // per small index: members of the cluster it roots, then fill cursor
  int* cl_off;                // per small index + 1: member offsets
  int* cl_mem;                // members (small indices), grouped by cluster
  int* gpar;                  // per root: merge union-find (group founder)
  int* gsize;                 // per root: group size
  int* next;                  // per small root: next member of its group, -1 at the end
  int* tail;                  // per small root founding a group: last member
  unsigned long long* cnt;    // counters: 0 small, 1 merged, 2 components, 3 edges, 4 error
  int* err;
};

__device__ __forceinline__ int find_root(const int* p, int x, int* err) {
  for (int h = 0; h < kMaxHops; ++h) {
    const int q = p[x];
    if (q == x) return x;
    x = q;
  }
  atomicExch(err, 1);
  return x;
}

// Lock-free union by the smaller index (atomicMin on the larger root): the
// final root of every set is its smallest member.
__device__ __forceinline__ void unite(int* p, int a, int b, int* err) {
  for (int h = 0; h < kMaxHops; ++h) {
    a = find_root(p, a, err);
    b = find_root(p, b, err);
    if (a == b) return;
    if (a < b) {
      const int old = atomicMin(p + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(p + a, b);
      if (old == a) return;
      a = old;
    }
  }
  atomicExch(err, 1);
}

__global__ void k_cc_init(int* __restrict__ p, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = int(i);
}

__global__ void k_cc_union(const int32_t* __restrict__ L, int W, int H, int* p, int* err) {
  const long long N = (long long)W * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int y = int(i / W), x = int(i - (long long)y * W);
    if (x + 1 < W && L[i] == L[i + 1]) unite(p, int(i), int(i + 1), err);
    if (y + 1 < H && L[i] == L[i + W]) unite(p, int(i), int(i + W), err);
  }
}

__global__ void k_cc_flatten(int* p, long long N, int* err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = find_root(p, int(i), err);
}

__global__ void k_comp_stats(const int* __restrict__ p, const float* __restrict__ lab, long long N,
                             int* __restrict__ size, long long* __restrict__ csum) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int r = p[i];
    atomicAdd(size + r, 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long f = llrint(double(lab[c * N + i]) * double(1 << kFixedShift));
      atomicAdd(reinterpret_cast<unsigned long long*>(csum + 3LL * r + c), (unsigned long long)f);
    }
  }
}

__device__ __forceinline__ bool small_size(long long s, int K, long long N) { return 4LL * K * s < N; }

// Small components get an index; every root starts its own group.
__global__ void k_small_index(const int* __restrict__ p, const int* __restrict__ size, long long N, int K,
                              int* __restrict__ sid, int* __restrict__ sroot, int* __restrict__ cpar,
                              int* __restrict__ gpar, int* __restrict__ gsize, int* __restrict__ next,
                              int* __restrict__ tail, unsigned long long* cnt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    sid[i] = -1;
    if (p[i] != int(i)) continue;
    atomicAdd(cnt + 2, 1ull);
    gpar[i] = int(i);
    gsize[i] = size[i];
    if (small_size(size[i], K, N)) {
      const int s = int(atomicAdd(cnt + 0, 1ull));
      sid[i] = s;
      sroot[s] = int(i);
      cpar[i] = int(i);
      next[i] = -1;
      tail[i] = int(i);
    }
  }
}

// Walks the 4-neighbour edges between different components; `mode` 0 unites
// small-small pairs into clusters, 1 counts each small side's adjacency, 2
// fills it.
__global__ void k_edges(const int* __restrict__ p, int W, int H, const int* __restrict__ sid, int* cpar,
                        int* deg, const int* __restrict__ aoff, int* __restrict__ adj, int mode, int* err) {
  const long long N = (long long)W * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int y = int(i / W), x = int(i - (long long)y * W);
    const int ri = p[i];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      long long j;
      if (d == 0) {
        if (x + 1 >= W) continue;
        j = i + 1;
      } else {
        if (y + 1 >= H) continue;
        j = i + W;
      }
      const int rj = p[j];
      if (ri == rj) continue;
      const int si = sid[ri], sj = sid[rj];
      if (mode == 0) {
        if (si >= 0 && sj >= 0) unite(cpar, ri, rj, err);
      } else if (mode == 1) {
        if (si >= 0) atomicAdd(deg + si, 1);
        if (sj >= 0) atomicAdd(deg + sj, 1);
      } else {
        if (si >= 0) adj[aoff[si] + atomicAdd(deg + si, 1)] = rj;
        if (sj >= 0) adj[aoff[sj] + atomicAdd(deg + sj, 1)] = ri;
      }
    }
  }
}

// Exclusive prefix sum of n ints into out[0..n] (one block; n up to a few million).
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int n, int* __restrict__ out) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int b = t * chunk, e = min(n, b + chunk);
  int s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the chunk sums
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t ? part[t - 1] : 0;
  for (int i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == 1023) out[n] = part[1023];
}

// Cluster root of every small component (flattened), member counts per cluster root.
__global__ void k_cluster_count(int* cpar, const int* __restrict__ sroot, const int* __restrict__ sid, int nsmall,
                                int* __restrict__ cl_count, int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsmall; s += gridDim.x * blockDim.x) {
    const int c = find_root(cpar, sroot[s], err);
    atomicAdd(cl_count + sid[c], 1);
  }
}

__global__ void k_cluster_fill(const int* cpar, const int* __restrict__ sroot, const int* __restrict__ sid, int nsmall,
                               const int* __restrict__ cl_off, int* cl_cur, int* __restrict__ cl_mem, int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsmall; s += gridDim.x * blockDim.x) {
    const int c = sid[find_root(cpar, sroot[s], err)];
    cl_mem[cl_off[c] + atomicAdd(cl_cur + c, 1)] = s;
  }
}

__device__ __forceinline__ double dist2(const long long* csum, const int* size, int a, int b) {
  double d = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double ma = double(csum[3LL * a + c]) / double(size[a]);
    const double mb = double(csum[3LL * b + c]) / double(size[b]);
    const double t = __dsub_rn(ma, mb);
    d = __dadd_rn(d, __dmul_rn(t, t));
  }
  return d;
}

// One thread per cluster: the sequential rule over the cluster's members in
// (size, root) order.
__global__ void k_cluster_merge(const int* __restrict__ sroot, int nsmall, const int* __restrict__ cpar,
                                const int* __restrict__ sid, const int* __restrict__ cl_off, int* cl_mem,
                                const int* __restrict__ size, const long long* __restrict__ csum,
                                const int* __restrict__ aoff, const int* __restrict__ adj, int* gpar, int* gsize,
                                int* next, int* tail, int K, long long N, unsigned long long* cnt, int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsmall; s += gridDim.x * blockDim.x) {
    const int r0 = sroot[s];
    if (cpar[r0] != r0) continue;  // not a cluster root
    int* mem = cl_mem + cl_off[s];
    const int n = cl_off[s + 1] - cl_off[s];
    if (n > kMaxCluster) {
      atomicExch(err, 1);
      continue;
    }
    // insertion sort of the members by (size, root)
    for (int a = 1; a < n; ++a) {
      const int v = mem[a];
      const int rv = sroot[v];
      const long long kv = ((long long)size[rv] << 32) | (unsigned)rv;
      int b = a - 1;
      while (b >= 0) {
        const int rb = sroot[mem[b]];
        const long long kb = ((long long)size[rb] << 32) | (unsigned)rb;
        if (kb <= kv) break;
        mem[b + 1] = mem[b];
        --b;
      }
      mem[b + 1] = v;
    }
    unsigned merged = 0;
    for (int a = 0; a < n; ++a) {
      const int r = sroot[mem[a]];
      if (gpar[r] != r || !small_size(gsize[r], K, N)) continue;
      int best = -1;
      double bd = 0.0;
      int hops = 0;
      for (int m = r; m >= 0 && hops < kMaxHops; m = next[m], ++hops) {
        const int sm = sid[m];
        for (int q = aoff[sm]; q < aoff[sm + 1]; ++q) {
          const int g = find_root(gpar, adj[q], err);
          if (g == r) continue;
          const double d = dist2(csum, size, r, g);
          if (best < 0 || d < bd || (d == bd && g < best)) {
            best = g;
            bd = d;
          }
        }
      }
      if (hops >= kMaxHops) atomicExch(err, 1);
      if (best < 0) continue;
      gpar[r] = best;
      atomicAdd(gsize + best, gsize[r]);  // a large destination may be shared with other clusters
      gsize[r] = 0;
      if (sid[best] >= 0) {  // a small founder keeps the member list of its group
        next[tail[best]] = r;
        tail[best] = tail[r];
      }
      ++merged;
    }
    if (merged) atomicAdd(cnt + 1, (unsigned long long)merged);
  }
}

__global__ void k_relabel(const int* __restrict__ p, const int* gpar, const int32_t* __restrict__ in, long long N,
                          int32_t* __restrict__ out, int* err) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[find_root(gpar, p[i], err)];
}

int grid_for(long long n, int block) {
  return int(std::max<long long>(1, std::min<long long>((n + block - 1) / block, 152LL * 16)));
}

}  // namespace conn

// Runs the post-processing on one image: labels_dev in place, lab three FP32
// planes of W H values.
gmmsp_status enforce_connectivity(int32_t* labels_dev, const float* lab, int W, int H, int K,
                                  gmmsp_conn_stats* stats, cudaStream_t s) {
  using namespace conn;
  const long long N = (long long)W * H;
  if (N >= (1LL << 30)) return GMMSP_E_INVALID;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t nI = up(size_t(N) * 4), nL = up(size_t(N) * 8);
  // per-pixel / per-root arrays: parent, size, cpar, sid, gpar, gsize, next, tail, sroot, deg, cl_count,
  // aoff (N + 1), cl_off (N + 1), csum (3 N long long), plus the copy of the input labels
  size_t off = 0;
  const size_t o_parent = off; off += nI;
  const size_t o_size = off; off += nI;
  const size_t o_cpar = off; off += nI;
  const size_t o_sid = off; off += nI;
  const size_t o_gpar = off; off += nI;
  const size_t o_gsize = off; off += nI;
  const size_t o_next = off; off += nI;
  const size_t o_tail = off; off += nI;
  const size_t o_sroot = off; off += nI;
  const size_t o_deg = off; off += nI;
  const size_t o_clc = off; off += nI;
  const size_t o_aoff = off; off += up(size_t(N + 1) * 4);
  const size_t o_cloff = off; off += up(size_t(N + 1) * 4);
  const size_t o_clmem = off; off += nI;
  const size_t o_in = off; off += nI;
  const size_t o_adj = off; off += up(size_t(N) * 16);  // <= 4 entries per pixel (2 edges, both sides)
  const size_t o_csum = off; off += 3 * nL;
  const size_t o_cnt = off; off += 256;
  void* slab = nullptr;
  cudaError_t e = cudaMalloc(&slab, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  }
  char* b = static_cast<char*>(slab);
  Scratch S{};
  S.parent = reinterpret_cast<int*>(b + o_parent);
  S.size = reinterpret_cast<int*>(b + o_size);
  S.cpar = reinterpret_cast<int*>(b + o_cpar);
  S.sid = reinterpret_cast<int*>(b + o_sid);
  S.gpar = reinterpret_cast<int*>(b + o_gpar);
  S.gsize = reinterpret_cast<int*>(b + o_gsize);
  S.next = reinterpret_cast<int*>(b + o_next);
  S.tail = reinterpret_cast<int*>(b + o_tail);
  S.sroot = reinterpret_cast<int*>(b + o_sroot);
  S.deg = reinterpret_cast<int*>(b + o_deg);
  S.cl_count = reinterpret_cast<int*>(b + o_clc);
  S.aoff = reinterpret_cast<int*>(b + o_aoff);
  S.cl_off = reinterpret_cast<int*>(b + o_cloff);
  S.cl_mem = reinterpret_cast<int*>(b + o_clmem);
  int32_t* in = reinterpret_cast<int32_t*>(b + o_in);
  S.adj = reinterpret_cast<int*>(b + o_adj);
  S.csum = reinterpret_cast<long long*>(b + o_csum);
  S.cnt = reinterpret_cast<unsigned long long*>(b + o_cnt);
  S.err = reinterpret_cast<int*>(b + o_cnt + 64);
  const int gb = grid_for(N, 256);
  unsigned long long host[8] = {};
  int herr = 0;
  int nsmall = 0;
  do {
    if ((e = cudaMemsetAsync(S.size, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.csum, 0, 3 * nL, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cnt, 0, 256, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(in, labels_dev, size_t(N) * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
    k_cc_init<<<gb, 256, 0, s>>>(S.parent, N);
    k_cc_union<<<gb, 256, 0, s>>>(in, W, H, S.parent, S.err);
    k_cc_flatten<<<gb, 256, 0, s>>>(S.parent, N, S.err);
    k_comp_stats<<<gb, 256, 0, s>>>(S.parent, lab, N, S.size, S.csum);
    k_small_index<<<gb, 256, 0, s>>>(S.parent, S.size, N, K, S.sid, S.sroot, S.cpar, S.gpar, S.gsize, S.next,
                                     S.tail, S.cnt);
    k_edges<<<gb, 256, 0, s>>>(S.parent, W, H, S.sid, S.cpar, S.deg, S.aoff, S.adj, 0, S.err);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(host, S.cnt, sizeof(host), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    nsmall = int(host[0]);
    // adjacency of the small components
    k_edges<<<gb, 256, 0, s>>>(S.parent, W, H, S.sid, S.cpar, S.deg, S.aoff, S.adj, 1, S.err);
    k_scan<<<1, 1024, 0, s>>>(S.deg, nsmall, S.aoff);
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    k_edges<<<gb, 256, 0, s>>>(S.parent, W, H, S.sid, S.cpar, S.deg, S.aoff, S.adj, 2, S.err);
    // clusters and their member lists
    const int gs = grid_for(std::max(nsmall, 1), 256);
    k_cluster_count<<<gs, 256, 0, s>>>(S.cpar, S.sroot, S.sid, nsmall, S.cl_count, S.err);
    k_scan<<<1, 1024, 0, s>>>(S.cl_count, nsmall, S.cl_off);
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    k_cluster_fill<<<gs, 256, 0, s>>>(S.cpar, S.sroot, S.sid, nsmall, S.cl_off, S.cl_count, S.cl_mem, S.err);
    k_cluster_merge<<<gs, 256, 0, s>>>(S.sroot, nsmall, S.cpar, S.sid, S.cl_off, S.cl_mem, S.size, S.csum, S.aoff,
                                       S.adj, S.gpar, S.gsize, S.next, S.tail, K, N, S.cnt, S.err);
    k_relabel<<<gb, 256, 0, s>>>(S.parent, S.gpar, in, N, labels_dev, S.err);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(host, S.cnt, sizeof(host), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(&herr, S.err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (false);
  cudaFree(slab);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  if (herr) return GMMSP_E_TIMEOUT;
  if (stats) {
    stats->components = (long long)host[2];
    stats->small = (long long)host[0];
    stats->merged = (long long)host[1];
  }
  return GMMSP_OK;
}

}  // namespace gmmsp

extern "C" gmmsp_status gmmsp_enforce_connectivity(int32_t* labels_dev, const float* lab_planes_dev, int W, int H,
                                                   int K, gmmsp_conn_stats* stats_host, void* stream) {
  if (!labels_dev || !lab_planes_dev || W < 1 || H < 1 || K < 1) return GMMSP_E_INVALID;
  return gmmsp::enforce_connectivity(labels_dev, lab_planes_dev, W, H, K, stats_host,
                                     static_cast<cudaStream_t>(stream));
}
