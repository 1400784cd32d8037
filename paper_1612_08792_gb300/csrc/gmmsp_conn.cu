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
// Kernels (all images of a call at once: blockIdx.y is the image): union-
// find component labelling (k_cc_*), component sizes and colour sums
// (k_comp_stats), small-component indices in pixel order (k_small_count /
// _scan / _assign), one edge walk
// (k_edges) three times -- small-small clusters, then the adjacency lists of
// the small components -- a three-kernel scan for the offsets (k_scan_*),
// the cluster member lists as (size, root) sort keys (k_cluster_count /
// _fill), the per-cluster merge -- one thread per cluster of at most
// kThreadCluster members (k_cluster_merge), one warp per larger cluster
// (k_cluster_merge_warp: the keys sorted in shared memory, the neighbours
// of each member's group scanned by the lanes) -- and the relabelling
// (k_relabel).  One allocation (kept by a context between calls) and one
// synchronisation per call.
// Every loop over a parent chain or a retry is bounded; running out sets the
// error word (reported as GMMSP_E_TIMEOUT).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_conn.h"
#include "gmmsp_internal.cuh"

namespace gmmsp {
namespace conn {

constexpr int kMaxHops = 1 << 24;      // bound on any parent-chain walk or union retry
constexpr int kFixedShift = 20;        // colour sums in units of 2^-20
constexpr int kMaxCluster = 1 << 16;   // bound on the members a cluster sorted in global memory may have
constexpr int kThreadCluster = 8;      // clusters up to this size: one thread; larger: one warp
constexpr int kWarpSortMax = 1024;     // members a warp sorts in shared memory
constexpr int kScanTile = 4096;        // elements per block of the scan (1024 threads x 4)

// One image of a call: pixels [off, off + W H) of the call's arrays.
struct Img {
  int W, H, K;
  long long off;
  const float* lab;   // three FP32 planes of W H values
  int32_t* labels;    // the caller's labels (rewritten)
};

struct Scratch {
  int* parent;                // per pixel: component union-find, then the component root
  int* size;                  // per root: component size
  long long* csum;            // per root: 3 fixed-point colour sums
  int* cpar;                  // per small root: cluster union-find over roots
  int* sid;                   // per root: index of the small component, or -1
  int* sroot;                 // per small index: its root
  int* simg;                  // per small index: its image
  int* deg;                   // per small index: adjacency count, then fill cursor
  int* aoff;                  // per small index + 1: adjacency offsets
  int* adj;                   // adjacency lists (roots of neighbouring components)
  int* cl_count;              // per small index: members of the cluster it roots, then fill cursor
  int* cl_off;                // per small index + 1: member offsets
  unsigned long long* cl_key; // members as (size << 32 | root), grouped by cluster
  int* big;                   // small indices of the roots of clusters above kThreadCluster
  int* tile_sum;              // scan: per tile sums, then their exclusive prefix
  int* gpar;                  // per root: merge union-find (group founder)
  int* gsize;                 // per root: group size
  int* next;                  // per small root: next member of its group, -1 at the end
  int* tail;                  // per small root founding a group: last member
  int32_t* in;                // the input labels of all images
  unsigned long long* cnt;    // counters: 0 small, 1 merged, 2 components
  int* nsmall;                // the small count as int (read by later kernels)
  int* nbig;                  // entries of `big`
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

// Root of x with path halving, for the union phase: every visited node is
// re-pointed at its grandparent, an ancestor in the same set, so no set
// changes; a concurrent link that such a store overwrites is redone by that
// link's own retry.
__device__ __forceinline__ int find_halve(int* p, int x, int* err) {
  for (int h = 0; h < kMaxHops; ++h) {
    const int q = p[x];
    if (q == x) return x;
    const int r = p[q];
    if (r == q) return q;
    p[x] = r;
    x = r;
  }
  atomicExch(err, 1);
  return x;
}

// Root of x in the merge union-find, with path compression.  Only the
// thread or warp that owns a cluster calls it, on that cluster's members and
// on large components (their own roots), so the compression writes touch no
// other cluster's nodes; lanes of one warp that compress the same node write
// the same root.
__device__ __forceinline__ int find_group(int* p, int x, int* err) {
  const int r = find_root(p, x, err);
  for (int h = 0; h < kMaxHops && p[x] != r; ++h) {
    const int q = p[x];
    p[x] = r;
    x = q;
  }
  return r;
}

// Lock-free union by the smaller index (atomicMin on the larger root): the
// final root of every set is its smallest member.
__device__ __forceinline__ void unite(int* p, int a, int b, int* err) {
  for (int h = 0; h < kMaxHops; ++h) {
    a = find_halve(p, a, err);
    b = find_halve(p, b, err);
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

// Per-image pixel loops: blockIdx.y is the image, x strides over its pixels.
#define FOR_PIXELS(im, i)                                                                    \
  const Img im = imgs[blockIdx.y];                                                           \
  const long long im##_N = (long long)im.W * im.H;                                           \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < im##_N;           \
       i += (long long)gridDim.x * blockDim.x)

__global__ void k_cc_init(const Img* __restrict__ imgs, int* __restrict__ p, int32_t* __restrict__ in) {
  FOR_PIXELS(im, i) {
    p[im.off + i] = int(im.off + i);
    in[im.off + i] = im.labels[i];
  }
}

__global__ void k_cc_union(const Img* __restrict__ imgs, const int32_t* __restrict__ in, int* p, int* err) {
  FOR_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    const long long g = im.off + i;
    if (x + 1 < im.W && in[g] == in[g + 1]) unite(p, int(g), int(g + 1), err);
    if (y + 1 < im.H && in[g] == in[g + im.W]) unite(p, int(g), int(g + im.W), err);
  }
}

// After the unions: every pixel points at its root.  The walks only read, so
// the one store per pixel (its root) cannot be overwritten by another
// thread's walk (a halving store here could leave a non-root behind).
__global__ void k_cc_flatten(const Img* __restrict__ imgs, int* p, int* err) {
  FOR_PIXELS(im, i) p[im.off + i] = find_root(p, int(im.off + i), err);
}

__global__ void k_comp_stats(const Img* __restrict__ imgs, const int* __restrict__ p, int* __restrict__ size,
                             long long* __restrict__ csum) {
  FOR_PIXELS(im, i) {
    const int r = p[im.off + i];
    atomicAdd(size + r, 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long f = llrint(double(im.lab[c * im_N + i]) * double(1 << kFixedShift));
      atomicAdd(reinterpret_cast<unsigned long long*>(csum + 3LL * r + c), (unsigned long long)f);
    }
  }
}

__device__ __forceinline__ bool small_size(long long s, int K, long long N) { return 4LL * K * s < N; }

// Exclusive scan of one int per thread over the block; total = the block sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < int(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  total = warp_sums[(blockDim.x >> 5) - 1];
  const int before = warp ? warp_sums[warp - 1] : 0;
  __syncthreads();  // warp_sums is reused by the next call
  return before + x - v;
}

// Image of pixel g of the call (binary search over the images' offsets).
__device__ __forceinline__ int image_of(const Img* __restrict__ imgs, int n, long long g) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (imgs[mid].off <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Small components get consecutive indices in pixel order, from a count per
// tile of kScanTile pixels (k_small_count), a scan of the counts
// (k_small_scan) and the assignment (k_small_assign): no counter that every
// block updates.  Every root starts its own group.
__device__ __forceinline__ bool small_root(const Img* __restrict__ imgs, int n, const Scratch& S, long long g,
                                           int* img) {
  if (S.parent[g] != int(g)) return false;
  const int i = image_of(imgs, n, g);
  *img = i;
  const Img im = imgs[i];
  return small_size(S.size[g], im.K, (long long)im.W * im.H);
}

__global__ void __launch_bounds__(1024) k_small_count(const Img* __restrict__ imgs, int n, long long T, Scratch S) {
  __shared__ int warp_sums[32];
  const long long g0 = (long long)blockIdx.x * kScanTile + 4LL * threadIdx.x;
  int c = 0, roots = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long g = g0 + j;
    if (g >= T) break;
    S.sid[g] = -1;
    if (S.parent[g] != int(g)) continue;
    ++roots;
    S.gpar[g] = int(g);
    S.gsize[g] = S.size[g];
    int img;
    c += small_root(imgs, n, S, g, &img);
  }
  int total, total_roots;
  block_exclusive_scan(c, warp_sums, total);
  block_exclusive_scan(roots, warp_sums, total_roots);
  if (threadIdx.x == 0) {
    S.tile_sum[blockIdx.x] = total;
    if (total_roots) atomicAdd(S.cnt + 2, (unsigned long long)total_roots);
  }
}

// Exclusive scan of the ntiles tile counts in place (one block); the total is
// the small count.
__global__ void __launch_bounds__(1024) k_small_scan(int ntiles, Scratch S) {
  __shared__ int warp_sums[32];
  int carry = 0;
  for (int c = 0; c < ntiles; c += 1024) {
    const int i = c + threadIdx.x;
    const int v = i < ntiles ? S.tile_sum[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, warp_sums, total);
    if (i < ntiles) S.tile_sum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) {
    *S.nsmall = carry;
    S.cnt[0] = (unsigned long long)carry;
  }
}

__global__ void __launch_bounds__(1024) k_small_assign(const Img* __restrict__ imgs, int n, long long T, Scratch S) {
  __shared__ int warp_sums[32];
  const long long g0 = (long long)blockIdx.x * kScanTile + 4LL * threadIdx.x;
  bool f[4];
  int img[4] = {0, 0, 0, 0};
  int c = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    f[j] = g0 + j < T && small_root(imgs, n, S, g0 + j, &img[j]);
    c += f[j];
  }
  int total;
  int s = S.tile_sum[blockIdx.x] + block_exclusive_scan(c, warp_sums, total);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!f[j]) continue;
    const int g = int(g0 + j);
    S.sid[g] = s;
    S.sroot[s] = g;
    S.simg[s] = img[j];
    S.cpar[g] = g;
    S.next[g] = -1;
    S.tail[g] = g;
    ++s;
  }
}


// Walks the 4-neighbour edges between different components; `mode` 0 unites
// small-small pairs into clusters, 1 counts each small side's adjacency, 2
// fills it.
__global__ void k_edges(const Img* __restrict__ imgs, Scratch S, int mode) {
  FOR_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    const long long g = im.off + i;
    const int ri = S.parent[g];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      long long j;
      if (d == 0) {
        if (x + 1 >= im.W) continue;
        j = g + 1;
      } else {
        if (y + 1 >= im.H) continue;
        j = g + im.W;
      }
      const int rj = S.parent[j];
      if (ri == rj) continue;
      const int si = S.sid[ri], sj = S.sid[rj];
      if (mode == 0) {
        if (si >= 0 && sj >= 0) unite(S.cpar, ri, rj, S.err);
      } else if (mode == 1) {
        if (si >= 0) atomicAdd(S.deg + si, 1);
        if (sj >= 0) atomicAdd(S.deg + sj, 1);
      } else {
        if (si >= 0) S.adj[S.aoff[si] + atomicAdd(S.deg + si, 1)] = rj;
        if (sj >= 0) S.adj[S.aoff[sj] + atomicAdd(S.deg + sj, 1)] = ri;
      }
    }
  }
}

// Exclusive prefix sum of the first n = *np ints of `in` into out[0..n]
// (out[n] = the total), in three kernels: tile scans (kScanTile elements per
// block), a scan of the tile sums (one block), the tile offsets added.  The
// grids cover the largest possible n; blocks past n return at once.
__global__ void __launch_bounds__(1024) k_scan_tiles(const int* __restrict__ in, const int* __restrict__ np,
                                                     int* __restrict__ out, int* __restrict__ tile_sum) {
  __shared__ int warp_sums[32];
  const int n = *np;
  const long long base = (long long)blockIdx.x * kScanTile;
  if (base >= n) return;
  const long long i0 = base + 4LL * threadIdx.x;
  int v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = (i0 + j < n) ? in[i0 + j] : 0;
  const int t = v[0] + v[1] + v[2] + v[3];
  int total;
  int run = block_exclusive_scan(t, warp_sums, total);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (i0 + j < n) out[i0 + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(int* __restrict__ tile_sum, const int* __restrict__ np,
                                                         int* __restrict__ out) {
  __shared__ int warp_sums[32];
  const int n = *np;
  const int ntiles = (n + kScanTile - 1) / kScanTile;
  int carry = 0;
  for (int c = 0; c < ntiles; c += 1024) {
    const int i = c + threadIdx.x;
    const int v = i < ntiles ? tile_sum[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, warp_sums, total);
    if (i < ntiles) tile_sum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void __launch_bounds__(1024) k_scan_add(int* __restrict__ out, const int* __restrict__ tile_sum,
                                                   const int* __restrict__ np) {
  const int n = *np;
  const long long base = (long long)blockIdx.x * kScanTile;
  if (base >= n || blockIdx.x == 0) return;
  const int add = tile_sum[blockIdx.x];
  const long long i0 = base + 4LL * threadIdx.x;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (i0 + j < n) out[i0 + j] += add;
}

// Cluster root of every small component, member counts per cluster root.
__global__ void k_cluster_count(Scratch S) {
  const int n = *S.nsmall;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int c = find_root(S.cpar, S.sroot[s], S.err);
    atomicAdd(S.cl_count + S.sid[c], 1);
  }
}

// Members of each cluster as sort keys (size << 32 | root): contiguous per
// cluster, so that the sort reads and writes no scattered data.
__global__ void k_cluster_fill(Scratch S) {
  const int n = *S.nsmall;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const int r = S.sroot[s];
    const int c = S.sid[find_root(S.cpar, r, S.err)];
    S.cl_key[S.cl_off[c] + atomicAdd(S.cl_count + c, 1)] =
        ((unsigned long long)(unsigned)S.size[r] << 32) | (unsigned)r;
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

// Merge of small component r (still its group's founder, still small) into
// the nearest group next to its group, under the sequential rule; the
// caller has found the nearest (best, or -1 for none).
__device__ __forceinline__ void merge_into(Scratch& S, int r, int best) {
  S.gpar[r] = best;
  atomicAdd(S.gsize + best, S.gsize[r]);  // a large destination may be shared with other clusters
  S.gsize[r] = 0;
  if (S.sid[best] >= 0) {  // a small founder keeps the member list of its group
    S.next[S.tail[best]] = r;
    S.tail[best] = S.tail[r];
  }
}

// Insertion sort of n keys (one thread).
__device__ __forceinline__ void sort_keys(unsigned long long* key, int n) {
  for (int a = 1; a < n; ++a) {
    const unsigned long long v = key[a];
    int b = a - 1;
    while (b >= 0 && key[b] > v) {
      key[b + 1] = key[b];
      --b;
    }
    key[b + 1] = v;
  }
}

// One thread per cluster of at most kThreadCluster members: the sequential
// rule over the members in (size, root) order.  Larger clusters go to the
// list of the warp kernel.
__global__ void k_cluster_merge(const Img* __restrict__ imgs, Scratch S) {
  const int nsm = *S.nsmall;
  unsigned merged = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsm; s += gridDim.x * blockDim.x) {
    const int r0 = S.sroot[s];
    if (S.cpar[r0] != r0) continue;  // not a cluster root
    const int n = S.cl_off[s + 1] - S.cl_off[s];
    if (n > kThreadCluster) {
      S.big[atomicAdd(S.nbig, 1)] = s;
      continue;
    }
    const Img im = imgs[S.simg[s]];
    const long long N = (long long)im.W * im.H;
    unsigned long long* key = S.cl_key + S.cl_off[s];
    sort_keys(key, n);
    for (int a = 0; a < n; ++a) {
      const int r = int(unsigned(key[a]));
      if (S.gpar[r] != r || !small_size(S.gsize[r], im.K, N)) continue;
      int best = -1;
      double bd = 0.0;
      int hops = 0;
      for (int m = r; m >= 0 && hops < kMaxHops; m = S.next[m], ++hops) {
        const int sm = S.sid[m];
        for (int q = S.aoff[sm]; q < S.aoff[sm + 1]; ++q) {
          const int g = find_group(S.gpar, S.adj[q], S.err);
          if (g == r) continue;
          const double d = dist2(S.csum, S.size, r, g);
          if (best < 0 || d < bd || (d == bd && g < best)) {
            best = g;
            bd = d;
          }
        }
      }
      if (hops >= kMaxHops) atomicExch(S.err, 1);
      if (best < 0) continue;
      merge_into(S, r, best);
      ++merged;
    }
  }
  merged = __reduce_add_sync(0xffffffffu, merged);
  if ((threadIdx.x & 31) == 0 && merged) atomicAdd(S.cnt + 1, (unsigned long long)merged);
}

// One warp per cluster above kThreadCluster members.  The keys are sorted in
// shared memory (bitonic; clusters above kWarpSortMax members are sorted in
// place by one lane), then the members are taken in order as above, with the
// adjacency entries of each member's group spread over the lanes and the
// nearest group found by a warp reduction on (distance, group index) -- the
// same minimum the sequential scan finds.  __syncwarp orders lane 0's merge
// writes before the next member's reads.
constexpr int kMergeWarps = 4;

__global__ void __launch_bounds__(kMergeWarps * 32) k_cluster_merge_warp(const Img* __restrict__ imgs, Scratch S) {
  __shared__ unsigned long long sk[kMergeWarps][kWarpSortMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbig = *S.nbig;
  unsigned merged = 0;
  for (int b = blockIdx.x * kMergeWarps + warp; b < nbig; b += gridDim.x * kMergeWarps) {
    const int s = S.big[b];
    const Img im = imgs[S.simg[s]];
    const long long N = (long long)im.W * im.H;
    unsigned long long* gkey = S.cl_key + S.cl_off[s];
    const int n = S.cl_off[s + 1] - S.cl_off[s];
    const unsigned long long* key = sk[warp];
    if (n <= kWarpSortMax) {
      int P = 32;
      while (P < n) P <<= 1;
      unsigned long long* k = sk[warp];
      for (int i = lane; i < P; i += 32) k[i] = i < n ? gkey[i] : ~0ull;
      __syncwarp();
      for (int w = 2; w <= P; w <<= 1)
        for (int j = w >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < P; i += 32) {
            const int l = i ^ j;
            if (l > i) {
              const unsigned long long x = k[i], y = k[l];
              if ((x > y) == ((i & w) == 0)) {
                k[i] = y;
                k[l] = x;
              }
            }
          }
          __syncwarp();
        }
    } else {
      if (lane == 0) {
        if (n > kMaxCluster) atomicExch(S.err, 1);
        else sort_keys(gkey, n);
      }
      __syncwarp();
      if (n > kMaxCluster) continue;
      key = gkey;
    }
    for (int a = 0; a < n; ++a) {
      const int r = int(unsigned(key[a]));
      if (S.gpar[r] != r || !small_size(S.gsize[r], im.K, N)) continue;  // warp-uniform
      int best = 0x7fffffff;
      double bd = INFINITY;
      int hops = 0;
      for (int m = r; m >= 0 && hops < kMaxHops; m = S.next[m], ++hops) {
        const int sm = S.sid[m];
        const int q1 = S.aoff[sm + 1];
        for (int q = S.aoff[sm] + lane; q < q1; q += 32) {
          const int g = find_group(S.gpar, S.adj[q], S.err);
          if (g == r) continue;
          const double d = dist2(S.csum, S.size, r, g);
          if (d < bd || (d == bd && g < best)) {
            best = g;
            bd = d;
          }
        }
      }
      if (hops >= kMaxHops && lane == 0) atomicExch(S.err, 1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double d2 = __shfl_xor_sync(0xffffffffu, bd, o);
        const int g2 = __shfl_xor_sync(0xffffffffu, best, o);
        if (d2 < bd || (d2 == bd && g2 < best)) {
          bd = d2;
          best = g2;
        }
      }
      if (best != 0x7fffffff) {
        if (lane == 0) {
          merge_into(S, r, best);
          ++merged;
        }
      }
      __syncwarp();
    }
    __syncwarp();  // sk[warp] is refilled by the next cluster
  }
  merged = __reduce_add_sync(0xffffffffu, merged);
  if (lane == 0 && merged) atomicAdd(S.cnt + 1, (unsigned long long)merged);
}

__global__ void k_relabel(const Img* __restrict__ imgs, Scratch S) {
  FOR_PIXELS(im, i) im.labels[i] = S.in[find_root(S.gpar, S.parent[im.off + i], S.err)];
}

}  // namespace conn

gmmsp_status enforce_connectivity_many(int n, const int* W, const int* H, const int* K, int32_t* const* labels,
                                       const float* const* lab, gmmsp_conn_stats* stats, cudaStream_t s,
                                       ConnScratch* cache) {
  using namespace conn;
  if (n < 1 || n > 65535) return GMMSP_E_INVALID;
  std::vector<Img> host(n);
  long long T = 0, maxN = 0;
  for (int i = 0; i < n; ++i) {
    if (W[i] < 1 || H[i] < 1 || K[i] < 1 || !labels[i] || !lab[i]) return GMMSP_E_INVALID;
    host[i] = Img{W[i], H[i], K[i], T, lab[i], labels[i]};
    T += (long long)W[i] * H[i];
    maxN = std::max(maxN, (long long)W[i] * H[i]);
  }
  if (T >= (1LL << 30)) return GMMSP_E_INVALID;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t nI = up(size_t(T) * 4), nI1 = up(size_t(T + 1) * 4);
  const long long ntiles = std::max<long long>(1, (T + kScanTile - 1) / kScanTile);
  size_t o[22];
  size_t off = 0;
  for (int j = 0; j < 14; ++j) { o[j] = off; off += nI; }          // 14 int arrays of T entries
  o[14] = off; off += nI1;                                          // aoff
  o[15] = off; off += nI1;                                          // cl_off
  o[16] = off; off += up(size_t(T) * 16);                           // adj (<= 4 entries per pixel)
  o[17] = off; off += up(size_t(T) * 24);                           // csum
  o[18] = off; off += up(sizeof(Img) * n);                          // image table
  o[19] = off; off += 256;                                          // counters
  o[20] = off; off += up(size_t(T) * 8);                            // cl_key
  o[21] = off; off += up(size_t(ntiles + 1) * 4);                   // tile_sum
  void* slab = nullptr;
  cudaError_t e = cudaSuccess;
  if (cache && cache->bytes >= off) {
    slab = cache->ptr;
  } else {
    if (cache && cache->ptr) {
      cudaStreamSynchronize(s);
      cudaFree(cache->ptr);
      cache->ptr = nullptr;
      cache->bytes = 0;
    }
    e = cudaMalloc(&slab, off);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
    }
    if (cache) {
      cache->ptr = slab;
      cache->bytes = off;
    }
  }
  char* b = static_cast<char*>(slab);
  int* ia[14];
  for (int j = 0; j < 14; ++j) ia[j] = reinterpret_cast<int*>(b + o[j]);
  Scratch S{};
  S.parent = ia[0]; S.size = ia[1]; S.cpar = ia[2]; S.sid = ia[3]; S.sroot = ia[4]; S.simg = ia[5];
  S.deg = ia[6]; S.cl_count = ia[7]; S.big = ia[8]; S.gpar = ia[9]; S.gsize = ia[10]; S.next = ia[11];
  S.tail = ia[12]; S.in = reinterpret_cast<int32_t*>(ia[13]);
  S.aoff = reinterpret_cast<int*>(b + o[14]);
  S.cl_off = reinterpret_cast<int*>(b + o[15]);
  S.adj = reinterpret_cast<int*>(b + o[16]);
  S.csum = reinterpret_cast<long long*>(b + o[17]);
  Img* table = reinterpret_cast<Img*>(b + o[18]);
  S.cnt = reinterpret_cast<unsigned long long*>(b + o[19]);
  S.nsmall = reinterpret_cast<int*>(b + o[19] + 64);
  S.err = reinterpret_cast<int*>(b + o[19] + 128);
  S.nbig = reinterpret_cast<int*>(b + o[19] + 192);
  S.cl_key = reinterpret_cast<unsigned long long*>(b + o[20]);
  S.tile_sum = reinterpret_cast<int*>(b + o[21]);
  // blocks per image: enough to fill the machine across the images
  const long long per = std::max<long long>(1, std::min<long long>((maxN + 255) / 256, (152LL * 16 + n - 1) / n));
  const dim3 gp{static_cast<unsigned>(per), static_cast<unsigned>(n)};
  const int gs = 152 * 8;
  unsigned long long hc[3] = {};
  int herr = 0;
  do {
    if ((e = cudaMemcpyAsync(table, host.data(), sizeof(Img) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.size, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.csum, 0, up(size_t(T) * 24), s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cnt, 0, 256, s)) != cudaSuccess) break;
    k_cc_init<<<gp, 256, 0, s>>>(table, S.parent, S.in);
    k_cc_union<<<gp, 256, 0, s>>>(table, S.in, S.parent, S.err);
    k_cc_flatten<<<gp, 256, 0, s>>>(table, S.parent, S.err);
    k_comp_stats<<<gp, 256, 0, s>>>(table, S.parent, S.size, S.csum);
    k_small_count<<<unsigned(ntiles), 1024, 0, s>>>(table, n, T, S);
    k_small_scan<<<1, 1024, 0, s>>>(int(ntiles), S);
    k_small_assign<<<unsigned(ntiles), 1024, 0, s>>>(table, n, T, S);
    k_edges<<<gp, 256, 0, s>>>(table, S, 0);
    k_edges<<<gp, 256, 0, s>>>(table, S, 1);
    k_scan_tiles<<<unsigned(ntiles), 1024, 0, s>>>(S.deg, S.nsmall, S.aoff, S.tile_sum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(S.tile_sum, S.nsmall, S.aoff);
    k_scan_add<<<unsigned(ntiles), 1024, 0, s>>>(S.aoff, S.tile_sum, S.nsmall);
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    k_edges<<<gp, 256, 0, s>>>(table, S, 2);
    k_cluster_count<<<gs, 256, 0, s>>>(S);
    k_scan_tiles<<<unsigned(ntiles), 1024, 0, s>>>(S.cl_count, S.nsmall, S.cl_off, S.tile_sum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(S.tile_sum, S.nsmall, S.cl_off);
    k_scan_add<<<unsigned(ntiles), 1024, 0, s>>>(S.cl_off, S.tile_sum, S.nsmall);
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    k_cluster_fill<<<gs, 256, 0, s>>>(S);
    k_cluster_merge<<<gs, 256, 0, s>>>(table, S);
    k_cluster_merge_warp<<<152 * 4, kMergeWarps * 32, 0, s>>>(table, S);
    k_relabel<<<gp, 256, 0, s>>>(table, S);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(hc, S.cnt, sizeof(hc), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(&herr, S.err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (false);
  if (!cache) cudaFree(slab);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GMMSP_E_NOMEM : GMMSP_E_CUDA;
  if (herr) return GMMSP_E_TIMEOUT;
  if (stats) {
    stats->components = (long long)hc[2];
    stats->small = (long long)hc[0];
    stats->merged = (long long)hc[1];
  }
  return GMMSP_OK;
}

gmmsp_status enforce_connectivity(int32_t* labels_dev, const float* lab, int W, int H, int K,
                                  gmmsp_conn_stats* stats, cudaStream_t s, ConnScratch* cache) {
  int32_t* l[1] = {labels_dev};
  const float* c[1] = {lab};
  return enforce_connectivity_many(1, &W, &H, &K, l, c, stats, s, cache);
}

}  // namespace gmmsp

extern "C" gmmsp_status gmmsp_enforce_connectivity(int32_t* labels_dev, const float* lab_planes_dev, int W, int H,
                                                   int K, gmmsp_conn_stats* stats_host, void* stream) {
  if (!labels_dev || !lab_planes_dev || W < 1 || H < 1 || K < 1) return GMMSP_E_INVALID;
  return gmmsp::enforce_connectivity(labels_dev, lab_planes_dev, W, H, K, stats_host,
                                     static_cast<cudaStream_t>(stream), nullptr);
}
