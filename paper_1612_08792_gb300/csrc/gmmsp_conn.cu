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
// over the whole image gives there.  One thread (or one warp) runs each
// cluster.
//
// Data layout.  After the pixel-level labelling every component gets a
// compact index c in the order of its smallest pixel (so ordering by c is
// ordering by that pixel), and every per-component array is indexed by c:
// about 1.6 M entries for 256 images of 481x321, a few MB each, which the
// L2 keeps while the merge reads them at random.
//
// Kernels (all images of a call at once; pixel loops take blockIdx.y as the
// image, tile loops cover all pixels of the call):
//   k_cc_init / _union / _flatten   union-find labelling, parent = root pixel
//   k_root_count / _scan / _assign  compact index per root (tile counts, scan)
//   k_comp_map                      parent := compact index; sizes and
//                                   fixed-point colour sums (atomics)
//   k_comp_flags                    small flag, mean colour, group state per component
//   k_edges (x2)                    small-small clusters and adjacency counts;
//                                   adjacency lists (of the small components)
//   k_scan_tiles / _tile_sums / _add  offsets (twice)
//   k_cluster_count / _fill         member lists as (size << 32 | c) keys
//   k_cluster_merge                 one thread per cluster of <= kThreadCluster
//   k_cluster_merge_warp            one warp per larger cluster (keys sorted
//                                   in shared memory, adjacency over the lanes)
//   k_relabel                       label of the group founder
// One allocation (kept by a context between calls) and one synchronisation
// per call.  Every loop over a parent chain or a retry is bounded; running
// out sets the error word (reported as GMMSP_E_TIMEOUT).
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
constexpr int kThreadCluster = 2;      // clusters up to this size: one thread; larger: one warp
constexpr int kHugeCluster = 32;       // warp clusters above this size are started first
constexpr int kWarpSortMax = 1024;     // members a warp sorts in shared memory
constexpr int kScanTile = 4096;        // elements per block of the tile kernels (1024 threads x 4)
constexpr int kMergeWarps = 4;

// One image of a call: pixels [off, off + W H) of the call's arrays.
struct Img {
  int W, H, K;
  long long off;
  const float* lab;   // three FP32 planes of W H values
  int32_t* labels;    // the caller's labels (read, then rewritten by k_relabel)
};

struct Scratch {
  // per pixel of the call
  int* parent;                // union-find, then the root pixel, then the compact index
  int* cidr;                  // at root pixels: the compact index
  // per component (compact index c < ncomp)
  int* size;                  // pixel count
  long long* csum;            // 3 fixed-point colour sums, then (k_comp_flags) ...
  double* mean;               // ... the 3 mean colours csum / size, in the same memory
  int* cimg;                  // image
  int32_t* clabel;            // its label
  int* small;                 // 1 for a small component
  int* cpar;                  // cluster union-find over small components
  int* deg;                   // adjacency count, then fill cursor
  int* aoff;                  // (ncomp + 1) adjacency offsets
  int* adj;                   // adjacency lists (compact indices of neighbouring components)
  int* cl_count;              // members of the cluster it roots, then fill cursor
  int* cl_off;                // (ncomp + 1) member offsets
  unsigned long long* cl_key; // members as (size << 32 | c), grouped by cluster
  int* big;                   // roots of clusters above kThreadCluster members: those above
                              // kHugeCluster from the front, the others from the back
  int* gpar;                  // merge union-find (group founder)
  int* gsize;                 // group size (kept for small founders)
  int* next;                  // next member of its group, -1 at the end
  int* tail;                  // of a group's founder: its last member
  int* tile_sum;              // tile kernels: per tile counts, then their exclusive prefix
  unsigned long long* cnt;    // counters: 0 small, 1 merged, 2 components
  int* ncomp;                 // the component count as int (read by later kernels)
  int* nbig;                  // [0] entries at the front of `big`, [1] at the back
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

// Root of x with path halving, for the union phases: every visited node is
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

__device__ __forceinline__ bool small_size(long long s, int K, long long N) { return 4LL * K * s < N; }

// Per-image pixel loops: blockIdx.y is the image, x strides over its pixels.
#define FOR_PIXELS(im, i)                                                                    \
  const Img im = imgs[blockIdx.y];                                                           \
  const long long im##_N = (long long)im.W * im.H;                                           \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < im##_N;           \
       i += (long long)gridDim.x * blockDim.x)

// Per-component loops over c < *S.ncomp.
#define FOR_COMPONENTS(c)      \
  const int ncomp_ = *S.ncomp; \
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp_; c += gridDim.x * blockDim.x)

// Warp-uniform pixel loop (32 consecutive pixels per warp and step, every
// lane taking part in the shuffles; `valid` marks the pixels of the image).
#define FOR_PIXEL_WARPS(im, i, valid)                                                          \
  const Img im = imgs[blockIdx.y];                                                             \
  const long long im##_N = (long long)im.W * im.H;                                             \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i - (threadIdx.x & 31) < im##_N; \
       i += (long long)gridDim.x * blockDim.x)                                                 \
    if (const bool valid = i < im##_N; true)

// Every pixel starts under the first pixel of its run: the pixels of one
// label that follow each other in a row within the warp's 32 (a ballot).  No
// union runs yet, so these plain stores race with nothing.
__global__ void k_cc_init(const Img* __restrict__ imgs, int* __restrict__ p) {
  const int lane = threadIdx.x & 31;
  FOR_PIXEL_WARPS(im, i, valid) {
    const int x = valid ? int(i % im.W) : 0;
    const int32_t l = valid ? im.labels[i] : 0;
    const int32_t lprev = __shfl_up_sync(0xffffffffu, l, 1);
    const bool head = !valid || lane == 0 || x == 0 || lprev != l;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    if (valid) p[im.off + i] = int(im.off + i - (lane - start));
  }
}

// The unions the runs leave: a run that begins at a warp's first lane with the
// same label to its left, and one vertical union per pair of vertically
// adjacent runs (at the leftmost pixel of their overlap).
__global__ void k_cc_union(const Img* __restrict__ imgs, int* p, int* err) {
  FOR_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    const long long g = im.off + i;
    const int32_t l = im.labels[i];
    const bool left_same = x > 0 && im.labels[i - 1] == l;
    if (left_same && (threadIdx.x & 31) == 0) unite(p, int(g), int(g - 1), err);
    if (y + 1 < im.H && l == im.labels[i + im.W] && !(left_same && im.labels[i - 1 + im.W] == l))
      unite(p, int(g), int(g + im.W), err);
  }
}

// After the unions: every pixel points at its root.  The walks only read, so
// the one store per pixel (its root) cannot be overwritten by another
// thread's walk (a halving store here could leave a non-root behind).
__global__ void k_cc_flatten(const Img* __restrict__ imgs, int* p, int* err) {
  FOR_PIXELS(im, i) p[im.off + i] = find_root(p, int(im.off + i), err);
}

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

// Compact indices of the components in the order of their roots (smallest
// pixels): a count per tile of kScanTile pixels, a scan of the counts, the
// assignment.  No counter that every block updates.
__global__ void __launch_bounds__(1024) k_root_count(long long T, Scratch S) {
  __shared__ int warp_sums[32];
  const long long g0 = (long long)blockIdx.x * kScanTile + 4LL * threadIdx.x;
  int c = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) c += (g0 + j < T && S.parent[g0 + j] == int(g0 + j));
  int total;
  block_exclusive_scan(c, warp_sums, total);
  if (threadIdx.x == 0) S.tile_sum[blockIdx.x] = total;
}

// Exclusive scan of the ntiles tile counts in place (one block); the total
// is the component count.
__global__ void __launch_bounds__(1024) k_root_scan(int ntiles, Scratch S) {
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
    *S.ncomp = carry;
    S.cnt[2] = (unsigned long long)carry;
  }
}

__global__ void __launch_bounds__(1024) k_root_assign(const Img* __restrict__ imgs, int n, long long T, Scratch S) {
  __shared__ int warp_sums[32];
  const long long g0 = (long long)blockIdx.x * kScanTile + 4LL * threadIdx.x;
  bool f[4];
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    f[j] = g0 + j < T && S.parent[g0 + j] == int(g0 + j);
    cnt += f[j];
  }
  int total;
  int c = S.tile_sum[blockIdx.x] + block_exclusive_scan(cnt, warp_sums, total);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!f[j]) continue;
    const long long g = g0 + j;
    const int i = image_of(imgs, n, g);
    S.cidr[g] = c;
    S.cimg[c] = i;
    S.clabel[c] = imgs[i].labels[g - imgs[i].off];
    ++c;
  }
}

// parent := compact index of the pixel's component; component sizes and
// fixed-point colour sums.  A warp takes 32 consecutive pixels; the lanes of
// a run of equal components (a row segment of one component) add their
// values to the run's first lane (a segmented reduction by shuffles), which
// alone updates the sums: one set of atomics per run instead of per pixel.
__global__ void k_comp_map(const Img* __restrict__ imgs, Scratch S) {
  const Img im = imgs[blockIdx.y];
  const long long N = (long long)im.W * im.H;
  const int lane = threadIdx.x & 31;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i - lane < N; i += step) {
    const bool valid = i < N;  // warp-uniform loop: every lane takes part in the shuffles
    int c = -1 - lane;         // distinct for invalid lanes: they form runs of their own
    long long v[4] = {0, 0, 0, 0};
    if (valid) {
      const long long g = im.off + i;
      c = S.cidr[S.parent[g]];
      S.parent[g] = c;
      v[0] = 1;
#pragma unroll
      for (int k = 0; k < 3; ++k)  // z 2^20 is exact in FP32 (a power-of-two scaling): round(2^20 z)
        v[1 + k] = __float2ll_rn(im.lab[k * N + i] * float(1 << kFixedShift));
    }
    const int cprev = __shfl_up_sync(0xffffffffu, c, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || cprev != c);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of my run
    const int run_end = (heads & (0xfffffffeu << lane)) ? __ffs(heads & (0xfffffffeu << lane)) - 1 : 32;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long w = __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane + o < run_end) v[k] += w;
      }
    }
    if (valid && lane == start) {
      atomicAdd(S.size + c, int(v[0]));
#pragma unroll
      for (int k = 0; k < 3; ++k)
        atomicAdd(reinterpret_cast<unsigned long long*>(S.csum + 3LL * c + k), (unsigned long long)v[1 + k]);
    }
  }
}

// Small flag, mean colour (the FP64 quotient csum / size, written over the
// sums) and the initial group state of every component (each is its own
// group); the small count takes one atomic per block.
__global__ void __launch_bounds__(256) k_comp_flags(const Img* __restrict__ imgs, Scratch S) {
  const int ncomp = *S.ncomp;
  for (int base = blockIdx.x * blockDim.x; base < ncomp; base += gridDim.x * blockDim.x) {
    const int c = base + threadIdx.x;
    bool sm = false;
    if (c < ncomp) {
      const Img im = imgs[S.cimg[c]];
      const int sz = S.size[c];
      sm = small_size(sz, im.K, (long long)im.W * im.H);
      S.small[c] = sm ? 1 : 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) S.mean[3LL * c + k] = double(S.csum[3LL * c + k]) / double(sz);
      S.gpar[c] = c;
      S.gsize[c] = sz;
      S.cpar[c] = c;
      S.next[c] = -1;
      S.tail[c] = c;
    }
    const int nsm = __syncthreads_count(sm);
    if (threadIdx.x == 0 && nsm) atomicAdd(S.cnt + 0, (unsigned long long)nsm);
  }
}

// Walks the 4-neighbour edges between different components; `mode` 0 unites
// small-small pairs into clusters and counts each small side's adjacency, 1
// fills the adjacency lists.  An edge whose pair of components the previous
// edge along the same line already gave (the pixel to the left for a vertical
// edge, the pixel above for a horizontal one) is skipped: the lists are
// neighbour sets, and most repeats go.
__global__ void k_edges(const Img* __restrict__ imgs, Scratch S, int mode) {
  FOR_PIXELS(im, i) {
    const int y = int(i / im.W), x = int(i - (long long)y * im.W);
    const long long g = im.off + i;
    const int ci = S.parent[g];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      long long j, back;  // back: the same edge one pixel earlier along the line, or -1
      if (d == 0) {
        if (x + 1 >= im.W) continue;
        j = g + 1;
        back = y > 0 ? g - im.W : -1;
      } else {
        if (y + 1 >= im.H) continue;
        j = g + im.W;
        back = x > 0 ? g - 1 : -1;
      }
      const int cj = S.parent[j];
      if (ci == cj) continue;
      if (back >= 0 && S.parent[back] == ci && S.parent[back + (j - g)] == cj) continue;
      const int si = S.small[ci], sj = S.small[cj];
      if (mode == 0) {
        if (si && sj) unite(S.cpar, ci, cj, S.err);
        if (si) atomicAdd(S.deg + ci, 1);
        if (sj) atomicAdd(S.deg + cj, 1);
      } else {
        if (si) S.adj[S.aoff[ci] + atomicAdd(S.deg + ci, 1)] = cj;
        if (sj) S.adj[S.aoff[cj] + atomicAdd(S.deg + cj, 1)] = ci;
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
  FOR_COMPONENTS(c) {
    if (!S.small[c]) continue;
    atomicAdd(S.cl_count + find_root(S.cpar, c, S.err), 1);
  }
}

// Members of each cluster as sort keys (size << 32 | c): contiguous per
// cluster, so that the sort reads and writes no scattered data.
__global__ void k_cluster_fill(Scratch S) {
  FOR_COMPONENTS(c) {
    if (!S.small[c]) continue;
    const int r = find_root(S.cpar, c, S.err);
    S.cl_key[S.cl_off[r] + atomicAdd(S.cl_count + r, 1)] =
        ((unsigned long long)(unsigned)S.size[c] << 32) | unsigned(c);
  }
}

// Squared distance of the mean colours of components a and b, in a fixed
// order without contractions.
__device__ __forceinline__ double dist2(const double* mean, int a, int b) {
  double d = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double t = __dsub_rn(mean[3LL * a + k], mean[3LL * b + k]);
    d = __dadd_rn(d, __dmul_rn(t, t));
  }
  return d;
}

// Merge of small component r (still its group's founder, still small) into
// the nearest group `best` next to its group.  A small destination belongs
// to the same cluster and gets r's size and members; a large destination is
// never a source, and no decision reads its size.
__device__ __forceinline__ void merge_into(Scratch& S, int r, int best) {
  S.gpar[r] = best;
  if (S.small[best]) {
    S.gsize[best] += S.gsize[r];
    S.next[S.tail[best]] = r;
    S.tail[best] = S.tail[r];
  }
  S.gsize[r] = 0;
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
// rule over the members in (size, index) order.  Larger clusters go to the
// list of the warp kernel.
__global__ void k_cluster_merge(const Img* __restrict__ imgs, Scratch S) {
  unsigned merged = 0;
  FOR_COMPONENTS(c) {
    if (!S.small[c] || S.cpar[c] != c) continue;  // not a cluster root
    const int n = S.cl_off[c + 1] - S.cl_off[c];
    if (n > kThreadCluster) {
      if (n > kHugeCluster) S.big[atomicAdd(S.nbig, 1)] = c;
      else S.big[*S.ncomp - 1 - atomicAdd(S.nbig + 1, 1)] = c;
      continue;
    }
    const Img im = imgs[S.cimg[c]];
    const long long N = (long long)im.W * im.H;
    unsigned long long* key = S.cl_key + S.cl_off[c];
    sort_keys(key, n);
    for (int a = 0; a < n; ++a) {
      const int r = int(unsigned(key[a]));
      if (S.gpar[r] != r || !small_size(S.gsize[r], im.K, N)) continue;
      int best = -1;
      double bd = 0.0;
      int hops = 0;
      for (int m = r; m >= 0 && hops < kMaxHops; m = S.next[m], ++hops) {
        for (int q = S.aoff[m]; q < S.aoff[m + 1]; ++q) {
          const int g = find_group(S.gpar, S.adj[q], S.err);
          if (g == r) continue;
          const double d = dist2(S.mean, r, g);
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

// One warp per cluster above kThreadCluster members, the clusters above
// kHugeCluster members first (the longest serial chains start earliest).
// The keys are sorted in
// shared memory (bitonic; clusters above kWarpSortMax members are sorted in
// place by one lane), then the members are taken in order as above, with the
// adjacency entries of each member's group spread over the lanes and the
// nearest group found by a warp reduction on (distance, group index) -- the
// same minimum the sequential scan finds.  __syncwarp orders lane 0's merge
// writes before the next member's reads.
__global__ void __launch_bounds__(kMergeWarps * 32) k_cluster_merge_warp(const Img* __restrict__ imgs, Scratch S) {
  __shared__ unsigned long long sk[kMergeWarps][kWarpSortMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nhuge = S.nbig[0], nbig = S.nbig[0] + S.nbig[1], ncomp = *S.ncomp;
  unsigned merged = 0;
  for (int b = blockIdx.x * kMergeWarps + warp; b < nbig; b += gridDim.x * kMergeWarps) {
    const int c = b < nhuge ? S.big[b] : S.big[ncomp - 1 - (b - nhuge)];
    const Img im = imgs[S.cimg[c]];
    const long long N = (long long)im.W * im.H;
    unsigned long long* gkey = S.cl_key + S.cl_off[c];
    const int n = S.cl_off[c + 1] - S.cl_off[c];
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
        const int q1 = S.aoff[m + 1];
        for (int q = S.aoff[m] + lane; q < q1; q += 32) {
          const int g = find_group(S.gpar, S.adj[q], S.err);
          if (g == r) continue;
          const double d = dist2(S.mean, r, g);
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
      if (best != 0x7fffffff && lane == 0) {
        merge_into(S, r, best);
        ++merged;
      }
      __syncwarp();
    }
    __syncwarp();  // sk[warp] is refilled by the next cluster
  }
  merged = __reduce_add_sync(0xffffffffu, merged);
  if (lane == 0 && merged) atomicAdd(S.cnt + 1, (unsigned long long)merged);
}

__global__ void k_relabel(const Img* __restrict__ imgs, Scratch S) {
  FOR_PIXELS(im, i) im.labels[i] = S.clabel[find_root(S.gpar, S.parent[im.off + i], S.err)];
}

}  // namespace conn

gmmsp_status enforce_connectivity_many(int n, const int* W, const int* H, const int* K, int32_t* const* labels,
                                       const float* const* lab, gmmsp_conn_stats* stats, cudaStream_t s,
                                       ConnScratch* cache) {
  GMMSP_NVTX("enforce_connectivity_many");
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
  // every per-component array has room for T components (one per pixel at most)
  const size_t nI = up(size_t(T) * 4), nI1 = up(size_t(T + 1) * 4);
  const long long ntiles = std::max<long long>(1, (T + kScanTile - 1) / kScanTile);
  enum { A_PARENT, A_CIDR, A_SIZE, A_CIMG, A_CLABEL, A_SMALL, A_CPAR, A_DEG, A_CLCOUNT, A_BIG, A_GPAR, A_GSIZE,
         A_NEXT, A_TAIL, kIntArrays };
  enum { O_AOFF = kIntArrays, O_CLOFF, O_ADJ, O_CSUM, O_TABLE, O_CNT, O_KEY, O_TILE, kRegions };
  size_t o[kRegions];
  size_t off = 0;
  for (int j = 0; j < kIntArrays; ++j) { o[j] = off; off += nI; }
  o[O_AOFF] = off; off += nI1;
  o[O_CLOFF] = off; off += nI1;
  o[O_ADJ] = off; off += up(size_t(T) * 16);   // <= 2 edges per pixel, 2 entries per edge
  o[O_CSUM] = off; off += up(size_t(T) * 24);
  o[O_TABLE] = off; off += up(sizeof(Img) * n);
  o[O_CNT] = off; off += 256;
  o[O_KEY] = off; off += up(size_t(T) * 8);
  o[O_TILE] = off; off += up(size_t(ntiles + 1) * 4);
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
  auto ia = [&](int j) { return reinterpret_cast<int*>(b + o[j]); };
  Scratch S{};
  S.parent = ia(A_PARENT); S.cidr = ia(A_CIDR); S.size = ia(A_SIZE); S.cimg = ia(A_CIMG);
  S.clabel = reinterpret_cast<int32_t*>(ia(A_CLABEL)); S.small = ia(A_SMALL); S.cpar = ia(A_CPAR);
  S.deg = ia(A_DEG); S.cl_count = ia(A_CLCOUNT); S.big = ia(A_BIG); S.gpar = ia(A_GPAR); S.gsize = ia(A_GSIZE);
  S.next = ia(A_NEXT); S.tail = ia(A_TAIL);
  S.aoff = ia(O_AOFF);
  S.cl_off = ia(O_CLOFF);
  S.adj = ia(O_ADJ);
  S.csum = reinterpret_cast<long long*>(b + o[O_CSUM]);
  S.mean = reinterpret_cast<double*>(b + o[O_CSUM]);
  Img* table = reinterpret_cast<Img*>(b + o[O_TABLE]);
  S.cnt = reinterpret_cast<unsigned long long*>(b + o[O_CNT]);
  S.ncomp = reinterpret_cast<int*>(b + o[O_CNT] + 64);
  S.err = reinterpret_cast<int*>(b + o[O_CNT] + 128);
  S.nbig = reinterpret_cast<int*>(b + o[O_CNT] + 192);
  S.cl_key = reinterpret_cast<unsigned long long*>(b + o[O_KEY]);
  S.tile_sum = ia(O_TILE);
  // blocks per image: enough to fill the machine across the images
  const long long per = std::max<long long>(1, std::min<long long>((maxN + 255) / 256, (152LL * 16 + n - 1) / n));
  const dim3 gp{static_cast<unsigned>(per), static_cast<unsigned>(n)};
  const int gs = 152 * 8;
  const unsigned nt = unsigned(ntiles);
  unsigned long long hc[3] = {};
  int herr = 0;
  do {
    if ((e = cudaMemcpyAsync(table, host.data(), sizeof(Img) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.size, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.csum, 0, up(size_t(T) * 24), s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(S.cnt, 0, 256, s)) != cudaSuccess) break;
    k_cc_init<<<gp, 256, 0, s>>>(table, S.parent);
    k_cc_union<<<gp, 256, 0, s>>>(table, S.parent, S.err);
    k_cc_flatten<<<gp, 256, 0, s>>>(table, S.parent, S.err);
    k_root_count<<<nt, 1024, 0, s>>>(T, S);
    k_root_scan<<<1, 1024, 0, s>>>(int(ntiles), S);
    k_root_assign<<<nt, 1024, 0, s>>>(table, n, T, S);
    k_comp_map<<<gp, 256, 0, s>>>(table, S);
    k_comp_flags<<<gs, 256, 0, s>>>(table, S);
    k_edges<<<gp, 256, 0, s>>>(table, S, 0);
    k_scan_tiles<<<nt, 1024, 0, s>>>(S.deg, S.ncomp, S.aoff, S.tile_sum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(S.tile_sum, S.ncomp, S.aoff);
    k_scan_add<<<nt, 1024, 0, s>>>(S.aoff, S.tile_sum, S.ncomp);
    if ((e = cudaMemsetAsync(S.deg, 0, nI, s)) != cudaSuccess) break;
    k_edges<<<gp, 256, 0, s>>>(table, S, 1);
    k_cluster_count<<<gs, 256, 0, s>>>(S);
    k_scan_tiles<<<nt, 1024, 0, s>>>(S.cl_count, S.ncomp, S.cl_off, S.tile_sum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(S.tile_sum, S.ncomp, S.cl_off);
    k_scan_add<<<nt, 1024, 0, s>>>(S.cl_off, S.tile_sum, S.ncomp);
    if ((e = cudaMemsetAsync(S.cl_count, 0, nI, s)) != cudaSuccess) break;
    k_cluster_fill<<<gs, 256, 0, s>>>(S);
    k_cluster_merge<<<gs, 256, 0, s>>>(table, S);
    k_cluster_merge_warp<<<152 * 16, kMergeWarps * 32, 0, s>>>(table, S);
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
