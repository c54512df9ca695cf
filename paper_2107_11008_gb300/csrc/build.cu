// build.cu -- LBVH construction on sm_103a.
//
// Steps (one kernel each, all on the caller's stream):
//   1. gather: triangles from the indexed arrays into float4 vertex triples, shading
//      attributes, centroids, and the centroid bounds (block reduce + sortable-int atomics).
//   2. morton: 63-bit Morton code of each centroid in the normalised bounds (21 bits/axis;
//      10 bits/axis would give ~2 cm cells over a 20 m backdrop, coarser than the glass
//      triangles, and a poor hierarchy over them), with bit 63 set for oversized triangles
//      (a size class in the key, after Vinkler et al. 2017, "Extended Morton codes").
//   3. radix sort of (code, index), least-significant digit first, 8 passes of 8 bits; each
//      pass is histogram -> exclusive scan -> stable scatter (the tile is ranked by 8 one-bit
//      stable splits in shared memory), so equal codes keep input order.
//   4. reorder: triangles into leaf order.
//   5. hierarchy: PLOC agglomerative clustering over the leaves in key order (below), which
//      writes every node's boxes as it makes it.  With SC_BVH_PLOC=0 instead: Karras (HPG 2012)
//      -- internal node i covers a key range found from the longest-common-prefix function
//      delta(i, j) (ties broken by index) -- and a refit in which each leaf climbs to the root and
//      the second arrival at a node merges both boxes (__threadfence + an atomic counter per node).
//   6. depth of the deepest leaf; the 4-wide collapse.
#include <cfloat>

#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace sc {

constexpr int kTile = kSortTile;

size_t sort_blocks(int32_t n) { return sort_blocks_for(n); }

// order-preserving float <-> uint32 map for atomic min/max
__device__ __forceinline__ uint32_t f2key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void k_init_bounds(uint32_t *bounds, int32_t *depth) {
  const int i = threadIdx.x;
  if (i < 3) bounds[i] = 0xFFFFFFFFu;
  else if (i < 6) bounds[i] = 0u;
  if (i == 0) *depth = 0;
}

__global__ void k_gather(BuildBuffers b) {
  __shared__ float red[6][32];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  if (t < b.n_tris) {
    const int i0 = b.indices[3 * t], i1 = b.indices[3 * t + 1], i2 = b.indices[3 * t + 2];
    const int vi[3] = {i0, i1, i2};
    float3 c = f3(0.f, 0.f, 0.f), plo = f3(FLT_MAX, FLT_MAX, FLT_MAX), phi = f3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
    for (int j = 0; j < 3; ++j) {
      const float3 p = f3(b.positions + 3 * vi[j]);
      b.tris_in[3 * t + j] = make_float4(p.x, p.y, p.z, j == 0 ? __int_as_float(t) : 0.0f);
      c = c + p;
      plo = f3(fminf(plo.x, p.x), fminf(plo.y, p.y), fminf(plo.z, p.z));
      phi = f3(fmaxf(phi.x, p.x), fmaxf(phi.y, p.y), fmaxf(phi.z, p.z));
      const float3 n = b.normals ? f3(b.normals + 3 * vi[j]) : f3(0.f, 0.f, 0.f);
      const float ux = b.uvs ? b.uvs[2 * vi[j]] : 0.0f;
      b.shade[3 * t + j] = make_float4(n.x, n.y, n.z, ux);
    }
    const int obj = b.tri_object[t];
    const int mat = (obj >= 0 && obj < b.n_objects) ? b.object_material[obj] : 0;
    b.shade2[t] = make_float4(b.uvs ? b.uvs[2 * i0 + 1] : 0.0f, b.uvs ? b.uvs[2 * i1 + 1] : 0.0f,
                              b.uvs ? b.uvs[2 * i2 + 1] : 0.0f, __int_as_float(mat));
    b.tri_obj[t] = obj;
    c = c * (1.0f / 3.0f);
    // w: the triangle's largest box extent (the size class of its Morton key)
    b.centroids[t] = make_float4(c.x, c.y, c.z, fmaxf(fmaxf(phi.x - plo.x, phi.y - plo.y), phi.z - plo.z));
    lo[0] = hi[0] = c.x;
    lo[1] = hi[1] = c.y;
    lo[2] = hi[2] = c.z;
  }
  // warp then block reduction of the centroid bounds
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 3; ++k) {
      red[k][warp] = lo[k];
      red[3 + k][warp] = hi[k];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    float v = red[k][0];
    for (int w = 1; w < nw; ++w) v = k < 3 ? fminf(v, red[k][w]) : fmaxf(v, red[k][w]);
    if (v != FLT_MAX && v != -FLT_MAX) {
      if (k < 3) atomicMin(&b.bounds[k], f2key(v));
      else atomicMax(&b.bounds[k], f2key(v));
    }
  }
}

// spread the low 21 bits of v to every third bit of a 64-bit word
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void k_morton(BuildBuffers b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.n_tris) return;
  const float3 lo = f3(key2f(b.bounds[0]), key2f(b.bounds[1]), key2f(b.bounds[2]));
  const float3 hi = f3(key2f(b.bounds[3]), key2f(b.bounds[4]), key2f(b.bounds[5]));
  const float4 c = b.centroids[t];
  const float cc[3] = {c.x, c.y, c.z}, l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
  uint32_t q[3];
  for (int k = 0; k < 3; ++k) {
    const float ext = h[k] - l[k];
    const float u = ext > 0.0f ? (cc[k] - l[k]) / ext : 0.5f;
    q[k] = (uint32_t)fminf(fmaxf(u * 2097152.0f, 0.0f), 2097151.0f);
  }
  // Bit 63 (above the 63 Morton bits) marks triangles whose box spans more than an eighth of the
  // largest centroid extent: they sort after all others, so the root separates them and their
  // boxes (a backdrop quad's is metres wide) stay out of the subtrees of the small triangles;
  // mixed into those subtrees by centroid, every ancestor box would span the backdrop.
  const float span = fmaxf(fmaxf(h[0] - l[0], h[1] - l[1]), h[2] - l[2]);
  const unsigned long long big = (span > 0.0f && c.w > 0.125f * span) ? (1ull << 63) : 0ull;
  b.keys[t] = big | (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  b.vals[t] = (uint32_t)t;
}

__global__ void k_sort_hist(const unsigned long long *keys, int32_t n, int shift, uint32_t *hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kTile;
  for (int j = 0; j < kSortItems; ++j) {
    const int i = base + j * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of a 256-thread block; returns the prefix, *total gets the sum
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  const uint32_t before = warp == 0 ? 0u : warp_sums[warp - 1];
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

// single-block exclusive scan over n words (digit-major histogram)
__global__ void k_scan(uint32_t *data, int n) {
  __shared__ uint32_t ws[32];
  uint32_t carry = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < n ? data[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_scan(v, ws, &total);
    if (i < n) data[i] = carry + ex;
    carry += total;
  }
}

__global__ void k_sort_scatter(const unsigned long long *keys, const uint32_t *vals, unsigned long long *keys_out,
                               uint32_t *vals_out, int32_t n, int shift, const uint32_t *hist, int nblocks) {
  __shared__ unsigned long long sk[2][kTile];
  __shared__ uint32_t sv[2][kTile];
  __shared__ uint32_t ws[32];
  __shared__ uint32_t start[256];
  __shared__ uint32_t cnt[256];
  const int base = blockIdx.x * kTile;
  const int count = min(kTile, n - base);
  // load; padding items get digit 0xFF so that they sort last and are never written
  for (int j = 0; j < kSortItems; ++j) {
    const int l = j * kSortThreads + threadIdx.x;
    const int i = base + l;
    sk[0][l] = i < n ? keys[i] : ~0ull;
    sv[0][l] = i < n ? vals[i] : 0xFFFFFFFFu;
  }
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int cur = 0;
  // 8 stable one-bit splits on the digit; thread t owns items 8t .. 8t+7 (in tile order)
  for (int bit = 0; bit < 8; ++bit) {
    uint32_t zeros = 0;
    unsigned long long k[kSortItems];
    uint32_t v[kSortItems];
    for (int j = 0; j < kSortItems; ++j) {
      k[j] = sk[cur][threadIdx.x * kSortItems + j];
      v[j] = sv[cur][threadIdx.x * kSortItems + j];
      zeros += ((k[j] >> (shift + bit)) & 1ull) ? 0u : 1u;
    }
    uint32_t total_zeros;
    const uint32_t zpre = block_scan(zeros, ws, &total_zeros);
    uint32_t z = zpre, o = total_zeros + threadIdx.x * kSortItems - zpre;
    for (int j = 0; j < kSortItems; ++j) {
      const bool one = (k[j] >> (shift + bit)) & 1ull;
      const uint32_t dst = one ? o++ : z++;
      sk[cur ^ 1][dst] = k[j];
      sv[cur ^ 1][dst] = v[j];
    }
    cur ^= 1;
    __syncthreads();
  }
  // local digit starts
  for (int j = 0; j < kSortItems; ++j) {
    const int l = threadIdx.x * kSortItems + j;
    if (l < count) atomicAdd(&cnt[(uint32_t)(sk[cur][l] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  uint32_t tot;
  const uint32_t ex = block_scan(cnt[threadIdx.x], ws, &tot);
  start[threadIdx.x] = ex;
  __syncthreads();
  for (int j = 0; j < kSortItems; ++j) {
    const int l = j * kSortThreads + threadIdx.x;
    if (l < count) {
      const unsigned long long key = sk[cur][l];
      const uint32_t d = (uint32_t)(key >> shift) & 0xFFu;
      const uint32_t pos = hist[d * nblocks + blockIdx.x] + (uint32_t)l - start[d];
      keys_out[pos] = key;
      vals_out[pos] = sv[cur][l];
    }
  }
}

__global__ void k_reorder(BuildBuffers b, const uint32_t *order) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.n_tris) return;
  const uint32_t t = order[k];
  b.tris[3 * k] = b.tris_in[3 * t];
  b.tris[3 * k + 1] = b.tris_in[3 * t + 1];
  b.tris[3 * k + 2] = b.tris_in[3 * t + 2];
}

// longest common prefix of sorted keys i and j (index bits break ties), -1 outside
__device__ __forceinline__ int delta(const unsigned long long *keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const unsigned long long a = keys[i], b = keys[j];
  if (a == b) return 64 + __clz((uint32_t)i ^ (uint32_t)j);
  return __clzll(a ^ b);
}

__global__ void k_karras(BuildBuffers b, const unsigned long long *keys) {
  const int n = b.n_tris;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(keys, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    const int t = (l + div - 1) / div;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
  }
  const int gamma = i + s * d + min(d, 0);
  const int lo = min(i, j), hi = max(i, j);
  const int left = (lo == gamma) ? ~gamma : gamma;
  const int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  b.nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.0f, 0.0f);
  // parents: internal nodes at [0, n-1), leaves at [n-1, 2n-1)
  const int pl = left < 0 ? (n - 1) + ~left : left;
  const int pr = right < 0 ? (n - 1) + ~right : right;
  b.parents[pl] = (i << 1) | 0;
  b.parents[pr] = (i << 1) | 1;
  b.flags[i] = 0;
}

__device__ __forceinline__ void store_box(float4 *nodes, int parent, int slot, float3 lo, float3 hi) {
  float4 *nd = nodes + 4 * parent;
  if (slot == 0) {
    nd[0] = make_float4(lo.x, hi.x, lo.y, hi.y);
    reinterpret_cast<float2 *>(&nd[2])[0] = make_float2(lo.z, hi.z);
  } else {
    nd[1] = make_float4(lo.x, hi.x, lo.y, hi.y);
    reinterpret_cast<float2 *>(&nd[2])[1] = make_float2(lo.z, hi.z);
  }
}

__global__ void k_refit(BuildBuffers b) {
  const int n = b.n_tris;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float3 v0 = xyz(b.tris[3 * k]), v1 = xyz(b.tris[3 * k + 1]), v2 = xyz(b.tris[3 * k + 2]);
  float3 lo = f3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
  float3 hi = f3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
  if (n == 1) {
    // a single triangle: a root whose two slots both hold that leaf (a slab test cannot
    // reject an inverted box, so no empty slot is used)
    store_box(b.nodes, 0, 0, lo, hi);
    store_box(b.nodes, 0, 1, lo, hi);
    b.nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), 0.0f, 0.0f);
    return;
  }
  int link = b.parents[(n - 1) + k];
  int depth = 1;
  for (;;) {
    const int parent = link >> 1, slot = link & 1;
    store_box(b.nodes, parent, slot, lo, hi);
    __threadfence();
    if (atomicAdd(&b.flags[parent], 1) == 0) return;  // the sibling finishes this node
    __threadfence();
    const float4 a = __ldcg(&b.nodes[4 * parent]), c = __ldcg(&b.nodes[4 * parent + 1]);
    const float4 z = __ldcg(&b.nodes[4 * parent + 2]);
    lo = f3(fminf(a.x, c.x), fminf(a.z, c.z), fminf(z.x, z.z));
    hi = f3(fmaxf(a.y, c.y), fmaxf(a.w, c.w), fmaxf(z.y, z.w));
    if (parent == 0) break;
    link = b.parents[parent];
    ++depth;
  }
}

// ---- PLOC: the binary tree by agglomerative clustering ----------------------------------------
// Meister & Bittner (2018), "Parallel locally-ordered clustering for bounding volume hierarchy
// construction": the leaves start as clusters in Morton order; every round, each cluster finds the
// neighbour within kPlocR places whose union box has the smallest surface area, mutual pairs merge
// into a new internal node (its boxes written as it is made, so no refit), and the clusters
// compact in order.  Against the Morton split of the LBVH the tree's summed internal-box area drops
// by about 40 % on the glass workloads.  A NaN area counts as infinite and ties are broken by keys
// symmetric in the pair (ploc_nearest), so the least pair is always mutual and every round merges
// at least once.  Internal nodes are numbered downward from n - 2 in merge order
// (ranks from prefix sums, not atomics: the tree is deterministic), so the last merge, the root, is
// node 0.  While many clusters remain a round is four grid-wide launches; a single block finishes
// the last ones.  The rounds run on the device from counters in device memory: no host sync.
#ifndef SC_BVH_PLOC
#define SC_BVH_PLOC 1
#endif
constexpr int kPlocR = 8;         // neighbour window (the tree's area changed by < 0.5 % from 8 to 25)
constexpr int kPlocBlock = 256;
constexpr int kPlocSmall = 1024;  // clusters below which one block finishes

// Views into scratch the sort no longer needs: cluster boxes ping-pong between tris_in (lo[0],
// hi[0], hi[1]) and centroids (lo[1]); references in keys, neighbours and per-block counts in
// keys_alt; control words in bounds: [0, 1] cluster count by round parity, [2, 3] first merge rank
// of the round by parity, [4] merges so far.
struct Ploc {
  float4 *lo[2], *hi[2];
  int32_t *ref[2];
  int32_t *nn;
  uint32_t *blk;
  uint32_t *ctl;
};

__host__ __device__ inline Ploc ploc_views(const BuildBuffers &b) {
  Ploc P;
  const int n = b.n_tris;
  P.lo[0] = b.tris_in;
  P.hi[0] = b.tris_in + n;
  P.hi[1] = b.tris_in + 2 * n;
  P.lo[1] = b.centroids;
  P.ref[0] = reinterpret_cast<int32_t *>(b.keys);
  P.ref[1] = reinterpret_cast<int32_t *>(b.keys) + n;
  P.nn = reinterpret_cast<int32_t *>(b.keys_alt);
  P.blk = reinterpret_cast<uint32_t *>(b.keys_alt) + n;
  P.ctl = b.bounds;
  return P;
}

__device__ __forceinline__ float ploc_area(float4 la, float4 ha, float4 lb, float4 hb) {
  const float dx = fmaxf(ha.x, hb.x) - fminf(la.x, lb.x), dy = fmaxf(ha.y, hb.y) - fminf(la.y, lb.y);
  const float dz = fmaxf(ha.z, hb.z) - fminf(la.z, lb.z);
  const float a = dx * dy + dy * dz + dz * dx;  // half the surface area
  return a == a ? a : __int_as_float(0x7f800000);
}

// The neighbour of cluster i (of m) whose union with it has the least area.  Ties go to the
// nearer index, then to the partner i ^ 1, then to the lower index: each of these keys is
// symmetric in the pair, so the pairs are totally ordered (the least one is mutual: progress), and
// equal boxes (duplicate triangles) pair off (2k, 2k + 1) into a balanced tree instead of a chain.
__device__ __forceinline__ int ploc_nearest(const float4 *lo, const float4 *hi, int i, int m) {
  const float4 li = lo[i], hi_ = hi[i];
  int bj = -1, bd = 0;
  bool bp = false;
  float best = 0.0f;
  const int j1 = min(m - 1, i + kPlocR);
  for (int j = max(0, i - kPlocR); j <= j1; ++j) {
    if (j == i) continue;
    const float a = ploc_area(li, hi_, lo[j], hi[j]);
    const int d = j > i ? j - i : i - j;
    const bool pf = j == (i ^ 1);
    if (bj < 0 || a < best || (a == best && (d < bd || (d == bd && pf && !bp)))) {
      best = a;
      bj = j;
      bd = d;
      bp = pf;
    }
  }
  return bj;
}

__device__ __forceinline__ int child_slot_index(int ref, int n) { return ref >= 0 ? ref : (n - 1) + ~ref; }

// cluster i and its mutual neighbour j > i become internal node p; the merged cluster is returned
__device__ __forceinline__ void ploc_make_node(const BuildBuffers &b, int n, int p, float4 li, float4 hi_, int ri,
                                               float4 lj, float4 hj, int rj, float4 &lo_out, float4 &hi_out) {
  store_box(b.nodes, p, 0, f3(li.x, li.y, li.z), f3(hi_.x, hi_.y, hi_.z));
  store_box(b.nodes, p, 1, f3(lj.x, lj.y, lj.z), f3(hj.x, hj.y, hj.z));
  b.nodes[4 * p + 3] = make_float4(__int_as_float(ri), __int_as_float(rj), 0.0f, 0.0f);
  b.parents[child_slot_index(ri, n)] = p << 1;
  b.parents[child_slot_index(rj, n)] = (p << 1) | 1;
  lo_out = make_float4(fminf(li.x, lj.x), fminf(li.y, lj.y), fminf(li.z, lj.z), 0.0f);
  hi_out = make_float4(fmaxf(hi_.x, hj.x), fmaxf(hi_.y, hj.y), fmaxf(hi_.z, hj.z), 0.0f);
}

__global__ void k_ploc_init(BuildBuffers b) {
  const Ploc P = ploc_views(b);
  const int n = b.n_tris;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    P.ctl[0] = (uint32_t)n;
    P.ctl[4] = 0u;
  }
  if (i >= n) return;
  const float3 v0 = xyz(b.tris[3 * i]), v1 = xyz(b.tris[3 * i + 1]), v2 = xyz(b.tris[3 * i + 2]);
  P.lo[0][i] = make_float4(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)),
                           fminf(v0.z, fminf(v1.z, v2.z)), 0.0f);
  P.hi[0][i] = make_float4(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)),
                           fmaxf(v0.z, fmaxf(v1.z, v2.z)), 0.0f);
  P.ref[0][i] = ~i;
}

__global__ void __launch_bounds__(kPlocBlock) k_ploc_nn(BuildBuffers b, int par) {
  const Ploc P = ploc_views(b);
  const int m = (int)P.ctl[par];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) P.nn[i] = ploc_nearest(P.lo[par], P.hi[par], i, m);
}

// per block: clusters that open a merge (the lower of a mutual pair) and clusters that stay
__global__ void __launch_bounds__(kPlocBlock) k_ploc_count(BuildBuffers b, int par) {
  const Ploc P = ploc_views(b);
  const int m = (int)P.ctl[par];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool merge = false, keep = false;
  if (i < m) {
    const int j = P.nn[i];
    const bool mutual = j >= 0 && P.nn[j] == i;
    merge = mutual && i < j;
    keep = !(mutual && j < i);
  }
  const int nm = __syncthreads_count(merge), nk = __syncthreads_count(keep);
  if (threadIdx.x == 0) {
    P.blk[2 * blockIdx.x] = (uint32_t)nm;
    P.blk[2 * blockIdx.x + 1] = (uint32_t)nk;
  }
}

// one block: exclusive prefixes of the per-block counts, the next round's cluster count, the
// round's first merge rank
__global__ void k_ploc_scan(BuildBuffers b, int nblk, int par) {
  __shared__ uint32_t ws[32];
  const Ploc P = ploc_views(b);
  uint32_t carry_m = 0, carry_k = 0;
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const uint32_t vm = k < nblk ? P.blk[2 * k] : 0u, vk = k < nblk ? P.blk[2 * k + 1] : 0u;
    uint32_t tm, tk;
    const uint32_t em = block_scan(vm, ws, &tm);
    const uint32_t ek = block_scan(vk, ws, &tk);
    if (k < nblk) {
      P.blk[2 * k] = carry_m + em;
      P.blk[2 * k + 1] = carry_k + ek;
    }
    carry_m += tm;
    carry_k += tk;
  }
  if (threadIdx.x == 0) {
    P.ctl[2 + par] = P.ctl[4];
    P.ctl[4] += carry_m;
    P.ctl[par ^ 1] = carry_k;
  }
}

__global__ void __launch_bounds__(kPlocBlock) k_ploc_merge(BuildBuffers b, int par) {
  __shared__ uint32_t ws[32];
  const Ploc P = ploc_views(b);
  const int n = b.n_tris;
  const int m = (int)P.ctl[par];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = -1;
  bool merge = false, keep = false;
  if (i < m) {
    j = P.nn[i];
    const bool mutual = j >= 0 && P.nn[j] == i;
    merge = mutual && i < j;
    keep = !(mutual && j < i);
  }
  uint32_t tm, tk;
  const uint32_t rm = block_scan(merge ? 1u : 0u, ws, &tm) + P.blk[2 * blockIdx.x];
  const uint32_t rk = block_scan(keep ? 1u : 0u, ws, &tk) + P.blk[2 * blockIdx.x + 1];
  if (!keep) return;
  float4 lo = P.lo[par][i], hi = P.hi[par][i];
  int ref = P.ref[par][i];
  if (merge) {
    const int p = (n - 2) - (int)(P.ctl[2 + par] + rm);
    float4 lo2, hi2;
    ploc_make_node(b, n, p, lo, hi, ref, P.lo[par][j], P.hi[par][j], P.ref[par][j], lo2, hi2);
    lo = lo2;
    hi = hi2;
    ref = p;
  }
  P.lo[par ^ 1][rk] = lo;
  P.hi[par ^ 1][rk] = hi;
  P.ref[par ^ 1][rk] = ref;
}

// One block of 1024 finishes the clusters left after the grid-wide rounds: the same round in
// chunks of the block's width, __syncthreads between the phases.  At least one merge per round,
// so at most m - 1 rounds.
__global__ void __launch_bounds__(1024) k_ploc_finish(BuildBuffers b, int par) {
  __shared__ uint32_t ws[32];
  const Ploc P = ploc_views(b);
  const int n = b.n_tris;
  int m = (int)P.ctl[par];
  uint32_t merged = P.ctl[4];
  for (int round = 0; m > 1 && round < n; ++round, par ^= 1) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) P.nn[i] = ploc_nearest(P.lo[par], P.hi[par], i, m);
    __syncthreads();
    uint32_t carry_m = 0, carry_k = 0;
    for (int base = 0; base < m; base += blockDim.x) {
      const int i = base + threadIdx.x;
      int j = -1;
      bool merge = false, keep = false;
      if (i < m) {
        j = P.nn[i];
        const bool mutual = j >= 0 && P.nn[j] == i;
        merge = mutual && i < j;
        keep = !(mutual && j < i);
      }
      uint32_t tm, tk;
      const uint32_t rm = carry_m + block_scan(merge ? 1u : 0u, ws, &tm);
      const uint32_t rk = carry_k + block_scan(keep ? 1u : 0u, ws, &tk);
      if (keep) {
        float4 lo = P.lo[par][i], hi = P.hi[par][i];
        int ref = P.ref[par][i];
        if (merge) {
          const int p = (n - 2) - (int)(merged + rm);
          float4 lo2, hi2;
          ploc_make_node(b, n, p, lo, hi, ref, P.lo[par][j], P.hi[par][j], P.ref[par][j], lo2, hi2);
          lo = lo2;
          hi = hi2;
          ref = p;
        }
        P.lo[par ^ 1][rk] = lo;
        P.hi[par ^ 1][rk] = hi;
        P.ref[par ^ 1][rk] = ref;
      }
      carry_m += tm;
      carry_k += tk;
    }
    merged += carry_m;
    m = (int)carry_k;
    __syncthreads();  // the next round reads what this one wrote
  }
}

// rounds of the grid-wide form: enough that ~1000 clusters are left, at the ~0.82 of clusters a
// round keeps on the glass workloads (0.84 assumed); extra rounds cost little, missing ones only
// leave more to the single block
int ploc_grid_rounds(int n) {
  if (n <= kPlocSmall) return 0;
  return (int)std::ceil(std::log((double)n / kPlocSmall) / std::log(1.0 / 0.84));
}

cudaError_t launch_ploc(const BuildBuffers &b, cudaStream_t s) {
  const int n = b.n_tris;
  const int G = (n + kPlocBlock - 1) / kPlocBlock;
  k_ploc_init<<<G, kPlocBlock, 0, s>>>(b);
  const int rounds = ploc_grid_rounds(n);
  int par = 0;
  for (int r = 0; r < rounds; ++r, par ^= 1) {
    k_ploc_nn<<<G, kPlocBlock, 0, s>>>(b, par);
    k_ploc_count<<<G, kPlocBlock, 0, s>>>(b, par);
    k_ploc_scan<<<1, 1024, 0, s>>>(b, G, par);
    k_ploc_merge<<<G, kPlocBlock, 0, s>>>(b, par);
  }
  k_ploc_finish<<<1, 1024, 0, s>>>(b, par);
  return cudaGetLastError();
}

// depth of every leaf (walk to the root); keeps the maximum
__global__ void k_depth(BuildBuffers b) {
  const int n = b.n_tris;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || n < 2) return;
  int node = (n - 1) + k, d = 0;
  while (true) {
    const int p = b.parents[node] >> 1;
    ++d;
    if (p == 0) break;
    node = p;
    if (d > 4 * 64) break;
  }
  atomicMax(b.depth, d);
}

// Collapse the binary LBVH into 4-wide nodes, one per binary internal node (stored at its
// index).  SC_COLLAPSE_GREEDY: starting from the node's two children, the internal child with the
// largest surface area is replaced by its two children until there are four (or only leaves):
// wide nodes then split space where the binary tree's big boxes are, wherever that is in depth.
// Otherwise the children of the node's children (every binary node at even depth becomes a wide
// node).  A record depends on its binary subtree alone, so all are built at once; traversal from
// the root reaches only the records its references name.
#ifndef SC_COLLAPSE_GREEDY
#define SC_COLLAPSE_GREEDY 1
#endif
__global__ void k_collapse4(BuildBuffers b) {
  const int n = b.n_tris;
  const int n_int = n > 1 ? n - 1 : 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  float lo[3][4], hi[3][4];
  int ref[4];
  // entry k <- child `slot` of binary node m
  auto put = [&](int m, int slot, int k) {
    const float4 *nd = b.nodes + 4 * m;
    const float4 xy = nd[slot], z = nd[2], r = nd[3];
    lo[0][k] = xy.x;
    hi[0][k] = xy.y;
    lo[1][k] = xy.z;
    hi[1][k] = xy.w;
    lo[2][k] = slot ? z.z : z.x;
    hi[2][k] = slot ? z.w : z.y;
    ref[k] = __float_as_int(slot ? r.y : r.x);
  };
  int cnt = 0;
#if SC_COLLAPSE_GREEDY
  put(i, 0, cnt++);
  put(i, 1, cnt++);
  while (cnt < 4) {
    int best = -1;
    float best_area = -1.0f;
    for (int k = 0; k < cnt; ++k) {
      if (ref[k] < 0) continue;
      const float dx = hi[0][k] - lo[0][k], dy = hi[1][k] - lo[1][k], dz = hi[2][k] - lo[2][k];
      const float area = dx * dy + dy * dz + dz * dx;
      if (area > best_area) {
        best_area = area;
        best = k;
      }
    }
    if (best < 0) break;
    const int m = ref[best];
    put(m, 1, cnt++);
    put(m, 0, best);
  }
#else
  const float4 r = b.nodes[4 * i + 3];
  for (int slot = 0; slot < 2; ++slot) {
    const int c = __float_as_int(slot ? r.y : r.x);
    if (c < 0) {
      put(i, slot, cnt++);
    } else {
      put(c, 0, cnt++);
      put(c, 1, cnt++);
    }
  }
#endif
  // empty slots: an inverted box (lo > hi on every axis), which no ray enters whatever the signs
  // of its direction, so traversal needs no test of the reference
  for (int k = cnt; k < 4; ++k) {
    lo[0][k] = lo[1][k] = lo[2][k] = 3.0e38f;
    hi[0][k] = hi[1][k] = hi[2][k] = -3.0e38f;
    ref[k] = kEmptyRef;
  }
  float4 *o = b.nodes4 + 8 * i;
  for (int a = 0; a < 3; ++a) {
    o[2 * a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
    o[2 * a + 1] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
  }
  o[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]), __int_as_float(ref[3]));
  o[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

#define SC_TRY(x)                              \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return e_;          \
  } while (0)

// Stable LSD radix sort of n (key, value) pairs on the byte digits first_byte .. first_byte +
// passes - 1 of the keys (an even number of passes leaves the result in keys / vals).
cudaError_t radix_sort_pairs(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                             uint32_t *vals_alt, uint32_t *hist, int32_t n, int first_byte, int passes,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (int)sort_blocks(n);
  unsigned long long *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * (first_byte + pass);
    k_sort_hist<<<nb, kSortThreads, 0, s>>>(ka, n, shift, hist, nb);
    k_scan<<<1, 1024, 0, s>>>(hist, 256 * nb);
    k_sort_scatter<<<nb, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
    unsigned long long *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  return cudaGetLastError();
}

cudaError_t launch_build(const BuildBuffers &b, cudaStream_t s) {
  const int n = b.n_tris;
  if (n <= 0) return cudaSuccess;
  const int T = 256, G = (n + T - 1) / T;
  k_init_bounds<<<1, 32, 0, s>>>(b.bounds, b.depth);
  k_gather<<<G, T, 0, s>>>(b);
  k_morton<<<G, T, 0, s>>>(b);
  SC_TRY(cudaGetLastError());
  const int nb = (int)sort_blocks(n);
  unsigned long long *ka = b.keys, *kb = b.keys_alt;
  uint32_t *va = b.vals, *vb = b.vals_alt;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    k_sort_hist<<<nb, kSortThreads, 0, s>>>(ka, n, shift, b.hist, nb);
    k_scan<<<1, 1024, 0, s>>>(b.hist, 256 * nb);
    k_sort_scatter<<<nb, kSortThreads, 0, s>>>(ka, va, kb, vb, n, shift, b.hist, nb);
    unsigned long long *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  SC_TRY(cudaGetLastError());
  // after an even number of passes the sorted data is back in keys / vals
  k_reorder<<<G, T, 0, s>>>(b, va);
#if SC_BVH_PLOC
  if (n > 1) {
    SC_TRY(launch_ploc(b, s));
  } else {
    k_refit<<<G, T, 0, s>>>(b);  // one triangle: the root holds it in both slots
  }
#else
  if (n > 1) {
    const int Gi = (n - 1 + T - 1) / T;
    k_karras<<<Gi, T, 0, s>>>(b, ka);
  }
  k_refit<<<G, T, 0, s>>>(b);
#endif
  k_depth<<<G, T, 0, s>>>(b);
  if (b.nodes4) {
    const int Gi = (std::max(n - 1, 1) + T - 1) / T;
    k_collapse4<<<Gi, T, 0, s>>>(b);
  }
  return cudaGetLastError();
}

}  // namespace sc
