// device.cuh -- device-side building blocks of the sm_103a path/light tracer.
//
// Layout in HBM (all 16-byte aligned):
//   nodes   float4[4 * n_nodes]  binary BVH node = both child boxes + child refs (64 B):
//           (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y) (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//           (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z) (child0, child1 as int bits, -, -)
//           a child >= 0 is an internal node, < 0 is leaf ~k (one triangle, leaf order k).
//   tris    float4[3 * n_tris]   vertices in leaf order; tris[3k].w = input triangle id bits.
//   shade   float4[3 * n_tris]   per input triangle: (normal_j.xyz, uv_j.x) for j = 0..2.
//   shade2  float4[n_tris]       (uv0.y, uv1.y, uv2.y, material id bits).
//   tri_obj int32[n_tris]        object id per input triangle.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "supercaustics.h"

namespace sc {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kStack = 96;   // 4-wide traversal (camera kernel) pushes up to 3 entries per visit
constexpr int kStack2 = 64;  // binary traversal (trace())
constexpr uint32_t kMiss = 0xFFFFFFFFu;
constexpr int kMaxBins = 64;
// traversal watchdog: node visits per query before the query is abandoned (default; the context's
// limits override it per launch, sc_set_limits)
constexpr int kMaxVisits = 1 << 22;

enum : uint32_t { EV_REFLECT = 1, EV_REFRACT = 2, EV_LIT = 3, EV_UNLIT = 4, EV_FIXUP = 7, EV_KILL = 9 };

// Checked builds (-DSC_CHECKED): SC_IN_RANGE(status, site, v, n) is false when v is outside
// [0, n); the first failure stores (site, v, thread) in status[8..10] and sets
// SC_STATUS_BOUNDS, and the caller skips the access.  Release builds compile it to `true`.
#ifdef SC_CHECKED
__device__ __forceinline__ bool sc_in_range(unsigned *status, unsigned site, long long v, long long n) {
  if (v >= 0 && v < n) return true;
  atomicOr(status, SC_STATUS_BOUNDS);
  if (atomicCAS(status + 8, 0u, site) == 0u) {
    status[9] = (unsigned)v;
    status[10] = blockIdx.x * blockDim.x + threadIdx.x;
  }
  return false;
}
#define SC_IN_RANGE(status, site, v, n) sc_in_range((status), (site), (long long)(v), (long long)(n))
#else
#define SC_IN_RANGE(status, site, v, n) true
#endif

// ------------------------------------------------------------------------------------------
// float3 algebra
// ------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 f3(const float *p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float3 xyz(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float length(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float maxabs(float3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }
__device__ __forceinline__ float comp(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies
// with Weyl key bumps.  Counter word 3 carries tag | scene << 8.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}
__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag,
                                      uint32_t scene) {
  return philox(make_uint4(c0, c1, c2, tag | (scene << 8)), (uint32_t)seed, (uint32_t)(seed >> 32));
}
// 24-bit uniform in [0,1), exact in FP32
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
// floor(u * n) in exact integer arithmetic
__device__ __forceinline__ int choose(uint32_t x, int n) {
  return (int)(((uint64_t)(x >> 8) * (uint64_t)n) >> 24);
}
__device__ __forceinline__ uint32_t fnv(uint32_t h, uint32_t w) { return (h ^ w) * 16777619u; }

// ------------------------------------------------------------------------------------------
// Spectrum: bin centres over 400-700 nm; RGB weight = linear sRGB of the multi-lobe CIE 1931
// fit (Wyman, Sloan, Shirley, JCGT 2013), normalised to mean 1 per channel over the bins.
// ------------------------------------------------------------------------------------------
// The table is tiny (one entry per bin, built once per block), so it is evaluated in FP64: the
// XYZ -> RGB rows cancel strongly for some bins and FP32 would leave ~1e-4 relative error there.
__host__ __device__ inline double lobe_hd(double lam, double mu, double s1, double s2) {
  const double t = (lam - mu) / (lam < mu ? s1 : s2);
  return exp(-0.5 * t * t);
}
__host__ __device__ inline void lambda_rgb(double lam, double out[3]) {
  const double X = 1.056 * lobe_hd(lam, 599.8, 37.9, 31.0) + 0.362 * lobe_hd(lam, 442.0, 16.0, 26.7) -
                   0.065 * lobe_hd(lam, 501.1, 20.4, 26.2);
  const double Y = 0.821 * lobe_hd(lam, 568.8, 46.9, 40.5) + 0.286 * lobe_hd(lam, 530.9, 16.3, 31.1);
  const double Z = 1.217 * lobe_hd(lam, 437.0, 11.8, 36.0) + 0.681 * lobe_hd(lam, 459.0, 26.0, 13.8);
  out[0] = 3.2404542 * X - 1.5371385 * Y - 0.4985314 * Z;
  out[1] = -0.9692660 * X + 1.8760108 * Y + 0.0415560 * Z;
  out[2] = 0.0556434 * X - 0.2040259 * Y + 1.0572252 * Z;
}
__device__ __forceinline__ void bin_rgb(int b, int nbins, double out[3]) {
  lambda_rgb(400.0 + (b + 0.5) * 300.0 / nbins, out);
}
// Fills w[0..nbins) (shared memory); call from every thread of the block.
__device__ __forceinline__ void spectral_table(float3 *w, int nbins) {
  if (nbins <= 1) {
    if (threadIdx.x == 0) w[0] = f3(1.f, 1.f, 1.f);
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    double mean[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nbins; ++b) {
      double c[3];
      bin_rgb(b, nbins, c);
      for (int k = 0; k < 3; ++k) mean[k] += c[k] / nbins;
    }
    for (int b = 0; b < nbins; ++b) {
      double c[3];
      bin_rgb(b, nbins, c);
      w[b] = f3((float)(c[0] / mean[0]), (float)(c[1] / mean[1]), (float)(c[2] / mean[2]));
    }
  }
  __syncthreads();
}
// A path keeps the uniform u of its bin draw (exact in FP32: u = (x >> 8) 2^-24); its bin is the
// exact integer floor(u B) and its wavelength the bin centre, or with SC_FLAG_WAVELENGTH_JITTER
// 400 + 300 u nm (continuous).
__device__ __forceinline__ int bin_of(float u, int nbins) {
  return (int)(((unsigned long long)(uint32_t)(u * 16777216.0f) * (unsigned)nbins) >> 24);
}
__device__ __forceinline__ float path_lambda(float u, int nbins, bool jitter) {
  return jitter ? 400.0f + 300.0f * u : 400.0f + (bin_of(u, nbins) + 0.5f) * 300.0f / nbins;
}
__device__ __forceinline__ float cauchy_at(float A, float B, float lam, int nbins) {
  if (nbins <= 1) return A;
  const float lum = lam * 1e-3f;
  return A + B / (lum * lum);
}
// Jitter: RGB weight at 400 + 300 u nm, the fit's sRGB there over its 400-700 nm mean (inv_mean
// = 1 / mean per channel, computed on the host), evaluated in FP64 like the bin table.
struct JitterNorm {
  double inv_mean[3];
};
static __device__ __noinline__ float3 jitter_weight(float u, const JitterNorm &jn) {
  double c[3];
  lambda_rgb(400.0 + 300.0 * (double)u, c);
  return make_float3((float)(c[0] * jn.inv_mean[0]), (float)(c[1] * jn.inv_mean[1]), (float)(c[2] * jn.inv_mean[2]));
}
// the normaliser, on the host: composite Simpson rule over 400-700 nm, 3000 intervals
inline JitterNorm jitter_norm_host() {
  const int n = 3000;
  const double h = 300.0 / n;
  double acc[3] = {0.0, 0.0, 0.0}, c[3];
  for (int i = 0; i <= n; ++i) {
    lambda_rgb(400.0 + i * h, c);
    const double w = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    for (int k = 0; k < 3; ++k) acc[k] += w * c[k];
  }
  JitterNorm jn;
  for (int k = 0; k < 3; ++k) jn.inv_mean[k] = 300.0 / (acc[k] * h / 3.0);
  return jn;
}

// ------------------------------------------------------------------------------------------
// Scene as seen by kernels
// ------------------------------------------------------------------------------------------
struct Cam {
  float3 eye, f, r, u;
  float th, aspect;
  int W, H;
};
__device__ __forceinline__ Cam make_cam(const sc_camera &c) {
  Cam k;
  k.eye = f3(c.eye);
  k.f = normalize(f3(c.look) - k.eye);
  k.r = normalize(cross(k.f, f3(c.up)));
  k.u = cross(k.r, k.f);
  k.th = tanf(0.5f * c.vfov_deg * (kPi / 180.0f));
  k.W = c.width;
  k.H = c.height;
  k.aspect = (float)c.width / (float)c.height;
  return k;
}
__device__ __forceinline__ float3 cam_dir(const Cam &c, float sx, float sy) {
  return normalize(c.r * ((2.0f * sx - 1.0f) * c.th * c.aspect) + c.u * ((1.0f - 2.0f * sy) * c.th) + c.f);
}

struct DevScene {
  const float4 *nodes;
  const float4 *nodes4;  // 4-wide nodes collapsed from the binary LBVH (NULL: traverse `nodes`)
  const float4 *tris;
  const float4 *shade;
  const float4 *shade2;
  const int32_t *tri_obj;
  const sc_material *mats;
  const sc_light *lights;
  int32_t n_tris, n_nodes, n_mats, n_lights;
  float env[3];
  sc_camera cam;
  // failure-detection limits of the traversals, filled from the context at each launch
  // (sc_set_limits): node visits per query, stack entries of the 4-wide / binary traversal
  int32_t max_visits, stack4, stack2, pad;
};

// Work tickets of a scene (32 per 8x4 pixel tile) and the blocks of a batched launch over it.
constexpr unsigned kBatchChunk = 512;  // tickets (16 tiles) per block of a batched launch
__host__ __device__ __forceinline__ unsigned scene_tickets(const sc_camera &c) {
  return (unsigned)(((c.width + 7) / 8) * ((c.height + 3) / 4)) * 32u;
}
__host__ __device__ __forceinline__ unsigned scene_blocks(const sc_camera &c) {
  return (scene_tickets(c) + kBatchChunk - 1) / kBatchChunk;
}

// One scene of a batched launch: its tables, its frame buffers, its first block (persistent
// engine) and its first pixel slot in the concatenation of all scenes' tile-order slots (wavefront).
struct BatchEntry {
  DevScene S;
  sc_frame F;
  unsigned begin;
  unsigned slot_begin;
  unsigned pad[2];
};

// ------------------------------------------------------------------------------------------
// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013), both faces, FP32 with an
// FP64 recomputation of an edge function that evaluates to exactly zero.
// ------------------------------------------------------------------------------------------
struct WRay {
  float3 o, d, inv;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};
__device__ __forceinline__ WRay make_wray(float3 o, float3 d) {
  WRay w;
  w.o = o;
  w.d = d;
  // a zero component gets a huge finite reciprocal: with 1/0 = inf, a ray lying in a box face
  // plane would give (l - o) * inf = NaN and the slab test would wrongly reject the box
  w.inv = f3(d.x != 0.0f ? 1.0f / d.x : copysignf(1e30f, d.x), d.y != 0.0f ? 1.0f / d.y : copysignf(1e30f, d.y),
             d.z != 0.0f ? 1.0f / d.z : copysignf(1e30f, d.z));
  const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  w.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  w.kx = w.kz == 2 ? 0 : w.kz + 1;
  w.ky = w.kx == 2 ? 0 : w.kx + 1;
  if (comp(d, w.kz) < 0.0f) {
    const int t = w.kx;
    w.kx = w.ky;
    w.ky = t;
  }
  const float dz = comp(d, w.kz);
  w.Sx = comp(d, w.kx) / dz;
  w.Sy = comp(d, w.ky) / dz;
  w.Sz = 1.0f / dz;
  return w;
}

// Returns true and (t, b1, b2) if the ray meets the triangle at 0 < t.
__device__ __forceinline__ bool tri_test(const WRay &w, float3 v0, float3 v1, float3 v2, float &t, float &b1,
                                         float &b2) {
  const float3 A = v0 - w.o, B = v1 - w.o, C = v2 - w.o;
  const float Akz = comp(A, w.kz), Bkz = comp(B, w.kz), Ckz = comp(C, w.kz);
  const float Ax = comp(A, w.kx) - w.Sx * Akz, Ay = comp(A, w.ky) - w.Sy * Akz;
  const float Bx = comp(B, w.kx) - w.Sx * Bkz, By = comp(B, w.ky) - w.Sy * Bkz;
  const float Cx = comp(C, w.kx) - w.Sx * Ckz, Cy = comp(C, w.ky) - w.Sy * Ckz;
  // edge functions without contraction so that a shared edge evaluates to exact negatives
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
  const float det = U + V + W;
  if (det == 0.0f) return false;
  const float T = U * (w.Sz * Akz) + V * (w.Sz * Bkz) + W * (w.Sz * Ckz);
  t = T / det;
  if (!(t > 0.0f)) return false;
  b1 = V / det;
  b2 = W / det;
  return true;
}

// slab test of one box against [0, tmax]
__device__ __forceinline__ bool box_test(const WRay &w, float lx, float hx, float ly, float hy, float lz, float hz,
                                         float tmax, float &tnear) {
  const float tx0 = (lx - w.o.x) * w.inv.x, tx1 = (hx - w.o.x) * w.inv.x;
  const float ty0 = (ly - w.o.y) * w.inv.y, ty1 = (hy - w.o.y) * w.inv.y;
  const float tz0 = (lz - w.o.z) * w.inv.z, tz1 = (hz - w.o.z) * w.inv.z;
  const float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  // Ize (2013): widen the far bound by 2*gamma(3) so rounding never culls a real hit
  const float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax)) * 1.0000004f;
  tnear = t0;
  return t0 <= t1;
}

// The same slab test with each axis's entry and exit planes already chosen by the sign of the
// ray's reciprocal direction (n* entry, f* exit): with inv >= 0, (lo - o) * inv <= (hi - o) * inv
// holds after rounding too, so the min / max that box_test takes per axis are exactly these, and
// the result is bit for bit box_test's.
__device__ __forceinline__ bool box_test_nf(const WRay &w, float nx, float fx, float ny, float fy, float nz, float fz,
                                            float tmax, float &tnear) {
  const float tnx = (nx - w.o.x) * w.inv.x, tfx = (fx - w.o.x) * w.inv.x;
  const float tny = (ny - w.o.y) * w.inv.y, tfy = (fy - w.o.y) * w.inv.y;
  const float tnz = (nz - w.o.z) * w.inv.z, tfz = (fz - w.o.z) * w.inv.z;
  const float t0 = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.0f));
  const float t1 = fminf(fminf(tfx, tfy), fminf(tfz, tmax)) * 1.0000004f;
  tnear = t0;
  return t0 <= t1;
}

struct Hit {
  float t, b1, b2;
  int prim;     // leaf order, -1 = miss
  uint32_t id;  // input triangle id
};

// Work done by traversal queries (node visits = 4-wide nodes loaded, each with four box tests).
struct TravCount {
  unsigned nodes = 0, tris = 0, queries = 0;
};

// Resumable form of trace(): the query's state lives with the caller and each call visits at
// most `budget` nodes, so a persistent kernel can interleave other lanes' shading with long
// traversals.  Results are identical to trace() (same visit order, same tie-break).
struct TravState {
  Hit h;
  int node, sp, visits;
  bool anyhit;
};
__device__ __forceinline__ void trav_begin(TravState &ts, float tmax, bool anyhit) {
  ts.h.t = tmax;
  ts.h.prim = -1;
  ts.h.id = kMiss;
  ts.h.b1 = ts.h.b2 = 0.0f;
  ts.node = 0;
  ts.sp = 0;
  ts.visits = 0;
  ts.anyhit = anyhit;
}
__device__ __forceinline__ bool trav_step4(const DevScene &S, const WRay &w, float tmax, TravState &ts, int *stack,
                                           int budget, unsigned *status, TravCount &tc);

// Closest hit (anyhit = false; ties on equal t go to the lowest input id) or any hit with
// 0 < t < tmax (anyhit = true; returns the first one found), over the binary LBVH: the kernels
// that trace whole paths per thread (light tracer, resolve, queries) run faster on it than on the
// 4-wide nodes the camera kernel's state machine uses.  One traversal loop serves both so
// that lanes of a warp tracing shadow rays and extension rays stay in the same loop.  Stack
// overflow and the visit watchdog latch a status bit and abandon the query (reported as a miss).
static __device__ __forceinline__ Hit trace(const DevScene &S, float3 o, float3 d, float tmax, bool anyhit,
                                         unsigned *status, TravCount &tc) {
  ++tc.queries;
  Hit h;
  h.t = tmax;
  h.prim = -1;
  h.id = kMiss;
  h.b1 = h.b2 = 0.0f;
  if (S.n_tris <= 0) return h;
  const WRay w = make_wray(o, d);
  int stack[kStack2];
  int sp = 0;
  int node = 0;
  int visits = 0;
  for (;;) {
    ++tc.nodes;
    if (++visits > S.max_visits) {
      atomicOr(status, SC_STATUS_WATCHDOG);
      h.prim = -1;
      h.id = kMiss;
      h.t = tmax;
      return h;
    }
    const float4 n0 = __ldg(&S.nodes[4 * node + 0]);
    const float4 n1 = __ldg(&S.nodes[4 * node + 1]);
    const float4 n2 = __ldg(&S.nodes[4 * node + 2]);
    const float4 n3 = __ldg(&S.nodes[4 * node + 3]);
    const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
    float ta, tb;
    bool ha = box_test(w, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, h.t, ta);
    bool hb = box_test(w, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, h.t, tb);
    // leaves (one triangle each) are tested right away
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool hit_box = side == 0 ? ha : hb;
      const int c = side == 0 ? c0 : c1;
      if (hit_box && c < 0) {
        const int k = ~c;
        const float4 a = __ldg(&S.tris[3 * k]), b = __ldg(&S.tris[3 * k + 1]), cc = __ldg(&S.tris[3 * k + 2]);
        float t, b1, b2;
        ++tc.tris;
        if (tri_test(w, xyz(a), xyz(b), xyz(cc), t, b1, b2)) {
          const uint32_t id = (uint32_t)__float_as_int(a.w);
          if (t < h.t || (!anyhit && t == h.t && id < h.id)) {
            h.t = t; h.b1 = b1; h.b2 = b2; h.prim = k; h.id = id;
            if (anyhit) return h;
          }
        }
        if (side == 0) ha = false;
        else hb = false;
      }
    }
    if (ha && hb) {
      const bool a_first = ta <= tb;
      if (sp >= S.stack2) {
        atomicOr(status, SC_STATUS_STACK_OVERFLOW);
        h.prim = -1;
        h.id = kMiss;
        h.t = tmax;
        return h;
      }
      stack[sp++] = a_first ? c1 : c0;
      node = a_first ? c0 : c1;
    } else if (ha) {
      node = c0;
    } else if (hb) {
      node = c1;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  if (h.prim < 0) h.t = tmax;
  return h;
}

// Returns true when the query is complete (ts.h holds the answer; prim < 0 = miss).
__device__ __forceinline__ bool trav_step(const DevScene &S, const WRay &w, float tmax, TravState &ts, int *stack,
                                          int budget, unsigned *status, TravCount &tc) {
  if (S.n_tris <= 0) return true;
  return trav_step4(S, w, tmax, ts, stack, budget, status, tc);
}

// ------------------------------------------------------------------------------------------
// 4-wide traversal.  Node j of nodes4 (8 float4, j = the index of the binary node it was
// collapsed from) holds, structure-of-arrays, the boxes of up to four children: x lo, x hi,
// y lo, y hi, z lo, z hi, then the four child references (>= 0: a 4-wide node, < 0: leaf ~k,
// kEmptyRef: no child, whose box is inverted so that it is never entered).  One visit tests the
// four boxes, tests the hit leaves' triangles at once, and continues with the nearest hit
// internal child, pushing the others farthest first.
// The closest hit (with its tie-break on the input id) does not depend on the visit order.
// ------------------------------------------------------------------------------------------
constexpr int kEmptyRef = 0x7FFFFFFF;

__device__ __forceinline__ float comp4(const float4 &v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ void sort_pair(float &ka, int &ra, float &kb, int &rb) {
  if (kb < ka) {
    const float tk = ka;
    ka = kb;
    kb = tk;
    const int tr = ra;
    ra = rb;
    rb = tr;
  }
}

__device__ __forceinline__ bool trav_step4(const DevScene &S, const WRay &w, float tmax, TravState &ts, int *stack,
                                           int budget, unsigned *status, TravCount &tc) {
  const float kInf = __int_as_float(0x7f800000);
  for (int it = 0; it < budget; ++it) {
    ++tc.nodes;
    if (++ts.visits > S.max_visits) {
      atomicOr(status, SC_STATUS_WATCHDOG);
      ts.h.prim = -1;
      ts.h.id = kMiss;
      ts.h.t = tmax;
      return true;
    }
    const int node = ts.node;
    if (!SC_IN_RANGE(status, 1, node, S.n_nodes)) {
      ts.h.prim = -1;
      ts.h.id = kMiss;
      ts.h.t = tmax;
      return true;
    }
    const float4 *nd = S.nodes4 + 8 * node;
    // entry / exit bounds of each axis, picked by the sign of the reciprocal direction
    const int sx = w.inv.x < 0.0f, sy = w.inv.y < 0.0f, sz = w.inv.z < 0.0f;
    const float4 nx = __ldg(nd + sx), fx = __ldg(nd + 1 - sx), ny = __ldg(nd + 2 + sy), fy = __ldg(nd + 3 - sy);
    const float4 nz = __ldg(nd + 4 + sz), fz = __ldg(nd + 5 - sz), rr = __ldg(nd + 6);
    int ref[4] = {__float_as_int(rr.x), __float_as_int(rr.y), __float_as_int(rr.z), __float_as_int(rr.w)};
    float key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float tn;
      // empty slots hold inverted boxes and never pass
      const bool hb = box_test_nf(w, comp4(nx, i), comp4(fx, i), comp4(ny, i), comp4(fy, i), comp4(nz, i), comp4(fz, i),
                                  ts.h.t, tn);
      key[i] = hb ? tn : kInf;
    }
    // leaves (one triangle each) are tested right away, the hit ones of this lane in one compact
    // loop (a warp runs as many triangle tests as its busiest lane, not one per child slot)
    unsigned leaves = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (key[i] < kInf && ref[i] < 0) {
        leaves |= 1u << i;
        key[i] = kInf;
      }
    while (leaves) {
      const int i = __ffs(leaves) - 1;
      leaves &= leaves - 1;
      {
        const int k = ~(i == 0 ? ref[0] : (i == 1 ? ref[1] : (i == 2 ? ref[2] : ref[3])));
        if (!SC_IN_RANGE(status, 2, k, S.n_tris)) {
          ts.h.prim = -1;
          ts.h.id = kMiss;
          ts.h.t = tmax;
          return true;
        }
        const float4 a = __ldg(&S.tris[3 * k]), b = __ldg(&S.tris[3 * k + 1]), cc = __ldg(&S.tris[3 * k + 2]);
        float t, b1, b2;
        ++tc.tris;
        if (tri_test(w, xyz(a), xyz(b), xyz(cc), t, b1, b2)) {
          const uint32_t id = (uint32_t)__float_as_int(a.w);
          if (t < ts.h.t || (!ts.anyhit && t == ts.h.t && id < ts.h.id)) {
            ts.h.t = t; ts.h.b1 = b1; ts.h.b2 = b2; ts.h.prim = k; ts.h.id = id;
            if (ts.anyhit) return true;
          }
        }
      }
    }
    // internal children by entry distance (misses sort last)
    sort_pair(key[0], ref[0], key[1], ref[1]);
    sort_pair(key[2], ref[2], key[3], ref[3]);
    sort_pair(key[0], ref[0], key[2], ref[2]);
    sort_pair(key[1], ref[1], key[3], ref[3]);
    sort_pair(key[1], ref[1], key[2], ref[2]);
    const int cnt = (key[0] < kInf) + (key[1] < kInf) + (key[2] < kInf) + (key[3] < kInf);
    if (cnt == 0) {
      if (ts.sp == 0) {
        if (ts.h.prim < 0) ts.h.t = tmax;
        return true;
      }
      ts.node = stack[--ts.sp];
      continue;
    }
    if (ts.sp + cnt - 1 > S.stack4) {
      atomicOr(status, SC_STATUS_STACK_OVERFLOW);
      ts.h.prim = -1;
      ts.h.id = kMiss;
      ts.h.t = tmax;
      return true;
    }
    if (cnt > 3) stack[ts.sp++] = ref[3];
    if (cnt > 2) stack[ts.sp++] = ref[2];
    if (cnt > 1) stack[ts.sp++] = ref[1];
    ts.node = ref[0];
  }
  return false;
}

__device__ __forceinline__ Hit closest_hit(const DevScene &S, float3 o, float3 d, float tmax, unsigned *status,
                                           TravCount &tc) {
  return trace(S, o, d, tmax, false, status, tc);
}
__device__ __forceinline__ bool any_hit(const DevScene &S, float3 o, float3 d, float tmax, unsigned *status,
                                        TravCount &tc) {
  return trace(S, o, d, tmax, true, status, tc).prim >= 0;
}

// ------------------------------------------------------------------------------------------
// Surface interaction
// ------------------------------------------------------------------------------------------
struct Surf {
  float3 p, ng, ns, ngf, nsf;
  float cosg;
  int mat;
  uint32_t id;
  float b1, b2;
};

__device__ __forceinline__ Surf interact(const DevScene &S, float3 d, const Hit &h) {
  Surf f;
  const float4 a = __ldg(&S.tris[3 * h.prim]), b = __ldg(&S.tris[3 * h.prim + 1]), c = __ldg(&S.tris[3 * h.prim + 2]);
  const float3 v0 = xyz(a), v1 = xyz(b), v2 = xyz(c);
  const float b0 = 1.0f - h.b1 - h.b2;
  f.b1 = h.b1;
  f.b2 = h.b2;
  f.id = h.id;
  f.p = v0 * b0 + v1 * h.b1 + v2 * h.b2;
  f.ng = normalize(cross(v1 - v0, v2 - v0));
  const float4 s0 = __ldg(&S.shade[3 * h.id]), s1 = __ldg(&S.shade[3 * h.id + 1]), s2 = __ldg(&S.shade[3 * h.id + 2]);
  const float4 m = __ldg(&S.shade2[h.id]);
  f.mat = __float_as_int(m.w);
  const float3 n0 = xyz(s0), n1 = xyz(s1), n2 = xyz(s2);
  const bool flat = (n0.x == 0.f && n0.y == 0.f && n0.z == 0.f) || (n1.x == 0.f && n1.y == 0.f && n1.z == 0.f) ||
                    (n2.x == 0.f && n2.y == 0.f && n2.z == 0.f);
  if (flat) {
    f.ns = f.ng;
  } else {
    f.ns = normalize(n0 * b0 + n1 * h.b1 + n2 * h.b2);
    if (dot(f.ns, f.ng) < 0.0f) f.ns = f.ns * -1.0f;
  }
  f.cosg = dot(d, f.ng);
  const float side = f.cosg < 0.0f ? 1.0f : -1.0f;
  f.ngf = f.ng * side;
  f.nsf = f.ns * side;
  return f;
}

__device__ __forceinline__ float eps_of(float3 p) { return 1e-4f * fmaxf(1.0f, maxabs(p)); }
__device__ __forceinline__ float3 offset_along(float3 p, float3 ng, float3 dir) {
  return p + ng * ((dot(dir, ng) >= 0.0f ? 1.0f : -1.0f) * eps_of(p));
}

__device__ __forceinline__ float3 albedo_at(const DevScene &S, const sc_material &m, const Surf &f) {
  if (!(m.checker_scale > 0.0f)) return f3(m.albedo);
  const float4 s0 = __ldg(&S.shade[3 * f.id]), s1 = __ldg(&S.shade[3 * f.id + 1]), s2 = __ldg(&S.shade[3 * f.id + 2]);
  const float4 m2 = __ldg(&S.shade2[f.id]);
  const float b0 = 1.0f - f.b1 - f.b2;
  const float su = (b0 * s0.w + f.b1 * s1.w + f.b2 * s2.w) * m.checker_scale;
  const float sv = (b0 * m2.x + f.b1 * m2.y + f.b2 * m2.z) * m.checker_scale;
  const long parity = ((long)floorf(su) + (long)floorf(sv)) & 1;
  return parity ? f3(m.albedo2) : f3(m.albedo);
}

// Fresnel reflectance of unpolarised light (average of s and p), Hecht "Optics" Sec. 4.6
__device__ __forceinline__ float fresnel(float cos_i, float cos_t, float n_i, float n_t) {
  const float rs = (n_i * cos_i - n_t * cos_t) / (n_i * cos_i + n_t * cos_t);
  const float rp = (n_i * cos_t - n_t * cos_i) / (n_i * cos_t + n_t * cos_i);
  return 0.5f * (rs * rs + rp * rp);
}

// Dielectric scatter: Snell refraction or reflection chosen with probability R (u0 < R);
// on the wrong side of the geometric normal, repeated with the geometric normal.
__device__ __forceinline__ float3 dielectric(const Surf &f, float3 d, float n_lambda, float u0, int flags,
                                             bool &reflected, bool &fixup) {
  const bool entering = f.cosg < 0.0f;
  const float n_i = entering ? 1.0f : n_lambda, n_t = entering ? n_lambda : 1.0f;
  const float eta = n_i / n_t;
  float3 out = d;
  fixup = false;
  reflected = false;
  for (int pass = 0; pass < 2; ++pass) {
    const float3 n = pass == 0 ? f.nsf : f.ngf;
    const float cos_i = -dot(d, n);
    if (pass == 0 && cos_i <= 0.0f) {
      fixup = true;
      continue;
    }
    const float k = 1.0f - eta * eta * (1.0f - cos_i * cos_i);
    float R = 1.0f;
    if (k >= 0.0f) R = fresnel(cos_i, sqrtf(k), n_i, n_t);
    const bool refl = (k < 0.0f) || (!(flags & SC_FLAG_FORCE_TRANSMIT) && u0 < R);
    if (refl)
      out = normalize(d + n * (2.0f * cos_i));
    else
      out = normalize(d * eta + n * (eta * cos_i - sqrtf(k)));
    reflected = refl;
    const float side = dot(out, f.ngf);
    const bool ok = refl ? side > 0.0f : side < 0.0f;
    if (ok || pass == 1) break;
    fixup = true;
  }
  return out;
}

// Beer-Lambert attenuation of a segment of length t inside a dielectric (per RGB channel)
__device__ __forceinline__ float3 absorb_over(const sc_material &m, float t) {
  return f3(expf(-m.absorption[0] * t), expf(-m.absorption[1] * t), expf(-m.absorption[2] * t));
}
__device__ __forceinline__ bool absorbs(const sc_material &m) {
  return m.absorption[0] != 0.0f || m.absorption[1] != 0.0f || m.absorption[2] != 0.0f;
}

// orthonormal basis around unit n (Duff et al., "Building an Orthonormal Basis, Revisited",
// JCGT 2017) and a cosine-weighted direction about n
__device__ __forceinline__ void onb(float3 n, float3 &t1, float3 &t2) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  t1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  t2 = f3(b, sign + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2) {
  float3 t1, t2;
  onb(n, t1, t2);
  const float r = sqrtf(u1);
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return normalize(t1 * (r * c) + t2 * (r * s) + n * sqrtf(fmaxf(0.0f, 1.0f - u1)));
}

// Smith masking of GGX at cosine cos_v to the macro normal (Walter et al. 2007, eq. 34)
__device__ __forceinline__ float ggx_g1(float cos_v, float alpha) {
  const float c2 = cos_v * cos_v;
  return 2.0f / (1.0f + sqrtf(1.0f + alpha * alpha * ((1.0f - c2) / c2)));
}

// Rough dielectric (Walter, Marschner, Li, Torrance, EGSR 2007, GGX of width alpha): macro normal
// n = shading normal facing the ray (geometric if it faces away); microfacet normal m drawn with
// density D(m)|m.n| (tan^2 theta_m = alpha^2 u1 / (1 - u1), phi = 2 pi u2 in the Duff frame of n);
// Fresnel choice at m as for smooth glass; weight = |i.m| G1(i) G1(o) / (|i.n| |m.n|) (eq. 41).
// Returns false (the path ends) for a facet turned away from the ray or an outgoing direction on
// the wrong side of the macro or the geometric surface.
static __device__ __noinline__ bool rough_dielectric(const Surf &f, float3 d, float n_lambda, float alpha, float u0,
                                                 float u1, float u2, int flags, float3 &out, float &weight,
                                                 bool &reflected, bool &fixup) {
  const bool entering = f.cosg < 0.0f;
  const float n_i = entering ? 1.0f : n_lambda, n_t = entering ? n_lambda : 1.0f;
  const float eta = n_i / n_t;
  float3 n = f.nsf;
  float cn = -dot(d, n);
  fixup = false;
  reflected = false;
  weight = 0.0f;
  if (!(cn > 0.0f)) {
    n = f.ngf;
    cn = -dot(d, n);
    fixup = true;
  }
  float3 t1, t2;
  onb(n, t1, t2);
  const float tan2 = alpha * alpha * u1 / (1.0f - u1);
  const float cm = 1.0f / sqrtf(1.0f + tan2);
  const float sm = sqrtf(tan2) * cm;  // sin theta_m without the cancellation of sqrt(1 - cm^2)
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  const float3 m = normalize(t1 * (sm * cp) + t2 * (sm * sp) + n * cm);
  const float c = -dot(d, m);
  if (!(c > 0.0f)) return false;
  const float k = 1.0f - eta * eta * (1.0f - c * c);
  float R = 1.0f;
  if (k >= 0.0f) R = fresnel(c, sqrtf(k), n_i, n_t);
  const bool refl = (k < 0.0f) || (!(flags & SC_FLAG_FORCE_TRANSMIT) && u0 < R);
  const float3 o = refl ? normalize(d + m * (2.0f * c)) : normalize(d * eta + m * (eta * c - sqrtf(k)));
  reflected = refl;
  const float sg = dot(o, f.ngf), sn = dot(o, n), om = dot(o, m);
  if (refl ? !(sg > 0.0f && sn > 0.0f) : !(sg < 0.0f && sn < 0.0f)) return false;
  if (!(om * sn > 0.0f)) return false;
  weight = c * ggx_g1(cn, alpha) * ggx_g1(fabsf(sn), alpha) / (cn * cm);
  out = o;
  return true;
}

}  // namespace sc
