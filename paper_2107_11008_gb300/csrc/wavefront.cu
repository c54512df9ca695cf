// wavefront.cu -- the camera estimator as a wavefront of paths regrouped by event.
//
// The per-lane state machine of render.cu mixes traversal with shading in one loop, so a warp
// runs its shading code with the few lanes whose query just ended.  Here the same paths advance
// one event at a time through kernels that each do one thing for every path that needs it:
//
//   generate  primary rays of a wave of whole pixels (all their samples), 8x4 pixel tiles
//   per bounce:
//     extend      closest-hit traversal (4-wide BVH): persistent lanes refilled from the extend
//                 queue as soon as their query ends; each hit is classified at once -- a miss or an
//                 emitter ends the path, a dielectric or a diffuse hit joins that material's queue
//     dielectric  Fresnel / Snell (or rough GGX) scatter, Beer-Lambert absorption
//     diffuse     next-event estimate (its shadow ray joins the shadow queue) and cosine bounce
//     shadow      any-hit traversal of the shadow queue, same persistent lanes
//   reduce    each pixel's samples weighted by their wavelength bin, summed in sample order and
//             added to the accumulator; path records written
//
// Every path draws the same random numbers, takes the same decisions in the same order and does
// the same float operations as in the per-lane state machine (both call the same device
// functions), so path records and accumulators are bit for bit the same.  Path state lives in
// HBM as structure of arrays.  Queues of large waves are kept in path-slot order (producers set
// a bit per path, a compaction emits the set bits in order); small waves append with
// warp-aggregated atomics.
#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "internal.h"

namespace sc {

namespace {

constexpr int kWfBlock = 128;
// node visits per traversal chunk before a lane whose query ended may take the next one
#ifndef SC_WF_CHUNK
#define SC_WF_CHUNK 12
#endif
// Launch bounds of the two persistent traversal kernels: by default the compiler's register
// choice; a build with SC_WF_TRAV_MINB set asks for that many resident blocks per SM instead
// (fewer registers each, more warps to hide node-fetch latency).
#ifdef SC_WF_TRAV_MINB
#define SC_WF_TRAV_BOUNDS __launch_bounds__(kWfBlock, SC_WF_TRAV_MINB)
#else
#define SC_WF_TRAV_BOUNDS __launch_bounds__(kWfBlock)
#endif
constexpr int kWfChunk = SC_WF_CHUNK;
enum : uint32_t {
  W_SPEC_ONLY = 1u, W_DIFFUSE_FIRST = 2u, W_LAST_SPECULAR = 4u, W_FIXUP = 8u, W_HAS_NEXT = 16u
};
// counters of a wave (device words): queue sizes and the persistent kernels' ticket
enum { C_EXT0 = 0, C_EXT1 = 1, C_DIEL = 2, C_DIFF = 3, C_SHADOW = 4, C_TICKET_EXT = 5, C_TICKET_SHADOW = 6, C_WORDS = 8 };
enum { BM_DIEL = 0, BM_DIFF = 1, BM_SHADOW = 2, BM_EXT = 3 };
// Queues in path-slot order: producers set the path's bit and a compaction emits the set bits in
// order, so that the kernels reading a queue touch path state in runs of neighbouring slots and a
// warp's rays come from neighbouring pixels (512^2 glass frame: camera phase 115.2 -> 99.7 ms).
// Used for waves of at least SC_WF_ORDERED_MIN paths: on small waves the compactions' nine
// launches per bounce cost more than they save (64^2 ball frame: 1.10 -> 1.39 ms), and the queues
// are appended in the order paths are produced.  0 = always appended.
#ifndef SC_WF_ORDERED_MIN
#define SC_WF_ORDERED_MIN (1 << 18)
#endif
constexpr int kBmWordsPerBlock = 1024;  // bitmap words per compaction block (256 threads x 4)

struct Wave {
  float4 *o;      // ray origin; w: the path's bin draw u
  float4 *d;      // ray direction; w: the path's scene in the batch (int bits)
  float4 *beta;   // throughput
  float4 *L;      // radiance so far; w: 1 once the path has ended
  float4 *nee;    // pending next-event contribution; w: shadow ray length limit
  float4 *so;     // shadow ray origin
  float4 *sd;     // shadow ray direction
  uint4 *m0;      // signature, first hit, closest-hit queries, dielectric events
  uint4 *m1;      // closest-hit depth k, diffuse vertices, flags, -
  float4 *hit;    // t, b1, b2, leaf index (int bits)
  uint32_t *hid;  // input triangle id of the hit
  uint32_t *q_ext[2], *q_diel, *q_diff, *q_shadow;
  // ordered queues: one bit per path slot for each queue being filled, emitted in slot order
  uint32_t *bm[4];  // BM_DIEL, BM_DIFF, BM_SHADOW, BM_EXT: contiguous, bm_words apart
  uint32_t *bmblk;  // per-block bit counts of the compaction (two bitmaps at a time)
  int bm_words;     // words of each bitmap (sized for the largest wave)
  int ordered;      // this wave's queues are ordered (bitmaps + compaction), else appended
  unsigned *cnt;
  int t0;         // first pixel of the wave in tile order
  int wave_px;    // tile-order pixel slots in the wave
  int n;          // paths = wave_px * spp
};

// One scene (S, F) or, for a batch, the scene table: tab[i].slot_begin is the first tile-order
// pixel slot of scene i in the batch's concatenation of all scenes' slots.
struct WfArgs {
  DevScene S;
  sc_trace_params P;
  sc_frame F;
  const BatchEntry *tab;
  int n_tab;
  unsigned *status;
  unsigned long long *counters;
  JitterNorm jn;
  int nb;
  int jitter;
};

// the scene, frame and random-stream scene index of scene sc (always the one scene without a batch)
template <bool B>
__device__ __forceinline__ const DevScene &scene_of(const WfArgs &a, int sc) {
  return B ? a.tab[sc].S : a.S;
}
template <bool B>
__device__ __forceinline__ const sc_frame &frame_of(const WfArgs &a, int sc) {
  return B ? a.tab[sc].F : a.F;
}
template <bool B>
__device__ __forceinline__ uint32_t stream_of(const WfArgs &a, int sc) {
  return (uint32_t)(a.P.scene_index + (B ? sc : 0));
}

// global tile-order slot -> scene and local slot (binary search over the slot starts)
template <bool B>
__device__ __forceinline__ int slot_scene(const WfArgs &a, int g, int &local) {
  if (!B) {
    local = g;
    return 0;
  }
  int lo = 0, hi = a.n_tab - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)a.tab[mid].slot_begin <= g) lo = mid;
    else hi = mid - 1;
  }
  local = g - (int)a.tab[lo].slot_begin;
  return lo;
}

__device__ __forceinline__ void pixel_of(const DevScene &S, int tslot, int &px, int &py) {
  const unsigned tiles_x = (unsigned)((S.cam.width + 7) / 8);
  const unsigned tile = (unsigned)tslot >> 5, in = (unsigned)tslot & 31u;
  px = (int)(tile % tiles_x) * 8 + (int)(in & 7u);
  py = (int)(tile / tiles_x) * 4 + (int)(in >> 3);
}

// Appends v for every lane with pred set; the whole warp must call it together.
__device__ __forceinline__ void warp_push(uint32_t *q, unsigned *count, bool pred, uint32_t v) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (pred) q[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

// Adds path p to a queue for every lane with pred set (the whole warp calls it together): its
// bit in the queue's bitmap (ordered queues), else warp_push.
__device__ __forceinline__ void enqueue(const Wave &w, int bm, uint32_t *q, unsigned *count, bool pred, int p) {
  if (w.ordered) {  // uniform over the launch
    if (pred) atomicOr(w.bm[bm] + (p >> 5), 1u << (p & 31));
  } else {
    warp_push(q, count, pred, (uint32_t)p);
  }
}

__device__ __forceinline__ void end_path(const Wave &w, int p, float3 L) {
  w.L[p] = make_float4(L.x, L.y, L.z, 1.0f);
}

__device__ __forceinline__ void flush_counts(const WfArgs &a, const TravCount &tc) {
  if (a.counters) {
    atomicAdd(&a.counters[0], (unsigned long long)tc.queries);
    atomicAdd(&a.counters[1], (unsigned long long)tc.nodes);
    atomicAdd(&a.counters[2], (unsigned long long)tc.tris);
  }
}

// ---- generate: one path per (sample, pixel slot) of the wave -----------------------------------
template <bool B>
__global__ void __launch_bounds__(kWfBlock) k_wf_generate(WfArgs a, Wave w) {
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < w.n; base += stride) {
    const int p = base + (threadIdx.x & 31);
    bool live = false;
    if (p < w.n) {
      const int s = p / w.wave_px, t = p - s * w.wave_px;
      int local;
      const int sc = slot_scene<B>(a, w.t0 + t, local);
      const DevScene &S = scene_of<B>(a, sc);
      const Cam cam = make_cam(S.cam);
      int px, py;
      pixel_of(S, local, px, py);
      live = px < cam.W && py < cam.H;
      w.L[p] = make_float4(0.f, 0.f, 0.f, live ? 0.0f : 1.0f);
      if (live) {
        const uint32_t pix = (uint32_t)(py * cam.W + px);
        const uint4 x0 = draw(a.P.seed, pix, (uint32_t)(a.P.sample_offset + s), 0u, 0u, stream_of<B>(a, sc));
        const float ul = u01(x0.z);
        const float3 d = cam_dir(cam, (px + u01(x0.x)) / cam.W, (py + u01(x0.y)) / cam.H);
        w.o[p] = make_float4(cam.eye.x, cam.eye.y, cam.eye.z, ul);
        w.d[p] = make_float4(d.x, d.y, d.z, __int_as_float(sc));
        w.beta[p] = make_float4(1.f, 1.f, 1.f, 0.f);
        w.m0[p] = make_uint4(2166136261u, kMiss, 0u, 0u);
        w.m1[p] = make_uint4(0u, 0u, W_SPEC_ONLY, (uint32_t)sc);
      }
    }
    warp_push(w.q_ext[0], w.cnt + C_EXT0, live, (uint32_t)p);
  }
}

// ---- extend: closest hits of the extend queue, classified by material ----------------------------
template <bool B>
__global__ void SC_WF_TRAV_BOUNDS k_wf_extend(WfArgs a, Wave w, int cur) {
  const uint32_t *q = w.q_ext[cur];
  const unsigned nq_total = w.cnt[cur ? C_EXT1 : C_EXT0];
  unsigned *ticket = w.cnt + C_TICKET_EXT;
  const int lane = threadIdx.x & 31;
  TravCount tc;
  TravState ts;
  int stack[kStack];
  int p = -1, sc = 0;
  bool tracing = false, exhausted = false;
  float3 o = f3(0.f, 0.f, 0.f), d = o;
  for (;;) {
    // refill lanes without a query from the queue (one atomic per warp)
    const bool want = !tracing && !exhausted;
    const unsigned wmask = __ballot_sync(0xFFFFFFFFu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ticket, (unsigned)__popc(wmask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (want) {
        const unsigned t = base + (unsigned)__popc(wmask & ((1u << lane) - 1u));
        if (t < nq_total) {
          p = (int)q[t];
          const float4 o4 = w.o[p], d4 = w.d[p];
          if (B) sc = __float_as_int(d4.w);
          o = f3(o4.x, o4.y, o4.z);
          d = f3(d4.x, d4.y, d4.z);
          trav_begin(ts, 3.0e38f, false);
          tracing = true;
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xFFFFFFFFu, !tracing && exhausted)) break;
    bool done = false;
    if (tracing) {
      done = trav_step(scene_of<B>(a, sc), make_wray(o, d), 3.0e38f, ts, stack, kWfChunk, a.status, tc);
      if (done) tracing = false;
    }
    // a finished query: record the hit and queue the path for its material, or end it (a miss, an
    // emitter); the hit's signature entry and query count are added by whichever kernel takes the hit
    bool to_diel = false, to_diff = false;
    if (done) {
      const DevScene &S = scene_of<B>(a, sc);
      ++tc.queries;
      const Hit h = ts.h;
      bool ends = true;
      float3 Ladd = f3(0.f, 0.f, 0.f);
      if (h.prim >= 0 && SC_IN_RANGE(a.status, 5, h.prim, S.n_tris) && SC_IN_RANGE(a.status, 6, h.id, S.n_tris)) {
        w.hit[p] = make_float4(h.t, h.b1, h.b2, __int_as_float(h.prim));
        w.hid[p] = h.id;
        const int mat = __float_as_int(__ldg(&S.shade2[h.id]).w);
        const sc_material m = S.mats[SC_IN_RANGE(a.status, 7, mat, S.n_mats) ? mat : 0];
        if (m.kind == SC_MAT_DIELECTRIC) {
          to_diel = true;
          ends = false;
        } else if (m.kind != SC_MAT_EMISSIVE) {
          to_diff = true;
          ends = false;
        } else {
          const uint4 m1 = w.m1[p];
          const Surf f = interact(S, d, h);
          const bool count = (m1.z & W_SPEC_ONLY) ||
                             ((a.P.flags & SC_FLAG_EMITTER_AFTER_DS) && (m1.z & W_DIFFUSE_FIRST) && m1.y == 1u &&
                              (m1.z & W_LAST_SPECULAR));
          if (f.cosg < 0.0f && count) Ladd = f3(w.beta[p].x, w.beta[p].y, w.beta[p].z) * f3(m.emission);
        }
      } else if (h.prim < 0) {
        const float4 b4 = w.beta[p];
        Ladd = f3(b4.x, b4.y, b4.z) * f3(S.env);
      }
      if (ends) {
        uint4 m0 = w.m0[p];
        m0.z += 1u;                          // closest-hit queries
        m0.x = fnv(m0.x, h.id);              // signature
        if (w.m1[p].x == 0u) m0.y = h.id;    // first hit
        w.m0[p] = m0;
        const float4 L4 = w.L[p];
        end_path(w, p, f3(L4.x, L4.y, L4.z) + Ladd);
      }
    }
    enqueue(w, BM_DIEL, w.q_diel, w.cnt + C_DIEL, to_diel, p);
    enqueue(w, BM_DIFF, w.q_diff, w.cnt + C_DIFF, to_diff, p);
  }
  flush_counts(a, tc);
}

// pixel index and sample number of path slot p (for its random numbers)
template <bool B>
__device__ __forceinline__ void path_pixel(const WfArgs &a, const Wave &w, int p, uint32_t &pix, uint32_t &smp) {
  const int s = p / w.wave_px, t = p - s * w.wave_px;
  int local;
  const int sc = slot_scene<B>(a, w.t0 + t, local);
  const DevScene &S = scene_of<B>(a, sc);
  int px, py;
  pixel_of(S, local, px, py);
  pix = (uint32_t)(py * S.cam.width + px);
  smp = (uint32_t)(a.P.sample_offset + s);
}

__device__ __forceinline__ Hit load_hit(const Wave &w, int p) {
  const float4 h4 = w.hit[p];
  Hit h;
  h.t = h4.x;
  h.b1 = h4.y;
  h.b2 = h4.z;
  h.prim = __float_as_int(h4.w);
  h.id = w.hid[p];
  return h;
}

// ---- dielectric events -----------------------------------------------------------------------
template <bool B>
__global__ void __launch_bounds__(kWfBlock) k_wf_dielectric(WfArgs a, Wave w, int next) {
  const unsigned n = w.cnt[C_DIEL];
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < (int)n; base += stride) {
    const int i = base + (threadIdx.x & 31);
    bool cont = false;
    int p = 0;
    if (i < (int)n) {
      p = (int)w.q_diel[i];
      uint4 m0 = w.m0[p], m1 = w.m1[p];
      const int sc = (int)m1.w;
      const DevScene &S = scene_of<B>(a, sc);
      const float4 o4 = w.o[p], d4 = w.d[p], b4 = w.beta[p];
      const float ul = o4.w;
      const float3 d = f3(d4.x, d4.y, d4.z);
      float3 beta = f3(b4.x, b4.y, b4.z);
      const Hit h = load_hit(w, p);
      m0.z += 1u;                        // closest-hit queries
      m0.x = fnv(m0.x, h.id);            // signature
      if (m1.x == 0u) m0.y = h.id;       // first hit
      const Surf f = interact(S, d, h);
      const sc_material m = S.mats[SC_IN_RANGE(a.status, 7, f.mat, S.n_mats) ? f.mat : 0];
      // the segment ended on the glass's inner side: it ran through the glass (Beer-Lambert)
      if (f.cosg > 0.0f && absorbs(m)) beta = beta * absorb_over(m, h.t);
      uint32_t pix, smp;
      path_pixel<B>(a, w, p, pix, smp);
      const uint4 xs = draw(a.P.seed, pix, smp, m1.x + 1u, 1u, stream_of<B>(a, sc));
      bool refl, fix, alive = true;
      const float nl = cauchy_at(m.cauchy_a, m.cauchy_b, path_lambda(ul, a.nb, a.jitter), a.P.n_bins);
      float3 nd;
      if (m.roughness > 0.0f) {
        float wgt;
        alive = rough_dielectric(f, d, nl, m.roughness, u01(xs.x), u01(xs.y), u01(xs.z), a.P.flags, nd, wgt, refl,
                                 fix);
        beta = beta * wgt;
      } else {
        nd = dielectric(f, d, nl, u01(xs.x), a.P.flags, refl, fix);
      }
      m0.w += 1u;  // dielectric events
      if (!alive) {
        m0.x = fnv(m0.x, EV_KILL);
        const float4 L4 = w.L[p];
        end_path(w, p, f3(L4.x, L4.y, L4.z));
      } else {
        m0.x = fnv(m0.x, refl ? EV_REFLECT : EV_REFRACT);
        if (fix) m0.x = fnv(m0.x, EV_FIXUP);
        m1.z |= W_LAST_SPECULAR;
        m1.x += 1u;
        const float3 no = offset_along(f.p, f.ng, nd);
        w.o[p] = make_float4(no.x, no.y, no.z, ul);
        w.d[p] = make_float4(nd.x, nd.y, nd.z, d4.w);
        w.m1[p] = m1;
        if ((int)m1.x >= a.P.max_depth) {
          const float4 L4 = w.L[p];
          end_path(w, p, f3(L4.x, L4.y, L4.z));
        } else {
          cont = true;
        }
      }
      w.beta[p] = make_float4(beta.x, beta.y, beta.z, 0.0f);
      w.m0[p] = m0;
    }
    enqueue(w, BM_EXT, w.q_ext[next], w.cnt + (next ? C_EXT1 : C_EXT0), cont, p);
  }
}

// ---- diffuse events: next-event estimate and cosine bounce -----------------------------------
template <bool B>
__global__ void __launch_bounds__(kWfBlock) k_wf_diffuse(WfArgs a, Wave w, int next) {
  const unsigned n = w.cnt[C_DIFF];
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < (int)n; base += stride) {
    const int i = base + (threadIdx.x & 31);
    bool cont = false, shadow = false;
    int p = 0;
    if (i < (int)n) {
      p = (int)w.q_diff[i];
      uint4 m0 = w.m0[p], m1 = w.m1[p];
      const int sc = (int)m1.w;
      const DevScene &S = scene_of<B>(a, sc);
      const float4 o4 = w.o[p], d4 = w.d[p], b4 = w.beta[p];
      const float ul = o4.w;
      const float3 d = f3(d4.x, d4.y, d4.z);
      float3 beta = f3(b4.x, b4.y, b4.z);
      const Hit h = load_hit(w, p);
      m0.z += 1u;                        // closest-hit queries
      m0.x = fnv(m0.x, h.id);            // signature
      if (m1.x == 0u) m0.y = h.id;       // first hit
      const Surf f = interact(S, d, h);
      const sc_material m = S.mats[SC_IN_RANGE(a.status, 7, f.mat, S.n_mats) ? f.mat : 0];
      uint32_t pix, smp;
      path_pixel<B>(a, w, p, pix, smp);
      const uint32_t k = m1.x;
      const uint4 xs = draw(a.P.seed, pix, smp, k + 1u, 1u, stream_of<B>(a, sc));
      const float3 alb = albedo_at(S, m, f);
      float3 so = f3(0.f, 0.f, 0.f), sd = so, nee = so;
      float sdist = 0.0f;
      if (S.n_lights > 0) {
        const uint4 xn = draw(a.P.seed, pix, smp, k + 1u, 2u, stream_of<B>(a, sc));
        const sc_light Lg = S.lights[choose(xn.x, S.n_lights)];
        float3 lp = f3(0.f, 0.f, 0.f);
        float geo = 0.0f;
        bool ok = false;
        if (Lg.kind == SC_LIGHT_POINT) {
          lp = f3(Lg.p);
          float3 wl = lp - f.p;
          const float d2l = dot(wl, wl);
          wl = wl * (1.0f / sqrtf(d2l));
          const float cs = dot(f.nsf, wl), cg = dot(f.ngf, wl);
          ok = cs > 0.0f && cg > 0.0f;
          geo = cs / d2l;
        } else if (Lg.kind == SC_LIGHT_RECT) {
          const float3 eu = f3(Lg.u), ev = f3(Lg.v);
          lp = f3(Lg.p) + eu * u01(xn.y) + ev * u01(xn.z);
          const float3 c = cross(eu, ev);
          const float area = length(c);
          const float3 nlt = c * (1.0f / area);
          float3 wl = lp - f.p;
          const float d2l = dot(wl, wl);
          wl = wl * (1.0f / sqrtf(d2l));
          const float cs = dot(f.nsf, wl), cg = dot(f.ngf, wl), cl = -dot(nlt, wl);
          ok = cs > 0.0f && cg > 0.0f && cl > 0.0f;
          geo = cs * cl * area / d2l;
        }
        if (ok) {
          so = f.p + f.ngf * eps_of(f.p);
          const float3 wv = lp - so;
          sdist = length(wv);
          sd = wv * (1.0f / sdist);
          nee = beta * (alb * f3(Lg.power)) * (geo * (float)S.n_lights / kPi);
          shadow = true;
        }
      }
      uint32_t fl = m1.z;
      if (k == 0u) fl |= W_DIFFUSE_FIRST;
      m1.y += 1u;  // diffuse vertices
      fl &= ~(W_SPEC_ONLY | W_LAST_SPECULAR | W_FIXUP | W_HAS_NEXT);
      if ((int)k < a.P.max_depth - 1) {
        float3 nd = cosine_dir(f.nsf, u01(xs.y), u01(xs.z));
        if (!(dot(nd, f.ngf) > 0.0f)) {
          nd = cosine_dir(f.ngf, u01(xs.y), u01(xs.z));
          fl |= W_FIXUP;
        }
        beta = beta * alb;
        const float3 no = f.p + f.ngf * eps_of(f.p);
        w.o[p] = make_float4(no.x, no.y, no.z, ul);
        w.d[p] = make_float4(nd.x, nd.y, nd.z, d4.w);
        w.beta[p] = make_float4(beta.x, beta.y, beta.z, 0.0f);
        fl |= W_HAS_NEXT;
      }
      m1.x = k + 1u;
      m1.z = fl;
      if (shadow) {
        w.so[p] = make_float4(so.x, so.y, so.z, 0.0f);
        w.sd[p] = make_float4(sd.x, sd.y, sd.z, d4.w);
        w.nee[p] = make_float4(nee.x, nee.y, nee.z, sdist * (1.0f - 1e-4f));
      } else {
        m0.x = fnv(m0.x, EV_UNLIT);
        if (fl & W_FIXUP) m0.x = fnv(m0.x, EV_FIXUP);
        if (fl & W_HAS_NEXT) {
          cont = true;
        } else {
          const float4 L4 = w.L[p];
          end_path(w, p, f3(L4.x, L4.y, L4.z));
        }
      }
      w.m0[p] = m0;
      w.m1[p] = m1;
    }
    enqueue(w, BM_SHADOW, w.q_shadow, w.cnt + C_SHADOW, shadow, p);
    enqueue(w, BM_EXT, w.q_ext[next], w.cnt + (next ? C_EXT1 : C_EXT0), cont, p);
  }
}

// ---- shadow rays of the next-event estimates -----------------------------------------------------
template <bool B>
__global__ void SC_WF_TRAV_BOUNDS k_wf_shadow(WfArgs a, Wave w, int next) {
  const unsigned nq_total = w.cnt[C_SHADOW];
  unsigned *ticket = w.cnt + C_TICKET_SHADOW;
  const int lane = threadIdx.x & 31;
  TravCount tc;
  TravState ts;
  int stack[kStack];
  int p = -1, sc = 0;
  bool tracing = false, exhausted = false;
  float3 o = f3(0.f, 0.f, 0.f), d = o;
  float tmax = 0.0f;
  for (;;) {
    const bool want = !tracing && !exhausted;
    const unsigned wmask = __ballot_sync(0xFFFFFFFFu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ticket, (unsigned)__popc(wmask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (want) {
        const unsigned t = base + (unsigned)__popc(wmask & ((1u << lane) - 1u));
        if (t < nq_total) {
          p = (int)w.q_shadow[t];
          const float4 o4 = w.so[p], d4 = w.sd[p];
          if (B) sc = __float_as_int(d4.w);
          o = f3(o4.x, o4.y, o4.z);
          d = f3(d4.x, d4.y, d4.z);
          tmax = w.nee[p].w;
          trav_begin(ts, tmax, true);
          tracing = true;
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xFFFFFFFFu, !tracing && exhausted)) break;
    bool done = false;
    if (tracing) {
      done = trav_step(scene_of<B>(a, sc), make_wray(o, d), tmax, ts, stack, kWfChunk, a.status, tc);
      if (done) tracing = false;
    }
    bool cont = false;
    if (done) {
      ++tc.queries;
      const bool lit = ts.h.prim < 0;
      const float4 L4 = w.L[p];
      float3 L = f3(L4.x, L4.y, L4.z);
      if (lit) {
        const float4 e4 = w.nee[p];
        L = L + f3(e4.x, e4.y, e4.z);
      }
      uint4 m0 = w.m0[p];
      const uint32_t fl = w.m1[p].z;
      m0.x = fnv(m0.x, lit ? EV_LIT : EV_UNLIT);
      if (fl & W_FIXUP) m0.x = fnv(m0.x, EV_FIXUP);
      w.m0[p] = m0;
      if (fl & W_HAS_NEXT) {
        w.L[p] = make_float4(L.x, L.y, L.z, 0.0f);
        cont = true;
      } else {
        end_path(w, p, L);
      }
    }
    enqueue(w, BM_EXT, w.q_ext[next], w.cnt + (next ? C_EXT1 : C_EXT0), cont, p);
  }
  flush_counts(a, tc);
}

// Between bounces: the next extend queue becomes current, the others are emptied.
// ---- ordered queues: compaction of a bitmap into the queue, in slot order ---------------------
// blockIdx.y picks one of up to two bitmaps compacted together (which[y]); a block covers
// kBmWordsPerBlock words, thread t words 4t .. 4t + 3 of them.
struct Compact {
  const uint32_t *bm[2];  // bitmap (cleared by the emit kernel)
  uint32_t *q[2];         // queue written in slot order
  unsigned *count[2];     // queue size
  int nwords;             // bitmap words of the wave
  int nblk;               // blocks per bitmap
};

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *ws, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) ws[lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp == 0 ? 0u : ws[warp - 1];
  *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(256) k_wf_compact_count(Compact c, uint32_t *blk) {
  __shared__ uint32_t ws[32];
  const int y = blockIdx.y;
  const int w0 = blockIdx.x * kBmWordsPerBlock + 4 * threadIdx.x;
  uint32_t n = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (w0 + k < c.nwords) n += (uint32_t)__popc(c.bm[y][w0 + k]);
  uint32_t total;
  block_excl_scan(n, ws, &total);
  if (threadIdx.x == 0) blk[y * c.nblk + blockIdx.x] = total;
}

// one block of 1024 per bitmap: exclusive prefix of the block counts, the queue size
__global__ void __launch_bounds__(1024) k_wf_compact_scan(Compact c, uint32_t *blk) {
  __shared__ uint32_t ws[32];
  uint32_t *b = blk + blockIdx.x * c.nblk;
  uint32_t carry = 0;
  for (int base = 0; base < c.nblk; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < c.nblk ? b[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan(v, ws, &total);
    if (i < c.nblk) b[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *c.count[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(256) k_wf_compact_emit(Compact c, const uint32_t *blk) {
  __shared__ uint32_t ws[32];
  const int y = blockIdx.y;
  uint32_t *bm = const_cast<uint32_t *>(c.bm[y]);
  const int w0 = blockIdx.x * kBmWordsPerBlock + 4 * threadIdx.x;
  uint32_t wd[4];
  uint32_t n = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wd[k] = w0 + k < c.nwords ? bm[w0 + k] : 0u;
    n += (uint32_t)__popc(wd[k]);
  }
  uint32_t total;
  uint32_t pos = block_excl_scan(n, ws, &total) + blk[y * c.nblk + blockIdx.x];
  uint32_t *q = c.q[y];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t v = wd[k];
    while (v) {
      const int bit = __ffs(v) - 1;
      v &= v - 1u;
      q[pos++] = (uint32_t)((w0 + k) * 32 + bit);
    }
    if (wd[k] && w0 + k < c.nwords) bm[w0 + k] = 0u;  // ready for the next round
  }
}

__global__ void k_wf_rotate(Wave w, int cur) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    w.cnt[cur ? C_EXT1 : C_EXT0] = 0u;
    w.cnt[C_DIEL] = 0u;
    w.cnt[C_DIFF] = 0u;
    w.cnt[C_SHADOW] = 0u;
    w.cnt[C_TICKET_EXT] = 0u;
    w.cnt[C_TICKET_SHADOW] = 0u;
  }
}

// Per pixel slot of the wave: its samples in order, each weighted by its wavelength (bin table or
// jitter), summed and added to the accumulator; records of every path.
template <bool B>
__global__ void __launch_bounds__(kWfBlock) k_wf_reduce(WfArgs a, Wave w) {
  __shared__ float3 wts[kMaxBins];
  spectral_table(wts, a.P.n_bins);  // ends with __syncthreads
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w.wave_px) return;
  int local;
  const int sc = slot_scene<B>(a, w.t0 + t, local);
  const DevScene &S = scene_of<B>(a, sc);
  const sc_frame &F = frame_of<B>(a, sc);
  int px, py;
  pixel_of(S, local, px, py);
  if (px >= S.cam.width || py >= S.cam.height) return;
  const int pix = py * S.cam.width + px;
  const int spp = a.P.spp;
  float3 acc = f3(0.f, 0.f, 0.f);
  for (int s = 0; s < spp; ++s) {
    const int p = s * w.wave_px + t;
    const float4 L4 = w.L[p];
    const float ul = w.o[p].w;
    const int bin = bin_of(ul, a.nb);
    const float3 Lw = f3(L4.x, L4.y, L4.z) * (a.jitter ? jitter_weight(ul, a.jn) : wts[bin]);
    acc = acc + Lw;
    if (F.path_records && SC_IN_RANGE(a.status, 9, (int64_t)pix * spp + s, (int64_t)S.cam.width * S.cam.height * spp)) {
      const uint4 m0 = w.m0[p];
      sc_path_record r;
      r.L[0] = Lw.x; r.L[1] = Lw.y; r.L[2] = Lw.z;
      r.first_tri = m0.y;
      r.signature = m0.x;
      r.n_queries = m0.z;
      r.bin = (uint32_t)bin;
      r.n_specular = m0.w;
      F.path_records[(int64_t)pix * spp + s] = r;
    }
  }
  if (F.accum_camera && SC_IN_RANGE(a.status, 4, pix, S.cam.width * S.cam.height)) {
    float4 *acp = reinterpret_cast<float4 *>(F.accum_camera) + pix;
    float4 v = *acp;
    v.x += acc.x; v.y += acc.y; v.z += acc.z;
    *acp = v;
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace of one wave of up to `max_paths` paths.
size_t wavefront_workspace_bytes(int64_t max_paths) {
  const size_t n = (size_t)max_paths;
  return 11 * a256(16 * n) + a256(4 * n) * 6 + a256(4 * C_WORDS);
}

int64_t wavefront_wave_pixels(int width, int height, int spp, int64_t max_paths) {
  const int64_t tiles = (int64_t)((width + 7) / 8) * ((height + 3) / 4);
  int64_t wave_tiles = std::max<int64_t>(1, max_paths / (32 * (int64_t)std::max(spp, 1)));
  wave_tiles = std::min(wave_tiles, tiles);
  return wave_tiles * 32;
}

namespace {

// Carves the wave's arrays out of the workspace (the layout wavefront_workspace_bytes sizes).
bool carve_wave(void *workspace, int64_t max_paths, Wave &w) {
  const size_t n = (size_t)max_paths;
  char *base = static_cast<char *>(workspace);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *r = base + off;
    off += a256(bytes);
    return r;
  };
  w.o = reinterpret_cast<float4 *>(take(16 * n));
  w.d = reinterpret_cast<float4 *>(take(16 * n));
  w.beta = reinterpret_cast<float4 *>(take(16 * n));
  w.L = reinterpret_cast<float4 *>(take(16 * n));
  w.nee = reinterpret_cast<float4 *>(take(16 * n));
  w.so = reinterpret_cast<float4 *>(take(16 * n));
  w.sd = reinterpret_cast<float4 *>(take(16 * n));
  w.m0 = reinterpret_cast<uint4 *>(take(16 * n));
  w.m1 = reinterpret_cast<uint4 *>(take(16 * n));
  w.hit = reinterpret_cast<float4 *>(take(16 * n));
  {  // the reserved 16 n bytes: four bitmaps of n bits and the compaction's block counts
    char *r = take(16 * n);
    const size_t words = (n + 31) / 32;
    for (int k = 0; k < 4; ++k) w.bm[k] = reinterpret_cast<uint32_t *>(r) + k * words;
    w.bm_words = (int)words;
    w.bmblk = reinterpret_cast<uint32_t *>(r) + 4 * words;  // 2 x blocks (n / 32768 + 1) words
  }
  w.hid = reinterpret_cast<uint32_t *>(take(4 * n));
  w.q_ext[0] = reinterpret_cast<uint32_t *>(take(4 * n));
  w.q_ext[1] = reinterpret_cast<uint32_t *>(take(4 * n));
  w.q_diel = reinterpret_cast<uint32_t *>(take(4 * n));
  w.q_diff = reinterpret_cast<uint32_t *>(take(4 * n));
  w.q_shadow = reinterpret_cast<uint32_t *>(take(4 * n));
  w.cnt = reinterpret_cast<unsigned *>(take(4 * C_WORDS));
  return off <= wavefront_workspace_bytes(max_paths);
}

// Emits bitmaps into their queues (one or two at a time), clearing the bitmaps.
cudaError_t compact(const Wave &w, int nq, const int *which, uint32_t *const *queues, const int *counts,
                    cudaStream_t s) {
  Compact c;
  c.nwords = (w.n + 31) / 32;
  c.nblk = (c.nwords + kBmWordsPerBlock - 1) / kBmWordsPerBlock;
  for (int k = 0; k < 2; ++k) {
    const int j = k < nq ? k : 0;
    c.bm[k] = w.bm[which[j]];
    c.q[k] = queues[j];
    c.count[k] = w.cnt + counts[j];
  }
  const dim3 g((unsigned)c.nblk, (unsigned)nq);
  k_wf_compact_count<<<g, 256, 0, s>>>(c, w.bmblk);
  k_wf_compact_scan<<<nq, 1024, 0, s>>>(c, w.bmblk);
  k_wf_compact_emit<<<g, 256, 0, s>>>(c, w.bmblk);
  return cudaGetLastError();
}

// Waves of whole pixel slots over [0, total_slots): each wave's kernels, bounce by bounce.
template <bool B>
cudaError_t run_waves(const WfArgs &a, Wave w, int64_t total_slots, int64_t wave_px, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wf_extend<B>, kWfBlock, 0);
  if (e != cudaSuccess || per_sm <= 0) {
    cudaGetLastError();
    per_sm = 4;
  }
  const int persistent = num_sms * per_sm;
  const int wide = num_sms * 16;
  for (int64_t t0 = 0; t0 < total_slots; t0 += wave_px) {
    w.t0 = (int)t0;
    w.wave_px = (int)std::min<int64_t>(wave_px, total_slots - t0);
    w.n = w.wave_px * a.P.spp;
    w.ordered = SC_WF_ORDERED_MIN > 0 && w.n >= SC_WF_ORDERED_MIN;
    e = cudaMemsetAsync(w.cnt, 0, 4 * C_WORDS, s);
    if (e != cudaSuccess) return e;
    if (w.ordered) {
      e = cudaMemsetAsync(w.bm[0], 0, 4 * sizeof(uint32_t) * (size_t)w.bm_words, s);  // the four bitmaps
      if (e != cudaSuccess) return e;
    }
    k_wf_generate<B><<<std::max(1, std::min(wide, (w.n + kWfBlock - 1) / kWfBlock)), kWfBlock, 0, s>>>(a, w);
    for (int b = 0; b < a.P.max_depth; ++b) {
      const int cur = b & 1, next = cur ^ 1;
      k_wf_extend<B><<<persistent, kWfBlock, 0, s>>>(a, w, cur);
      if (w.ordered) {
        const int which[2] = {BM_DIEL, BM_DIFF}, counts[2] = {C_DIEL, C_DIFF};
        uint32_t *const queues[2] = {w.q_diel, w.q_diff};
        if ((e = compact(w, 2, which, queues, counts, s)) != cudaSuccess) return e;
      }
      k_wf_dielectric<B><<<wide, kWfBlock, 0, s>>>(a, w, next);
      k_wf_diffuse<B><<<wide, kWfBlock, 0, s>>>(a, w, next);
      if (w.ordered) {
        const int which[1] = {BM_SHADOW}, counts[1] = {C_SHADOW};
        uint32_t *const queues[1] = {w.q_shadow};
        if ((e = compact(w, 1, which, queues, counts, s)) != cudaSuccess) return e;
      }
      k_wf_shadow<B><<<persistent, kWfBlock, 0, s>>>(a, w, next);
      if (w.ordered) {
        const int which[1] = {BM_EXT}, counts[1] = {next ? C_EXT1 : C_EXT0};
        uint32_t *const queues[1] = {w.q_ext[next]};
        if ((e = compact(w, 1, which, queues, counts, s)) != cudaSuccess) return e;
      }
      k_wf_rotate<<<1, 32, 0, s>>>(w, cur);
    }
    k_wf_reduce<B><<<(w.wave_px + kWfBlock - 1) / kWfBlock, kWfBlock, 0, s>>>(a, w);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

WfArgs make_args(const sc_trace_params &p, unsigned *status, unsigned long long *counters) {
  static const JitterNorm jn = jitter_norm_host();
  WfArgs a;
  memset(&a, 0, sizeof(a));
  a.P = p;
  a.status = status;
  a.counters = counters;
  a.jn = jn;
  a.nb = p.n_bins > 0 ? p.n_bins : 1;
  a.jitter = (p.flags & SC_FLAG_WAVELENGTH_JITTER) && a.nb > 1;
  return a;
}

}  // namespace

cudaError_t launch_trace_camera_wavefront(const DevScene &S, const sc_trace_params &p, const sc_frame &f,
                                          unsigned *status, unsigned long long *counters, void *workspace,
                                          int64_t max_paths, int num_sms, cudaStream_t s) {
  WfArgs a = make_args(p, status, counters);
  a.S = S;
  a.F = f;
  Wave w;
  if (!carve_wave(workspace, max_paths, w)) return cudaErrorInvalidValue;
  const int64_t total_slots = (int64_t)scene_tickets(S.cam);
  const int64_t wave_px = wavefront_wave_pixels(S.cam.width, S.cam.height, p.spp, max_paths);
  return run_waves<false>(a, w, total_slots, wave_px, num_sms, s);
}

cudaError_t launch_trace_batch_wavefront(const BatchEntry *tab, int n, int64_t total_slots, const sc_trace_params &p,
                                         unsigned *status, unsigned long long *counters, void *workspace,
                                         int64_t max_paths, int num_sms, cudaStream_t s) {
  WfArgs a = make_args(p, status, counters);
  a.tab = tab;
  a.n_tab = n;
  Wave w;
  if (!carve_wave(workspace, max_paths, w)) return cudaErrorInvalidValue;
  const int64_t wave_px = std::max<int64_t>(32, max_paths / (32 * (int64_t)std::max(p.spp, 1)) * 32);
  return run_waves<true>(a, w, total_slots, wave_px, num_sms, s);
}

}  // namespace sc
