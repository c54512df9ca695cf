// render.cu -- camera path tracer, light tracer (caustic splats), resolve and test queries.
//
// Transport rules (identical in every kernel; the paper's renderer is an engine, so these are
// the readings this library implements, stated in the header of each function):
//   * camera path: pinhole ray with uniform pixel jitter; at a dielectric, Fresnel-chosen
//     reflection or Snell refraction (throughput unchanged); at a diffuse surface, next-event
//     estimation to one uniformly chosen light (glass blocks shadow rays) then a cosine bounce
//     (throughput times albedo); emitters count only along purely specular prefixes.
//   * light path: emitted from a uniformly chosen light, traced through glass; at its first
//     diffuse vertex after at least one specular event it is connected to the pinhole and
//     splatted with weight beta * albedo/pi * cos / (d^2 * A_pix * cos^3(theta_c)).
#include "device.cuh"
#include "internal.h"

namespace sc {

constexpr int kBlock = 128;
// resident blocks per SM the camera kernel is compiled for (register budget = 64K / (128 * this))
#ifndef SC_CAM_MIN_BLOCKS
#define SC_CAM_MIN_BLOCKS 4
#endif
// node visits per traversal chunk in the camera kernel
#ifndef SC_TRAV_CHUNK
#define SC_TRAV_CHUNK 12
#endif

// Camera paths as a per-lane state machine.  Every loop iteration each live lane traces exactly
// one ray -- an extension ray or the shadow ray of its pending next-event estimate -- through the
// same traversal call, then advances its path by one event.  A lane whose path ends starts its
// pixel's next sample at once, and a lane whose pixel is done takes the next pixel from a global
// ticket (warp-aggregated), so lanes never wait for the longest path of their warp.  The event
// order, and therefore every random number, decision and signature, is that of the
// straightforward per-path loop: hit -> (emission | dielectric scatter | NEE -> shadow result
// -> bounce).
enum : int { M_IDLE = 0, M_EXTEND = 1, M_SHADOW = 2 };
enum : uint32_t {
  F_SPEC_ONLY = 1u, F_DIFFUSE_FIRST = 2u, F_LAST_SPECULAR = 4u, F_FIXUP = 8u, F_HAS_NEXT = 16u
};

// BATCH = false: one scene (S0, F0), persistent grid, tickets from the global counter.
// BATCH = true: one block per chunk of kBatchChunk tickets of one scene of tab[0..n_tab):
// tab[i].begin is the first block of scene i.  The block loads its scene's record into shared
// memory once and its lanes take tickets of the chunk from a shared counter, so the per-lane
// work is exactly the single-scene path; the block scheduler balances scenes of uneven size.
// Scene i draws its random numbers with scene index P.scene_index + i.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock, SC_CAM_MIN_BLOCKS)
    k_trace_camera_t(DevScene S0, sc_trace_params P, sc_frame F0, const BatchEntry *tab, int n_tab,
                     unsigned total_tickets, unsigned *status, unsigned *ticket, unsigned long long *counters,
                     JitterNorm jn) {
  TravCount tc;
  __shared__ float3 wts[kMaxBins];
  __shared__ BatchEntry blk;
  __shared__ unsigned blk_scene, blk_ticket, blk_end;
  if (BATCH && threadIdx.x == 0) {
    int lo = 0, hi = n_tab - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].begin <= blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    blk = tab[lo];
    blk_scene = (unsigned)lo;
    const unsigned first = (blockIdx.x - blk.begin) * kBatchChunk;
    blk_ticket = first;
    blk_end = min(first + kBatchChunk, scene_tickets(blk.S.cam));
  }
  spectral_table(wts, P.n_bins);  // ends with __syncthreads
  const DevScene S = BATCH ? blk.S : S0;
  const sc_frame F = BATCH ? blk.F : F0;
  const Cam cam = make_cam(S.cam);
  const int tiles_x = (cam.W + 7) / 8;
  const unsigned n_tickets = BATCH ? blk_end : (unsigned)(tiles_x * ((cam.H + 3) / 4)) * 32u;
  if (BATCH) ticket = &blk_ticket;
  const int lane = threadIdx.x & 31;
  const float3 env = f3(S.env);
  const int nb = P.n_bins > 0 ? P.n_bins : 1;
  const bool jitter = (P.flags & SC_FLAG_WAVELENGTH_JITTER) && nb > 1;
  const int scene_index = BATCH ? P.scene_index + (int)blk_scene : P.scene_index;

  // pixel state
  int px = 0, py = 0, pix = -1, s = 0;
  bool done = false;
  float3 acc = f3(0.f, 0.f, 0.f);
  // path state
  int mode = M_IDLE, k = 0, n_diffuse = 0;
  float ul = 0.0f;  // the path's bin draw u: bin floor(u B), wavelength (path_lambda)
  uint32_t fl = 0, sig = 0, first = kMiss, nq = 0, nspec = 0;
  float3 o = f3(0.f, 0.f, 0.f), d = o, beta = o, L = o, nee = o, o2 = o, d2 = o;
  float tmax = 3.0e38f;
  // traversal state, kept across chunks
  TravState ts;
  bool tracing = false;
  int stack[kStack];

  for (;;) {
    // ---- refill: next sample of this pixel, or the next pixel ----
    if (mode == M_IDLE && pix >= 0 && s >= P.spp) {
      if (F.accum_camera && SC_IN_RANGE(status, 4, pix, cam.W * cam.H)) {
        float4 *a = reinterpret_cast<float4 *>(F.accum_camera) + pix;
        float4 v = *a;
        v.x += acc.x; v.y += acc.y; v.z += acc.z;
        *a = v;
      }
      pix = -1;
    }
    const bool want = mode == M_IDLE && pix < 0 && !done;
    const unsigned wmask = __ballot_sync(0xFFFFFFFFu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(ticket, (unsigned)__popc(wmask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (want) {
        const unsigned t = base + (unsigned)__popc(wmask & ((1u << lane) - 1u));
        bool got = false;
        if (t < n_tickets) {
          const unsigned tile = t >> 5, in = t & 31u;
          px = (int)(tile % tiles_x) * 8 + (int)(in & 7u);
          py = (int)(tile / tiles_x) * 4 + (int)(in >> 3);
          got = px < cam.W && py < cam.H;
        } else {
          done = true;
        }
        if (got) {
          pix = py * cam.W + px;
          s = 0;
          acc = f3(0.f, 0.f, 0.f);
        }
      }
    }
    if (mode == M_IDLE && pix >= 0 && s < P.spp) {
      // start sample s: primary ray (tag 0: jitter x, jitter y, wavelength bin)
      const uint4 x0 = draw(P.seed, (uint32_t)pix, (uint32_t)(P.sample_offset + s), 0u, 0u, (uint32_t)scene_index);
      ul = u01(x0.z);
      o = cam.eye;
      d = cam_dir(cam, (px + u01(x0.x)) / cam.W, (py + u01(x0.y)) / cam.H);
      tmax = 3.0e38f;
      beta = f3(1.f, 1.f, 1.f);
      L = f3(0.f, 0.f, 0.f);
      fl = F_SPEC_ONLY;
      n_diffuse = 0;
      sig = 2166136261u;
      first = kMiss;
      nq = 0;
      nspec = 0;
      k = 0;
      mode = M_EXTEND;
    }
    if (__all_sync(0xFFFFFFFFu, mode == M_IDLE && done)) break;
    if (mode == M_IDLE) continue;  // a lane whose ticket fell outside the image retries

    // ---- advance this lane's ray by at most SC_TRAV_CHUNK node visits; lanes whose query
    // completes shade below while the others keep traversing on the next iteration ----
    if (!tracing) {
      trav_begin(ts, tmax, mode == M_SHADOW);
      tracing = true;
    }
    if (!trav_step(S, make_wray(o, d), tmax, ts, stack, SC_TRAV_CHUNK, status, tc)) continue;
    tracing = false;
    ++tc.queries;
    const Hit h = ts.h;

    bool finish = false;
    if (mode == M_SHADOW) {
      const bool lit = h.prim < 0;
      if (lit) L = L + nee;
      sig = fnv(sig, lit ? EV_LIT : EV_UNLIT);
      if (fl & F_FIXUP) sig = fnv(sig, EV_FIXUP);
      if (fl & F_HAS_NEXT) {
        o = o2;
        d = d2;
        tmax = 3.0e38f;
        mode = M_EXTEND;
      } else {
        finish = true;
      }
    } else {
      ++nq;
      sig = fnv(sig, h.id);
      if (k == 0) first = h.id;
      if (h.prim < 0) {
        L = L + beta * env;
        finish = true;
      } else if (!SC_IN_RANGE(status, 5, h.prim, S.n_tris) || !SC_IN_RANGE(status, 6, h.id, S.n_tris)) {
        finish = true;
      } else {
        const Surf f = interact(S, d, h);
        const sc_material m = S.mats[SC_IN_RANGE(status, 7, f.mat, S.n_mats) ? f.mat : 0];
        // a segment that ends on a dielectric's inner side ran through that glass (Beer-Lambert)
        if (m.kind == SC_MAT_DIELECTRIC && f.cosg > 0.0f && absorbs(m)) beta = beta * absorb_over(m, h.t);
        if (m.kind == SC_MAT_EMISSIVE) {
          const bool count = (fl & F_SPEC_ONLY) || ((P.flags & SC_FLAG_EMITTER_AFTER_DS) && (fl & F_DIFFUSE_FIRST) &&
                                                    n_diffuse == 1 && (fl & F_LAST_SPECULAR));
          if (f.cosg < 0.0f && count) L = L + beta * f3(m.emission);
          finish = true;
        } else {
          const uint32_t pixu = (uint32_t)pix, smp = (uint32_t)(P.sample_offset + s);
          const uint4 xs = draw(P.seed, pixu, smp, (uint32_t)(k + 1), 1u, (uint32_t)scene_index);
          if (m.kind == SC_MAT_DIELECTRIC) {
            bool refl, fix, alive = true;
            const float nl = cauchy_at(m.cauchy_a, m.cauchy_b, path_lambda(ul, nb, jitter), P.n_bins);
            float3 nd;
            if (m.roughness > 0.0f) {
              float w;
              alive = rough_dielectric(f, d, nl, m.roughness, u01(xs.x), u01(xs.y), u01(xs.z), P.flags, nd, w, refl,
                                       fix);
              beta = beta * w;
            } else {
              nd = dielectric(f, d, nl, u01(xs.x), P.flags, refl, fix);
            }
            ++nspec;
            if (!alive) {
              sig = fnv(sig, EV_KILL);
              finish = true;
            } else {
              sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
              if (fix) sig = fnv(sig, EV_FIXUP);
              fl |= F_LAST_SPECULAR;
              o = offset_along(f.p, f.ng, nd);
              d = nd;
              ++k;
              if (k >= P.max_depth) finish = true;
            }
          } else {
            // diffuse: next-event estimate (shadow ray traced next iteration), then the bounce
            const float3 alb = albedo_at(S, m, f);
            bool need_shadow = false;
            float3 so = f3(0.f, 0.f, 0.f), sd = so;
            float sdist = 0.0f;
            if (S.n_lights > 0) {
              const uint4 xn = draw(P.seed, pixu, smp, (uint32_t)(k + 1), 2u, (uint32_t)scene_index);
              const sc_light Lg = S.lights[choose(xn.x, S.n_lights)];
              float3 lp = f3(0.f, 0.f, 0.f);
              float geo = 0.0f;
              bool ok = false;
              if (Lg.kind == SC_LIGHT_POINT) {
                lp = f3(Lg.p);
                float3 w = lp - f.p;
                const float d2l = dot(w, w);
                w = w * (1.0f / sqrtf(d2l));
                const float cs = dot(f.nsf, w), cg = dot(f.ngf, w);
                ok = cs > 0.0f && cg > 0.0f;
                geo = cs / d2l;
              } else if (Lg.kind == SC_LIGHT_RECT) {
                const float3 eu = f3(Lg.u), ev = f3(Lg.v);
                lp = f3(Lg.p) + eu * u01(xn.y) + ev * u01(xn.z);
                const float3 c = cross(eu, ev);
                const float area = length(c);
                const float3 nlt = c * (1.0f / area);
                float3 w = lp - f.p;
                const float d2l = dot(w, w);
                w = w * (1.0f / sqrtf(d2l));
                const float cs = dot(f.nsf, w), cg = dot(f.ngf, w), cl = -dot(nlt, w);
                ok = cs > 0.0f && cg > 0.0f && cl > 0.0f;
                geo = cs * cl * area / d2l;
              }
              if (ok) {
                so = f.p + f.ngf * eps_of(f.p);
                const float3 wv = lp - so;
                sdist = length(wv);
                sd = wv * (1.0f / sdist);
                nee = beta * (alb * f3(Lg.power)) * (geo * (float)S.n_lights / kPi);
                need_shadow = true;
              }
            }
            if (k == 0) fl |= F_DIFFUSE_FIRST;
            ++n_diffuse;
            fl &= ~(F_SPEC_ONLY | F_LAST_SPECULAR | F_FIXUP | F_HAS_NEXT);
            if (k < P.max_depth - 1) {
              float3 nd = cosine_dir(f.nsf, u01(xs.y), u01(xs.z));
              if (!(dot(nd, f.ngf) > 0.0f)) {
                nd = cosine_dir(f.ngf, u01(xs.y), u01(xs.z));
                fl |= F_FIXUP;
              }
              beta = beta * alb;
              o2 = f.p + f.ngf * eps_of(f.p);
              d2 = nd;
              fl |= F_HAS_NEXT;
            }
            ++k;
            if (need_shadow) {
              o = so;
              d = sd;
              tmax = sdist * (1.0f - 1e-4f);
              mode = M_SHADOW;
            } else {
              sig = fnv(sig, EV_UNLIT);
              if (fl & F_FIXUP) sig = fnv(sig, EV_FIXUP);
              if (fl & F_HAS_NEXT) {
                o = o2;
                d = d2;
                tmax = 3.0e38f;
              } else {
                finish = true;
              }
            }
          }
        }
      }
    }
    if (finish) {
      const int bin = bin_of(ul, nb);
      const float3 Lw = L * (jitter ? jitter_weight(ul, jn) : wts[bin]);
      acc = acc + Lw;
      if (F.path_records && SC_IN_RANGE(status, 9, (int64_t)pix * P.spp + s, (int64_t)cam.W * cam.H * P.spp)) {
        sc_path_record r;
        r.L[0] = Lw.x; r.L[1] = Lw.y; r.L[2] = Lw.z;
        r.first_tri = first;
        r.signature = sig;
        r.n_queries = nq;
        r.bin = (uint32_t)bin;
        r.n_specular = nspec;
        F.path_records[(int64_t)pix * P.spp + s] = r;
      }
      ++s;
      mode = M_IDLE;
    }
  }
  if (counters) {
    atomicAdd(&counters[0], (unsigned long long)tc.queries);
    atomicAdd(&counters[1], (unsigned long long)tc.nodes);
    atomicAdd(&counters[2], (unsigned long long)tc.tris);
  }
}

// ---- the light tracer ------------------------------------------------------------------------
// Light path emission: light chosen by xe.x, position from xe.y / xe.z, direction from xd (the
// emission draws of the path); guided emission into the cone subtending the guide sphere.
// Returns false when the sampled direction leaves a one-sided emitter (nothing is traced).
__device__ __forceinline__ bool light_emit(const DevScene &S, const sc_light_params &P, uint4 xe, uint4 xd, float3 &o,
                                           float3 &d, float3 &beta) {
  const int j = choose(xe.x, S.n_lights);
  const sc_light Lg = S.lights[j];
  const float3 gc = f3(P.guide[0], P.guide[1], P.guide[2]);
  const float gr = P.guide[3];
  // direction uniform in the cone subtending the guide sphere from x; returns the cone's solid
  // angle, or 0 when x lies inside the sphere (then unguided)
  auto guided = [&](float3 x, float3 &dir) -> float {
    if (!(gr > 0.0f)) return 0.0f;
    const float3 v = gc - x;
    const float dist = length(v);
    if (!(dist > gr)) return 0.0f;
    const float3 wz = v * (1.0f / dist);
    const float sin2 = (gr / dist) * (gr / dist);
    const float cmax = sqrtf(fmaxf(0.0f, 1.0f - sin2));
    const float omc = sin2 / (1.0f + cmax);  // 1 - cos(theta_max) without cancellation
    const float ct = 1.0f - u01(xd.x) * omc;
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincospif(2.0f * u01(xd.y), &sp, &cp);
    float3 t1, t2;
    onb(wz, t1, t2);
    dir = normalize(t1 * (st * cp) + t2 * (st * sp) + wz * ct);
    return 2.0f * kPi * omc;
  };
  bool emitted = true;
  if (Lg.kind == SC_LIGHT_POINT) {
    const float z = 1.0f - 2.0f * u01(xd.x);
    float s, c;
    sincospif(2.0f * u01(xd.y), &s, &c);
    const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    o = f3(Lg.p);
    const float omega = guided(o, d);
    if (omega > 0.0f) {
      beta = f3(Lg.power) * (omega * S.n_lights);
    } else {
      d = normalize(f3(rr * c, rr * s, z));
      beta = f3(Lg.power) * (4.0f * kPi * S.n_lights);
    }
  } else if (Lg.kind == SC_LIGHT_RECT) {
    const float3 eu = f3(Lg.u), ev = f3(Lg.v);
    const float3 c = cross(eu, ev);
    const float area = length(c);
    const float3 nlt = c * (1.0f / area);
    const float3 x = f3(Lg.p) + eu * u01(xe.y) + ev * u01(xe.z);
    const float omega = guided(x, d);
    if (omega > 0.0f) {
      const float cl = dot(d, nlt);
      emitted = cl > 0.0f;  // one-sided emitter
      beta = f3(Lg.power) * (area * S.n_lights * cl * omega);
    } else {
      d = cosine_dir(nlt, u01(xd.x), u01(xd.y));
      beta = f3(Lg.power) * (kPi * area * S.n_lights);
    }
    o = x + nlt * eps_of(x);
  } else {
    const float3 dir = normalize(f3(Lg.u));
    float3 t1, t2;
    onb(dir, t1, t2);
    const float rad = Lg.radius * sqrtf(u01(xe.y));
    float s, c;
    sincospif(2.0f * u01(xe.z), &s, &c);
    o = f3(Lg.p) + t1 * (rad * c) + t2 * (rad * s);
    d = dir;
    beta = f3(Lg.power) * (kPi * Lg.radius * Lg.radius * S.n_lights);
  }
  return emitted;
}

// Light paths: emission, specular chain, splat at the first diffuse vertex after glass.
// photons (optional): three float4 per path -- (position, bin as int bits), (shading normal on the
// side the light arrived from, 1 if deposited), (throughput, 0) -- at that same vertex.
// One bounce per loop turn: a lane whose path has ended takes the next path at once (tickets for
// all such lanes of a warp in one atomic) instead of waiting for the longest path of a batch of
// 32 (32M guided light paths through the dense glass scene: 82.0 -> 58.9 ms).
__global__ void __launch_bounds__(kBlock) k_trace_lights(DevScene S, sc_light_params P, sc_frame F,
                                                            unsigned *status, unsigned long long *ticket,
                                                            unsigned long long *counters, JitterNorm jn,
                                                            float4 *photons) {
  TravCount tc;
  __shared__ float3 wts[kMaxBins];
  spectral_table(wts, P.n_bins);
  const Cam cam = make_cam(S.cam);
  const float apix = (2.0f * cam.th * cam.aspect / cam.W) * (2.0f * cam.th / cam.H);
  const int lane = threadIdx.x & 31;
  const int nbl = P.n_bins > 0 ? P.n_bins : 1;
  const bool jitter = (P.flags & SC_FLAG_WAVELENGTH_JITTER) && nbl > 1;
  const float kNaN = __int_as_float(0x7FC00000);
  unsigned long long li = 0;
  uint32_t lo = 0, hi = 0, sig = 0, nspec = 0;
  int k = 0, bin = 0, pixel = -1;
  float ul = 0.0f;
  float3 o = f3(0.f, 0.f, 0.f), d = o, beta = o, C = o, X = o, phn = o, phb = o;
  bool active = false, exhausted = false, had_spec = false, ph = false;
  for (;;) {
    bool fin = false;
    const bool want = !active && !exhausted;
    const unsigned wmask = __ballot_sync(0xFFFFFFFFu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(ticket, (unsigned long long)__popc(wmask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (want) {
        const unsigned long long tk = base + (unsigned long long)__popc(wmask & ((1u << lane) - 1u));
        if (tk < (unsigned long long)P.n_paths) {
          li = tk;
          const int64_t idx = P.path_offset + (int64_t)li;
          lo = (uint32_t)idx;
          hi = (uint32_t)((uint64_t)idx >> 32);
          const uint4 xe = draw(P.seed, lo, hi, 0u, 4u, (uint32_t)P.scene_index);
          const uint4 xd = draw(P.seed, lo, hi, 0u, 3u, (uint32_t)P.scene_index);
          ul = u01(xe.w);
          bin = bin_of(ul, nbl);
          sig = 2166136261u;
          nspec = 0;
          pixel = -1;
          C = f3(0.f, 0.f, 0.f);
          X = f3(kNaN, kNaN, kNaN);
          ph = false;
          phn = phb = f3(0.f, 0.f, 0.f);
          had_spec = false;
          k = 0;
          active = true;
          if (!(S.n_lights > 0 && light_emit(S, P, xe, xd, o, d, beta))) fin = true;  // nothing to trace
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xFFFFFFFFu, !active && exhausted)) break;
    if (active && !fin) {
      if (k >= P.max_depth) {
        fin = true;
      } else {
        const Hit h = closest_hit(S, o, d, 3.0e38f, status, tc);
        sig = fnv(sig, h.id);
        if (h.prim < 0) {
          fin = true;
        } else {
          const Surf f = interact(S, d, h);
          const sc_material m = S.mats[f.mat];
          if (m.kind == SC_MAT_DIELECTRIC && f.cosg > 0.0f && absorbs(m)) beta = beta * absorb_over(m, h.t);
          if (m.kind == SC_MAT_EMISSIVE) {
            fin = true;
          } else if (m.kind == SC_MAT_DIELECTRIC) {
            const uint4 xs = draw(P.seed, lo, hi, (uint32_t)(k + 1), 3u, (uint32_t)P.scene_index);
            bool refl, fix, alive = true;
            const float nl = cauchy_at(m.cauchy_a, m.cauchy_b, path_lambda(ul, nbl, jitter), P.n_bins);
            float3 nd;
            if (m.roughness > 0.0f) {
              float wgt;
              alive = rough_dielectric(f, d, nl, m.roughness, u01(xs.x), u01(xs.y), u01(xs.z), P.flags, nd, wgt, refl,
                                       fix);
              if (alive) beta = beta * wgt;
            } else {
              nd = dielectric(f, d, nl, u01(xs.x), P.flags, refl, fix);
            }
            ++nspec;
            if (!alive) {
              sig = fnv(sig, EV_KILL);
              fin = true;
            } else {
              sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
              if (fix) sig = fnv(sig, EV_FIXUP);
              had_spec = true;
              o = offset_along(f.p, f.ng, nd);
              d = nd;
              ++k;
            }
          } else if (!had_spec && !(P.flags & SC_FLAG_SPLAT_DIRECT)) {
            fin = true;
          } else {
            // the first diffuse vertex after glass: photon, and the splat toward the camera
            fin = true;
            X = f.p;
            if (had_spec) {
              ph = true;
              phn = f.nsf;
              phb = beta;
            }
            const float3 alb = albedo_at(S, m, f);
            float3 wc = cam.eye - f.p;
            const float dc = length(wc);
            wc = wc * (1.0f / dc);
            const float cs = dot(f.nsf, wc), cg = dot(f.ngf, wc);
            const float3 wv = wc * -1.0f;
            const float cc = dot(wv, cam.f);
            bool lit = cs > 0.0f && cg > 0.0f && cc > 0.0f;
            float sx = 0.0f, sy = 0.0f;
            if (lit) {
              sx = (dot(wv, cam.r) / cc / (cam.th * cam.aspect) + 1.0f) * 0.5f;
              sy = (1.0f - dot(wv, cam.u) / cc / cam.th) * 0.5f;
              lit = sx >= 0.0f && sx < 1.0f && sy >= 0.0f && sy < 1.0f;
            }
            if (lit) {
              const float3 so = f.p + f.ngf * eps_of(f.p);
              const float3 wsv = cam.eye - so;
              const float dist = length(wsv);
              lit = !any_hit(S, so, wsv * (1.0f / dist), dist * (1.0f - 1e-4f), status, tc);
            }
            if (!lit) {
              sig = fnv(sig, EV_UNLIT);
            } else {
              sig = fnv(sig, EV_LIT);
              const int ix = min((int)floorf(sx * cam.W), cam.W - 1), iy = min((int)floorf(sy * cam.H), cam.H - 1);
              const float g = cs / (dc * dc * apix * cc * cc * cc) / kPi;
              C = beta * g * alb * (jitter ? jitter_weight(ul, jn) : wts[bin]);
              pixel = iy * cam.W + ix;
              if (F.accum_caustic)  // one 16-byte vector atomic per splat (the entry's 4th word gets +0)
                atomicAdd(reinterpret_cast<float4 *>(F.accum_caustic) + pixel, make_float4(C.x, C.y, C.z, 0.0f));
            }
          }
        }
      }
    }
    if (fin) {
      if (photons) {
        float4 *q = photons + 3 * li;
        q[0] = make_float4(X.x, X.y, X.z, __int_as_float(bin));
        q[1] = make_float4(phn.x, phn.y, phn.z, ph ? 1.0f : 0.0f);
        q[2] = make_float4(phb.x, phb.y, phb.z, 0.0f);
      }
      if (F.light_records) {
        sc_light_record r;
        r.C[0] = C.x; r.C[1] = C.y; r.C[2] = C.z;
        r.pixel = pixel;
        r.x[0] = X.x; r.x[1] = X.y; r.x[2] = X.z;
        r.signature = sig;
        r.n_specular = nspec;
        r.bin = (uint32_t)bin;
        r.pad[0] = r.pad[1] = 0;
        F.light_records[li] = r;
      }
      active = false;
    }
  }
  if (counters) {
    atomicAdd(&counters[0], (unsigned long long)tc.queries);
    atomicAdd(&counters[1], (unsigned long long)tc.nodes);
    atomicAdd(&counters[2], (unsigned long long)tc.tris);
  }
}

// Resolve: normalised images and the ground-truth buffers from a pixel-centre primary ray.
__global__ void k_resolve(DevScene S, sc_resolve_params P, sc_frame F, unsigned *status) {
  const Cam cam = make_cam(S.cam);
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= cam.W * cam.H) return;
  const int px = pix % cam.W, py = pix / cam.W;
  const float inv_spp = P.spp_total > 0 ? (float)(1.0 / P.spp_total) : 0.0f;
  const float inv_nl = P.light_paths_total > 0 ? (float)(1.0 / P.light_paths_total) : 0.0f;
  float3 D = f3(0.f, 0.f, 0.f), C = f3(0.f, 0.f, 0.f);
  if (F.accum_camera) D = xyz(reinterpret_cast<const float4 *>(F.accum_camera)[pix]) * inv_spp;
  if (F.accum_caustic) C = xyz(reinterpret_cast<const float4 *>(F.accum_caustic)[pix]) * inv_nl;
  float3 Lc = f3(0.f, 0.f, 0.f);
  if (F.accum_local_caustic) Lc = xyz(reinterpret_cast<const float4 *>(F.accum_local_caustic)[pix]) * inv_spp;
  if (F.direct) reinterpret_cast<float4 *>(F.direct)[pix] = make_float4(D.x, D.y, D.z, 1.0f);
  if (F.caustic) reinterpret_cast<float4 *>(F.caustic)[pix] = make_float4(C.x, C.y, C.z, 1.0f);
  if (F.local_caustic) reinterpret_cast<float4 *>(F.local_caustic)[pix] = make_float4(Lc.x, Lc.y, Lc.z, 1.0f);
  if (F.rgb)
    reinterpret_cast<float4 *>(F.rgb)[pix] = make_float4(D.x + C.x + Lc.x, D.y + C.y + Lc.y, D.z + C.z + Lc.z, 1.0f);
  const float3 d = cam_dir(cam, (px + 0.5f) / cam.W, (py + 0.5f) / cam.H);
  TravCount tc;
  const Hit h = closest_hit(S, cam.eye, d, 3.0e38f, status, tc);
  int inst = -1, tri = -1;
  uint8_t mask = 0, cmask = 0, lmask = 0;
  float depth = __int_as_float(0x7F800000), dn = 1.0f;
  float4 nw = make_float4(0.f, 0.f, 0.f, 0.f), nc = nw, alb = nw;
  if (h.prim >= 0) {
    const Surf f = interact(S, d, h);
    const sc_material m = S.mats[f.mat];
    inst = S.tri_obj[h.id];
    tri = (int)h.id;
    mask = m.kind == SC_MAT_DIELECTRIC;
    depth = length(f.p - cam.eye);
    dn = fminf(depth / P.depth_range, 1.0f);
    const float3 n = f.nsf;
    nw = make_float4(n.x, n.y, n.z, 1.0f);
    nc = make_float4(dot(n, cam.r), dot(n, cam.u), -dot(n, cam.f), 1.0f);
    const float3 a = m.kind == SC_MAT_DIFFUSE ? albedo_at(S, m, f) : f3(1.f, 1.f, 1.f);
    alb = make_float4(a.x, a.y, a.z, 1.0f);
    const float yc = 0.2126f * C.x + 0.7152f * C.y + 0.0722f * C.z;
    const float yd = 0.2126f * D.x + 0.7152f * D.y + 0.0722f * D.z;
    cmask = (m.kind != SC_MAT_DIELECTRIC) && (yc > P.tau_rel * fmaxf(yd, 1e-3f));
    const float yl = 0.2126f * Lc.x + 0.7152f * Lc.y + 0.0722f * Lc.z;
    lmask = (m.kind == SC_MAT_DIELECTRIC) && (yl > P.tau_rel * fmaxf(yd, 1e-3f));
  }
  if (F.instance_id) F.instance_id[pix] = inst;
  if (F.tri_id) F.tri_id[pix] = tri;
  if (F.mask) F.mask[pix] = mask;
  if (F.caustic_mask) F.caustic_mask[pix] = cmask;
  if (F.local_caustic_mask) F.local_caustic_mask[pix] = lmask;
  if (F.depth) F.depth[pix] = depth;
  if (F.depth_norm) F.depth_norm[pix] = dn;
  if (F.normal_world) reinterpret_cast<float4 *>(F.normal_world)[pix] = nw;
  if (F.normal_camera) reinterpret_cast<float4 *>(F.normal_camera)[pix] = nc;
  if (F.albedo) reinterpret_cast<float4 *>(F.albedo)[pix] = alb;
}

// Outline and occlusion-boundary ground truth (Sec. III-D) from the buffers k_resolve wrote:
// instance ids, transparency mask, depth.  One block per 32 x 8 pixels.  The block stages the ids
// of its tile plus a halo of R = max(T, 1) pixels in shared memory (coordinates clamped to the
// image, which leaves every clipped window's minimum and maximum unchanged), takes per halo row the
// minimum and maximum id over each output column's 2T+1 wide window, then per output pixel the
// minimum and maximum of those over 2T+1 rows: the pixel is on the outline when either differs from
// its own id (the Chebyshev window of radius T holds another id) and it is transparent.  Occlusion
// codes compare each transparent pixel with its four in-image neighbours: 1 when it is the nearer
// side of a depth jump |d_p - d_q| > jump_rel * min(d_p, d_q) (a miss, d = inf, always jumps),
// else 2 when a neighbour shows another id, else 0.
constexpr int kEdgeTX = 32, kEdgeTY = 8;
__global__ void __launch_bounds__(kEdgeTX * kEdgeTY) k_gt_edges(sc_frame F, int T, float jump_rel) {
  extern __shared__ int edge_sm[];
  const int W = F.width, H = F.height;
  const int R = T > 1 ? T : 1;
  const int SW = kEdgeTX + 2 * R, SH = kEdgeTY + 2 * R;
  int *ids = edge_sm;               // SH x SW
  int *rmin = ids + SH * SW;        // SH x kEdgeTX
  int *rmax = rmin + SH * kEdgeTX;  // SH x kEdgeTX
  const int x0 = blockIdx.x * kEdgeTX, y0 = blockIdx.y * kEdgeTY;
  const int tid = threadIdx.y * kEdgeTX + threadIdx.x;
  constexpr int nt = kEdgeTX * kEdgeTY;
  for (int i = tid; i < SH * SW; i += nt) {
    const int r = i / SW, c = i - r * SW;
    const int y = min(max(y0 - R + r, 0), H - 1), x = min(max(x0 - R + c, 0), W - 1);
    ids[i] = F.instance_id[y * W + x];
  }
  __syncthreads();
  if (F.outline) {
    for (int i = tid; i < SH * kEdgeTX; i += nt) {
      const int r = i / kEdgeTX, c = i - r * kEdgeTX;
      const int *row = ids + r * SW + c + R - T;  // smem columns c + R - T .. c + R + T
      int mn = row[0], mx = row[0];
      for (int k = 1; k <= 2 * T; ++k) {
        mn = min(mn, row[k]);
        mx = max(mx, row[k]);
      }
      rmin[i] = mn;
      rmax[i] = mx;
    }
    __syncthreads();
  }
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (x >= W || y >= H) return;
  const int p = y * W + x;
  const int cy = threadIdx.y + R, cx = threadIdx.x + R;
  const int id = ids[cy * SW + cx];
  const bool transparent = F.mask[p] != 0;
  if (F.outline) {
    bool edge = false;
    if (transparent) {
      int mn = id, mx = id;
      for (int k = -T; k <= T; ++k) {
        const int i = (cy + k) * kEdgeTX + threadIdx.x;
        mn = min(mn, rmin[i]);
        mx = max(mx, rmax[i]);
      }
      edge = mn != id || mx != id;
    }
    F.outline[p] = edge ? 1 : 0;
  }
  if (F.occlusion) {
    uint8_t code = 0;
    if (transparent) {
      const float dp = F.depth[p];
      bool nearer = false, contact = false;
      const int ox[4] = {-1, 1, 0, 0}, oy[4] = {0, 0, -1, 1};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int qx = x + ox[k], qy = y + oy[k];
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        const float dq = F.depth[qy * W + qx];
        const bool jump = fabsf(dp - dq) > jump_rel * fminf(dp, dq);
        nearer |= jump && dp < dq;
        contact |= ids[(cy + oy[k]) * SW + cx + ox[k]] != id;
      }
      code = nearer ? 1 : (contact ? 2 : 0);
    }
    F.occlusion[p] = code;
  }
}

__global__ void k_intersect(DevScene S, const float4 *rays, int64_t n, float4 *hits, unsigned *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = rays[2 * i], b = rays[2 * i + 1];
  TravCount tc;
  const Hit h = closest_hit(S, xyz(a), xyz(b), a.w, status, tc);
  hits[i] = make_float4(h.prim >= 0 ? h.t : a.w, __int_as_float(h.prim >= 0 ? (int)h.id : -1), h.b1, h.b2);
}

__global__ void k_occluded(DevScene S, const float4 *rays, int64_t n, int32_t *occ, unsigned *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = rays[2 * i], b = rays[2 * i + 1];
  TravCount tc;
  occ[i] = any_hit(S, xyz(a), xyz(b), a.w, status, tc) ? 1 : 0;
}

__global__ void k_philox(const uint4 *ctr, uint64_t key, int64_t n, uint4 *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = philox(ctr[i], (uint32_t)key, (uint32_t)(key >> 32));
}

const void *camera_kernel_ptr() { return reinterpret_cast<const void *>(&k_trace_camera_t<false>); }
const void *light_kernel_ptr() { return reinterpret_cast<const void *>(&k_trace_lights); }

static int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

cudaError_t launch_trace_camera(const DevScene &S, const sc_trace_params &p, const sc_frame &f, unsigned *status,
                                unsigned *ticket, unsigned long long *counters, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  static const JitterNorm jn = jitter_norm_host();
  k_trace_camera_t<false><<<grid, kBlock, 0, s>>>(S, p, f, nullptr, 0, 0u, status, ticket, counters, jn);
  return cudaGetLastError();
}

cudaError_t launch_trace_batch(const BatchEntry *tab, int n, unsigned total_blocks, const sc_trace_params &p,
                               unsigned *status, unsigned long long *counters, cudaStream_t s) {
  if (total_blocks == 0) return cudaSuccess;
  DevScene none{};
  sc_frame nof{};
  static const JitterNorm jn = jitter_norm_host();
  k_trace_camera_t<true><<<total_blocks, kBlock, 0, s>>>(none, p, nof, tab, n, 0u, status, nullptr, counters, jn);
  return cudaGetLastError();
}

cudaError_t launch_trace_lights(const DevScene &S, const sc_light_params &p, const sc_frame &f, unsigned *status,
                                unsigned long long *ticket, unsigned long long *counters, int grid,
                                cudaStream_t s, float4 *photons) {
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  static const JitterNorm jn = jitter_norm_host();
  k_trace_lights<<<grid, kBlock, 0, s>>>(S, p, f, status, ticket, counters, jn, photons);
  return cudaGetLastError();
}

cudaError_t launch_resolve(const DevScene &S, const sc_resolve_params &p, const sc_frame &f, unsigned *status,
                           cudaStream_t s) {
  const int n = f.width * f.height;
  k_resolve<<<blocks_for(n, 128), 128, 0, s>>>(S, p, f, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || (!f.outline && !f.occlusion) || n == 0) return e;
  const int T = f.outline && p.outline_px > 0 ? p.outline_px : 1;  // the halo only the outline needs
  const float jump = p.depth_jump_rel > 0.0f ? p.depth_jump_rel : 0.05f;
  const int R = T > 1 ? T : 1;
  const size_t smem = sizeof(int) * ((size_t)(kEdgeTY + 2 * R) * (kEdgeTX + 2 * R) + 2 * (kEdgeTY + 2 * R) * kEdgeTX);
  const dim3 grid((f.width + kEdgeTX - 1) / kEdgeTX, (f.height + kEdgeTY - 1) / kEdgeTY);
  k_gt_edges<<<grid, dim3(kEdgeTX, kEdgeTY), smem, s>>>(f, T, jump);
  return cudaGetLastError();
}

cudaError_t launch_intersect(const DevScene &S, const float *rays, int64_t n, float *hits, unsigned *status,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_intersect<<<blocks_for(n, 128), 128, 0, s>>>(S, reinterpret_cast<const float4 *>(rays), n,
                                                   reinterpret_cast<float4 *>(hits), status);
  return cudaGetLastError();
}

cudaError_t launch_occluded(const DevScene &S, const float *rays, int64_t n, int32_t *occ, unsigned *status,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_occluded<<<blocks_for(n, 128), 128, 0, s>>>(S, reinterpret_cast<const float4 *>(rays), n, occ, status);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_philox<<<blocks_for(n, 256), 256, 0, s>>>(reinterpret_cast<const uint4 *>(ctr), key, n,
                                              reinterpret_cast<uint4 *>(out));
  return cudaGetLastError();
}

}  // namespace sc
