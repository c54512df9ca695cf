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

struct PathOut {
  float3 L;
  uint32_t first, sig, nq, nspec;
};

// One camera path of pixel (px, py), global sample index `sample`.
__device__ __forceinline__ PathOut camera_path(const DevScene &S, const Cam &cam, const float3 *wts,
                                               const sc_trace_params &P, int px, int py, uint32_t sample,
                                               unsigned *status, uint32_t &bin_out, TravCount &tc) {
  const uint32_t pix = (uint32_t)(py * cam.W + px);
  const uint4 x0 = draw(P.seed, pix, sample, 0u, 0u, (uint32_t)P.scene_index);
  const int bin = choose(x0.z, P.n_bins > 0 ? P.n_bins : 1);
  bin_out = (uint32_t)bin;
  float3 o = cam.eye;
  float3 d = cam_dir(cam, (px + u01(x0.x)) / cam.W, (py + u01(x0.y)) / cam.H);
  float3 beta = f3(1.f, 1.f, 1.f), L = f3(0.f, 0.f, 0.f);
  bool spec_only = true, diffuse_first = false, last_specular = false;
  int n_diffuse = 0;
  PathOut out;
  out.sig = 2166136261u;
  out.first = kMiss;
  out.nq = 0;
  out.nspec = 0;
  const float3 env = f3(S.env);
  for (int k = 0; k < P.max_depth; ++k) {
    const Hit h = closest_hit(S, o, d, 3.0e38f, status, tc);
    ++out.nq;
    out.sig = fnv(out.sig, h.id);
    if (k == 0) out.first = h.id;
    if (h.prim < 0) {
      L = L + beta * env;
      break;
    }
    const Surf f = interact(S, d, h);
    const sc_material m = S.mats[f.mat];
    if (m.kind == SC_MAT_EMISSIVE) {
      const bool count = spec_only || ((P.flags & SC_FLAG_EMITTER_AFTER_DS) && diffuse_first && n_diffuse == 1 &&
                                       last_specular);
      if (f.cosg < 0.0f && count) L = L + beta * f3(m.emission);
      break;
    }
    const uint4 xs = draw(P.seed, pix, sample, (uint32_t)(k + 1), 1u, (uint32_t)P.scene_index);
    if (m.kind == SC_MAT_DIELECTRIC) {
      bool refl, fix;
      const float nl = cauchy(m.cauchy_a, m.cauchy_b, bin, P.n_bins);
      const float3 nd = dielectric(f, d, nl, u01(xs.x), P.flags, refl, fix);
      out.sig = fnv(out.sig, refl ? EV_REFLECT : EV_REFRACT);
      if (fix) out.sig = fnv(out.sig, EV_FIXUP);
      ++out.nspec;
      last_specular = true;
      o = offset_along(f.p, f.ng, nd);
      d = nd;
      continue;
    }
    // diffuse: next-event estimation
    const float3 alb = albedo_at(S, m, f);
    bool lit = false;
    if (S.n_lights > 0) {
      const uint4 xn = draw(P.seed, pix, sample, (uint32_t)(k + 1), 2u, (uint32_t)P.scene_index);
      const int j = choose(xn.x, S.n_lights);
      const sc_light Lg = S.lights[j];
      float3 lp, le = f3(Lg.power);
      float geo = 0.0f;
      bool ok = false;
      if (Lg.kind == SC_LIGHT_POINT) {
        lp = f3(Lg.p);
        float3 w = lp - f.p;
        const float d2 = dot(w, w);
        w = w * (1.0f / sqrtf(d2));
        const float cs = dot(f.nsf, w), cg = dot(f.ngf, w);
        ok = cs > 0.0f && cg > 0.0f;
        geo = cs / d2;
      } else if (Lg.kind == SC_LIGHT_RECT) {
        const float3 eu = f3(Lg.u), ev = f3(Lg.v);
        lp = f3(Lg.p) + eu * u01(xn.y) + ev * u01(xn.z);
        const float3 c = cross(eu, ev);
        const float area = length(c);
        const float3 nlt = c * (1.0f / area);
        float3 w = lp - f.p;
        const float d2 = dot(w, w);
        w = w * (1.0f / sqrtf(d2));
        const float cs = dot(f.nsf, w), cg = dot(f.ngf, w), cl = -dot(nlt, w);
        ok = cs > 0.0f && cg > 0.0f && cl > 0.0f;
        geo = cs * cl * area / d2;
      }
      if (ok) {
        const float3 so = f.p + f.ngf * eps_of(f.p);
        const float3 wv = lp - so;
        const float dist = length(wv);
        if (!any_hit(S, so, wv * (1.0f / dist), dist * (1.0f - 1e-4f), status, tc)) {
          lit = true;
          L = L + beta * (alb * le) * (geo * (float)S.n_lights / kPi);
        }
      }
    }
    out.sig = fnv(out.sig, lit ? EV_LIT : EV_UNLIT);
    if (k == 0) diffuse_first = true;
    ++n_diffuse;
    spec_only = false;
    last_specular = false;
    if (k == P.max_depth - 1) break;
    float3 nd = cosine_dir(f.nsf, u01(xs.y), u01(xs.z));
    if (!(dot(nd, f.ngf) > 0.0f)) {
      nd = cosine_dir(f.ngf, u01(xs.y), u01(xs.z));
      out.sig = fnv(out.sig, EV_FIXUP);
    }
    beta = beta * alb;
    o = f.p + f.ngf * eps_of(f.p);
    d = nd;
  }
  out.L = L * wts[bin];
  return out;
}

// Persistent camera kernel: each warp takes 8x4 pixel tiles from a global ticket and each
// lane traces every sample of its pixel, accumulating in registers (no atomics, fixed order).
__global__ void __launch_bounds__(kBlock) k_trace_camera(DevScene S, sc_trace_params P, sc_frame F,
                                                         unsigned *status, unsigned *ticket,
                                                         unsigned long long *counters) {
  TravCount tc;
  __shared__ float3 wts[kMaxBins];
  spectral_table(wts, P.n_bins);
  const Cam cam = make_cam(S.cam);
  const int tiles_x = (cam.W + 7) / 8, tiles_y = (cam.H + 3) / 4;
  const unsigned n_tiles = (unsigned)(tiles_x * tiles_y);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(ticket, 1u);
    tile = __shfl_sync(0xFFFFFFFFu, tile, 0);
    if (tile >= n_tiles) break;
    const int px = (int)(tile % tiles_x) * 8 + (lane & 7);
    const int py = (int)(tile / tiles_x) * 4 + (lane >> 3);
    if (px >= cam.W || py >= cam.H) continue;
    float3 acc = f3(0.f, 0.f, 0.f);
    const int pix = py * cam.W + px;
    for (int s = 0; s < P.spp; ++s) {
      uint32_t bin;
      const PathOut po = camera_path(S, cam, wts, P, px, py, (uint32_t)(P.sample_offset + s), status, bin, tc);
      acc = acc + po.L;
      if (F.path_records) {
        sc_path_record r;
        r.L[0] = po.L.x; r.L[1] = po.L.y; r.L[2] = po.L.z;
        r.first_tri = po.first;
        r.signature = po.sig;
        r.n_queries = po.nq;
        r.bin = bin;
        r.n_specular = po.nspec;
        F.path_records[(int64_t)pix * P.spp + s] = r;
      }
    }
    if (F.accum_camera) {
      float4 *a = reinterpret_cast<float4 *>(F.accum_camera) + pix;
      float4 v = *a;
      v.x += acc.x; v.y += acc.y; v.z += acc.z;
      *a = v;
    }
  }
  if (counters) {
    atomicAdd(&counters[0], (unsigned long long)tc.queries);
    atomicAdd(&counters[1], (unsigned long long)tc.nodes);
    atomicAdd(&counters[2], (unsigned long long)tc.tris);
  }
}

// One light path: emission, specular chain, splat at the first diffuse vertex after glass.
__global__ void __launch_bounds__(kBlock) k_trace_lights(DevScene S, sc_light_params P, sc_frame F,
                                                         unsigned *status, unsigned long long *ticket,
                                                         unsigned long long *counters) {
  TravCount tc;
  __shared__ float3 wts[kMaxBins];
  spectral_table(wts, P.n_bins);
  const Cam cam = make_cam(S.cam);
  const float apix = (2.0f * cam.th * cam.aspect / cam.W) * (2.0f * cam.th / cam.H);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(ticket, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= (unsigned long long)P.n_paths) break;
    const unsigned long long li = base + lane;
    if (li >= (unsigned long long)P.n_paths) continue;
    const int64_t idx = P.path_offset + (int64_t)li;
    const uint32_t lo = (uint32_t)idx, hi = (uint32_t)((uint64_t)idx >> 32);
    const uint4 xe = draw(P.seed, lo, hi, 0u, 4u, (uint32_t)P.scene_index);
    const uint4 xd = draw(P.seed, lo, hi, 0u, 3u, (uint32_t)P.scene_index);
    const int bin = choose(xe.w, P.n_bins > 0 ? P.n_bins : 1);
    uint32_t sig = 2166136261u, nspec = 0;
    int pixel = -1;
    float3 C = f3(0.f, 0.f, 0.f), X = f3(__int_as_float(0x7FC00000), __int_as_float(0x7FC00000),
                                         __int_as_float(0x7FC00000));
    if (S.n_lights > 0) {
      const int j = choose(xe.x, S.n_lights);
      const sc_light Lg = S.lights[j];
      float3 o, d, beta;
      if (Lg.kind == SC_LIGHT_POINT) {
        const float z = 1.0f - 2.0f * u01(xd.x);
        float s, c;
        sincospif(2.0f * u01(xd.y), &s, &c);
        const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
        o = f3(Lg.p);
        d = normalize(f3(rr * c, rr * s, z));
        beta = f3(Lg.power) * (4.0f * kPi * S.n_lights);
      } else if (Lg.kind == SC_LIGHT_RECT) {
        const float3 eu = f3(Lg.u), ev = f3(Lg.v);
        const float3 c = cross(eu, ev);
        const float area = length(c);
        const float3 nlt = c * (1.0f / area);
        const float3 x = f3(Lg.p) + eu * u01(xe.y) + ev * u01(xe.z);
        d = cosine_dir(nlt, u01(xd.x), u01(xd.y));
        o = x + nlt * eps_of(x);
        beta = f3(Lg.power) * (kPi * area * S.n_lights);
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
      bool had_spec = false;
      for (int k = 0; k < P.max_depth; ++k) {
        const Hit h = closest_hit(S, o, d, 3.0e38f, status, tc);
        sig = fnv(sig, h.id);
        if (h.prim < 0) break;
        const Surf f = interact(S, d, h);
        const sc_material m = S.mats[f.mat];
        if (m.kind == SC_MAT_EMISSIVE) break;
        if (m.kind == SC_MAT_DIELECTRIC) {
          const uint4 xs = draw(P.seed, lo, hi, (uint32_t)(k + 1), 3u, (uint32_t)P.scene_index);
          bool refl, fix;
          const float nl = cauchy(m.cauchy_a, m.cauchy_b, bin, P.n_bins);
          const float3 nd = dielectric(f, d, nl, u01(xs.x), P.flags, refl, fix);
          sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
          if (fix) sig = fnv(sig, EV_FIXUP);
          ++nspec;
          had_spec = true;
          o = offset_along(f.p, f.ng, nd);
          d = nd;
          continue;
        }
        if (!had_spec && !(P.flags & SC_FLAG_SPLAT_DIRECT)) break;
        X = f.p;
        const float3 alb = albedo_at(S, m, f);
        float3 wc = cam.eye - f.p;
        const float dc = length(wc);
        wc = wc * (1.0f / dc);
        const float cs = dot(f.nsf, wc), cg = dot(f.ngf, wc);
        if (!(cs > 0.0f && cg > 0.0f)) { sig = fnv(sig, EV_UNLIT); break; }
        const float3 wv = wc * -1.0f;
        const float cc = dot(wv, cam.f);
        if (!(cc > 0.0f)) { sig = fnv(sig, EV_UNLIT); break; }
        const float sx = (dot(wv, cam.r) / cc / (cam.th * cam.aspect) + 1.0f) * 0.5f;
        const float sy = (1.0f - dot(wv, cam.u) / cc / cam.th) * 0.5f;
        if (!(sx >= 0.0f && sx < 1.0f && sy >= 0.0f && sy < 1.0f)) { sig = fnv(sig, EV_UNLIT); break; }
        const int ix = min((int)floorf(sx * cam.W), cam.W - 1), iy = min((int)floorf(sy * cam.H), cam.H - 1);
        const float3 so = f.p + f.ngf * eps_of(f.p);
        const float3 wsv = cam.eye - so;
        const float dist = length(wsv);
        if (any_hit(S, so, wsv * (1.0f / dist), dist * (1.0f - 1e-4f), status, tc)) {
          sig = fnv(sig, EV_UNLIT);
          break;
        }
        sig = fnv(sig, EV_LIT);
        const float g = cs / (dc * dc * apix * cc * cc * cc) / kPi;
        C = beta * g * alb * wts[bin];
        pixel = iy * cam.W + ix;
        if (F.accum_caustic) {
          float *a = F.accum_caustic + 4 * (int64_t)pixel;
          atomicAdd(a + 0, C.x);
          atomicAdd(a + 1, C.y);
          atomicAdd(a + 2, C.z);
        }
        break;
      }
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
  if (F.direct) reinterpret_cast<float4 *>(F.direct)[pix] = make_float4(D.x, D.y, D.z, 1.0f);
  if (F.caustic) reinterpret_cast<float4 *>(F.caustic)[pix] = make_float4(C.x, C.y, C.z, 1.0f);
  if (F.rgb) reinterpret_cast<float4 *>(F.rgb)[pix] = make_float4(D.x + C.x, D.y + C.y, D.z + C.z, 1.0f);
  const float3 d = cam_dir(cam, (px + 0.5f) / cam.W, (py + 0.5f) / cam.H);
  TravCount tc;
  const Hit h = closest_hit(S, cam.eye, d, 3.0e38f, status, tc);
  int inst = -1, tri = -1;
  uint8_t mask = 0, cmask = 0;
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
  }
  if (F.instance_id) F.instance_id[pix] = inst;
  if (F.tri_id) F.tri_id[pix] = tri;
  if (F.mask) F.mask[pix] = mask;
  if (F.caustic_mask) F.caustic_mask[pix] = cmask;
  if (F.local_caustic_mask) F.local_caustic_mask[pix] = 0;
  if (F.depth) F.depth[pix] = depth;
  if (F.depth_norm) F.depth_norm[pix] = dn;
  if (F.normal_world) reinterpret_cast<float4 *>(F.normal_world)[pix] = nw;
  if (F.normal_camera) reinterpret_cast<float4 *>(F.normal_camera)[pix] = nc;
  if (F.albedo) reinterpret_cast<float4 *>(F.albedo)[pix] = alb;
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

const void *camera_kernel_ptr() { return reinterpret_cast<const void *>(&k_trace_camera); }
const void *light_kernel_ptr() { return reinterpret_cast<const void *>(&k_trace_lights); }

static int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

cudaError_t launch_trace_camera(const DevScene &S, const sc_trace_params &p, const sc_frame &f, unsigned *status,
                                unsigned *ticket, unsigned long long *counters, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_trace_camera<<<grid, kBlock, 0, s>>>(S, p, f, status, ticket, counters);
  return cudaGetLastError();
}

cudaError_t launch_trace_lights(const DevScene &S, const sc_light_params &p, const sc_frame &f, unsigned *status,
                                unsigned long long *ticket, unsigned long long *counters, int grid,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_trace_lights<<<grid, kBlock, 0, s>>>(S, p, f, status, ticket, counters);
  return cudaGetLastError();
}

cudaError_t launch_resolve(const DevScene &S, const sc_resolve_params &p, const sc_frame &f, unsigned *status,
                           cudaStream_t s) {
  const int n = f.width * f.height;
  k_resolve<<<blocks_for(n, 128), 128, 0, s>>>(S, p, f, status);
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
