// photons.cu -- local caustics: caustics seen through glass (Sec. III-D "Local & Non-local Caustics
// Mask": the local mask covers caustics inside the transparent objects).
//
// The splatting light tracer connects a caustic receiver to the pinhole only along a straight,
// unoccluded line, so a caustic seen through glass (E S+ D S+ L) is missing from it and the
// camera estimator cannot find it either (its next-event rays are blocked by the glass).  A photon
// map estimates it:
//   1. light paths traced by the light tracer deposit a photon (position, normal on the lit side,
//      throughput, wavelength bin) at their first diffuse vertex after at least one glass event;
//   2. photons are hashed into cells of twice the gather radius (Teschner et al. 2003 spatial
//      hashing) and sorted by bucket with the LBVH's stable radix sort, so each bucket lists its
//      photons in light-path order;
//   3. camera paths follow their specular prefix exactly as the camera estimator does (same draws,
//      same decisions) to their first diffuse vertex; reached through glass, they gather the photons
//      of their own bin within the radius whose normal faces the same side:
//        L = beta * albedo / pi * W(lambda) * B * sum(photon throughput) / (N_L * pi * r^2)
//      (B bins, each photon bin has probability 1/B; N_L light paths traced).
// Each pixel sums its samples in order and adds them to accum_local_caustic: deterministic.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>

#include "device.cuh"
#include "internal.h"

struct sc_photon_map {
  void *block = nullptr;      // photons (sorted) | order | cell starts | cell ends
  float4 *photons = nullptr;  // 3 float4 per light path, in bucket order (not deposited ones last)
  uint32_t *order = nullptr;  // light path of each sorted slot
  uint32_t *start = nullptr, *end = nullptr;
  uint32_t table = 0;         // buckets (power of two)
  int64_t n_paths = 0;        // light paths traced: N_L
  int32_t n_bins = 1;
  float radius = 0.0f, inv_cell = 0.0f;
};

namespace sc {
int ctx_device(const sc_ctx *c);
cudaStream_t ctx_stream(const sc_ctx *c);
void ctx_set_error(sc_ctx *c, const std::string &msg);
void *ctx_alloc(sc_ctx *c, size_t bytes);
void ctx_free(sc_ctx *c, void *p);
unsigned *ctx_status(sc_ctx *c);
unsigned long long *ctx_counters(sc_ctx *c);
bool scene_valid(const sc_scene *s);
DevScene scene_launch_view(const sc_ctx *c, const sc_scene *s);
int trace_light_photons(sc_ctx *c, const sc_scene *s, const sc_light_params *p, float4 *photons);

namespace {

__device__ __forceinline__ uint32_t cell_hash(int cx, int cy, int cz, uint32_t table) {
  return (((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u)) & (table - 1u);
}

// key = bucket << 32 | light path (buckets of not-deposited slots: 0xFFFFFFFF, sorted last)
__global__ void k_photon_keys(const float4 *ph, int32_t n, float inv_cell, uint32_t table, unsigned long long *keys,
                              uint32_t *vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p0 = ph[3 * i], p1 = ph[3 * i + 1];
  uint32_t b = 0xFFFFFFFFu;
  if (p1.w != 0.0f)
    b = cell_hash((int)floorf(p0.x * inv_cell), (int)floorf(p0.y * inv_cell), (int)floorf(p0.z * inv_cell), table);
  keys[i] = ((unsigned long long)b << 32) | (unsigned long long)(uint32_t)i;
  vals[i] = (uint32_t)i;
}

// bucket ranges of the sorted keys, and the photons copied into bucket order
__global__ void k_photon_ranges(const unsigned long long *keys, const uint32_t *vals, const float4 *ph_in, int32_t n,
                                uint32_t table, uint32_t *start, uint32_t *end, float4 *ph_out, uint32_t *order) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t b = (uint32_t)(keys[j] >> 32);
  const uint32_t i = vals[j];
  ph_out[3 * j] = ph_in[3 * i];
  ph_out[3 * j + 1] = ph_in[3 * i + 1];
  ph_out[3 * j + 2] = ph_in[3 * i + 2];
  order[j] = i;
  if (b >= table) return;
  if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != b) start[b] = (uint32_t)j;
  if (j == n - 1 || (uint32_t)(keys[j + 1] >> 32) != b) end[b] = (uint32_t)j + 1u;
}

struct MapView {
  const float4 *ph;
  const uint32_t *start, *end;
  uint32_t table;
  float r, inv_cell, norm;  // norm = B / (N_L pi r^2)
};

// Sum of the throughputs of the photons of bin `bin` within r of x whose normal faces n's side.
__device__ __forceinline__ float3 gather_photons(const MapView &M, float3 x, float3 n, int bin) {
  const float r2 = M.r * M.r;
  const int lx = (int)floorf((x.x - M.r) * M.inv_cell), hx = (int)floorf((x.x + M.r) * M.inv_cell);
  const int ly = (int)floorf((x.y - M.r) * M.inv_cell), hy = (int)floorf((x.y + M.r) * M.inv_cell);
  const int lz = (int)floorf((x.z - M.r) * M.inv_cell), hz = (int)floorf((x.z + M.r) * M.inv_cell);
  uint32_t seen[27];
  int ns = 0;
  float3 sum = f3(0.f, 0.f, 0.f);
  for (int cz = lz; cz <= min(hz, lz + 2); ++cz)
    for (int cy = ly; cy <= min(hy, ly + 2); ++cy)
      for (int cx = lx; cx <= min(hx, lx + 2); ++cx) {
        const uint32_t b = cell_hash(cx, cy, cz, M.table);
        bool dup = false;
        for (int k = 0; k < ns; ++k) dup |= seen[k] == b;
        if (dup) continue;  // two cells in one bucket: its photons are visited once
        seen[ns++] = b;
        const uint32_t e = M.end[b];
        for (uint32_t j = M.start[b]; j < e; ++j) {
          const float4 p0 = M.ph[3 * j];
          if (__float_as_int(p0.w) != bin) continue;
          const float3 dx = f3(p0.x, p0.y, p0.z) - x;
          if (!(dot(dx, dx) < r2)) continue;
          const float4 p1 = M.ph[3 * j + 1];
          if (!(p1.x * n.x + p1.y * n.y + p1.z * n.z > 0.0f)) continue;
          const float4 p2 = M.ph[3 * j + 2];
          sum = sum + f3(p2.x, p2.y, p2.z);
        }
      }
  return sum;
}

// One thread per pixel; its samples in order.  The prefix is the camera estimator's.
__global__ void __launch_bounds__(128) k_gather_local(DevScene S, sc_trace_params P, sc_frame F, MapView M,
                                                      unsigned *status, JitterNorm jn) {
  __shared__ float3 wts[kMaxBins];
  spectral_table(wts, P.n_bins);  // ends with __syncthreads
  const Cam cam = make_cam(S.cam);
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= cam.W * cam.H) return;
  const int px = pix % cam.W, py = pix / cam.W;
  const int nb = P.n_bins > 0 ? P.n_bins : 1;
  const bool jitter = (P.flags & SC_FLAG_WAVELENGTH_JITTER) && nb > 1;
  TravCount tc;
  float3 acc = f3(0.f, 0.f, 0.f);
  for (int s = 0; s < P.spp; ++s) {
    const uint32_t smp = (uint32_t)(P.sample_offset + s);
    const uint4 x0 = draw(P.seed, (uint32_t)pix, smp, 0u, 0u, (uint32_t)P.scene_index);
    const float ul = u01(x0.z);
    const int bin = bin_of(ul, nb);
    float3 d = cam_dir(cam, (px + u01(x0.x)) / cam.W, (py + u01(x0.y)) / cam.H);
    float3 o = cam.eye, beta = f3(1.f, 1.f, 1.f), L = f3(0.f, 0.f, 0.f);
    uint32_t sig = 2166136261u, first = kMiss, nq = 0, nspec = 0;
    for (int k = 0; k < P.max_depth; ++k) {
      const Hit h = closest_hit(S, o, d, 3.0e38f, status, tc);
      ++nq;
      sig = fnv(sig, h.id);
      if (k == 0) first = h.id;
      if (h.prim < 0) break;
      if (!SC_IN_RANGE(status, 5, h.prim, S.n_tris) || !SC_IN_RANGE(status, 6, h.id, S.n_tris)) break;
      const Surf f = interact(S, d, h);
      const sc_material m = S.mats[SC_IN_RANGE(status, 7, f.mat, S.n_mats) ? f.mat : 0];
      if (m.kind == SC_MAT_DIELECTRIC && f.cosg > 0.0f && absorbs(m)) beta = beta * absorb_over(m, h.t);
      if (m.kind == SC_MAT_EMISSIVE) break;
      if (m.kind == SC_MAT_DIELECTRIC) {
        const uint4 xs = draw(P.seed, (uint32_t)pix, smp, (uint32_t)(k + 1), 1u, (uint32_t)P.scene_index);
        bool refl, fix, alive = true;
        const float nl = cauchy_at(m.cauchy_a, m.cauchy_b, path_lambda(ul, nb, jitter), P.n_bins);
        float3 nd;
        if (m.roughness > 0.0f) {
          float wgt;
          alive = rough_dielectric(f, d, nl, m.roughness, u01(xs.x), u01(xs.y), u01(xs.z), P.flags, nd, wgt, refl,
                                   fix);
          beta = beta * wgt;
        } else {
          nd = dielectric(f, d, nl, u01(xs.x), P.flags, refl, fix);
        }
        ++nspec;
        if (!alive) {
          sig = fnv(sig, EV_KILL);
          break;
        }
        sig = fnv(sig, refl ? EV_REFLECT : EV_REFRACT);
        if (fix) sig = fnv(sig, EV_FIXUP);
        o = offset_along(f.p, f.ng, nd);
        d = nd;
        continue;
      }
      // diffuse: the gather vertex when reached through glass
      if (nspec > 0) {
        const float3 alb = albedo_at(S, m, f);
        const float3 W = jitter ? jitter_weight(ul, jn) : wts[bin];
        const float3 w = beta * alb * W * (1.0f / kPi);
        L = w * (gather_photons(M, f.p, f.nsf, bin) * M.norm);
      }
      break;
    }
    acc = acc + L;
    if (F.path_records && SC_IN_RANGE(status, 9, (int64_t)pix * P.spp + s, (int64_t)cam.W * cam.H * P.spp)) {
      sc_path_record r;
      r.L[0] = L.x; r.L[1] = L.y; r.L[2] = L.z;
      r.first_tri = first;
      r.signature = sig;
      r.n_queries = nq;
      r.bin = (uint32_t)bin;
      r.n_specular = nspec;
      F.path_records[(int64_t)pix * P.spp + s] = r;
    }
  }
  if (F.accum_local_caustic) {
    float4 *a = reinterpret_cast<float4 *>(F.accum_local_caustic) + pix;
    float4 v = *a;
    v.x += acc.x; v.y += acc.y; v.z += acc.z;
    *a = v;
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int fail(sc_ctx *c, int code, const std::string &m) {
  if (c) ctx_set_error(c, m);
  return code;
}

}  // namespace
}  // namespace sc

extern "C" {

int sc_photon_map_create(sc_ctx *c, const sc_scene *s, const sc_light_params *p, float radius, sc_photon_map **out) {
  using namespace sc;
  if (!c || !out) return SC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!scene_valid(s) || !p) return fail(c, SC_ERR_INVALID_ARG, "sc_photon_map_create: null argument");
  if (!(radius > 0.0f) || !std::isfinite(radius))
    return fail(c, SC_ERR_INVALID_ARG, "sc_photon_map_create: the gather radius must be positive and finite");
  if (p->n_paths < 1 || p->n_paths > (int64_t(1) << 30))
    return fail(c, SC_ERR_INVALID_ARG, "sc_photon_map_create: n_paths must be in [1, 2^30]");
  const int32_t n = (int32_t)p->n_paths;
  uint32_t table = 1024;
  while (table < (uint32_t)n) table <<= 1;
  cudaStream_t st = ctx_stream(c);
  // persistent block: sorted photons | order | bucket starts | bucket ends
  const size_t pbytes = a256(48 * (size_t)n) + a256(4 * (size_t)n) + 2 * a256(4 * (size_t)table);
  // temporary block: photons in light-path order | keys x 2 | values x 2 | digit histograms
  const size_t tbytes = a256(48 * (size_t)n) + 2 * a256(8 * (size_t)n) + 2 * a256(4 * (size_t)n) +
                        a256(4 * 256 * sort_blocks(n));
  sc_photon_map *m = new (std::nothrow) sc_photon_map;
  if (!m) return SC_ERR_OOM;
  m->block = ctx_alloc(c, pbytes);
  char *tmp = static_cast<char *>(ctx_alloc(c, tbytes));
  if (!m->block || !tmp) {
    if (m->block) ctx_free(c, m->block);
    if (tmp) ctx_free(c, tmp);
    delete m;
    return fail(c, SC_ERR_OOM, "sc_photon_map_create: out of device memory");
  }
  char *pb = static_cast<char *>(m->block);
  m->photons = reinterpret_cast<float4 *>(pb);
  m->order = reinterpret_cast<uint32_t *>(pb + a256(48 * (size_t)n));
  m->start = reinterpret_cast<uint32_t *>(pb + a256(48 * (size_t)n) + a256(4 * (size_t)n));
  m->end = m->start + a256(4 * (size_t)table) / 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *r = tmp + off;
    off += a256(bytes);
    return r;
  };
  float4 *raw = reinterpret_cast<float4 *>(take(48 * (size_t)n));
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(take(8 * (size_t)n));
  unsigned long long *keys_alt = reinterpret_cast<unsigned long long *>(take(8 * (size_t)n));
  uint32_t *vals = reinterpret_cast<uint32_t *>(take(4 * (size_t)n));
  uint32_t *vals_alt = reinterpret_cast<uint32_t *>(take(4 * (size_t)n));
  uint32_t *hist = reinterpret_cast<uint32_t *>(take(4 * 256 * sort_blocks(n)));
  m->table = table;
  m->n_paths = p->n_paths;
  m->n_bins = p->n_bins;
  m->radius = radius;
  m->inv_cell = 1.0f / (2.0f * radius);
  int rc = trace_light_photons(c, s, p, raw);
  cudaError_t e = cudaSuccess;
  if (rc == SC_OK) {
    const int G = (n + 255) / 256;
    k_photon_keys<<<G, 256, 0, st>>>(raw, n, m->inv_cell, table, keys, vals);
    e = cudaGetLastError();
    // bytes 4..7 of the key: the bucket (the light-path index in bytes 0..3 is already in order)
    if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, keys_alt, vals_alt, hist, n, 4, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->start, 0, 2 * a256(4 * (size_t)table), st);
    if (e == cudaSuccess) {
      k_photon_ranges<<<G, 256, 0, st>>>(keys, vals, raw, n, table, m->start, m->end, m->photons, m->order);
      e = cudaGetLastError();
    }
  }
  ctx_free(c, tmp);
  if (rc != SC_OK || e != cudaSuccess) {
    ctx_free(c, m->block);
    delete m;
    if (rc != SC_OK) return rc;
    return fail(c, SC_ERR_CUDA, std::string("sc_photon_map_create: ") + cudaGetErrorString(e));
  }
  *out = m;
  return SC_OK;
}

int sc_photon_map_destroy(sc_ctx *c, sc_photon_map *m) {
  if (!c || !m) return SC_ERR_INVALID_ARG;
  sc::ctx_free(c, m->block);
  delete m;
  return SC_OK;
}

int sc_photon_map_export(sc_ctx *c, const sc_photon_map *m, float *photons_host, uint32_t *order_host) {
  if (!c || !m || !photons_host || !order_host) return SC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(sc::ctx_stream(c));
  if (e == cudaSuccess) e = cudaMemcpy(photons_host, m->photons, 48 * (size_t)m->n_paths, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(order_host, m->order, 4 * (size_t)m->n_paths, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return sc::fail(c, SC_ERR_CUDA, std::string("sc_photon_map_export: ") + cudaGetErrorString(e));
  return SC_OK;
}

int sc_gather_local_caustics(sc_ctx *c, const sc_scene *s, const sc_photon_map *m, const sc_trace_params *p,
                             const sc_frame *f) {
  using namespace sc;
  if (!c || !scene_valid(s) || !m || !p || !f) return SC_ERR_INVALID_ARG;
  const DevScene S = scene_launch_view(c, s);
  if (f->width != S.cam.width || f->height != S.cam.height)
    return fail(c, SC_ERR_INVALID_ARG, "sc_gather_local_caustics: frame size differs from the scene camera");
  if (!frame_vectors_aligned(f))
    return fail(c, SC_ERR_INVALID_ARG, "sc_gather_local_caustics: float4 frame buffers must be 16-byte aligned");
  if (p->spp < 0 || p->sample_offset < 0 || p->max_depth < 0 || p->n_bins < 1 || p->n_bins > kMaxBins)
    return fail(c, SC_ERR_INVALID_ARG, "sc_gather_local_caustics: bad parameters (n_bins must be 1..64)");
  if (p->n_bins != m->n_bins)
    return fail(c, SC_ERR_INVALID_ARG, "sc_gather_local_caustics: the photon map was traced with other bins");
  if (p->spp == 0) return SC_OK;
  static const JitterNorm jn = jitter_norm_host();
  MapView v;
  v.ph = m->photons;
  v.start = m->start;
  v.end = m->end;
  v.table = m->table;
  v.r = m->radius;
  v.inv_cell = m->inv_cell;
  v.norm = (float)((double)std::max(m->n_bins, 1) / ((double)m->n_paths * 3.14159265358979323846 *
                                                      (double)m->radius * (double)m->radius));
  const int npx = f->width * f->height;
  k_gather_local<<<(npx + 127) / 128, 128, 0, ctx_stream(c)>>>(S, *p, *f, v, ctx_status(c), jn);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(c, SC_ERR_CUDA, std::string("sc_gather_local_caustics: ") + cudaGetErrorString(e));
  return SC_OK;
}

}  // extern "C"
