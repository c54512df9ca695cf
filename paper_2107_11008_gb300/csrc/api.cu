// api.cu -- the C ABI (include/supercaustics.h): contexts, scenes, launches, status.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "device.cuh"
#include "internal.h"

struct sc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  sc_alloc_fn alloc = nullptr;
  sc_free_fn free_fn = nullptr;
  void *user = nullptr;
  std::string err;
  unsigned *d_words = nullptr;  // [0] status, [1] camera ticket, [2..3] light ticket (64-bit)
  int num_sms = 0;
  int cam_blocks_per_sm = 0, light_blocks_per_sm = 0;
  unsigned long long *counters = nullptr;  // optional traversal work counters (device)
  // failure-detection limits of the traversals (sc_set_limits)
  int32_t max_visits = sc::kMaxVisits, stack4 = sc::kStack, stack2 = sc::kStack2;
  int32_t camera_engine = SC_CAMERA_WAVEFRONT;  // sc_set_camera_engine
};

struct sc_scene {
  sc::DevScene dev{};
  void *persist = nullptr;  // one allocation: nodes | nodes4 | tris | shade | shade2 | tri_obj | mats | lights | depth
  size_t persist_bytes = 0;
  int32_t *d_depth = nullptr;
  int n_tris = 0, n_nodes = 0;
};

namespace {

int fail(sc_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(sc_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, SC_ERR_OOM, std::string(where) + ": out of device memory");
  return fail(c, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void *dalloc(sc_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->alloc) return c->alloc(bytes, c->user);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dfree(sc_ctx *c, void *p) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, c->user);
  else cudaFreeAsync(p, c->stream);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// carve consecutive 256-byte-aligned sub-buffers out of one allocation
struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t bytes) {
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += align256(bytes);
    return p;
  }
};

bool valid_scene(const sc_scene *s) { return s && s->dev.nodes; }

// the scene's device record with the context's traversal limits, as every launch passes it
sc::DevScene launch_scene(const sc_ctx *c, const sc_scene *s) {
  sc::DevScene d = s->dev;
  d.max_visits = c->max_visits;
  d.stack4 = c->stack4;
  d.stack2 = c->stack2;
  return d;
}

}  // namespace

namespace sc {
// context accessors for the other translation units
int ctx_device(const sc_ctx *c) { return c->device; }
cudaStream_t ctx_stream(const sc_ctx *c) { return c->stream; }
void ctx_set_error(sc_ctx *c, const std::string &msg) { c->err = msg; }
void *ctx_alloc(sc_ctx *c, size_t bytes) { return dalloc(c, bytes); }
void ctx_free(sc_ctx *c, void *p) { dfree(c, p); }
unsigned *ctx_status(sc_ctx *c) { return c->d_words; }
unsigned long long *ctx_counters(sc_ctx *c) { return c->counters; }
int ctx_num_sms(const sc_ctx *c) { return c->num_sms; }
bool scene_valid(const sc_scene *s) { return valid_scene(s); }
DevScene scene_launch_view(const sc_ctx *c, const sc_scene *s) { return launch_scene(c, s); }
// the light tracer for the photon map: no frame outputs, photons written to `photons`
int trace_light_photons(sc_ctx *c, const sc_scene *s, const sc_light_params *p, float4 *photons);
}  // namespace sc

namespace sc {
// float4 buffers are read and written (and splatted into) as 16-byte vectors
bool frame_vectors_aligned(const sc_frame *f) {
  const float *vec[] = {f->accum_camera, f->accum_caustic, f->rgb, f->direct, f->caustic, f->normal_world,
                        f->normal_camera, f->albedo, f->accum_local_caustic, f->local_caustic};
  for (const float *v : vec)
    if (reinterpret_cast<uintptr_t>(v) % 16 != 0) return false;
  return true;
}
}  // namespace sc

extern "C" {

int sc_abi_version(void) { return SC_ABI_VERSION; }

int sc_struct_sizes(int32_t *out, int32_t n) {
  const int32_t sizes[] = {(int32_t)sizeof(sc_material),    (int32_t)sizeof(sc_light),
                           (int32_t)sizeof(sc_camera),      (int32_t)sizeof(sc_scene_desc),
                           (int32_t)sizeof(sc_trace_params), (int32_t)sizeof(sc_light_params),
                           (int32_t)sizeof(sc_resolve_params), (int32_t)sizeof(sc_path_record),
                           (int32_t)sizeof(sc_light_record), (int32_t)sizeof(sc_frame),
                           (int32_t)sizeof(sc_scene_info)};
  const int32_t m = (int32_t)(sizeof(sizes) / sizeof(sizes[0]));
  int32_t k = 0;
  for (; k < m && k < n; ++k) out[k] = sizes[k];
  return k;
}

int sc_create(int device, void *stream, sc_alloc_fn alloc, sc_free_fn free_fn, void *user, sc_ctx **out) {
  if (!out) return SC_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return SC_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return SC_ERR_CUDA;
  }
  sc_ctx *c = new (std::nothrow) sc_ctx;
  if (!c) return SC_ERR_OOM;
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return SC_ERR_CUDA;
  }
  c->d_words = static_cast<unsigned *>(dalloc(c, 256));
  if (!c->d_words) {
    delete c;
    return SC_ERR_OOM;
  }
  if (cudaMemsetAsync(c->d_words, 0, 256, c->stream) != cudaSuccess) {
    dfree(c, c->d_words);
    delete c;
    return SC_ERR_CUDA;
  }
  *out = c;
  return SC_OK;
}

int sc_destroy(sc_ctx *c) {
  if (!c) return SC_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  dfree(c, c->d_words);
  cudaStreamSynchronize(c->stream);
  delete c;
  return SC_OK;
}

int sc_set_stream(sc_ctx *c, void *stream) {
  if (!c) return SC_ERR_INVALID_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return SC_OK;
}

int sc_set_counters(sc_ctx *c, uint64_t *counters) {
  if (!c) return SC_ERR_INVALID_ARG;
  c->counters = reinterpret_cast<unsigned long long *>(counters);
  return SC_OK;
}

const char *sc_last_error(const sc_ctx *c) { return c ? c->err.c_str() : "null context"; }

int sc_sync_status(sc_ctx *c) {
  if (!c) return SC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "sc_sync_status");
  unsigned w[16] = {0};
  e = cudaMemcpy(w, c->d_words, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "sc_sync_status");
  const unsigned st = w[0];
  if (st) {
    cudaMemsetAsync(c->d_words, 0, sizeof(unsigned), c->stream);
    cudaMemsetAsync(c->d_words + 8, 0, 3 * sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    if (st & SC_STATUS_BOUNDS)
      return fail(c, SC_ERR_BOUNDS, "range check failed at site " + std::to_string(w[8]) + ": value " +
                                        std::to_string((int)w[9]) + ", thread " + std::to_string(w[10]));
    if (st & SC_STATUS_STACK_OVERFLOW) return fail(c, SC_ERR_STACK_OVERFLOW, "traversal stack overflow");
    if (st & SC_STATUS_WATCHDOG)
      return fail(c, SC_ERR_TIMEOUT, "watchdog: a traversal exceeded its visit budget or a tensor-core wait gave up");
    if (st & SC_STATUS_QUEUE_OVERFLOW) return fail(c, SC_ERR_QUEUE_OVERFLOW, "work queue overflow");
  }
  return SC_OK;
}

int sc_set_limits(sc_ctx *c, const sc_limits *l) {
  if (!c) return SC_ERR_INVALID_ARG;
  if (!l) {
    c->max_visits = sc::kMaxVisits;
    c->stack4 = sc::kStack;
    c->stack2 = sc::kStack2;
    return SC_OK;
  }
  if (l->max_visits < 0 || l->stack_depth4 < 0 || l->stack_depth4 > sc::kStack || l->stack_depth2 < 0 ||
      l->stack_depth2 > sc::kStack2)
    return fail(c, SC_ERR_INVALID_ARG, "sc_set_limits: max_visits >= 0, stack_depth4 in [0, " +
                                           std::to_string(sc::kStack) + "], stack_depth2 in [0, " +
                                           std::to_string(sc::kStack2) + "]");
  c->max_visits = l->max_visits == 0 ? sc::kMaxVisits : (int32_t)std::min<int64_t>(l->max_visits, INT32_MAX);
  c->stack4 = l->stack_depth4 == 0 ? sc::kStack : l->stack_depth4;
  c->stack2 = l->stack_depth2 == 0 ? sc::kStack2 : l->stack_depth2;
  return SC_OK;
}

int sc_set_camera_engine(sc_ctx *c, int32_t engine) {
  if (!c) return SC_ERR_INVALID_ARG;
  if (engine != SC_CAMERA_WAVEFRONT && engine != SC_CAMERA_PERSISTENT)
    return fail(c, SC_ERR_INVALID_ARG, "sc_set_camera_engine: unknown engine");
  c->camera_engine = engine;
  return SC_OK;
}

int sc_get_camera_engine(const sc_ctx *c, int32_t *engine) {
  if (!c || !engine) return SC_ERR_INVALID_ARG;
  *engine = c->camera_engine;
  return SC_OK;
}

int sc_get_limits(const sc_ctx *c, sc_limits *l) {
  if (!c || !l) return SC_ERR_INVALID_ARG;
  l->max_visits = c->max_visits;
  l->stack_depth4 = c->stack4;
  l->stack_depth2 = c->stack2;
  return SC_OK;
}

int sc_build_scene(sc_ctx *c, const sc_scene_desc *d, sc_scene **out) {
  if (!c || !d || !out) return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: null argument");
  *out = nullptr;
  const int n = d->n_tris;
  if (n < 0 || d->n_verts < 0 || (n > 0 && (!d->positions || !d->indices || !d->tri_object)))
    return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: bad geometry arrays");
  if (n > (1 << 28)) return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: too many triangles");
  if (d->n_materials <= 0 || !d->materials || d->n_objects < 0 || (d->n_objects > 0 && !d->object_material))
    return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: bad materials");
  if (d->n_lights < 0 || (d->n_lights > 0 && !d->lights))
    return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: bad lights");
  if (d->camera.width <= 0 || d->camera.height <= 0 || !(d->camera.vfov_deg > 0.0f && d->camera.vfov_deg < 180.0f))
    return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: bad camera");
  for (int m = 0; m < d->n_materials; ++m)
    if (d->materials[m].kind < SC_MAT_DIFFUSE || d->materials[m].kind > SC_MAT_EMISSIVE)
      return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: unknown material kind");
  for (int o = 0; o < d->n_objects; ++o)
    if (d->object_material[o] < 0 || d->object_material[o] >= d->n_materials)
      return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: object material out of range");
  for (int l = 0; l < d->n_lights; ++l)
    if (d->lights[l].kind < SC_LIGHT_POINT || d->lights[l].kind > SC_LIGHT_DISK)
      return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: unknown light kind");
  if (!d->geometry_on_device) {
    for (int64_t i = 0; i < 3 * (int64_t)n; ++i)
      if (d->indices[i] < 0 || d->indices[i] >= d->n_verts)
        return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: vertex index out of range");
    for (int i = 0; i < n; ++i)
      if (d->tri_object[i] < 0 || d->tri_object[i] >= d->n_objects)
        return fail(c, SC_ERR_INVALID_ARG, "sc_build_scene: triangle object out of range");
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "sc_build_scene");

  sc_scene *s = new (std::nothrow) sc_scene;
  if (!s) return fail(c, SC_ERR_OOM, "sc_build_scene: host allocation");
  const int nn = n > 1 ? n - 1 : 1;
  const int nt = n > 0 ? n : 1;
  // persistent block
  Carver P{nullptr};
  P.take<float4>(sizeof(float4) * 4 * nn);
  P.take<float4>(sizeof(float4) * 8 * nn);
  P.take<float4>(sizeof(float4) * 3 * nt);
  P.take<float4>(sizeof(float4) * 3 * nt);
  P.take<float4>(sizeof(float4) * nt);
  P.take<int32_t>(sizeof(int32_t) * nt);
  P.take<sc_material>(sizeof(sc_material) * d->n_materials);
  P.take<sc_light>(sizeof(sc_light) * (d->n_lights > 0 ? d->n_lights : 1));
  P.take<int32_t>(sizeof(int32_t));
  s->persist_bytes = P.off;
  s->persist = dalloc(c, P.off);
  if (!s->persist) {
    delete s;
    return fail(c, SC_ERR_OOM, "sc_build_scene: scene allocation");
  }
  Carver Q{static_cast<char *>(s->persist)};
  sc::BuildBuffers b{};
  b.nodes = Q.take<float4>(sizeof(float4) * 4 * nn);
  b.nodes4 = Q.take<float4>(sizeof(float4) * 8 * nn);
  b.tris = Q.take<float4>(sizeof(float4) * 3 * nt);
  b.shade = Q.take<float4>(sizeof(float4) * 3 * nt);
  b.shade2 = Q.take<float4>(sizeof(float4) * nt);
  b.tri_obj = Q.take<int32_t>(sizeof(int32_t) * nt);
  sc_material *mats = Q.take<sc_material>(sizeof(sc_material) * d->n_materials);
  sc_light *lights = Q.take<sc_light>(sizeof(sc_light) * (d->n_lights > 0 ? d->n_lights : 1));
  s->d_depth = Q.take<int32_t>(sizeof(int32_t));
  b.depth = s->d_depth;

  // scratch block (inputs when on the host, plus the sort and hierarchy work arrays)
  const size_t nb = sc::sort_blocks(nt);
  const bool host_geo = !d->geometry_on_device;
  const int nv = d->n_verts > 0 ? d->n_verts : 1;
  Carver T{nullptr};
  if (host_geo) {
    T.take<float>(sizeof(float) * 3 * nv);
    T.take<float>(sizeof(float) * 3 * nv);
    T.take<float>(sizeof(float) * 2 * nv);
    T.take<int32_t>(sizeof(int32_t) * 3 * nt);
    T.take<int32_t>(sizeof(int32_t) * nt);
  }
  T.take<int32_t>(sizeof(int32_t) * (d->n_objects > 0 ? d->n_objects : 1));
  T.take<float4>(sizeof(float4) * 3 * nt);
  T.take<float4>(sizeof(float4) * nt);
  T.take<uint32_t>(sizeof(uint32_t) * 8);
  for (int k = 0; k < 4; ++k) T.take<unsigned long long>(sizeof(unsigned long long) * nt);
  T.take<uint32_t>(sizeof(uint32_t) * 256 * nb);
  T.take<int32_t>(sizeof(int32_t) * 2 * nt);
  T.take<int32_t>(sizeof(int32_t) * nt);
  void *scratch = dalloc(c, T.off);
  if (!scratch) {
    dfree(c, s->persist);
    delete s;
    return fail(c, SC_ERR_OOM, "sc_build_scene: scratch allocation");
  }
  Carver U{static_cast<char *>(scratch)};
  const float *pos = d->positions, *nrm = d->normals, *uv = d->uvs;
  const int32_t *idx = d->indices, *tobj = d->tri_object;
  cudaStream_t st = c->stream;
  if (host_geo) {
    float *dp = U.take<float>(sizeof(float) * 3 * nv);
    float *dn = U.take<float>(sizeof(float) * 3 * nv);
    float *du = U.take<float>(sizeof(float) * 2 * nv);
    int32_t *di = U.take<int32_t>(sizeof(int32_t) * 3 * nt);
    int32_t *dt = U.take<int32_t>(sizeof(int32_t) * nt);
    if (n > 0) {
      e = cudaMemcpyAsync(dp, pos, sizeof(float) * 3 * d->n_verts, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && nrm) e = cudaMemcpyAsync(dn, nrm, sizeof(float) * 3 * d->n_verts, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && uv) e = cudaMemcpyAsync(du, uv, sizeof(float) * 2 * d->n_verts, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(di, idx, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tobj, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    }
    pos = dp;
    nrm = nrm ? dn : nullptr;
    uv = uv ? du : nullptr;
    idx = di;
    tobj = dt;
  }
  int32_t *dobj = U.take<int32_t>(sizeof(int32_t) * (d->n_objects > 0 ? d->n_objects : 1));
  if (e == cudaSuccess && d->n_objects > 0)
    e = cudaMemcpyAsync(dobj, d->object_material, sizeof(int32_t) * d->n_objects, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mats, d->materials, sizeof(sc_material) * d->n_materials, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && d->n_lights > 0)
    e = cudaMemcpyAsync(lights, d->lights, sizeof(sc_light) * d->n_lights, cudaMemcpyHostToDevice, st);
  b.positions = pos;
  b.normals = nrm;
  b.uvs = uv;
  b.indices = idx;
  b.tri_object = tobj;
  b.object_material = dobj;
  b.n_tris = n;
  b.n_objects = d->n_objects;
  b.tris_in = U.take<float4>(sizeof(float4) * 3 * nt);
  b.centroids = U.take<float4>(sizeof(float4) * nt);
  b.bounds = U.take<uint32_t>(sizeof(uint32_t) * 8);
  b.keys = U.take<unsigned long long>(sizeof(unsigned long long) * nt);
  b.keys_alt = U.take<unsigned long long>(sizeof(unsigned long long) * nt);
  b.vals = U.take<uint32_t>(sizeof(uint32_t) * nt);
  b.vals_alt = U.take<uint32_t>(sizeof(uint32_t) * nt);
  b.hist = U.take<uint32_t>(sizeof(uint32_t) * 256 * nb);
  b.parents = U.take<int32_t>(sizeof(int32_t) * 2 * nt);
  b.flags = U.take<int32_t>(sizeof(int32_t) * nt);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_depth, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = sc::launch_build(b, st);
  dfree(c, scratch);
  if (e != cudaSuccess) {
    dfree(c, s->persist);
    delete s;
    return cuda_fail(c, e, "sc_build_scene");
  }
  s->n_tris = n;
  s->n_nodes = nn;
  s->dev.nodes = b.nodes;
  s->dev.nodes4 = b.nodes4;
  s->dev.tris = b.tris;
  s->dev.shade = b.shade;
  s->dev.shade2 = b.shade2;
  s->dev.tri_obj = b.tri_obj;
  s->dev.mats = mats;
  s->dev.lights = lights;
  s->dev.n_tris = n;
  s->dev.n_nodes = nn;
  s->dev.n_mats = d->n_materials;
  s->dev.n_lights = d->n_lights;
  for (int k = 0; k < 3; ++k) s->dev.env[k] = d->env[k];
  s->dev.cam = d->camera;
  *out = s;
  return SC_OK;
}

int sc_free_scene(sc_ctx *c, sc_scene *s) {
  if (!c || !s) return fail(c, SC_ERR_INVALID_ARG, "sc_free_scene: null argument");
  dfree(c, s->persist);
  delete s;
  return SC_OK;
}

int sc_scene_get_info(const sc_scene *s, sc_scene_info *info) {
  if (!valid_scene(s) || !info) return SC_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n_tris = s->n_tris;
  info->n_nodes = s->n_nodes;
  info->n_materials = s->dev.n_mats;
  info->n_lights = s->dev.n_lights;
  info->bvh_bytes = (int64_t)s->n_nodes * (64 + 128) + (int64_t)s->n_tris * (48 + 48 + 16 + 4);
  info->bvh_width = s->dev.nodes4 ? 4 : 2;
  int32_t depth = -1;
  if (cudaMemcpy(&depth, s->d_depth, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    depth = -1;
  }
  info->max_depth = depth;
  return SC_OK;
}

int sc_scene_export_bvh(sc_ctx *c, const sc_scene *s, void *nodes_host, void *tris_host) {
  if (!c || !valid_scene(s)) return fail(c, SC_ERR_INVALID_ARG, "sc_scene_export_bvh: null argument");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && nodes_host)
    e = cudaMemcpy(nodes_host, s->dev.nodes, (size_t)s->n_nodes * 64, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && tris_host && s->n_tris > 0)
    e = cudaMemcpy(tris_host, s->dev.tris, (size_t)s->n_tris * 48, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_scene_export_bvh");
}

int sc_scene_export_bvh4(sc_ctx *c, const sc_scene *s, void *nodes4_host) {
  if (!c || !valid_scene(s) || !nodes4_host) return fail(c, SC_ERR_INVALID_ARG, "sc_scene_export_bvh4: null argument");
  if (!s->dev.nodes4) return fail(c, SC_ERR_UNSUPPORTED, "sc_scene_export_bvh4: the scene has no 4-wide nodes");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(nodes4_host, s->dev.nodes4, (size_t)s->n_nodes * 128, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_scene_export_bvh4");
}

int sc_intersect(sc_ctx *c, const sc_scene *s, const float *rays, int64_t n, float *hits) {
  if (!c || !valid_scene(s) || n < 0 || (n > 0 && (!rays || !hits)))
    return fail(c, SC_ERR_INVALID_ARG, "sc_intersect: bad argument");
  cudaError_t e = sc::launch_intersect(launch_scene(c, s), rays, n, hits, c->d_words, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_intersect");
}

int sc_occluded(sc_ctx *c, const sc_scene *s, const float *rays, int64_t n, int32_t *occ) {
  if (!c || !valid_scene(s) || n < 0 || (n > 0 && (!rays || !occ)))
    return fail(c, SC_ERR_INVALID_ARG, "sc_occluded: bad argument");
  cudaError_t e = sc::launch_occluded(launch_scene(c, s), rays, n, occ, c->d_words, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_occluded");
}

int sc_philox4x32_10(sc_ctx *c, const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out) {
  if (!c || n < 0 || (n > 0 && (!ctr || !out))) return fail(c, SC_ERR_INVALID_ARG, "sc_philox4x32_10: bad argument");
  cudaError_t e = sc::launch_philox(ctr, key, n, out, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_philox4x32_10");
}

static int check_frame(sc_ctx *c, const sc_scene *s, const sc_frame *f, const char *who) {
  if (!c || !valid_scene(s) || !f) return fail(c, SC_ERR_INVALID_ARG, std::string(who) + ": null argument");
  if (f->width != s->dev.cam.width || f->height != s->dev.cam.height)
    return fail(c, SC_ERR_INVALID_ARG, std::string(who) + ": frame size differs from the scene camera");
  if (!sc::frame_vectors_aligned(f))
    return fail(c, SC_ERR_INVALID_ARG, std::string(who) + ": float4 frame buffers must be 16-byte aligned");
  return SC_OK;
}

static int persistent_grid(sc_ctx *c, const void *kernel, int *cache) {
  if (*cache == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess || per_sm <= 0) {
      cudaGetLastError();
      per_sm = 4;
    }
    *cache = per_sm;
  }
  return c->num_sms * *cache;
}

int sc_trace_camera(sc_ctx *c, const sc_scene *s, const sc_trace_params *p, const sc_frame *f) {
  int r = check_frame(c, s, f, "sc_trace_camera");
  if (r) return r;
  if (!p || p->spp < 0 || p->sample_offset < 0 || p->max_depth < 0 || p->n_bins < 1 || p->n_bins > sc::kMaxBins)
    return fail(c, SC_ERR_INVALID_ARG, "sc_trace_camera: bad parameters (n_bins must be 1..64)");
  if (p->spp == 0) return SC_OK;
  if (c->camera_engine == SC_CAMERA_WAVEFRONT) {
    // waves of whole pixels of up to 2^24 paths (at least one 8x4 tile with all its samples)
    const int64_t tiles = (int64_t)((f->width + 7) / 8) * ((f->height + 3) / 4);
    const int64_t one_tile = 32 * (int64_t)p->spp;
    const int64_t max_paths = std::max<int64_t>(one_tile, std::min<int64_t>(tiles * one_tile, sc::kWfMaxWavePaths));
    if (max_paths > INT32_MAX / 2) return fail(c, SC_ERR_INVALID_ARG, "sc_trace_camera: spp too large");
    void *ws = dalloc(c, sc::wavefront_workspace_bytes(max_paths));
    if (!ws) return fail(c, SC_ERR_OOM, "sc_trace_camera: no device memory for the path wavefront");
    cudaError_t e = sc::launch_trace_camera_wavefront(launch_scene(c, s), *p, *f, c->d_words, c->counters, ws,
                                                      max_paths, c->num_sms, c->stream);
    dfree(c, ws);
    return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_trace_camera");
  }
  const int grid = persistent_grid(c, sc::camera_kernel_ptr(), &c->cam_blocks_per_sm);
  cudaError_t e = sc::launch_trace_camera(launch_scene(c, s), *p, *f, c->d_words, c->d_words + 1, c->counters, grid, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_trace_camera");
}

int sc_trace_lights(sc_ctx *c, const sc_scene *s, const sc_light_params *p, const sc_frame *f) {
  int r = check_frame(c, s, f, "sc_trace_lights");
  if (r) return r;
  if (!p || p->n_paths < 0 || p->path_offset < 0 || p->max_depth < 0 || p->n_bins < 1 || p->n_bins > sc::kMaxBins)
    return fail(c, SC_ERR_INVALID_ARG, "sc_trace_lights: bad parameters (n_bins must be 1..64)");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(p->guide[k])) return fail(c, SC_ERR_INVALID_ARG, "sc_trace_lights: guide sphere not finite");
  if (p->guide[3] > 0.0f && (p->flags & SC_FLAG_SPLAT_DIRECT))
    return fail(c, SC_ERR_INVALID_ARG, "sc_trace_lights: a guide sphere cannot be combined with SC_FLAG_SPLAT_DIRECT");
  if (p->n_paths == 0) return SC_OK;
  const int grid = persistent_grid(c, sc::light_kernel_ptr(), &c->light_blocks_per_sm);
  cudaError_t e = sc::launch_trace_lights(launch_scene(c, s), *p, *f, c->d_words,
                                          reinterpret_cast<unsigned long long *>(c->d_words + 2), c->counters, grid,
                                          c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_trace_lights");
}


// ---- batched camera tracing -----------------------------------------------------------------
struct sc_batch {
  sc::BatchEntry *table = nullptr;  // device
  int n = 0;
  unsigned total = 0;         // blocks of the persistent engine
  int64_t total_slots = 0;    // pixel slots of the wavefront engine
  int engine = SC_CAMERA_WAVEFRONT;
  void *workspace = nullptr;  // wavefront path state, kept for the graph's lifetime
  int64_t max_paths = 0;
  sc_trace_params params{};
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static int batch_table(sc_ctx *c, const sc_scene *const *scenes, const sc_frame *frames, int32_t n,
                       const sc_trace_params *p, sc::BatchEntry **out, unsigned *total, int64_t *total_slots) {
  if (!c || !scenes || !frames || n < 1 || !p) return fail(c, SC_ERR_INVALID_ARG, "batch: null argument or n < 1");
  if (p->spp < 0 || p->sample_offset < 0 || p->max_depth < 0 || p->n_bins < 1 || p->n_bins > sc::kMaxBins)
    return fail(c, SC_ERR_INVALID_ARG, "batch: bad parameters (n_bins must be 1..64)");
  sc::BatchEntry *h = new (std::nothrow) sc::BatchEntry[n];
  if (!h) return fail(c, SC_ERR_OOM, "batch: host table");
  unsigned begin = 0;
  int64_t slots = 0;
  for (int i = 0; i < n; ++i) {
    const sc_scene *s = scenes[i];
    if (!valid_scene(s) || frames[i].width != s->dev.cam.width || frames[i].height != s->dev.cam.height ||
        !sc::frame_vectors_aligned(&frames[i])) {
      delete[] h;
      return fail(c, SC_ERR_INVALID_ARG, "batch: scene " + std::to_string(i) + " invalid, its frame size differs or a float4 buffer is not 16-byte aligned");
    }
    const unsigned t = sc::scene_blocks(s->dev.cam);
    if (begin > 0x7FFFFFFFu - t) {
      delete[] h;
      return fail(c, SC_ERR_INVALID_ARG, "batch: more than 2^31 - 1 blocks of work");
    }
    std::memset(&h[i], 0, sizeof(h[i]));
    h[i].S = launch_scene(c, s);
    h[i].F = frames[i];
    h[i].begin = begin;
    h[i].slot_begin = (unsigned)slots;
    begin += t;
    slots += sc::scene_tickets(s->dev.cam);
    if (slots > 0x7FFFFFFF) {
      delete[] h;
      return fail(c, SC_ERR_INVALID_ARG, "batch: more than 2^31 - 1 pixel slots");
    }
  }
  sc::BatchEntry *d = static_cast<sc::BatchEntry *>(dalloc(c, sizeof(sc::BatchEntry) * n));
  if (!d) {
    delete[] h;
    return fail(c, SC_ERR_OOM, "batch: device table");
  }
  cudaError_t e = cudaMemcpyAsync(d, h, sizeof(sc::BatchEntry) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host table is freed below
  delete[] h;
  if (e != cudaSuccess) {
    dfree(c, d);
    return cuda_fail(c, e, "batch");
  }
  *out = d;
  *total = begin;
  *total_slots = slots;
  return SC_OK;
}

// wavefront workspace of a batch: waves of up to 2^24 paths, at least one 32-slot tile of all samples
static int64_t batch_wave_paths(const sc_trace_params *p, int64_t total_slots) {
  const int64_t one_tile = 32 * (int64_t)std::max(p->spp, 1);
  return std::max<int64_t>(one_tile, std::min<int64_t>(total_slots * (int64_t)std::max(p->spp, 1), sc::kWfMaxWavePaths));
}

int sc_trace_batch(sc_ctx *c, const sc_scene *const *scenes, const sc_frame *frames, int32_t n,
                   const sc_trace_params *p) {
  sc::BatchEntry *tab = nullptr;
  unsigned total = 0;
  int64_t slots = 0;
  int r = batch_table(c, scenes, frames, n, p, &tab, &total, &slots);
  if (r) return r;
  cudaError_t e = cudaSuccess;
  if (p->spp > 0 && c->camera_engine == SC_CAMERA_WAVEFRONT) {
    const int64_t max_paths = batch_wave_paths(p, slots);
    void *ws = dalloc(c, sc::wavefront_workspace_bytes(max_paths));
    if (!ws) {
      dfree(c, tab);
      return fail(c, SC_ERR_OOM, "sc_trace_batch: no device memory for the path wavefront");
    }
    e = sc::launch_trace_batch_wavefront(tab, n, slots, *p, c->d_words, c->counters, ws, max_paths, c->num_sms,
                                         c->stream);
    dfree(c, ws);
  } else if (p->spp > 0) {
    e = sc::launch_trace_batch(tab, n, total, *p, c->d_words, c->counters, c->stream);
  }
  dfree(c, tab);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_trace_batch");
}

int sc_batch_create(sc_ctx *c, const sc_scene *const *scenes, const sc_frame *frames, int32_t n,
                    const sc_trace_params *p, sc_batch **out) {
  if (!out) return fail(c, SC_ERR_INVALID_ARG, "sc_batch_create: null output");
  *out = nullptr;
  sc_batch *b = new (std::nothrow) sc_batch;
  if (!b) return fail(c, SC_ERR_OOM, "sc_batch_create: host allocation");
  int r = batch_table(c, scenes, frames, n, p, &b->table, &b->total, &b->total_slots);
  if (r) {
    delete b;
    return r;
  }
  b->n = n;
  b->params = *p;
  b->engine = c->camera_engine;
  if (b->engine == SC_CAMERA_WAVEFRONT && p->spp > 0) {
    b->max_paths = batch_wave_paths(p, b->total_slots);
    b->workspace = dalloc(c, sc::wavefront_workspace_bytes(b->max_paths));
    cudaError_t es = b->workspace ? cudaStreamSynchronize(c->stream) : cudaErrorMemoryAllocation;
    if (es != cudaSuccess) {
      if (b->workspace) dfree(c, b->workspace);
      dfree(c, b->table);
      delete b;
      return cuda_fail(c, es, "sc_batch_create: path wavefront");
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t el = cudaSuccess;
    if (b->params.spp > 0 && b->engine == SC_CAMERA_WAVEFRONT)
      el = sc::launch_trace_batch_wavefront(b->table, n, b->total_slots, b->params, c->d_words, c->counters,
                                            b->workspace, b->max_paths, c->num_sms, b->capture);
    else if (b->params.spp > 0)
      el = sc::launch_trace_batch(b->table, n, b->total, b->params, c->d_words, c->counters, b->capture);
    e = cudaStreamEndCapture(b->capture, &b->graph);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->workspace) dfree(c, b->workspace);
    dfree(c, b->table);
    delete b;
    return cuda_fail(c, e, "sc_batch_create");
  }
  *out = b;
  return SC_OK;
}

int sc_batch_launch(sc_ctx *c, sc_batch *b) {
  if (!c || !b || !b->exec) return fail(c, SC_ERR_INVALID_ARG, "sc_batch_launch: null argument");
  cudaError_t e = cudaGraphLaunch(b->exec, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_batch_launch");
}

int sc_batch_destroy(sc_ctx *c, sc_batch *b) {
  if (!c || !b) return fail(c, SC_ERR_INVALID_ARG, "sc_batch_destroy: null argument");
  cudaStreamSynchronize(c->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->workspace) dfree(c, b->workspace);
  dfree(c, b->table);
  delete b;
  return SC_OK;
}

int sc_resolve(sc_ctx *c, const sc_scene *s, const sc_resolve_params *p, const sc_frame *f) {
  int r = check_frame(c, s, f, "sc_resolve");
  if (r) return r;
  if (!p || p->spp_total < 0 || p->light_paths_total < 0 || !(p->depth_range > 0))
    return fail(c, SC_ERR_INVALID_ARG, "sc_resolve: bad parameters");
  if (p->outline_px < 0 || p->outline_px > 32 || !(p->depth_jump_rel >= 0.0f) || !std::isfinite(p->depth_jump_rel))
    return fail(c, SC_ERR_INVALID_ARG, "sc_resolve: outline_px must be in [0, 32], depth_jump_rel finite and >= 0");
  if ((f->outline || f->occlusion) && (!f->instance_id || !f->mask))
    return fail(c, SC_ERR_INVALID_ARG, "sc_resolve: outline and occlusion buffers need instance_id and mask");
  if (f->occlusion && !f->depth)
    return fail(c, SC_ERR_INVALID_ARG, "sc_resolve: the occlusion buffer needs depth");
  cudaError_t e = sc::launch_resolve(launch_scene(c, s), *p, *f, c->d_words, c->stream);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "sc_resolve");
}

}  // extern "C"

namespace sc {
int trace_light_photons(sc_ctx *c, const sc_scene *s, const sc_light_params *p, float4 *photons) {
  if (!p || p->n_paths <= 0 || p->path_offset < 0 || p->max_depth < 0 || p->n_bins < 1 || p->n_bins > kMaxBins)
    return fail(c, SC_ERR_INVALID_ARG, "photon map: bad light parameters (n_paths >= 1, n_bins 1..64)");
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(p->guide[k])) return fail(c, SC_ERR_INVALID_ARG, "photon map: guide sphere not finite");
  if (p->guide[3] > 0.0f && (p->flags & SC_FLAG_SPLAT_DIRECT))
    return fail(c, SC_ERR_INVALID_ARG, "photon map: a guide sphere cannot be combined with SC_FLAG_SPLAT_DIRECT");
  sc_frame f{};
  f.width = s->dev.cam.width;
  f.height = s->dev.cam.height;
  const int grid = persistent_grid(c, light_kernel_ptr(), &c->light_blocks_per_sm);
  cudaError_t e = launch_trace_lights(launch_scene(c, s), *p, f, c->d_words,
                                      reinterpret_cast<unsigned long long *>(c->d_words + 2), c->counters, grid,
                                      c->stream, photons);
  return e == cudaSuccess ? SC_OK : cuda_fail(c, e, "photon map: light tracing");
}
}  // namespace sc
