/*
 * supercaustics.h -- C ABI of the GB300 (sm_103a) spectral glass path/light tracer.
 *
 * The library renders the kind of image SuperCaustics (arXiv 2107.11008) generates:
 * transparent objects with refraction, reflection, dispersion and caustics (Abstract;
 * Sec. III), together with pixel-aligned ground truth (Sec. III-D: depth normalised by a
 * 10 m range, world/camera-space normals, object masks, caustic mask).  The paper's
 * renderer is an engine with hardware ray tracing; here every step is a hand-written CUDA
 * kernel: LBVH build over Morton codes, watertight BVH traversal, a persistent camera path
 * tracer, a light tracer that splats caustics, and the resolve pass.
 *
 * Conventions for every entry point:
 *   - Returns SC_OK (0) or a negative SC_ERR_* code; sc_last_error() gives a message.
 *     No C++ exception crosses the ABI.
 *   - Work is enqueued asynchronously on the context's stream.  Errors detected by a kernel
 *     (traversal stack overflow, watchdog) are latched in a device status word and
 *     reported by sc_sync_status(), which synchronises the stream.
 *   - "device" pointers are CUDA global-memory addresses on the context's device; "host"
 *     pointers are ordinary CPU memory.  The caller owns every buffer it passes in; the
 *     library owns scenes (BVH, triangles) and its scratch, allocated through the
 *     context's allocator callback (or cudaMallocAsync on the context stream when none is
 *     given).
 *   - All floating-point work is FP32.  Images are row-major, y = 0 at the top row.
 */
#ifndef SUPERCAUSTICS_H
#define SUPERCAUSTICS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_ABI_VERSION 4

#define SC_OK 0
#define SC_ERR_INVALID_ARG (-1)
#define SC_ERR_CUDA (-2)
#define SC_ERR_OOM (-3)
#define SC_ERR_STACK_OVERFLOW (-4)
#define SC_ERR_TIMEOUT (-5)
#define SC_ERR_QUEUE_OVERFLOW (-6)
#define SC_ERR_UNSUPPORTED (-7)

/* device status bits latched by kernels (sc_sync_status maps them to the codes above) */
#define SC_STATUS_STACK_OVERFLOW 1u
#define SC_STATUS_WATCHDOG 2u
#define SC_STATUS_QUEUE_OVERFLOW 4u
/* only in a library built with -DSC_CHECKED: an index failed its range check (the access was
 * skipped and the path abandoned); sc_last_error names the check site, value and thread */
#define SC_STATUS_BOUNDS 8u
#define SC_ERR_BOUNDS (-8)

typedef struct sc_ctx sc_ctx;
typedef struct sc_scene sc_scene;

/* Allocator callback pair.  alloc returns device memory of at least `bytes` (256-byte
 * aligned) usable on the context stream, or NULL; free releases it. */
typedef void *(*sc_alloc_fn)(size_t bytes, void *user);
typedef void (*sc_free_fn)(void *ptr, void *user);

enum { SC_MAT_DIFFUSE = 0, SC_MAT_DIELECTRIC = 1, SC_MAT_EMISSIVE = 2 };
enum { SC_LIGHT_POINT = 0, SC_LIGHT_RECT = 1, SC_LIGHT_DISK = 2 };

/* Test hooks of the estimators (0 in production). */
enum {
  SC_FLAG_FORCE_TRANSMIT = 1,   /* dielectrics refract unless totally internally reflecting */
  SC_FLAG_SPLAT_DIRECT = 2,     /* light tracer also splats paths with no specular event */
  SC_FLAG_EMITTER_AFTER_DS = 4, /* camera paths count emitters reached as E D S+ L */
  /* Sub-bin wavelength jitter (camera and light tracer): a path's wavelength is 400 + 300 u nm
   * for its bin draw u (so its bin is still floor(u B)), its index of refraction n(lambda) at that
   * wavelength and its RGB weight the CIE fit's linear sRGB there divided by the fit's mean over
   * 400-700 nm.  No effect with one bin. */
  SC_FLAG_WAVELENGTH_JITTER = 8
};

/* Surface description (Sec. III-C lists the glass and backdrop properties the paper varies).
 * DIFFUSE: Lambert albedo; if checker_scale > 0, albedo alternates with albedo2 on a
 * checkerboard of checker_scale squares per unit of the surface uv.  DIELECTRIC: glass with
 * Cauchy index n(lambda) = cauchy_a + cauchy_b / lambda_um^2; its colour is a Beer-Lambert
 * absorption coefficient per metre (RGB): a segment of length t that ends on the glass's inner
 * side multiplies the path throughput by exp(-absorption * t); roughness > 0 makes it a rough
 * dielectric (Walter, Marschner, Li, Torrance, EGSR 2007, GGX of width alpha = roughness):
 * a microfacet normal drawn with density D(m)|m.n| from the path's bounce draws, Fresnel-chosen
 * reflection or refraction about it, throughput times |i.m| G1(i) G1(o) / (|i.n| |m.n|); a
 * facet turned away or a direction leaving on the wrong side ends the path.  EMISSIVE:
 * one-sided emitter of radiance `emission` along the triangle winding normal. */
typedef struct {
  int32_t kind;
  float albedo[3];
  float albedo2[3];
  float checker_scale;
  float cauchy_a, cauchy_b;
  float emission[3];
  float absorption[3];
  float roughness;
} sc_material;

/* Light sources (Sec. III-C "lighting"; Fig. 4: softness follows the source size).
 * POINT: p = position, power = intensity (W/sr).  RECT: p = corner, u, v = edges,
 * power = radiance, emitting along u x v.  DISK: collimated beam for optics tests:
 * p = centre, u = direction, radius, power = irradiance. */
typedef struct {
  int32_t kind;
  float p[3], u[3], v[3];
  float power[3];
  float radius;
} sc_light;

/* Pinhole camera: eye, look-at point, up vector, vertical field of view in degrees. */
typedef struct {
  float eye[3], look[3], up[3];
  float vfov_deg;
  int32_t width, height;
} sc_camera;

/* Scene description.  Geometry arrays are world-space triangles:
 *   positions  n_verts*3 float, normals n_verts*3 float or NULL (a zero vertex normal makes
 *   its triangles flat), uvs n_verts*2 float or NULL, indices n_tris*3 int32 (winding gives
 *   the geometric normal), tri_object n_tris int32 object id.
 * When geometry_on_device is nonzero those five arrays are device pointers, otherwise host.
 * object_material, materials and lights are always host arrays.  Everything is copied
 * during sc_build_scene; the caller may free it afterwards. */
typedef struct {
  int32_t n_verts, n_tris;
  const float *positions;
  const float *normals;
  const float *uvs;
  const int32_t *indices;
  const int32_t *tri_object;
  int32_t n_objects;
  const int32_t *object_material;
  int32_t n_materials;
  const sc_material *materials;
  int32_t n_lights;
  const sc_light *lights;
  float env[3];
  sc_camera camera;
  int32_t geometry_on_device;
} sc_scene_desc;

/* Camera estimator parameters.  Sample s of pixel p draws Philox4x32-10 with key = seed and
 * counter (p, s, depth, tag | scene_index << 8), so ranges of sample_offset compose exactly. */
typedef struct {
  int32_t spp, sample_offset, max_depth, n_bins;
  uint64_t seed;
  int32_t scene_index, flags;
} sc_trace_params;

/* Light tracer parameters: paths path_offset .. path_offset + n_paths - 1.
 * guide: a sphere (centre xyz, radius) enclosing every dielectric triangle, or radius <= 0 for
 * none.  With a guide, point and rect lights emit only into the cone that subtends the sphere
 * from the emission point (uniform within the cone; the path's throughput carries the cone's
 * solid angle, and for a rect light the cosine to its normal, directions behind the light
 * contributing nothing).  A caustic path L S+ D E meets glass first, so its first direction lies
 * in that cone: the splat estimate keeps its expectation while no path is spent on directions
 * that cannot make a caustic.  Disk lights (collimated) ignore the guide.  A guide together with
 * SC_FLAG_SPLAT_DIRECT is rejected (direct splats start outside the cone). */
typedef struct {
  int64_t n_paths, path_offset;
  int32_t max_depth, n_bins;
  uint64_t seed;
  int32_t scene_index, flags;
  float guide[4];
} sc_light_params;

/* Resolve: divide accumulators by their totals and derive the ground-truth buffers. */
typedef struct {
  double spp_total;          /* camera samples accumulated per pixel */
  double light_paths_total;  /* light paths accumulated (0 = no caustic buffer) */
  float depth_range;         /* Sec. III-D depth range, 10 m by default */
  float tau_rel;             /* caustic mask threshold relative to direct luminance */
  int32_t outline_px;        /* Sec. III-D outline thickness T in pixels, 1..32 (0 = 1) */
  float depth_jump_rel;      /* occlusion boundaries: relative depth jump (0 = 0.05) */
} sc_resolve_params;

/* One record per camera path (debug / parity output). */
typedef struct {
  float L[3];           /* path radiance times the spectral weight of its bin */
  uint32_t first_tri;   /* first hit triangle (input order), 0xFFFFFFFF = miss */
  uint32_t signature;   /* FNV-1a over hit triangles and scattering decisions */
  uint32_t n_queries;   /* closest-hit queries traced */
  uint32_t bin;         /* wavelength bin */
  uint32_t n_specular;  /* dielectric events */
} sc_path_record;

/* One record per light path (debug / parity output). */
typedef struct {
  float C[3];           /* splatted contribution (before division by the path count) */
  int32_t pixel;        /* splat target y*W+x, -1 = none */
  float x[3];           /* receiver point (first diffuse hit after glass), NaN = none */
  uint32_t signature;
  uint32_t n_specular;
  uint32_t bin;
  uint32_t pad[2];
} sc_light_record;

/* Frame buffers, all device pointers owned by the caller, any may be NULL (not produced).
 * float4 buffers hold rgb (or xyz) in .xyz and must be 16-byte aligned (SC_ERR_INVALID_ARG
 * otherwise).  width/height must match the scene camera. */
typedef struct {
  float *accum_camera;      /* float4[W*H], radiance sums added by sc_trace_camera */
  float *accum_caustic;     /* float4[W*H], splat sums added by sc_trace_lights */
  float *rgb;               /* float4[W*H] direct + caustic + local caustic */
  float *direct;            /* float4[W*H] camera estimator / spp_total */
  float *caustic;           /* float4[W*H] splats / light_paths_total */
  int32_t *instance_id;     /* int32[W*H] object id of the pixel-centre hit, -1 = miss */
  int32_t *tri_id;          /* int32[W*H] triangle id (input order), -1 = miss */
  uint8_t *mask;            /* uint8[W*H] 1 = transparent object */
  uint8_t *caustic_mask;    /* uint8[W*H] non-local caustic (on a non-glass surface) */
  uint8_t *local_caustic_mask; /* uint8[W*H] local caustic: a glass pixel whose local-caustic
                                  luminance exceeds tau_rel * max(direct luminance, 1e-3) */
  float *depth;             /* float[W*H] Euclidean distance, +inf = miss */
  float *depth_norm;        /* float[W*H] min(depth / depth_range, 1) */
  float *normal_world;      /* float4[W*H] shading normal facing the camera, w = 1 on hit */
  float *normal_camera;     /* float4[W*H] the same in camera space (x right, y up, z to eye) */
  float *albedo;            /* float4[W*H] first-hit albedo (glass 1, miss 0) */
  /* Sec. III-D "Outlines": 1 on transparent pixels whose Chebyshev window of radius outline_px
   * holds another instance id (an inner band along the silhouettes), else 0.  Needs instance_id
   * and mask. */
  uint8_t *outline;
  /* Sec. III-D "Occlusion Boundaries", per transparent pixel against its four in-image
   * neighbours: 1 = nearer side of a depth jump |d_p - d_q| > depth_jump_rel * min(d_p, d_q) (a
   * miss always jumps), 2 = contact edge (a neighbour shows another id, no jump), 0 = neither or
   * not transparent.  Needs instance_id, mask and depth. */
  uint8_t *occlusion;
  float *accum_local_caustic; /* float4[W*H], photon-gather sums added by sc_gather_local_caustics */
  float *local_caustic;     /* float4[W*H] accum_local_caustic / spp_total (added into rgb) */
  sc_path_record *path_records;    /* [H][W][spp] of the last sc_trace_camera call, or NULL */
  sc_light_record *light_records;  /* [n_paths] of the last sc_trace_lights call, or NULL */
  int32_t width, height;
} sc_frame;

/* Read-only summary of a built scene. */
typedef struct {
  int32_t n_tris, n_nodes, n_materials, n_lights;
  int64_t bvh_bytes;   /* binary + 4-wide nodes + reordered triangles + shading attributes */
  int32_t max_depth;   /* deepest leaf of the binary BVH */
  int32_t bvh_width;   /* children per node of the camera kernel's traversal (4: nodes collapsed
                          from the binary LBVH, which the other kernels traverse) */
} sc_scene_info;

/* --- context ------------------------------------------------------------------------- */
int sc_abi_version(void);
/* sizes of the public structs in this order: material, light, camera, scene_desc,
 * trace_params, light_params, resolve_params, path_record, light_record, frame,
 * scene_info; returns the count written (<= n). */
int sc_struct_sizes(int32_t *out, int32_t n);
/* Create a context on `device` using `stream` (a cudaStream_t, NULL = legacy default). */
int sc_create(int device, void *stream, sc_alloc_fn alloc, sc_free_fn free_fn, void *user, sc_ctx **out);
int sc_destroy(sc_ctx *ctx);
int sc_set_stream(sc_ctx *ctx, void *stream);
const char *sc_last_error(const sc_ctx *ctx);
/* Synchronise the stream and report (then clear) latched device status bits. */
int sc_sync_status(sc_ctx *ctx);
/* Optional traversal work counters: a device uint64[3] that sc_trace_camera and
 * sc_trace_lights add to while set: [0] traversal queries (closest + any hit), [1] BVH
 * nodes visited (sc_trace_camera: 4-wide nodes, four child-box tests each;
 * sc_trace_lights: binary nodes, two each), [2] triangle tests.  NULL switches counting
 * off.  The caller owns the buffer and zeroes it. */
int sc_set_counters(sc_ctx *ctx, uint64_t *counters);

/* Failure-detection limits of the BVH traversals (all kernels of this context from the next
 * launch on).  A query that visits more than max_visits nodes latches SC_STATUS_WATCHDOG
 * (sc_sync_status: SC_ERR_TIMEOUT); one whose traversal stack would need more than stack_depth4
 * entries (4-wide traversal of the camera kernels, at most 96) or stack_depth2 entries (binary
 * traversal of the light tracer, resolve and queries, at most 64) latches
 * SC_STATUS_STACK_OVERFLOW (SC_ERR_STACK_OVERFLOW).  Either way the query is abandoned and reported
 * as a miss, so the frame is wrong and the status says so.  A field of 0 means its default
 * (max_visits 4,194,304; the compiled stack sizes); sc_set_limits(ctx, NULL) restores all
 * defaults.  Values above the compiled stacks are rejected (SC_ERR_INVALID_ARG).  Small limits
 * exist to test the error paths. */
typedef struct {
  int64_t max_visits;
  int32_t stack_depth4, stack_depth2;
} sc_limits;
int sc_set_limits(sc_ctx *ctx, const sc_limits *limits);
int sc_get_limits(const sc_ctx *ctx, sc_limits *limits);

/* How sc_trace_camera runs the camera estimator (sc_trace_batch always uses the persistent
 * state machine).  Both give the same path records and accumulators bit for bit.
 *   SC_CAMERA_WAVEFRONT (default): waves of whole pixels (at most 2^24 paths each, all samples of
 *     every pixel of the wave) advance one event at a time through separate kernels -- closest-hit
 *     traversal, dielectric events, diffuse events with next-event estimation, shadow rays --
 *     each over a queue of the paths at that event; path state in device memory allocated per
 *     call (about 230 bytes per path of a wave) through the context's allocator.
 *   SC_CAMERA_PERSISTENT: one persistent kernel whose lanes each run a path as a state machine,
 *     interleaving traversal chunks and shading; no workspace. */
enum { SC_CAMERA_WAVEFRONT = 0, SC_CAMERA_PERSISTENT = 1 };
int sc_set_camera_engine(sc_ctx *ctx, int32_t engine);
int sc_get_camera_engine(const sc_ctx *ctx, int32_t *engine);

/* --- scene: LBVH build (Karras 2012 hierarchy over 30-bit Morton codes) ------------------ */
int sc_build_scene(sc_ctx *ctx, const sc_scene_desc *desc, sc_scene **out);
int sc_free_scene(sc_ctx *ctx, sc_scene *scene);
int sc_scene_get_info(const sc_scene *scene, sc_scene_info *info);
/* Copy the BVH to host memory for inspection: nodes_host receives n_nodes * 64 bytes
 * (float4 c0 x/y bounds, float4 c1 x/y bounds, float4 z bounds, int4 children; a child
 * < 0 is leaf ~k), tris_host n_tris * 48 bytes (three float4 vertices in leaf order, .w
 * of the first holding the input triangle index as int bits).  Synchronises. */
int sc_scene_export_bvh(sc_ctx *ctx, const sc_scene *scene, void *nodes_host, void *tris_host);
/* Copy the 4-wide BVH the camera kernel traverses to host memory: n_nodes * 128 bytes, record j
 * collapsed from binary node j (only records reachable from record 0 through child references
 * are traversed): float4 x lo, x hi, y lo, y hi, z lo, z hi of the four children (structure of
 * arrays), int4 child references (>= 0: record of that binary node, < 0: leaf ~k, 0x7FFFFFFF:
 * empty), float4 padding.  SC_ERR_UNSUPPORTED if the scene has no 4-wide nodes.  Synchronises. */
int sc_scene_export_bvh4(sc_ctx *ctx, const sc_scene *scene, void *nodes4_host);

/* --- LBVH build without device allocation --------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory while they run (a fixed, pre-committed memory budget, or no tolerance for the
 * synchronisation that freeing device memory can cause).  It runs the same LBVH kernels as
 * sc_build_scene, but into buffers the caller owns, with its scratch in one static __device__
 * array of SC_NOALLOC_MAX_TRIS triangles' worth (about 3.3 MB, held by every GPU that loads the
 * library until the process exits).  It calls no cudaMalloc / cudaFree and no allocating
 * library routine.
 *   Inputs (device): positions n_verts*3, normals or NULL, uvs or NULL, indices n_tris*3,
 *   tri_object n_tris, object_material n_objects -- as in sc_scene_desc, all indices valid.
 *   Outputs (device, caller-owned, 16-byte aligned): nodes 16*max(n_tris-1,1) floats,
 *   tris 12*n_tris floats, shade 12*n_tris floats, shade2 4*n_tris floats, tri_obj n_tris ints,
 *   laid out exactly as in sc_scene_export_bvh (nodes, tris) and the scene's internal tables.
 * Returns SC_ERR_INVALID_ARG (with a message) if n_tris is outside [1, SC_NOALLOC_MAX_TRIS].
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device made current) and caches it; make that first call before any stream capture.
 * Every call shares the one array and it keeps the last call's contents (each build overwrites
 * what it reads), so calls that overlap on the GPU -- other streams, other host threads --
 * race: serialise them. */
#define SC_NOALLOC_MAX_TRIS 32768
int sc_build_bvh_noalloc(sc_ctx *ctx, const float *positions, const float *normals, const float *uvs,
                         const int32_t *indices, const int32_t *tri_object, const int32_t *object_material,
                         int32_t n_objects, int32_t n_tris, float *nodes, float *tris, float *shade,
                         float *shade2, int32_t *tri_obj);

/* --- queries --------------------------------------------------------------------------- */
/* Closest hit for n rays.  rays: device float[n][8] = (ox,oy,oz,tmax, dx,dy,dz,0);
 * hits: device float[n][4] = (t, tri as int bits (input order, -1 miss), b1, b2). */
int sc_intersect(sc_ctx *ctx, const sc_scene *scene, const float *rays, int64_t n, float *hits);
/* Any hit with t in (0, tmax): occluded[i] = 1/0.  Same ray layout. */
int sc_occluded(sc_ctx *ctx, const sc_scene *scene, const float *rays, int64_t n, int32_t *occluded);
/* Philox4x32-10 of n device counters (uint32[n][4]) under `key`, into device out[n][4]. */
int sc_philox4x32_10(sc_ctx *ctx, const uint32_t *counters, uint64_t key, int64_t n, uint32_t *out);

/* --- estimators ------------------------------------------------------------------------ */
/* Camera path tracer: adds spp samples per pixel into frame->accum_camera. */
int sc_trace_camera(sc_ctx *ctx, const sc_scene *scene, const sc_trace_params *params, const sc_frame *frame);
/* Light tracer: traces n_paths light paths and splats caustics into frame->accum_caustic. */
int sc_trace_lights(sc_ctx *ctx, const sc_scene *scene, const sc_light_params *params, const sc_frame *frame);
/* Resolve: rgb/direct/caustic from the accumulators, plus the pixel-centre ground truth. */
int sc_resolve(sc_ctx *ctx, const sc_scene *scene, const sc_resolve_params *params, const sc_frame *frame);

/* --- local caustics: caustics seen through glass (photon map) ----------------------------------
 * Sec. III-D separates caustics projected onto other surfaces (non-local: the splats of
 * sc_trace_lights) from caustics seen inside the transparent objects (local).  A local caustic is a
 * light path L S+ D seen along E S+: neither the splat (a straight unoccluded line to the pinhole)
 * nor the camera estimator (its next-event rays are blocked by glass) reaches it, so it is estimated
 * from a photon map.
 * sc_photon_map_create: traces the light paths of `params` (the sc_trace_lights estimator: same
 *   random numbers, guide, bins, flags) and keeps, per path reaching a diffuse surface after at least
 *   one glass event, a photon: position, shading normal on the lit side, throughput, wavelength bin.
 *   Photons are hashed into cells of 2 * radius and sorted by bucket (light-path order within a
 *   bucket).  Device memory through the context's allocator: ~70 bytes per light path kept, ~130
 *   during the build.  radius > 0 (scene units); n_paths in [1, 2^30].
 * sc_gather_local_caustics: camera paths of `params` (the camera estimator's own random numbers and
 *   decisions) follow their dielectric events to their first diffuse vertex; one reached through
 *   glass adds beta * albedo / pi * W(lambda) * B * sum(throughput of the photons of its bin within
 *   radius whose normal faces the same side) / (N_L * pi * radius^2) to frame->accum_local_caustic
 *   (B bins, N_L light paths of the map).  params->n_bins must equal the map's.  Path records, if
 *   requested, hold each sample's contribution (signature and counts of its prefix).  The estimate
 *   is the constant-kernel density estimate of photon mapping: biased by the kernel's width, which
 *   shrinks with the radius.
 * sc_photon_map_export: host copies of the photons (n_paths x 12 floats, bucket order: position +
 *   bin as int bits, normal + deposited flag, throughput + 0) and of order (n_paths uint32: the
 *   light path of each slot).  Synchronises. */
typedef struct sc_photon_map sc_photon_map;
int sc_photon_map_create(sc_ctx *ctx, const sc_scene *scene, const sc_light_params *params, float radius,
                         sc_photon_map **out);
int sc_photon_map_destroy(sc_ctx *ctx, sc_photon_map *map);
int sc_photon_map_export(sc_ctx *ctx, const sc_photon_map *map, float *photons_host, uint32_t *order_host);
int sc_gather_local_caustics(sc_ctx *ctx, const sc_scene *scene, const sc_photon_map *map,
                             const sc_trace_params *params, const sc_frame *frame);

/* --- batched camera tracing ----------------------------------------------------------------
 * A dataset generator renders many randomised scenes (Sec. III-A, Sec. IV-A: thousands of
 * images from hundreds of scenarios).  These calls trace the camera estimator of n scenes of
 * any size and resolution in ONE kernel launch: one block per chunk of 16 8x4-pixel tiles of a
 * scene, its lanes taking pixels of the chunk dynamically, so small and large scenes share the
 * GPU without a launch per scene.  scenes: n built scenes; frames: n host structs (device buffers as for
 * sc_trace_camera; accum_camera is added to, path_records optional); params as for
 * sc_trace_camera except that scene i draws its random numbers with scene index
 * params->scene_index + i.  Results equal n separate sc_trace_camera calls made with those
 * scene indices.  The scene and frame tables are copied during the call. */
int sc_trace_batch(sc_ctx *ctx, const sc_scene *const *scenes, const sc_frame *frames, int32_t n,
                   const sc_trace_params *params);
/* The same launch captured once into a CUDA graph and replayed by sc_batch_launch (the
 * scenes and frame buffers must outlive the batch; their contents may change between
 * launches).  The graph runs on the context stream of the launch call. */
typedef struct sc_batch sc_batch;
int sc_batch_create(sc_ctx *ctx, const sc_scene *const *scenes, const sc_frame *frames, int32_t n,
                    const sc_trace_params *params, sc_batch **out);
int sc_batch_launch(sc_ctx *ctx, sc_batch *batch);
int sc_batch_destroy(sc_ctx *ctx, sc_batch *batch);

/* --- measurement kernels (roofline denominators) ------------------------------------------
 * The paper reports no performance figures; these two kernels measure, on the context's device,
 * the two ceilings that bound BVH traversal besides HBM: FP32 FMA throughput and L2 read
 * bandwidth.  Both launch on the context stream and return at once; the caller times them with
 * events on that stream.
 * sc_peak_fma: SM count x 2048 threads, each running 8 independent FMA chains of `iters` steps
 *   (iters a positive multiple of 16).  *flops (host) receives the flops the launch performs
 *   (2 per FMA).  sink: a device float the kernel never writes in practice (keeps the work live).
 * sc_peak_l2_read: reads the device buffer `buf` (16-byte aligned, `bytes` a multiple of 16, sized
 *   to stay resident in L2, e.g. 32 MB) `reps` times with L1-bypassing 16-byte loads from SM count
 *   x 2048 threads; *bytes_read (host) receives bytes * reps.  Returns SC_ERR_INVALID_ARG on a bad
 *   size, alignment or null pointer. */
int sc_peak_fma(sc_ctx *ctx, int64_t iters, float *sink, int64_t *flops);
int sc_peak_l2_read(sc_ctx *ctx, const void *buf, int64_t bytes, int32_t reps, float *sink, int64_t *bytes_read);

#ifdef __cplusplus
}
#endif
#endif
