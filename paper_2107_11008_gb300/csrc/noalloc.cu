// noalloc.cu -- LBVH build into caller-owned buffers with no device allocation at all.
//
// sc_build_scene gets its scratch (Morton keys, sort buffers, hierarchy links) from the
// context's allocator.  Some callers cannot allocate device memory once they are running: a
// renderer whose whole memory budget is committed at start-up, or one that must not trigger
// the device-wide synchronisation that freeing device memory can cause in the middle of a
// frame.  sc_build_bvh_noalloc serves them: its scratch is one statically sized __device__
// array that lives in every GPU that loads this library, so the call itself allocates nothing.
#include <cstring>
#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxTris = SC_NOALLOC_MAX_TRIS;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
// radix-sort blocks of the largest accepted build: sized from the sort's own tile (internal.h)
constexpr size_t kBlocksMax = sc::sort_blocks_for(kNoAllocMaxTris);
constexpr size_t kScratchBytes = al(sizeof(float4) * 3 * kNoAllocMaxTris)   // triangles in input order
                                 + al(sizeof(float4) * kNoAllocMaxTris)      // centroids
                                 + al(sizeof(uint32_t) * 8)                  // centroid bounds
                                 + 2 * al(sizeof(unsigned long long) * kNoAllocMaxTris)  // keys, ping-pong
                                 + 2 * al(sizeof(uint32_t) * kNoAllocMaxTris)  // values, ping-pong
                                 + al(sizeof(uint32_t) * 256 * kBlocksMax)   // digit histograms
                                 + al(sizeof(int32_t) * 2 * kNoAllocMaxTris)   // parent links
                                 + al(sizeof(int32_t) * kNoAllocMaxTris)     // refit counters
                                 + al(sizeof(int32_t));                      // deepest leaf

// The regions carved below, in order; the carve is checked against kScratchBytes at run time.
constexpr size_t kCarvedBytes = al(sizeof(float4) * 3 * kNoAllocMaxTris) + al(sizeof(float4) * kNoAllocMaxTris) +
                                al(sizeof(uint32_t) * 8) + al(sizeof(unsigned long long) * kNoAllocMaxTris) +
                                al(sizeof(unsigned long long) * kNoAllocMaxTris) +
                                al(sizeof(uint32_t) * kNoAllocMaxTris) + al(sizeof(uint32_t) * kNoAllocMaxTris) +
                                al(sizeof(uint32_t) * 256 * kBlocksMax) + al(sizeof(int32_t) * 2 * kNoAllocMaxTris) +
                                al(sizeof(int32_t) * kNoAllocMaxTris) + al(sizeof(int32_t));
static_assert(kCarvedBytes == kScratchBytes, "scratch carve and scratch size disagree");

// The scratch array.  In host code its name is only a stand-in for the device symbol; the real
// device address comes from cudaGetSymbolAddress (below) and is what the kernels receive.
static __device__ __align__(256) unsigned char g_build_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current), looked up once per
// device and kept for the life of the process.  This assumes the device's primary context (the
// one the CUDA runtime uses) also lives as long as the process: after cudaDeviceReset the cached
// address would be stale, so a process that resets a device must not call this entry point again.
cudaError_t scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_build_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

struct Carve {
  char *p;
  template <class T>
  T *take(size_t bytes) {
    T *r = reinterpret_cast<T *>(p);
    p += al(bytes);
    return r;
  }
};

}  // namespace

// context fields used here (defined in api.cu)
struct sc_ctx;
namespace sc {
int ctx_device(const sc_ctx *c);
cudaStream_t ctx_stream(const sc_ctx *c);
void ctx_set_error(sc_ctx *c, const std::string &msg);
}  // namespace sc

extern "C" int sc_build_bvh_noalloc(sc_ctx *ctx, const float *positions, const float *normals, const float *uvs,
                                    const int32_t *indices, const int32_t *tri_object,
                                    const int32_t *object_material, int32_t n_objects, int32_t n_tris,
                                    float *nodes, float *tris, float *shade, float *shade2, int32_t *tri_obj) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (n_tris < 1 || n_tris > kNoAllocMaxTris) {
    sc::ctx_set_error(ctx, "sc_build_bvh_noalloc: n_tris must be in [1, " + std::to_string(kNoAllocMaxTris) +
                               "] (the size of its static scratch); use sc_build_scene for larger scenes");
    return SC_ERR_INVALID_ARG;
  }
  if (!positions || !indices || !tri_object || !object_material || n_objects < 1 || !nodes || !tris || !shade ||
      !shade2 || !tri_obj) {
    sc::ctx_set_error(ctx, "sc_build_bvh_noalloc: null buffer or no objects");
    return SC_ERR_INVALID_ARG;
  }
  const int dev = sc::ctx_device(ctx);
  if (dev < 0 || dev >= kMaxDevices) {
    sc::ctx_set_error(ctx, "sc_build_bvh_noalloc: device index out of range");
    return SC_ERR_INVALID_ARG;
  }
  // The symbol lookup needs the context's device current; the caller's current device is put
  // back before returning, on every path.
  int prev_dev = -1;
  cudaError_t e = cudaGetDevice(&prev_dev);
  if (e == cudaSuccess && prev_dev != dev) e = cudaSetDevice(dev);
  void *base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    if (prev_dev >= 0 && prev_dev != dev) cudaSetDevice(prev_dev);
    sc::ctx_set_error(ctx, std::string("sc_build_bvh_noalloc: ") + cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  Carve c{static_cast<char *>(base)};
  sc::BuildBuffers b{};
  b.positions = positions;
  b.normals = normals;
  b.uvs = uvs;
  b.indices = indices;
  b.tri_object = tri_object;
  b.object_material = object_material;
  b.n_tris = n_tris;
  b.n_objects = n_objects;
  b.nodes = reinterpret_cast<float4 *>(nodes);
  b.tris = reinterpret_cast<float4 *>(tris);
  b.shade = reinterpret_cast<float4 *>(shade);
  b.shade2 = reinterpret_cast<float4 *>(shade2);
  b.tri_obj = tri_obj;
  b.tris_in = c.take<float4>(sizeof(float4) * 3 * kNoAllocMaxTris);
  b.centroids = c.take<float4>(sizeof(float4) * kNoAllocMaxTris);
  b.bounds = c.take<uint32_t>(sizeof(uint32_t) * 8);
  b.keys = c.take<unsigned long long>(sizeof(unsigned long long) * kNoAllocMaxTris);
  b.keys_alt = c.take<unsigned long long>(sizeof(unsigned long long) * kNoAllocMaxTris);
  b.vals = c.take<uint32_t>(sizeof(uint32_t) * kNoAllocMaxTris);
  b.vals_alt = c.take<uint32_t>(sizeof(uint32_t) * kNoAllocMaxTris);
  b.hist = c.take<uint32_t>(sizeof(uint32_t) * 256 * kBlocksMax);
  b.parents = c.take<int32_t>(sizeof(int32_t) * 2 * kNoAllocMaxTris);
  b.flags = c.take<int32_t>(sizeof(int32_t) * kNoAllocMaxTris);
  b.depth = c.take<int32_t>(sizeof(int32_t));
  // Whatever a previous call left in the array is overwritten before it is read: the first
  // kernel resets the centroid bounds and the depth word, the hierarchy kernel zeroes the refit
  // counters, and every other scratch word is written before use.
  if (static_cast<size_t>(c.p - static_cast<char *>(base)) != kScratchBytes) {
    if (prev_dev != dev) cudaSetDevice(prev_dev);
    sc::ctx_set_error(ctx, "sc_build_bvh_noalloc: internal scratch layout mismatch");
    return SC_ERR_INVALID_ARG;
  }
  e = sc::launch_build(b, sc::ctx_stream(ctx));
  if (prev_dev != dev) {
    const cudaError_t e2 = cudaSetDevice(prev_dev);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) {
    sc::ctx_set_error(ctx, std::string("sc_build_bvh_noalloc: ") + cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  return SC_OK;
}
