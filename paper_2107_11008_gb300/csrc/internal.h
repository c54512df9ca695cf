// internal.h -- launchers shared between the CUDA translation units (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "supercaustics.h"

namespace sc {

struct DevScene;
bool frame_vectors_aligned(const sc_frame *f);  // every float4 buffer 16-byte aligned (or NULL)
struct BatchEntry;

// ---- LBVH build (build.cu) ----------------------------------------------------------------
// Radix sort geometry: each sort block ranks kSortThreads * kSortItems keys, and the digit
// histograms hold 256 words per block (sort_blocks(n) blocks for n keys).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr size_t sort_blocks_for(int64_t n) { return (size_t)((n + kSortTile - 1) / kSortTile); }
struct BuildBuffers {
  // inputs (device)
  const float *positions, *normals, *uvs;
  const int32_t *indices, *tri_object, *object_material;
  int32_t n_tris, n_objects;
  // outputs (device, owned by the scene)
  float4 *nodes;   // 4 * max(n_tris - 1, 1)
  float4 *nodes4;  // 8 * max(n_tris - 1, 1): 4-wide nodes at the indices of the binary nodes they
                   // were collapsed from (NULL: not built)
  float4 *tris;    // 3 * n_tris (leaf order)
  float4 *shade;   // 3 * n_tris (input order)
  float4 *shade2;  // n_tris
  int32_t *tri_obj;
  // scratch (device)
  float4 *tris_in;       // 3 * n_tris (input order)
  float4 *centroids;     // n_tris
  uint32_t *bounds;      // 6 sortable words (min xyz, max xyz)
  unsigned long long *keys, *keys_alt;  // 63-bit Morton codes
  uint32_t *vals, *vals_alt;
  uint32_t *hist;        // 256 * sort_blocks
  int32_t *parents;      // (n_tris - 1) internal + n_tris leaves, parent << 1 | slot
  int32_t *flags;        // n_tris - 1
  int32_t *depth;        // 1 word: deepest leaf
};
size_t sort_blocks(int32_t n);
cudaError_t launch_build(const BuildBuffers &b, cudaStream_t s);
// stable LSD radix sort on key bytes first_byte .. first_byte + passes - 1 (hist: 256 *
// sort_blocks(n) words); with an even number of passes the result is back in keys / vals
cudaError_t radix_sort_pairs(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                             uint32_t *vals_alt, uint32_t *hist, int32_t n, int first_byte, int passes,
                             cudaStream_t s);

// ---- renderer (render.cu) -----------------------------------------------------------------
cudaError_t launch_trace_camera(const DevScene &S, const sc_trace_params &p, const sc_frame &f, unsigned *status,
                                unsigned *ticket, unsigned long long *counters, int grid, cudaStream_t s);
cudaError_t launch_trace_lights(const DevScene &S, const sc_light_params &p, const sc_frame &f, unsigned *status,
                                unsigned long long *ticket, unsigned long long *counters, int grid,
                                cudaStream_t s, float4 *photons = nullptr);
cudaError_t launch_resolve(const DevScene &S, const sc_resolve_params &p, const sc_frame &f, unsigned *status,
                           cudaStream_t s);
cudaError_t launch_intersect(const DevScene &S, const float *rays, int64_t n, float *hits, unsigned *status,
                             cudaStream_t s);
cudaError_t launch_occluded(const DevScene &S, const float *rays, int64_t n, int32_t *occ, unsigned *status,
                            cudaStream_t s);
// the camera estimator as a wavefront (wavefront.cu): waves of whole pixels of at most max_paths
// paths, path state and queues in `workspace` (wavefront_workspace_bytes(max_paths) bytes)
// paths of one wave at most (whole pixels of all their samples; the path state is ~230 B a path,
// 7.7 GB at 2^25).  Larger waves measured faster down the line (512^2 glass frame at 256 spp,
// camera phase: 2^21 165 ms, 2^22 134, 2^23 123, 2^24 117, 2^25 115.4, 2^26 115.7): fewer waves
// mean fewer bounces whose last queries leave the GPU idle.
#ifndef SC_WF_MAX_WAVE_LOG2
#define SC_WF_MAX_WAVE_LOG2 25
#endif
constexpr int64_t kWfMaxWavePaths = int64_t(1) << SC_WF_MAX_WAVE_LOG2;
size_t wavefront_workspace_bytes(int64_t max_paths);
cudaError_t launch_trace_camera_wavefront(const DevScene &S, const sc_trace_params &p, const sc_frame &f,
                                          unsigned *status, unsigned long long *counters, void *workspace,
                                          int64_t max_paths, int num_sms, cudaStream_t s);
// the batched launch on the wavefront engine: tab[i].slot_begin = first tile-order pixel slot of
// scene i, total_slots = their sum
cudaError_t launch_trace_batch_wavefront(const BatchEntry *tab, int n, int64_t total_slots, const sc_trace_params &p,
                                         unsigned *status, unsigned long long *counters, void *workspace,
                                         int64_t max_paths, int num_sms, cudaStream_t s);
const void *camera_kernel_ptr();
const void *light_kernel_ptr();
struct BatchEntry;
// one block per kBatchChunk tickets of each scene; tab[i].begin = first block of scene i
cudaError_t launch_trace_batch(const BatchEntry *tab, int n, unsigned total_blocks, const sc_trace_params &p,
                               unsigned *status, unsigned long long *counters, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr, uint64_t key, int64_t n, uint32_t *out, cudaStream_t s);

}  // namespace sc
