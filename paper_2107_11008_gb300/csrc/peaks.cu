// peaks.cu -- measurement kernels for the roofline denominators of the traversal kernels.
//
// BVH traversal runs on the CUDA cores' FP32 pipes and reads its nodes and triangles from L2
// (the 512^2 scene's 14 MB of BVH stays resident).  A STREAM-style copy and a BF16 GEMM give the
// HBM and tensor ceilings; these two kernels measure the other two on the device they run on:
// FP32 fused multiply-add throughput and L2 read bandwidth.
#include <string>

#include "internal.h"

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 8;  // independent FMA chains per thread: hides the FMA latency
constexpr int kL2Threads = 512;

// Every thread runs kFmaChains chains of a = a * b + c for `iters` steps; b and c are kernel
// arguments, so nothing folds.  The sum is stored only if it equals a value no input produces,
// which keeps the chains live without a store per thread.
__global__ void __launch_bounds__(kFmaThreads) k_peak_fma(int64_t iters, float b, float c, float *sink) {
  float a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k);
  for (int64_t i = 0; i < iters; i += 16) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (s == -1234.5f) sink[0] = s;
}

// Grid-stride float4 reads through L2 only (ld.global.cg: L1 bypassed), `reps` passes over the
// buffer.  Each block's share of the buffer is the same on every pass.
__global__ void __launch_bounds__(kL2Threads) k_peak_l2_read(const float4 *__restrict__ buf, int64_t n, int reps,
                                                             float *sink) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == -1234.5f) sink[0] = acc;
}

int sm_count(int device) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return n;
}

}  // namespace

struct sc_ctx;
namespace sc {
int ctx_device(const sc_ctx *c);
cudaStream_t ctx_stream(const sc_ctx *c);
void ctx_set_error(sc_ctx *c, const std::string &msg);
}  // namespace sc

extern "C" int sc_peak_fma(sc_ctx *ctx, int64_t iters, float *sink, int64_t *flops) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (iters < 16 || iters % 16 != 0 || !sink || !flops) {
    sc::ctx_set_error(ctx, "sc_peak_fma: iters must be a positive multiple of 16; sink and flops non-null");
    return SC_ERR_INVALID_ARG;
  }
  const int sms = sm_count(sc::ctx_device(ctx));
  if (sms <= 0) {
    sc::ctx_set_error(ctx, "sc_peak_fma: cannot read the SM count");
    return SC_ERR_CUDA;
  }
  const int blocks = sms * 8;  // 2048 threads per SM
  k_peak_fma<<<blocks, kFmaThreads, 0, sc::ctx_stream(ctx)>>>(iters, 0.999f, 0.001f, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sc::ctx_set_error(ctx, std::string("sc_peak_fma: ") + cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  *flops = 2ll * kFmaChains * iters * (int64_t)blocks * kFmaThreads;
  return SC_OK;
}

extern "C" int sc_peak_l2_read(sc_ctx *ctx, const void *buf, int64_t bytes, int32_t reps, float *sink,
                               int64_t *bytes_read) {
  if (!ctx) return SC_ERR_INVALID_ARG;
  if (!buf || bytes < 16 || bytes % 16 != 0 || (reinterpret_cast<uintptr_t>(buf) & 15) != 0 || reps < 1 || !sink ||
      !bytes_read) {
    sc::ctx_set_error(ctx, "sc_peak_l2_read: buf 16-byte aligned, bytes a positive multiple of 16, reps >= 1, "
                           "sink and bytes_read non-null");
    return SC_ERR_INVALID_ARG;
  }
  const int sms = sm_count(sc::ctx_device(ctx));
  if (sms <= 0) {
    sc::ctx_set_error(ctx, "sc_peak_l2_read: cannot read the SM count");
    return SC_ERR_CUDA;
  }
  const int blocks = sms * 4;  // 2048 threads per SM
  k_peak_l2_read<<<blocks, kL2Threads, 0, sc::ctx_stream(ctx)>>>(static_cast<const float4 *>(buf), bytes / 16,
                                                                  reps, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sc::ctx_set_error(ctx, std::string("sc_peak_l2_read: ") + cudaGetErrorString(e));
    return SC_ERR_CUDA;
  }
  *bytes_read = bytes * (int64_t)reps;
  return SC_OK;
}
