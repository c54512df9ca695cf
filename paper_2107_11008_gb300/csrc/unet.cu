// unet.cu -- the BF16 U-Net denoiser (include/sc_unet.h): forward, L1 + SSIM loss, backward,
// Adam, all on the GPU.  Every 3x3 convolution (forward, data gradient, weight gradient) and the
// transposed convolutions run on the tensor cores (tcgen05: the TMA kernels of unet_conv.cuh and
// unet_wgrad_mn.cuh, else the gathering GEMM of unet_gemm.cuh); the 1x1 output layer (HBM-bound),
// pooling, the loss, the weight-gradient reduction and Adam are plain CUDA.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "internal.h"
#include "sc_unet.h"
#include "unet_conv.cuh"
#include "unet_gemm.cuh"
#include "unet_wgrad_mn.cuh"

namespace sc {
int ctx_device(const sc_ctx *c);
cudaStream_t ctx_stream(const sc_ctx *c);
void ctx_set_error(sc_ctx *c, const std::string &msg);
void *ctx_alloc(sc_ctx *c, size_t bytes);
void ctx_free(sc_ctx *c, void *p);
unsigned *ctx_status(sc_ctx *c);
}  // namespace sc

namespace sc {
namespace unet {

constexpr int kLevels = 4;
constexpr int kChans[kLevels] = {32, 48, 64, 128};
constexpr int kInCh = 11, kInPad = 16, kOutCh = 3, kGyCh = 8;
constexpr double kL1W = 0.16, kSsimW = 0.84;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// ---------------------------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------------------------

// x [P][11] FP32 -> 16 BF16 channels (11..15 zero), row-blocked with rows of w pixels
__global__ void k_pack_input(const float *x, bf16 *out, int64_t P, int w) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = i < kInCh ? x[p * kInCh + i] : 0.0f;
  const int64_t r = p / w;
  bf16 *o = out + rb_off(r, (int)(p - r * w), 0, kInPad, w);
  *reinterpret_cast<uint4 *>(o) = pack8(v);
  *reinterpret_cast<uint4 *>(o + 8 * w) = pack8(v + 8);
}

// a channel slice of a row-blocked BF16 tensor -> dense [rows * w][ch] (test inspection)
__global__ void k_rb_to_dense(const bf16 *src, int cs, int co, int ch, int64_t rows, int w, bf16 *dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * w * ch) return;
  const int c = (int)(i % ch);
  const int64_t p = i / ch, r = p / w;
  dst[i] = src[rb_off(r, (int)(p - r * w), co + c, cs, w)];
}

// 11-channel network input from a frame's buffers
__global__ void k_pack_frame(const float4 *rgb, const float4 *albedo, const float4 *normal, const float *depth_norm,
                             const uint8_t *mask, float *x, int64_t P) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float4 c = rgb[p], a = albedo[p], n = normal[p];
  float *o = x + p * kInCh;
  o[0] = log1pf(fmaxf(c.x, 0.0f));
  o[1] = log1pf(fmaxf(c.y, 0.0f));
  o[2] = log1pf(fmaxf(c.z, 0.0f));
  o[3] = a.x;
  o[4] = a.y;
  o[5] = a.z;
  o[6] = n.x;
  o[7] = n.y;
  o[8] = n.z;
  o[9] = depth_norm[p];
  o[10] = mask[p] ? 1.0f : 0.0f;
}

__global__ void k_pack_target(const float4 *rgb, float *t, int64_t P) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float4 c = rgb[p];
  t[p * 3 + 0] = log1pf(fmaxf(c.x, 0.0f));
  t[p * 3 + 1] = log1pf(fmaxf(c.y, 0.0f));
  t[p * 3 + 2] = log1pf(fmaxf(c.z, 0.0f));
}

__global__ void k_output_rgb(const float *y, int64_t P, const float4 *add, float4 *rgb) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float4 o = make_float4(fmaxf(expm1f(y[p * 3]), 0.0f), fmaxf(expm1f(y[p * 3 + 1]), 0.0f),
                         fmaxf(expm1f(y[p * 3 + 2]), 0.0f), 1.0f);
  if (add) {
    const float4 a = add[p];
    o.x += a.x;
    o.y += a.y;
    o.z += a.z;
  }
  rgb[p] = o;
}

// 2x2 stride-2 max pool of a channel slice: src (row-blocked, h x w, cs channels, slice at co)
// -> dst (row-blocked, h/2 x w/2, C channels).  Thread order: pixel fastest, then channel group,
// then output row, so that a warp reads and writes contiguous runs.
__global__ void k_pool(const bf16 *src, int cs, int co, int C, int n, int h, int w, bf16 *dst) {
  const int groups = C / 8;
  const int ho = h / 2, wo = w / 2;
  const int64_t total = (int64_t)n * ho * wo * groups;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int x = (int)(i % wo);
  const int64_t t = i / wo;
  const int g = (int)(t % groups);
  const int64_t ro = t / groups;  // img * ho + y
  const int64_t ri = ro / ho * h + 2 * (ro % ho);
  float best[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float v[8];
    unpack8(ldg16(src + rb_off(ri + (k >> 1), 2 * x + (k & 1), co + g * 8, cs, w)), v);
#pragma unroll
    for (int j = 0; j < 8; ++j) best[j] = k == 0 ? v[j] : fmaxf(best[j], v[j]);
  }
  *reinterpret_cast<uint4 *>(dst + rb_off(ro, x, g * 8, C, wo)) = pack8(best);
}

// gradient through the 2x2 max pool, the inverse routing of k_pool: gp, the FP32 gradient of the
// pooled tensor ([pooled pixel][N]), goes to the first maximum of each window in row-major order,
// plus the FP32 skip gradient of the pool input ([pixel][scs], may be null), times the pool
// input's ReLU mask, rounded once to BF16 into out (row-blocked, N channels, rows of 2 wo pixels).
// e: the pool input (row-blocked slice: ecs channels, slice at eco).
__global__ void k_pool_back(const float *gp, int N, const bf16 *e, int ecs, int eco, const float *skip, int scs,
                            bf16 *out, int n, int ho, int wo) {
  const int groups = N / 8;
  const int w = 2 * wo;
  const int64_t total = (int64_t)n * ho * wo * groups;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  // channel group fastest: the lanes of a warp read whole 128-byte rows of the FP32 tensors
  const int g = (int)(i % groups);
  const int64_t t = i / groups;
  const int x = (int)(t % wo);
  const int64_t ro = t / wo;  // img * ho + y
  const int64_t ri = ro / ho * (2 * ho) + 2 * (ro % ho);
  const int c = 8 * g;
  float gv[8];
  {
    const float4 *p = reinterpret_cast<const float4 *>(gp + (ro * wo + x) * N + c);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    gv[0] = a.x;
    gv[1] = a.y;
    gv[2] = a.z;
    gv[3] = a.w;
    gv[4] = b.x;
    gv[5] = b.y;
    gv[6] = b.z;
    gv[7] = b.w;
  }
  float ev[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) unpack8(ldg16(e + rb_off(ri + (q >> 1), 2 * x + (q & 1), eco + c, ecs, w)), ev[q]);
  int win[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int b = 0;
    float best = ev[0][j];
#pragma unroll
    for (int q = 1; q < 4; ++q)
      if (ev[q][j] > best) {
        best = ev[q][j];
        b = q;
      }
    win[j] = b;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r2 = ri + (q >> 1);
    const int x2 = 2 * x + (q & 1);
    float o[8];
    if (skip) {
      const float4 *sp = reinterpret_cast<const float4 *>(skip + (r2 * w + x2) * scs + c);
      const float4 f0 = __ldg(sp), f1 = __ldg(sp + 1);
      o[0] = f0.x;
      o[1] = f0.y;
      o[2] = f0.z;
      o[3] = f0.w;
      o[4] = f1.x;
      o[5] = f1.y;
      o[6] = f1.z;
      o[7] = f1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) o[j] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (win[j] == q) o[j] += gv[j];
      if (!(ev[q][j] > 0.0f)) o[j] = 0.0f;
    }
    *reinterpret_cast<uint4 *>(out + rb_off(r2, x2, c, N, w)) = pack8(o);
  }
}

enum { KIND_BIAS = 0, KIND_CONV = 1, KIND_UP = 2, KIND_OUT = 3 };

// ---- the 1x1 output layer (32 -> 3): HBM-bound, so plain CUDA-core kernels ------------------
// Weights are the BF16 copy the rest of the network uses, W[o][c] (o < 3, c < 32); products and
// sums in FP32.  x, the layer input, is row-blocked with 32 channels and rows of w pixels.
constexpr int kOutBlock = 256;

__device__ __forceinline__ void load_out_w(const bf16 *W, float *sw) {
  for (int i = threadIdx.x; i < kOutCh * 32; i += blockDim.x) sw[i] = __bfloat162float(W[i]);
}

// y[p][o] = sum_c W[o][c] x[p][c] + b[o]
__global__ void __launch_bounds__(kOutBlock) k_out_fwd(const bf16 *x, int w, int64_t P, const bf16 *W,
                                                        const float *b, float *y) {
  __shared__ float sw[kOutCh * 32];
  load_out_w(W, sw);
  __syncthreads();
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int64_t r = p / w;
  const int xx = (int)(p - r * w);
  float a[kOutCh] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    float v[8];
    unpack8(ldg16(x + rb_off(r, xx, 8 * g, 32, w)), v);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int o = 0; o < kOutCh; ++o) a[o] = fmaf(sw[o * 32 + 8 * g + j], v[j], a[o]);
  }
#pragma unroll
  for (int o = 0; o < kOutCh; ++o) y[p * kOutCh + o] = a[o] + __ldg(b + o);
}

// gx[p][c] = (sum_o W[o][c] gy[p][o]) * (x[p][c] > 0): the data gradient through the layer and
// the ReLU of its input.  gy: [p][8] BF16 (3 used); gx row-blocked like x.
__global__ void __launch_bounds__(kOutBlock) k_out_dgrad(const bf16 *gy8, const bf16 *x, int w, int64_t P,
                                                          const bf16 *W, bf16 *gx) {
  __shared__ float sw[kOutCh * 32];
  load_out_w(W, sw);
  __syncthreads();
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int64_t r = p / w;
  const int xx = (int)(p - r * w);
  float gy[8];
  unpack8(ldg16(gy8 + p * kGyCh), gy);
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    float m[8], t[8];
    const int64_t off = rb_off(r, xx, 8 * g, 32, w);
    unpack8(ldg16(x + off), m);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * g + j;
      const float v = fmaf(sw[64 + c], gy[2], fmaf(sw[32 + c], gy[1], sw[c] * gy[0]));
      t[j] = m[j] > 0.0f ? v : 0.0f;
    }
    *reinterpret_cast<uint4 *>(gx + off) = pack8(t);
  }
}

// Weight and bias gradient, stage 1: block b sums gy[p][o] x[p][c] and gy[p][o] over its pixel
// range [b * span, (b + 1) * span) in a fixed order (thread (lane, group) takes every 64th pixel,
// then a fixed shared-memory tree over the 64 lanes) -> part[b][99] (96 weights o * 32 + c, then
// 3 biases; thread group g < 3 also sums the bias of output g).
constexpr int kOutParts = kOutCh * 32 + kOutCh;
__global__ void __launch_bounds__(kOutBlock) k_out_wgrad(const bf16 *gy8, const bf16 *x, int w, int64_t P,
                                                          int64_t span, float *part) {
  __shared__ float red[kOutBlock][kOutCh * 8 + 1];
  const int pl = threadIdx.x & 63, g = threadIdx.x >> 6;  // pixel lane, channel group
  float acc[kOutCh * 8 + 1];
#pragma unroll
  for (int i = 0; i < kOutCh * 8 + 1; ++i) acc[i] = 0.0f;
  const int64_t p0 = blockIdx.x * span, p1 = min(P, p0 + span);
  int64_t r = (p0 + pl) / w;
  int xx = (int)(p0 + pl - r * w);
  for (int64_t p = p0 + pl; p < p1; p += 64) {
    float gy[8], v[8];
    unpack8(ldg16(gy8 + p * kGyCh), gy);
    unpack8(ldg16(x + rb_off(r, xx, 8 * g, 32, w)), v);
#pragma unroll
    for (int o = 0; o < kOutCh; ++o)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[o * 8 + j] = fmaf(gy[o], v[j], acc[o * 8 + j]);
    acc[kOutCh * 8] += g == 0 ? gy[0] : (g == 1 ? gy[1] : (g == 2 ? gy[2] : 0.0f));
    for (xx += 64; xx >= w; xx -= w) ++r;  // next pixel of this lane: p + 64
  }
#pragma unroll
  for (int i = 0; i < kOutCh * 8 + 1; ++i) red[threadIdx.x][i] = acc[i];
  __syncthreads();
  for (int s = 32; s > 0; s >>= 1) {
    if (pl < s)
#pragma unroll
      for (int i = 0; i < kOutCh * 8 + 1; ++i) red[threadIdx.x][i] += red[threadIdx.x + s][i];
    __syncthreads();
  }
  if (pl == 0) {
    float *o = part + (int64_t)blockIdx.x * kOutParts;
#pragma unroll
    for (int oo = 0; oo < kOutCh; ++oo)
#pragma unroll
      for (int j = 0; j < 8; ++j) o[oo * 32 + 8 * g + j] = red[threadIdx.x][oo * 8 + j];
    if (g < kOutCh) o[kOutCh * 32 + g] = red[threadIdx.x][kOutCh * 8];
  }
}

// stage 2: block i of kOutParts sums entry i of the block partials in a fixed order (thread t
// takes partials t, t + 128, ..., then a fixed shared-memory tree) -> gw[o * 32 + c], gb[o]
__global__ void __launch_bounds__(128) k_out_wgrad_final(const float *part, int nblk, float *gw, float *gb) {
  __shared__ float red[128];
  const int i = blockIdx.x, t = threadIdx.x;
  float v = 0.0f;
  for (int b = t; b < nblk; b += 128) v += part[(int64_t)b * kOutParts + i];
  red[t] = v;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) {
    if (i < kOutCh * 32) gw[i] = red[0];
    else gb[i - kOutCh * 32] = red[0];
  }
}



// Sum of the K-split partial products in a fixed order, scattered to the flat FP32 gradient.
// part[(s * Mpad + r) * np + n]; rows r: conv (tap * cin_p + c) | ones; up: c | ones.
// Block = 32 lanes x 4 consecutive entries (r, n..n+3; np is a multiple of 16) x 8 split groups;
// group g sums splits g, g + 8, ... (one 16-byte load per lane, 512 bytes per warp), then the 8
// group sums are added in order.
constexpr int kRedEntries = 32, kRedVec = 4, kRedGroups = 8;
constexpr int kRedBlockEntries = kRedEntries * kRedVec;

__device__ __forceinline__ float4 split_sum4(const float *part, int splits, int Mpad, int np, int r, int n, int g) {
  float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
  for (int k = g; k < splits; k += kRedGroups) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(part + ((int64_t)k * Mpad + r) * np + n));
    s.x += v.x;
    s.y += v.y;
    s.z += v.z;
    s.w += v.w;
  }
  return s;
}
__device__ __forceinline__ void add4(float4 &a, const float4 &b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

// One launch reduces the split-K partials of every layer of a backward pass: segment t covers
// blocks [first_block, next first_block) and its own partial region of the workspace.
struct RedSeg {
  int64_t part_off, w_off, b_off;  // floats into the workspace / into the flat gradient
  int splits, Mpad, np, rows, kind, cout, cin, cin_p, first_block;
  int col, cgb, nu, cpb, ncopy;  // conv rows in the MN-major kernel's column order (col = 1)
};
constexpr int kMaxRedSegs = 20;
struct RedTable {
  int n;
  RedSeg s[kMaxRedSegs];
};

__global__ void __launch_bounds__(kRedEntries *kRedGroups) k_wgrad_reduce(const __grid_constant__ RedTable T,
                                                                           const float *wpart, float *grads) {
  __shared__ float4 sh[kRedGroups][kRedEntries];
  int lo = 0, hi = T.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.s[mid].first_block <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const RedSeg &S = T.s[lo];
  const float *part = wpart + S.part_off;
  float *gw = grads + S.w_off, *gb = grads + S.b_off;
  const int splits = S.splits, Mpad = S.Mpad, np = S.np, rows = S.rows, kind = S.kind, cout = S.cout, cin = S.cin,
            cin_p = S.cin_p;
  const int e = threadIdx.x % kRedEntries, g = threadIdx.x / kRedEntries;
  const int64_t i = ((int64_t)((int)blockIdx.x - S.first_block) * kRedEntries + e) * kRedVec;
  const int64_t total = (int64_t)(rows + 1) * np;
  const int r = (int)(i / np), n = (int)(i % np);
  const bool valid = i < total;
  // the bias of a transposed conv sums its four (a, e) column blocks of the ones row (cout is a
  // multiple of 4, so the 4 entries are all below cout or all at or above it)
  float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  // padding rows of a column-ordered block were never written: skip them (r == rows, the bias row,
  // is not padding)
  bool pad = false;
  if (S.col && r < rows) {
    const int p = (r >> 3) & 15, kk = p / (3 * S.cgb);
    pad = kk >= S.cpb || (r >> 7) * S.cpb + kk >= S.ncopy;
  }
  if (valid && !pad) {
    if (kind == KIND_UP && r == rows) {
      if (n < cout)
        for (int ae = 0; ae < 4; ++ae) add4(v, split_sum4(part, splits, Mpad, np, r, ae * cout + n, g));
    } else {
      v = split_sum4(part, splits, Mpad, np, r, n, g);
    }
  }
  sh[g][e] = v;
  __syncthreads();
  if (g != 0 || !valid) return;
  float4 t4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int k = 0; k < kRedGroups; ++k) add4(t4, sh[k][e]);
  const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
  for (int q = 0; q < kRedVec; ++q) {
    const int nq = n + q;
    const float t = tv[q];
    if (kind == KIND_CONV) {
      if (nq >= cout) continue;
      if (r == rows) {
        gb[nq] = t;
        continue;
      }
      int tap, c;
      if (S.col) {
        // pair j = r / 8 of block j / 16: copy k = block * cpb + (j % 16) / (3 cgb), then (group, dy)
        const int j = r >> 3, m = j >> 4, p = j & 15, kk = p / (3 * S.cgb), rem = p - kk * 3 * S.cgb;
        const int k = m * S.cpb + kk;
        if (kk >= S.cpb || k >= S.ncopy) continue;  // padding of a block
        const int gi = rem / 3, dy = rem - 3 * gi, dx = k / S.nu, un = k - dx * S.nu;
        tap = 3 * dy + dx;
        c = 8 * (un * S.cgb + gi) + (r & 7);
      } else {
        tap = r / cin_p;
        c = r - tap * cin_p;
      }
      if (c < cin) gw[((int64_t)nq * 9 + tap) * cin + c] = t;
    } else {  // KIND_UP
      if (r == rows) {
        if (nq < cout) gb[nq] = t;
        continue;
      }
      if (nq >= 4 * cout) continue;
      const int ae = nq / cout, o = nq - ae * cout;
      gw[((int64_t)r * 4 + ae) * cout + o] = t;
    }
  }
}

struct Seg {
  int64_t off;
  int32_t count, kind, cout, cin, cin_p, first_block;
  bf16 *wf, *wd;    // B layouts of the gathering GEMM (forward, data gradient)
  bf16 *wtf, *wtd;  // B layouts of the TMA convolution: [tap][k-group][n][8]
  bf16 *wtf2, *wtd2;  // the same split in two halves of n, [half][tap][k-group][n/2][8] (or null)
};

// One bias-corrected Adam step over every parameter (update != 0), then the BF16 copies:
// wf = the layout the forward GEMM reads as B, wd = the layout of the data-gradient GEMM.
__global__ void k_adam(const Seg *segs, int nseg, float *p, const float *g, float *m, float *v, float lr, float bc1,
                       float bc2, int update) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].first_block <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const Seg S = segs[lo];
  const int i = ((int)blockIdx.x - S.first_block) * blockDim.x + threadIdx.x;
  if (i >= S.count) return;
  const int64_t k = S.off + i;
  float w = p[k];
  if (update) {
    const float gk = g[k];
    const float mk = 0.9f * m[k] + 0.1f * gk;
    const float vk = 0.999f * v[k] + 0.001f * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w -= lr * (mk / bc1) / (sqrtf(vk / bc2) + 1e-8f);
    p[k] = w;
  }
  const bf16 b = __float2bfloat16_rn(w);
  if (S.kind == KIND_CONV) {
    const int o = i / (9 * S.cin), rem = i - o * 9 * S.cin, tap = rem / S.cin, c = rem - tap * S.cin;
    S.wf[((int64_t)o * 9 + tap) * S.cin_p + c] = b;
    S.wtf[(((int64_t)tap * (S.cin_p / 8) + c / 8) * S.cout + o) * 8 + (c & 7)] = b;
    if (S.wd) {
      S.wd[((int64_t)c * 9 + tap) * S.cout + o] = b;
      S.wtd[(((int64_t)tap * (S.cout / 8) + o / 8) * S.cin + c) * 8 + (o & 7)] = b;
    }
    if (S.wtf2) {
      const int hn = S.cout / 2, hf = o / hn, oo = o - hf * hn;
      S.wtf2[((((int64_t)hf * 9 + tap) * (S.cin_p / 8) + c / 8) * hn + oo) * 8 + (c & 7)] = b;
    }
    if (S.wtd2) {
      const int hc = S.cin / 2, hf = c / hc, cc = c - hf * hc;
      S.wtd2[((((int64_t)hf * 9 + tap) * (S.cout / 8) + o / 8) * hc + cc) * 8 + (o & 7)] = b;
    }
  } else if (S.kind == KIND_UP) {
    const int c = i / (4 * S.cout), rem = i - c * 4 * S.cout;
    S.wf[(int64_t)rem * S.cin + c] = b;
    S.wd[i] = b;
    S.wtf[((int64_t)(c / 8) * (4 * S.cout) + rem) * 8 + (c & 7)] = b;
    if (S.wtd) S.wtd[((int64_t)(rem / 8) * S.cin + c) * 8 + (rem & 7)] = b;  // [(a, e, o) group][c][8]
  } else if (S.kind == KIND_OUT) {
    S.wf[i] = b;
  }
}

// ---- loss --------------------------------------------------------------------------------
constexpr int kSTW = 32, kSTH = 8, kWin = 11;
__constant__ float c_gauss[kWin];

__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// SSIM of each valid 11x11 window and d SSIM / d (mu_x, E[x^2], E[xy]) of that window.
// Grid: (ceil(Wv / 32), ceil(Hv / 8), n), 256 threads; Wv = w - 10, Hv = h - 10.
__global__ void __launch_bounds__(256) k_ssim_fwd(const float *p, const float *t, int h, int w, float *dmx,
                                                  float *dexx, float *dexy, double *part) {
  __shared__ float sp[kSTH + 10][kSTW + 10], st[kSTH + 10][kSTW + 10];
  __shared__ float hz[5][kSTH + 10][kSTW];
  __shared__ double red[256];
  const int Hv = h - 10, Wv = w - 10;
  const int x0 = blockIdx.x * kSTW, y0 = blockIdx.y * kSTH, img = blockIdx.z;
  const int tx = threadIdx.x % kSTW, ty = threadIdx.x / kSTW;
  const int wx = x0 + tx, wy = y0 + ty;
  double acc = 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    for (int i = threadIdx.x; i < (kSTH + 10) * (kSTW + 10); i += 256) {
      const int r = i / (kSTW + 10), cc = i % (kSTW + 10);
      const int yy = y0 + r, xx = x0 + cc;
      const bool in = yy < h && xx < w;
      const int64_t idx = ((int64_t)(img * h + yy) * w + xx) * 3 + ch;
      sp[r][cc] = in ? p[idx] : 0.0f;
      st[r][cc] = in ? t[idx] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (kSTH + 10) * kSTW; i += 256) {
      const int r = i / kSTW, cc = i % kSTW;
      float a = 0, b = 0, aa = 0, bb = 0, ab = 0;
#pragma unroll
      for (int k = 0; k < kWin; ++k) {
        const float g = c_gauss[k], u = sp[r][cc + k], q = st[r][cc + k];
        a += g * u;
        b += g * q;
        aa += g * u * u;
        bb += g * q * q;
        ab += g * u * q;
      }
      hz[0][r][cc] = a;
      hz[1][r][cc] = b;
      hz[2][r][cc] = aa;
      hz[3][r][cc] = bb;
      hz[4][r][cc] = ab;
    }
    __syncthreads();
    float mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const float g = c_gauss[k];
      mx += g * hz[0][ty + k][tx];
      my += g * hz[1][ty + k][tx];
      exx += g * hz[2][ty + k][tx];
      eyy += g * hz[3][ty + k][tx];
      exy += g * hz[4][ty + k][tx];
    }
    if (wx < Wv && wy < Hv) {
      const float a1 = 2.0f * mx * my + kC1;
      const float a2 = 2.0f * (exy - mx * my) + kC2;
      const float b1 = mx * mx + my * my + kC1;
      const float b2 = (exx - mx * mx) + (eyy - my * my) + kC2;
      const float S = a1 * a2 / (b1 * b2);
      const int64_t o = ((int64_t)(img * Hv + wy) * Wv + wx) * 3 + ch;
      dmx[o] = (2.0f * my * a2 - 2.0f * my * a1) / (b1 * b2) - S * (2.0f * mx / b1 - 2.0f * mx / b2);
      dexx[o] = -S / b2;
      dexy[o] = 2.0f * a1 / (b1 * b2);
      acc += S;
    }
    __syncthreads();
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// d loss / d pred per pixel: the adjoint of the window blurs applied to the three coefficient
// maps plus the L1 term.  Grid: (ceil(w / 32), ceil(h / 8), n), 256 threads.
__global__ void __launch_bounds__(256) k_ssim_bwd(const float *p, const float *t, int h, int w, const float *dmx,
                                                  const float *dexx, const float *dexy, float inv_px, float inv_win,
                                                  float *grad, bf16 *gy8, double *part) {
  __shared__ float wm[3][kSTH + 10][kSTW + 10];
  __shared__ float hz[3][kSTH + 10][kSTW];
  __shared__ double red[256];
  const int Hv = h - 10, Wv = w - 10;
  const int x0 = blockIdx.x * kSTW, y0 = blockIdx.y * kSTH, img = blockIdx.z;
  const int tx = threadIdx.x % kSTW, ty = threadIdx.x / kSTW;
  const int x = x0 + tx, y = y0 + ty;
  const bool in = x < w && y < h;
  const int64_t pix = ((int64_t)(img * h + y) * w + x);
  float gout[3] = {0.0f, 0.0f, 0.0f};
  double acc = 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    // window maps over rows y0-10 .. y0+7, cols x0-10 .. x0+31
    for (int i = threadIdx.x; i < (kSTH + 10) * (kSTW + 10); i += 256) {
      const int r = i / (kSTW + 10), cc = i % (kSTW + 10);
      const int wy = y0 - 10 + r, wx = x0 - 10 + cc;
      const bool ok = wy >= 0 && wy < Hv && wx >= 0 && wx < Wv;
      const int64_t o = ((int64_t)(img * Hv + wy) * Wv + wx) * 3 + ch;
      wm[0][r][cc] = ok ? dmx[o] : 0.0f;
      wm[1][r][cc] = ok ? dexx[o] : 0.0f;
      wm[2][r][cc] = ok ? dexy[o] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (kSTH + 10) * kSTW; i += 256) {
      const int r = i / kSTW, cc = i % kSTW;
      float a = 0, b = 0, c = 0;
#pragma unroll
      for (int k = 0; k < kWin; ++k) {
        const float g = c_gauss[k];
        a += g * wm[0][r][cc + 10 - k];
        b += g * wm[1][r][cc + 10 - k];
        c += g * wm[2][r][cc + 10 - k];
      }
      hz[0][r][cc] = a;
      hz[1][r][cc] = b;
      hz[2][r][cc] = c;
    }
    __syncthreads();
    if (in) {
      float G0 = 0, G1 = 0, G2 = 0;
#pragma unroll
      for (int k = 0; k < kWin; ++k) {
        const float g = c_gauss[k];
        G0 += g * hz[0][ty + 10 - k][tx];
        G1 += g * hz[1][ty + 10 - k][tx];
        G2 += g * hz[2][ty + 10 - k][tx];
      }
      const float pv = p[pix * 3 + ch], tv = t[pix * 3 + ch];
      const float d = pv - tv;
      const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
      const float gs = G0 + 2.0f * pv * G1 + tv * G2;
      const float gr = (float)kL1W * sgn * inv_px - (float)kSsimW * gs * inv_win;
      gout[ch] = gr;
      if (grad) grad[pix * 3 + ch] = gr;
      acc += fabs((double)d);
    }
    __syncthreads();
  }
  if (in && gy8) {
    float v[8] = {gout[0], gout[1], gout[2], 0, 0, 0, 0, 0};
    *reinterpret_cast<uint4 *>(gy8 + pix * kGyCh) = pack8(v);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

__global__ void k_loss_final(const double *ps, int nps, const double *pl, int npl, double n_px, double n_win,
                             float *loss) {
  __shared__ double red[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nps; i += 256) a += ps[i];
  for (int i = threadIdx.x; i < npl; i += 256) b += pl[i];
  const double S = block_sum(a, red);
  __syncthreads();
  const double L = block_sum(b, red);
  if (threadIdx.x == 0 && loss) *loss = (float)(kL1W * L / n_px + kSsimW * (1.0 - S / n_win));
}

// Segmentation loss: binary cross-entropy with the logit in output channel 0 and a label in [0, 1]
// in target channel 0 (channels 1 and 2 take no part: zero gradient).  Per pixel
// softplus(y) - t y = max(y, 0) - t y + log1p(exp(-|y|)); d / d y = (sigmoid(y) - t) / n_px.
// One block per 256 pixels; block partial sums in FP64, summed in a fixed order.
__global__ void __launch_bounds__(256) k_bce(const float *p, const float *t, int64_t n_px, float inv_px, float *grad,
                                             bf16 *gy8, double *part) {
  __shared__ double red[256];
  const int64_t pix = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double acc = 0.0;
  if (pix < n_px) {
    const float y = p[pix * 3], tv = t[pix * 3];
    const float g = (1.0f / (1.0f + expf(-y)) - tv) * inv_px;
    const double yd = (double)y;
    acc = fmax(yd, 0.0) - (double)tv * yd + log1p(exp(-fabs(yd)));
    if (grad) {
      grad[pix * 3] = g;
      grad[pix * 3 + 1] = 0.0f;
      grad[pix * 3 + 2] = 0.0f;
    }
    if (gy8) {
      float v[8] = {g, 0, 0, 0, 0, 0, 0, 0};
      *reinterpret_cast<uint4 *>(gy8 + pix * kGyCh) = pack8(v);
    }
  }
  const double sblk = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = sblk;
}

// Squared error in linear radiance on log1p-domain values: per element e = expm1(y) - expm1(t),
// loss = mean of e^2 over pixels and channels, d / d y = 2 e exp(y) / (3 n_px).  Its minimiser over
// noisy targets is their linear mean.  Same block partials as k_bce (k_bce_final sums them; the
// mean there divides by 3 n_px).
__global__ void __launch_bounds__(256) k_l2lin(const float *p, const float *t, int64_t n_px, float inv_n, float *grad,
                                               bf16 *gy8, double *part) {
  __shared__ double red[256];
  const int64_t pix = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double acc = 0.0;
  if (pix < n_px) {
    float g[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
      const float y = p[pix * 3 + ch], tv = t[pix * 3 + ch];
      const float e = expm1f(y) - expm1f(tv);
      g[ch] = 2.0f * e * expf(y) * inv_n;
      const double ed = expm1((double)y) - expm1((double)tv);
      acc += ed * ed;
      if (grad) grad[pix * 3 + ch] = g[ch];
    }
    if (gy8) *reinterpret_cast<uint4 *>(gy8 + pix * kGyCh) = pack8(g);
  }
  const double sblk = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = sblk;
}

__global__ void k_bce_final(const double *part, int np, double n_px, float *loss) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < np; i += 256) a += part[i];
  const double S = block_sum(a, red);
  if (threadIdx.x == 0 && loss) *loss = (float)(S / n_px);
}

// ---------------------------------------------------------------------------------------------
// GEMM launcher
// ---------------------------------------------------------------------------------------------
constexpr int kMaxDev = 16;

template <class AL, class BL, class EP>
cudaError_t gemm(const AL &a, const BL &b, const EP &e, int M, int N, int K, int splits, int k_split,
                 unsigned *status, cudaStream_t s) {
  if (M <= 0 || N <= 0 || N > 256 || K < 0 || splits < 1) return cudaErrorInvalidValue;
  const int np = pad16(N);
  auto kern = k_gemm<AL, BL, EP>;
  // per instantiation: dynamic shared memory per padded N such that the CTAs resident on one SM
  // never ask for more than the 512 TMEM columns
  static int smem_cache[kMaxDev][17];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  int smem = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    smem = smem_cache[dev][np / 16];
    if (smem == 0) {
      cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (err != cudaSuccess) return err;
      int bytes = (int)gemm_smem_bytes(np);
      for (;;) {
        int nb = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, bytes);
        if (err != cudaSuccess) return err;
        if (nb >= 1 && (uint32_t)nb * tmem_cols(np) <= 512u) break;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        bytes += 4096;
      }
      smem = smem_cache[dev][np / 16] = bytes;
    }
  }
  dim3 grid((unsigned)((M + kTM - 1) / kTM), (unsigned)splits);
  kern<<<grid, kThreads, smem, s>>>(a, b, e, M, N, K, k_split, status);
  return cudaGetLastError();
}

}  // namespace unet
}  // namespace sc

// =============================================================================================
// the network object
// =============================================================================================
using namespace sc::unet;

namespace {

struct Layer {
  int kind = 0, cout = 0, cin = 0, cin_p = 0;
  int64_t w_off = 0, b_off = 0, w_count = 0;
  bf16 *wf = nullptr, *wd = nullptr, *wtf = nullptr, *wtd = nullptr;
  bf16 *wtf2 = nullptr, *wtd2 = nullptr;  // n-split TMA layouts, for layers whose weights do not fit whole
  size_t part_off = 0, part_floats = 0;   // this layer's region of the weight-gradient partials
  int64_t wf_elems = 0, wd_elems = 0;
};

int enc_layer(int l, int j) { return 2 * l + j; }
int up_layer(int l) { return 8 + (2 - l) * 3; }
int dec_layer(int l, int j) { return up_layer(l) + 1 + j; }
constexpr int kOutLayer = 17, kNumLayers = 18;
// 3x3 layers whose TMA weight image is larger than this also get an n-split copy
constexpr uint32_t kConvSplitBytes = 200u * 1024u;

struct Wgrad {
  int rows = 0, Mtiles = 0, np = 0;
};

}  // namespace

struct sc_unet {
  int max_batch = 0, H = 0, W = 0;
  int n = 0;  // images of the last call
  int hl[kLevels], wl[kLevels];
  int64_t n_params = 0;
  Layer L[kNumLayers];
  void *block = nullptr;  // one allocation for everything
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  Seg *segs = nullptr;
  int nseg = 0, adam_blocks = 0;
  int step = 0;
  // activations
  bf16 *x0 = nullptr, *a1[kLevels] = {}, *cat[kLevels] = {}, *h3 = nullptr, *pool[kLevels] = {};
  bf16 *d1[kLevels] = {}, *d2[kLevels] = {};
  float *y = nullptr;
  // gradients
  bf16 *gy8 = nullptr, *gd2[kLevels] = {}, *gd1[kLevels] = {}, *gup[kLevels] = {}, *ge2[kLevels] = {},
       *ge1[kLevels] = {};
  float *gskip[kLevels] = {};
  float *gpool = nullptr;  // FP32 gradient of one level's pool output (backward)
  // loss
  float *smap[3] = {};
  double *lpart = nullptr;
  int lpart_n = 0;
  int loss_kind = SC_UNET_LOSS_L1_SSIM;  // sc_unet_set_loss
  float *loss = nullptr;
  // weight-gradient partials
  float *wpart = nullptr;
  size_t wpart_floats = 0;
  int num_sms = 0;
  // the backward pass runs the weight gradients (and their reductions, which share `wpart`) in
  // order on a second stream, forked from the context stream once each layer's output gradient
  // is enqueued and joined before it returns: they are needed only by Adam
  cudaStream_t side = nullptr;
  cudaEvent_t fork[24] = {};
  cudaEvent_t join = nullptr;
};

namespace {

int fail(sc_ctx *c, int code, const std::string &m) {
  if (c) sc::ctx_set_error(c, m);
  return code;
}
int cuda_fail(sc_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, SC_ERR_OOM, std::string(where) + ": out of device memory");
  return fail(c, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// the weight-gradient stream and its events, created on device `dev` (the caller's current device
// is restored); release_streams undoes whatever was created
cudaError_t create_streams(sc_unet *u, int dev) {
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return e;
  if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  e = cudaStreamCreateWithFlags(&u->side, cudaStreamNonBlocking);
  for (cudaEvent_t &ev : u->fork)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&u->join, cudaEventDisableTiming);
  if (prev != dev) cudaSetDevice(prev);
  return e;
}
void release_streams(sc_unet *u) {
  for (cudaEvent_t &ev : u->fork)
    if (ev) cudaEventDestroy(ev);
  if (u->join) cudaEventDestroy(u->join);
  if (u->side) cudaStreamDestroy(u->side);
}

struct Carve {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += a256(count * sizeof(T));
    return p;
  }
};

// flat parameter layout in the order of sc_unet.h
int64_t layout_params(Layer *L) {
  int64_t off = 0;
  auto add = [&](Layer &ly, int kind, int cout, int cin, int64_t wcount) {
    ly.kind = kind;
    ly.cout = cout;
    ly.cin = cin;
    ly.cin_p = (cin + 7) & ~7;
    ly.w_off = off;
    ly.w_count = wcount;
    off += wcount;
    ly.b_off = off;
    off += cout;
  };
  int cin = kInCh;
  for (int l = 0; l < kLevels; ++l) {
    add(L[enc_layer(l, 0)], KIND_CONV, kChans[l], cin, (int64_t)kChans[l] * 9 * cin);
    add(L[enc_layer(l, 1)], KIND_CONV, kChans[l], kChans[l], (int64_t)kChans[l] * 9 * kChans[l]);
    cin = kChans[l];
  }
  for (int l = kLevels - 2; l >= 0; --l) {
    add(L[up_layer(l)], KIND_UP, kChans[l], kChans[l + 1], (int64_t)kChans[l + 1] * 4 * kChans[l]);
    add(L[dec_layer(l, 0)], KIND_CONV, kChans[l], 2 * kChans[l], (int64_t)kChans[l] * 9 * 2 * kChans[l]);
    add(L[dec_layer(l, 1)], KIND_CONV, kChans[l], kChans[l], (int64_t)kChans[l] * 9 * kChans[l]);
  }
  add(L[kOutLayer], KIND_OUT, kOutCh, kChans[0], (int64_t)kOutCh * kChans[0]);
  for (int i = 0; i < kNumLayers; ++i) {
    Layer &ly = L[i];
    if (ly.kind == KIND_CONV) {
      ly.wf_elems = (int64_t)ly.cout * 9 * ly.cin_p;
      ly.wd_elems = ly.cin % 8 == 0 ? (int64_t)ly.cin * 9 * ly.cout : 0;
    } else if (ly.kind == KIND_UP) {
      ly.wf_elems = ly.wd_elems = (int64_t)ly.cin * 4 * ly.cout;
    } else {
      ly.wf_elems = (int64_t)ly.cout * ly.cin;
      ly.wd_elems = 0;
    }
  }
  return off;
}

// weight-gradient GEMM shape of a layer: rows of A (data rows + the ones row), tiles, padded N
Wgrad wgrad_shape(const Layer &ly) {
  Wgrad g;
  if (ly.kind == KIND_CONV) {
    g.rows = 9 * ly.cin_p;
    g.np = pad16(ly.cout);
  } else if (ly.kind == KIND_UP) {
    g.rows = ly.cin;
    g.np = pad16(4 * ly.cout);
  } else {
    g.rows = ly.cin;
    g.np = pad16(ly.cout);
  }
  g.Mtiles = (g.rows + 1 + kTM - 1) / kTM;
  return g;
}
void split_k(int Mtiles, int64_t K, int num_sms, int *splits, int *k_split) {
  int s = (4 * num_sms + Mtiles - 1) / Mtiles;
  const int64_t max_s = (K + 511) / 512;
  if (s > max_s) s = (int)max_s;
  if (s < 1) s = 1;
  int64_t ks = (K + s - 1) / s;
  ks = (ks + kKC - 1) / kKC * kKC;
  *k_split = (int)ks;
  *splits = (int)((K + ks - 1) / ks);
}

int check_geom(int n, int h, int w) { return n >= 1 && h >= 16 && w >= 16 && h % 8 == 0 && w % 8 == 0; }

}  // namespace

// ---------------------------------------------------------------------------------------------
// forward / backward drivers
// ---------------------------------------------------------------------------------------------
namespace {

#define UCHK(expr)                                 \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

ANbr nbr(const bf16 *src, int cs, int co, int h, int w, int cin, int ntaps, int sign, int M) {
  ANbr a;
  a.src = src;
  a.cs = cs;
  a.co = co;
  a.h = h;
  a.w = w;
  a.cin = cin;
  a.ntaps = ntaps;
  a.sign = sign;
  a.M = M;
  return a;
}
BDense dense(const bf16 *W, int ldk, int N) {
  BDense b;
  b.W = W;
  b.ldk = ldk;
  b.N = N;
  return b;
}
EBiasAct bias_act(bf16 *out, int cs, int co, const float *bias, int N, int relu, int w) {
  EBiasAct e;
  e.out = out;
  e.cs = cs;
  e.co = co;
  e.bias = bias;
  e.N = N;
  e.relu = relu;
  e.w = w;
  return e;
}
EGrad egrad(bf16 *out, int ocs, const bf16 *mask, int mcs, int mco, int N, int w) {
  EGrad e;
  e.w = w;
  e.out = out;
  e.ocs = ocs;
  e.oco = 0;
  e.mask = mask;
  e.mcs = mcs;
  e.mco = mco;
  e.N = N;
  e.split = N;
  e.out2 = nullptr;
  e.o2cs = 0;
  return e;
}
TPix tpix(const bf16 *src, int cs, int co, int h, int w, int cin, int ntaps, int mode, int rows, int ones, int R) {
  TPix t;
  t.src = src;
  t.cs = cs;
  t.co = co;
  t.h = h;
  t.w = w;
  t.cin = cin;
  t.ntaps = ntaps;
  t.mode = mode;
  t.rows = rows;
  t.ones = ones;
  t.R = R;
  return t;
}

// the skip tensor of level l (encoder conv 2 output): a slice of the concatenation buffer, or
// its own buffer at the deepest level
struct View {
  bf16 *p;
  int cs, co;
};
View enc_out(const sc_unet *u, int l) {
  if (l == kLevels - 1) return {u->h3, kChans[l], 0};
  return {u->cat[l], 2 * kChans[l], kChans[l]};
}
View up_in(const sc_unet *u, int l) {  // input of the transposed conv that produces level l
  if (l + 1 == kLevels - 1) return {u->h3, kChans[l + 1], 0};
  return {u->d2[l + 1], kChans[l + 1], 0};
}

// ---- 3x3 convolution: TMA halo-tile kernel where the row width allows, gathering GEMM otherwise
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 5-D tensor map of the channel slice [co, co + channels) of a row-blocked BF16 tensor (cs
// channels, rows of w pixels, h rows, n images).  blocked: dims (64, w / 8, groups, h, n) -- the
// innermost 128 bytes are 8 pixels x 8 channels, so a box row of whole 8-pixel blocks is one
// contiguous run -- with box (64, box_w / 8, 1, box_h, 1); otherwise dims (8, w, groups, h, n)
// and box (8, box_w, 1, box_h, 1) for boxes that start at any pixel.
bool encode_rb_map(CUtensorMap *map, const bf16 *src, int co, int channels, int cs, int w, int h, int n, bool blocked,
                   int box_w, int box_h) {
  const cuuint64_t e0 = blocked ? 64 : 8;
  const cuuint64_t row = (cuuint64_t)cs * w * 2;  // bytes of one image row, all channel groups
  const cuuint64_t dims[5] = {e0, (cuuint64_t)(blocked ? w / 8 : w), (cuuint64_t)(channels / 8), (cuuint64_t)h,
                              (cuuint64_t)n};
  const cuuint64_t strides[4] = {e0 * 2, (cuuint64_t)w * 16, row, row * h};
  const cuuint32_t box[5] = {(cuuint32_t)e0, (cuuint32_t)(blocked ? box_w / 8 : box_w), 1, (cuuint32_t)box_h, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  auto enc = tensor_map_encoder();
  return enc && enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(src + (int64_t)co * w), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A row-blocked BF16 slice (cs channels, slice at co, `channels` of them) seen with 8-byte elements
// (half a pixel's 8 channels) as (2 w, h, channel groups, n, 1), box (2 box_w, box_h, box_g, 1, 1):
// a one-pixel shift is an element offset of 2 (16 bytes), and one copy brings box_g channel groups
// of box_h rows of box_w pixels, each group's pixels contiguous (box_h box_w x 16 bytes).
bool encode_px_map(CUtensorMap *map, const bf16 *src, int co, int channels, int cs, int w, int h, int n, int box_w,
                   int box_h, int box_g) {
  const cuuint64_t row = (cuuint64_t)cs * w * 2;
  const cuuint64_t dims[5] = {(cuuint64_t)2 * w, (cuuint64_t)h, (cuuint64_t)(channels / 8), (cuuint64_t)n, 1};
  const cuuint64_t strides[4] = {row, (cuuint64_t)w * 16, row * h, row * h * n};
  const cuuint32_t box[5] = {(cuuint32_t)(2 * box_w), (cuuint32_t)box_h, (cuuint32_t)box_g, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  auto enc = tensor_map_encoder();
  return enc && enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<bf16 *>(src + (int64_t)co * w), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The output gradient of a 2x2 stride-2 transposed conv (row-blocked BF16, cs channels, rows of wc
// pixels, hc rows per image) seen as (2 half-pixels, pixel parity e, parent column, row, channel
// group) with 8-byte elements: one copy with e and the row parity a fixed brings, for bw parent
// columns of th parent rows (rows 2y + a, a row stride of 2), the children (2y + a, 2x + e) of
// box_g channel groups, each group's 128 children contiguous.
bool encode_parity_map(CUtensorMap *map, const bf16 *src, int channels, int cs, int wc, int hc, int n, int bw, int th,
                       int box_g) {
  const cuuint64_t dims[5] = {2, 2, (cuuint64_t)(wc / 2), (cuuint64_t)n * hc, (cuuint64_t)(channels / 8)};
  const cuuint64_t strides[4] = {16, 32, (cuuint64_t)cs * wc * 2, (cuuint64_t)wc * 16};
  const cuuint32_t box[5] = {2, 1, (cuuint32_t)bw, (cuuint32_t)(th > 1 ? 2 * th : 1), (cuuint32_t)box_g};
  const cuuint32_t estr[5] = {1, 1, 1, (cuuint32_t)(th > 1 ? 2 : 1), 1};
  auto enc = tensor_map_encoder();
  return enc && enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<bf16 *>(src), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// groups of 8 input channels per A stage (0: the layer does not fit in 227 KB next to its
// resident weights).  Among the even divisors of cin / 8 that fit, the one that lets the most CTAs
// share an SM (shared memory, TMEM, at most 4 by registers) when SC_CONV_MAXOCC, else the largest;
// ties go to the larger (fewer chunks per tile).  More co-resident CTAs overlap one CTA's loads
// with another's MMAs and epilogue, which pays more than fewer chunks per tile.
#ifndef SC_CONV_MAXOCC
#define SC_CONV_MAXOCC 1
#endif
int conv_stage_groups(int cin, int N, uint32_t gstride, int taps = 9) {
  const int ng = cin / 8;
  int best = 0, best_occ = 0;
  for (int gs = ng; gs >= 2; gs -= 2) {
    const int bytes = (int)conv_smem_bytes(cin, N, gs, gstride, taps);
    if (ng % gs != 0 || bytes > 227 * 1024) continue;
    if (!SC_CONV_MAXOCC) return gs;
    const int occ = std::min(std::min(228 * 1024 / (bytes + 1024), 512 / (2 * (int)conv_acc_cols(N))), 4);
    if (occ > best_occ) {
      best = gs;
      best_occ = occ;
    }
  }
  return best;
}

bool conv_rows_ok(int w, int h) {
  if (w % 128 == 0) return true;
  return w >= 16 && w < 128 && 128 % w == 0 && h % (128 / w) == 0;
}

// taps 9: 3x3 convolution (N <= 128); taps 1: pointwise (N <= 256, two 256-column accumulators)
bool conv_tma_ok(int cin, int N, int w, int h, int taps = 9) {
  return conv_rows_ok(w, h) && cin % 16 == 0 && N % 16 == 0 && N <= (taps == 1 ? 256 : 128) &&
         conv_stage_groups(cin, N, conv_geo(1, h, w, taps).gstride, taps) > 0 && tensor_map_encoder() != nullptr;
}

// Output columns [off, off + n) of a convolution's epilogue (the n-split TMA path).
template <class EP>
struct ColSplit {
  static constexpr bool ok = false;
  static EP shift(const EP &e, int, int) { return e; }
};
template <>
struct ColSplit<EBiasAct> {
  static constexpr bool ok = true;
  static EBiasAct shift(EBiasAct e, int off, int n) {
    e.co += off;
    e.bias += off;
    e.N = n;
    return e;
  }
};
template <>
struct ColSplit<EGrad> {  // BF16 columns only (split == N)
  static constexpr bool ok = true;
  static EGrad shift(EGrad e, int off, int n) {
    e.oco += off;
    e.mco += off;
    e.N = n;
    e.split = n;
    return e;
  }
};
bool col_splittable(const EBiasAct &, int) { return true; }
bool col_splittable(const EGrad &e, int N) { return e.split == N && !e.out2; }

template <class EP>
cudaError_t conv3x3_tma(sc_unet *u, const bf16 *src, int cs, int co, int cin, int h, int w, int n, int N,
                        const bf16 *wtma, int sign, const EP &e, unsigned *st, cudaStream_t s, int taps = 9,
                        int up_ngc = 0);

// src: row-blocked BF16 slice (cs channels, slice at co) with `cin` channels per tap; N output
// channels; wdense: [N][9][cin] (gathering GEMM), wtma: [tap][cin/8][N][8] (TMA kernel), wtma2:
// the same in two halves of N (or null), used when the whole weights do not fit next to the
// stages but half of them do; sign -1 = data gradient
template <class EP>
cudaError_t conv3x3(sc_unet *u, const bf16 *src, int cs, int co, int cin, int h, int w, int n, int N,
                    const bf16 *wdense, const bf16 *wtma, const bf16 *wtma2, int sign, const EP &e, unsigned *st,
                    cudaStream_t s) {
  const int M = n * h * w;
  if (conv_tma_ok(cin, N, w, h)) return conv3x3_tma(u, src, cs, co, cin, h, w, n, N, wtma, sign, e, st, s);
  if (ColSplit<EP>::ok && wtma2 && N % 32 == 0 && col_splittable(e, N) && conv_tma_ok(cin, N / 2, w, h)) {
    for (int hf = 0; hf < 2; ++hf) {
      const cudaError_t err = conv3x3_tma(u, src, cs, co, cin, h, w, n, N / 2, wtma2 + (size_t)hf * 9 * cin * (N / 2),
                                          sign, ColSplit<EP>::shift(e, hf * (N / 2), N / 2), st, s);
      if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
  }
  return gemm(nbr(src, cs, co, h, w, cin, 9, sign, M), dense(wdense, 9 * cin, N), e, M, N, 9 * cin, 1, 9 * cin, st,
              s);
}

// The TMA kernel for a 3x3 convolution (taps 9) or a pointwise contraction of each pixel's
// channels (taps 1; wtma [cin/8][N][8]).  up_ngc > 0: the data gradient of a 2x2 stride-2
// transposed conv, src = its output gradient at the children's resolution (2h x 2w, cs channels,
// up_ngc groups of 8), h x w the parents', cin = 4 * 8 up_ngc, wtma [(a, e, o) group][N][8].
template <class EP>
cudaError_t conv3x3_tma(sc_unet *u, const bf16 *src, int cs, int co, int cin, int h, int w, int n, int N,
                        const bf16 *wtma, int sign, const EP &e, unsigned *st, cudaStream_t s, int taps, int up_ngc) {
  CUtensorMap map;
  ConvGeo G = conv_geo(n, h, w, taps);
  G.up = up_ngc > 0 ? 1 : 0;
  G.ngc = up_ngc;
  const bool mapped = up_ngc > 0 ? encode_parity_map(&map, src, 8 * up_ngc, cs, 2 * w, 2 * h, n, G.narrow ? w : 128,
                                                     G.th, 1)
                      : taps == 1 ? encode_rb_map(&map, src, co, cin, cs, w, h, n, true, G.narrow ? w : 128, G.th)
                      : G.narrow ? encode_rb_map(&map, src, co, cin, cs, w, h, n, false, w, G.th + 2)
                                 : encode_rb_map(&map, src, co, cin, cs, w, h, n, true, kHaloW, kHaloH);
  if (!mapped) return cudaErrorInvalidValue;
  auto kern = k_conv_tma<EP>;
  const int gs = conv_stage_groups(cin, N, G.gstride, taps);
  const int smem = (int)conv_smem_bytes(cin, N, gs, G.gstride, taps);
  static std::mutex mu;
  static bool attr_set[kMaxDev] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr_set[dev]) {
      cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (err == cudaSuccess)
        err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
      if (err != cudaSuccess) return err;
      attr_set[dev] = true;
    }
  }
  // CTAs resident per SM: shared memory, registers and threads, capped by TMEM (the dynamic
  // shared memory is padded so that no more than the TMEM cap can ever be co-resident)
  cudaFuncAttributes fa;
  cudaError_t err = cudaFuncGetAttributes(&fa, kern);
  if (err != cudaSuccess) return err;
  const int cols = 2 * (int)conv_acc_cols(N);
  const int by_tmem = 512 / cols;
  const int regs = ((fa.numRegs + 7) / 8) * 8 * kConvThreads;
  const int by_regs = regs > 0 ? 65536 / regs : 1;
  const int kSmemPerSM = 228 * 1024, kSmemPerBlockReserve = 1024;
  int smem_launch = smem;
  if (kSmemPerSM / (smem_launch + kSmemPerBlockReserve) > by_tmem)
    smem_launch = kSmemPerSM / (by_tmem + 1) - kSmemPerBlockReserve + 16;
  const int by_smem = kSmemPerSM / (smem_launch + kSmemPerBlockReserve);
  int occ = std::min(std::min(by_smem, by_regs), std::min(by_tmem, 2048 / kConvThreads));
  if (occ < 1) occ = 1;
  const int ntiles = G.narrow ? n * (h / G.th) : n * h * (w / 128);
  const int grid = std::min(ntiles, u->num_sms * occ);
  kern<<<grid, kConvThreads, smem_launch, s>>>(map, wtma, cin, N, gs, G, sign, e, st);
  return cudaGetLastError();
}

int run_forward(sc_ctx *c, sc_unet *u, const float *x, int n) {
  const char *where = "sc_unet_forward";
  cudaStream_t s = sc::ctx_stream(c);
  unsigned *st = sc::ctx_status(c);
  u->n = n;
  int64_t P[kLevels];
  for (int l = 0; l < kLevels; ++l) P[l] = (int64_t)n * u->hl[l] * u->wl[l];
  k_pack_input<<<(unsigned)((P[0] + 255) / 256), 256, 0, s>>>(x, u->x0, P[0], u->wl[0]);
  UCHK(cudaGetLastError());
  const float *prm = u->params;
  for (int l = 0; l < kLevels; ++l) {
    const int h = u->hl[l], w = u->wl[l], cl = kChans[l];
    const Layer &c1 = u->L[enc_layer(l, 0)], &c2 = u->L[enc_layer(l, 1)];
    const bf16 *src = l == 0 ? u->x0 : u->pool[l];
    const int scs = l == 0 ? kInPad : kChans[l - 1];
    UCHK(conv3x3(u, src, scs, 0, c1.cin_p, h, w, n, cl, c1.wf, c1.wtf, c1.wtf2, 1,
                 bias_act(u->a1[l], cl, 0, prm + c1.b_off, cl, 1, w), st, s));
    const View e = enc_out(u, l);
    UCHK(conv3x3(u, u->a1[l], cl, 0, cl, h, w, n, cl, c2.wf, c2.wtf, c2.wtf2, 1,
                 bias_act(e.p, e.cs, e.co, prm + c2.b_off, cl, 1, w), st, s));
    if (l + 1 < kLevels) {
      const int64_t tot = P[l + 1] * (cl / 8);
      k_pool<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(e.p, e.cs, e.co, cl, n, h, w, u->pool[l + 1]);
      UCHK(cudaGetLastError());
    }
  }
  for (int l = kLevels - 2; l >= 0; --l) {
    const int h = u->hl[l], w = u->wl[l], cl = kChans[l], cn = kChans[l + 1];
    const Layer &up = u->L[up_layer(l)], &c1 = u->L[dec_layer(l, 0)], &c2 = u->L[dec_layer(l, 1)];
    const View ui = up_in(u, l);
    EUpFwd eu;
    eu.out = u->cat[l];
    eu.cs = 2 * cl;
    eu.co = 0;
    eu.bias = prm + up.b_off;
    eu.cu = cl;
    eu.h = u->hl[l + 1];
    eu.w = u->wl[l + 1];
    if (conv_tma_ok(cn, 4 * cl, u->wl[l + 1], u->hl[l + 1], 1))
      UCHK(conv3x3_tma(u, ui.p, ui.cs, ui.co, cn, u->hl[l + 1], u->wl[l + 1], n, 4 * cl, up.wtf, 1, eu, st, s, 1));
    else
      UCHK(gemm(nbr(ui.p, ui.cs, ui.co, u->hl[l + 1], u->wl[l + 1], cn, 1, 1, (int)P[l + 1]),
                dense(up.wf, cn, 4 * cl), eu, (int)P[l + 1], 4 * cl, cn, 1, cn, st, s));
    UCHK(conv3x3(u, u->cat[l], 2 * cl, 0, 2 * cl, h, w, n, cl, c1.wf, c1.wtf, c1.wtf2, 1,
                 bias_act(u->d1[l], cl, 0, prm + c1.b_off, cl, 1, w), st, s));
    UCHK(conv3x3(u, u->d1[l], cl, 0, cl, h, w, n, cl, c2.wf, c2.wtf, c2.wtf2, 1,
                 bias_act(u->d2[l], cl, 0, prm + c2.b_off, cl, 1, w), st, s));
  }
  const Layer &o = u->L[kOutLayer];
  k_out_fwd<<<(unsigned)((P[0] + kOutBlock - 1) / kOutBlock), kOutBlock, 0, s>>>(u->d2[0], u->wl[0], P[0], o.wf,
                                                                                 prm + o.b_off, u->y);
  UCHK(cudaGetLastError());
  return SC_OK;
}

int run_loss(sc_ctx *c, sc_unet *u, const float *pred, const float *target, int n, int h, int w, float *loss,
             float *grad, bf16 *gy8, const char *where) {
  cudaStream_t s = sc::ctx_stream(c);
  if (u->loss_kind == SC_UNET_LOSS_BCE || u->loss_kind == SC_UNET_LOSS_L2_LINEAR) {
    const int64_t n_px = (int64_t)n * h * w;
    const int nb = (int)((n_px + 255) / 256);
    if (nb > u->lpart_n) return fail(c, SC_ERR_INVALID_ARG, std::string(where) + ": loss workspace too small");
    if (u->loss_kind == SC_UNET_LOSS_BCE) {
      k_bce<<<nb, 256, 0, s>>>(pred, target, n_px, (float)(1.0 / (double)n_px), grad, gy8, u->lpart);
      UCHK(cudaGetLastError());
      k_bce_final<<<1, 256, 0, s>>>(u->lpart, nb, (double)n_px, loss);
    } else {
      k_l2lin<<<nb, 256, 0, s>>>(pred, target, n_px, (float)(1.0 / (3.0 * (double)n_px)), grad, gy8, u->lpart);
      UCHK(cudaGetLastError());
      k_bce_final<<<1, 256, 0, s>>>(u->lpart, nb, 3.0 * (double)n_px, loss);
    }
    UCHK(cudaGetLastError());
    return SC_OK;
  }
  const int Hv = h - 10, Wv = w - 10;
  dim3 gf((Wv + kSTW - 1) / kSTW, (Hv + kSTH - 1) / kSTH, n);
  dim3 gb((w + kSTW - 1) / kSTW, (h + kSTH - 1) / kSTH, n);
  const int nf = (int)(gf.x * gf.y * gf.z), nb = (int)(gb.x * gb.y * gb.z);
  if (nf + nb > u->lpart_n) return fail(c, SC_ERR_INVALID_ARG, std::string(where) + ": loss workspace too small");
  double *pf = u->lpart, *pb = u->lpart + nf;
  k_ssim_fwd<<<gf, 256, 0, s>>>(pred, target, h, w, u->smap[0], u->smap[1], u->smap[2], pf);
  UCHK(cudaGetLastError());
  const double n_px = (double)n * h * w * 3, n_win = (double)n * Hv * Wv * 3;
  k_ssim_bwd<<<gb, 256, 0, s>>>(pred, target, h, w, u->smap[0], u->smap[1], u->smap[2], (float)(1.0 / n_px),
                                (float)(1.0 / n_win), grad, gy8, pb);
  UCHK(cudaGetLastError());
  k_loss_final<<<1, 256, 0, s>>>(pf, nf, pb, nb, n_px, n_win, loss);
  UCHK(cudaGetLastError());
  return SC_OK;
}

// ring slots of the MN-major weight-gradient kernel that fit next to its two gz tiles at `ctas`
// CTAs per SM.  Rows of 128k pixels run two CTAs per SM (two or three slots each): the copies of
// one CTA are served about one after another, so two CTAs stream nearly twice the bytes (2.25 ->
// 2.08 ms per 16 x 256^2 step, e.g. 105 -> 70 us for a 32 -> 32 layer); narrow rows, with few tiles
// per CTA and more TMEM chunks at two CTAs, keep one CTA per SM with more slots.
#ifndef SC_WG_MN_CTAS
#define SC_WG_MN_CTAS 2
#endif
int wgrad_mn_slots(int cout, int ctas) {
  const int budget = ctas == 1 ? 227 * 1024 : 228 * 1024 / ctas - 1024;  // 1 KB per CTA is the system's
  for (int s = kMnMaxSlots; s >= 2; --s)
    if ((int)mn_smem_bytes(cout, s) <= budget) return s;
  return 0;
}

// weight gradient of one layer: A (rows = (tap, c) | c, + ones row), B (rows = output channels),
// contracted over the pixels, reduced deterministically into the flat gradient.  3x3 layers on
// rows of 128k pixels (or 128 / w whole rows) with at least 64 tiles take the MN-major TMA kernel
// (x: the layer input, gz: its output gradient), everything else the gathering GEMM.
int wgrad(sc_ctx *c, sc_unet *u, const Layer &ly, const TPix &A, const TPix &B, int64_t K, cudaStream_t ws,
          RedTable &red, int &red_blocks) {
  const char *where = "sc_unet wgrad";
  float *part = u->wpart + ly.part_off;
  const Wgrad g = wgrad_shape(ly);
  const int Mpad = g.Mtiles * kTM;
  const ConvGeo G = conv_geo((int)(K / ((int64_t)A.h * A.w)), A.h, A.w);
  const int64_t tiles = K / 128;
  const bool tma_ok = ly.kind == KIND_CONV && A.mode == 0 && A.ntaps == 9 && conv_rows_ok(A.w, A.h) && B.co == 0 &&
                      B.cs == ly.cout && A.cin * 9 == g.rows && tensor_map_encoder() != nullptr;
  // the transposed conv (A: its input at the parents' resolution; B: the children's gradients)
  const bool up_ok = ly.kind == KIND_UP && A.mode == 0 && A.ntaps == 1 && conv_rows_ok(A.w, A.h) && B.co == 0 &&
                     B.cs == ly.cout && A.cin == g.rows && 4 * ly.cout <= 256 && tensor_map_encoder() != nullptr;
  const int Nmn = up_ok ? 4 * ly.cout : ly.cout;  // accumulator columns
  const int mctas = A.w >= 128 && SC_WG_MN_CTAS > 1 && wgrad_mn_slots(Nmn, SC_WG_MN_CTAS) > 0 ? SC_WG_MN_CTAS : 1;
  const int mslots = (tma_ok || up_ok) && tiles >= 64 ? wgrad_mn_slots(Nmn, mctas) : 0;
  // the MN-major kernel's row layout (columns on rows of 128k pixels with at most 48 input
  // channels) sets the partials' rows
  const MnLayout L = up_ok ? mn_layout_up(A.cin) : mn_layout(A.cin, A.w >= 128 && A.cin <= 48);
  const int seg_Mpad = mslots > 0 ? L.mtiles * kTM : Mpad;
  const int seg_rows = mslots > 0 ? 8 * L.jones : g.rows;
  int splits;
  if (mslots > 0) {
    const int n_img = G.n_img;
    const int ntiles = G.narrow ? n_img * (A.h / G.th) : n_img * A.h * (A.w / 128);
    splits = std::min(ntiles, u->num_sms * mctas);
    if ((size_t)splits * seg_Mpad * g.np > ly.part_floats)
      return fail(c, SC_ERR_INVALID_ARG, "sc_unet: weight-gradient workspace too small");
    CUtensorMap xm, gm;
    // x: a column copy (3 rows of L.gb channel groups) or L.gb groups of one tap (a tap's shift is an
    // element offset); gz: the whole tile
    const int bw = G.narrow ? A.w : 128;
    const bool gok = up_ok ? encode_parity_map(&gm, B.src, ly.cout, ly.cout, 2 * A.w, 2 * A.h, n_img, bw, G.th,
                                               ly.cout / 8)
                           : encode_px_map(&gm, B.src, 0, ly.cout, ly.cout, A.w, A.h, n_img, bw, G.th, ly.cout / 8);
    if (!encode_px_map(&xm, A.src, A.co, A.cin, A.cs, A.w, A.h, n_img, bw, L.col ? 3 : G.th, L.gb) || !gok)
      return fail(c, SC_ERR_CUDA, "sc_unet wgrad: tensor map encoding failed");
    const int smem = (int)mn_smem_bytes(Nmn, mslots);
    static bool attr[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (dev >= 0 && dev < kMaxDev && !attr[dev]) {
        UCHK(cudaFuncSetAttribute(k_wgrad_mn<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        UCHK(cudaFuncSetAttribute(k_wgrad_mn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr[dev] = true;
      }
    }
    // 128-row blocks per CTA: as many accumulators as fit in TMEM, in balanced chunks
    const int per = 512 / mctas / (int)wg_cstride(Nmn);
    const int nchunk = (L.mtiles + per - 1) / per;
    const int mchunk = (L.mtiles + nchunk - 1) / nchunk;
    auto kern = G.narrow ? k_wgrad_mn<true> : k_wgrad_mn<false>;
    kern<<<dim3(splits, nchunk), kMnThreads, smem, ws>>>(xm, gm, A.cin, Nmn, L.mtiles, mchunk, mslots, L, G, part,
                                                         sc::ctx_status(c));
    UCHK(cudaGetLastError());
  } else {
    int ks;
    split_k(g.Mtiles, K, u->num_sms, &splits, &ks);
    if ((size_t)splits * Mpad * g.np > ly.part_floats)
      return fail(c, SC_ERR_INVALID_ARG, "sc_unet: weight-gradient workspace too small");
    EPartial ep;
    ep.part = part;
    ep.ld = g.np;
    ep.Mpad = Mpad;
    const int N = ly.kind == KIND_UP ? 4 * ly.cout : ly.cout;
    UCHK(gemm(A, B, ep, g.rows + 1, N, (int)K, splits, ks, sc::ctx_status(c), ws));
  }
  // the reduction of this layer's partials joins the pass's single reduce launch
  if (red.n >= kMaxRedSegs) return fail(c, SC_ERR_INVALID_ARG, "sc_unet: too many weight-gradient segments");
  RedSeg &sg = red.s[red.n++];
  sg.part_off = (int64_t)ly.part_off;
  sg.w_off = ly.w_off;
  sg.b_off = ly.b_off;
  sg.splits = splits;
  sg.Mpad = seg_Mpad;
  sg.np = g.np;
  sg.rows = seg_rows;
  sg.col = mslots > 0 ? L.col : 0;
  sg.cgb = L.gb;
  sg.nu = L.nu;
  sg.cpb = L.cpb;
  sg.ncopy = L.ncopy;
  sg.kind = ly.kind;
  sg.cout = ly.cout;
  sg.cin = ly.cin;
  sg.cin_p = ly.cin_p;
  sg.first_block = red_blocks;
  red_blocks += (int)(((int64_t)(seg_rows + 1) * g.np + kRedBlockEntries - 1) / kRedBlockEntries);
  UCHK(cudaGetLastError());
  return SC_OK;
}

int backward_body(sc_ctx *c, sc_unet *u) {
  const char *where = "sc_unet backward";
  cudaStream_t s = sc::ctx_stream(c);
  cudaStream_t ws = u->side;
  unsigned *st = sc::ctx_status(c);
  const int n = u->n;
  int64_t P[kLevels];
  for (int l = 0; l < kLevels; ++l) P[l] = (int64_t)n * u->hl[l] * u->wl[l];
  int rc;
  RedTable red;
  red.n = 0;
  int red_blocks = 0;
  // the side stream waits for everything enqueued on the context stream so far
  int nfork = 0;
  auto fork = [&]() -> cudaError_t {
    if (nfork >= (int)(sizeof(u->fork) / sizeof(u->fork[0]))) return cudaErrorInvalidValue;
    cudaError_t e = cudaEventRecord(u->fork[nfork], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ws, u->fork[nfork], 0);
    ++nfork;
    return e;
  };
  // output layer: weight and bias gradient (two fixed-order stages), data gradient into gd2[0]
  {
    const Layer &o = u->L[kOutLayer];
    const int w0 = u->wl[0];
    const int nblk = 2 * u->num_sms;
    if ((size_t)nblk * kOutParts > o.part_floats)
      return fail(c, SC_ERR_INVALID_ARG, "sc_unet: weight-gradient workspace too small");
    const int64_t span = (P[0] + nblk - 1) / nblk;
    UCHK(fork());
    float *opart = u->wpart + o.part_off;
    k_out_wgrad<<<nblk, kOutBlock, 0, ws>>>(u->gy8, u->d2[0], w0, P[0], span, opart);
    UCHK(cudaGetLastError());
    k_out_wgrad_final<<<kOutParts, 128, 0, ws>>>(opart, nblk, u->grads + o.w_off, u->grads + o.b_off);
    UCHK(cudaGetLastError());
    k_out_dgrad<<<(unsigned)((P[0] + kOutBlock - 1) / kOutBlock), kOutBlock, 0, s>>>(u->gy8, u->d2[0], w0, P[0],
                                                                                   o.wf, u->gd2[0]);
    UCHK(cudaGetLastError());
  }
  // decoder, shallow to deep
  for (int l = 0; l < kLevels - 1; ++l) {
    const int h = u->hl[l], w = u->wl[l], cl = kChans[l], cn = kChans[l + 1];
    const Layer &c2 = u->L[dec_layer(l, 1)], &c1 = u->L[dec_layer(l, 0)], &up = u->L[up_layer(l)];
    // dec conv 2: input d1, output gradient gd2
    UCHK(fork());
    rc = wgrad(c, u, c2, tpix(u->d1[l], cl, 0, h, w, cl, 9, 0, 9 * cl, 1, kTM),
               tpix(u->gd2[l], cl, 0, h, w, cl, 1, 0, cl, 0, pad16(cl)), P[l], ws, red, red_blocks);
    if (rc) return rc;
    UCHK(conv3x3(u, u->gd2[l], cl, 0, cl, h, w, n, cl, c2.wd, c2.wtd, c2.wtd2, -1, egrad(u->gd1[l], cl, u->d1[l], cl, 0, cl, w),
                 st, s));
    // dec conv 1: input cat = [up, skip], output gradient gd1 -> gup (BF16) | gskip (FP32)
    UCHK(fork());
    rc = wgrad(c, u, c1, tpix(u->cat[l], 2 * cl, 0, h, w, 2 * cl, 9, 0, 18 * cl, 1, kTM),
               tpix(u->gd1[l], cl, 0, h, w, cl, 1, 0, cl, 0, pad16(cl)), P[l], ws, red, red_blocks);
    if (rc) return rc;
    EGrad es = egrad(u->gup[l], cl, nullptr, 0, 0, 2 * cl, w);
    es.split = cl;
    es.out2 = u->gskip[l];
    es.o2cs = cl;
    UCHK(conv3x3(u, u->gd1[l], cl, 0, cl, h, w, n, 2 * cl, c1.wd, c1.wtd, c1.wtd2, -1, es, st, s));
    // transposed conv: input up_in (level l+1), output gradient gup (level l)
    const View ui = up_in(u, l);
    const int hn = u->hl[l + 1], wn = u->wl[l + 1];
    UCHK(fork());
    rc = wgrad(c, u, up, tpix(ui.p, ui.cs, ui.co, hn, wn, cn, 1, 0, cn, 1, kTM),
               tpix(u->gup[l], cl, 0, hn, wn, cl, 4, 1, 4 * cl, 0, pad16(4 * cl)), P[l + 1], ws, red, red_blocks);
    if (rc) return rc;
    AUpGrad ag;
    ag.g = u->gup[l];
    ag.gcs = cl;
    ag.h = hn;
    ag.w = wn;
    ag.cu = cl;
    ag.M = (int)P[l + 1];
    // gradient w.r.t. up_in, masked by its ReLU: the next decoder conv 2's output gradient,
    // or at the deepest level the encoder's last conv output gradient
    bf16 *dst = l + 1 == kLevels - 1 ? u->ge2[l + 1] : u->gd2[l + 1];
    const EGrad eu = egrad(dst, cn, ui.p, ui.cs, ui.co, cn, wn);
    if (conv_tma_ok(4 * cl, cn, wn, hn, 1)) {
      // the TMA convolution's pointwise mode over the children (K = (a, e, output channel))
      UCHK(conv3x3_tma(u, u->gup[l], cl, 0, 4 * cl, hn, wn, n, cn, up.wtd, 1, eu, st, s, 1, cl / 8));
    } else {
      UCHK(gemm(ag, dense(up.wd, 4 * cl, cn), eu, (int)P[l + 1], cn, 4 * cl, 1, 4 * cl, st, s));
    }
  }
  // encoder, deep to shallow; ge2[l] holds d loss / d (pre-ReLU) encoder conv 2 output
  for (int l = kLevels - 1; l >= 0; --l) {
    const int h = u->hl[l], w = u->wl[l], cl = kChans[l];
    const Layer &c2 = u->L[enc_layer(l, 1)], &c1 = u->L[enc_layer(l, 0)];
    UCHK(fork());
    rc = wgrad(c, u, c2, tpix(u->a1[l], cl, 0, h, w, cl, 9, 0, 9 * cl, 1, kTM),
               tpix(u->ge2[l], cl, 0, h, w, cl, 1, 0, cl, 0, pad16(cl)), P[l], ws, red, red_blocks);
    if (rc) return rc;
    UCHK(conv3x3(u, u->ge2[l], cl, 0, cl, h, w, n, cl, c2.wd, c2.wtd, c2.wtd2, -1, egrad(u->ge1[l], cl, u->a1[l], cl, 0, cl, w),
                 st, s));
    const bf16 *src = l == 0 ? u->x0 : u->pool[l];
    const int scs = l == 0 ? kInPad : kChans[l - 1];
    UCHK(fork());
    rc = wgrad(c, u, c1, tpix(src, scs, 0, h, w, c1.cin_p, 9, 0, 9 * c1.cin_p, 1, kTM),
               tpix(u->ge1[l], cl, 0, h, w, cl, 1, 0, cl, 0, pad16(cl)), P[l], ws, red, red_blocks);
    if (rc) return rc;
    if (l > 0) {
      // the gradient of the pool output (FP32), then through the pool into the level above, plus
      // its skip gradient, times its ReLU mask
      const int cp = kChans[l - 1];
      const View e = enc_out(u, l - 1);
      EGrad eg = egrad(nullptr, cp, nullptr, 0, 0, cp, w);
      eg.split = 0;
      eg.out2 = u->gpool;
      eg.o2cs = cp;
      UCHK(conv3x3(u, u->ge1[l], cl, 0, cl, h, w, n, cp, c1.wd, c1.wtd, c1.wtd2, -1, eg, st, s));
      const int64_t tot = P[l] * (cp / 8);
      k_pool_back<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(u->gpool, cp, e.p, e.cs, e.co, u->gskip[l - 1], cp,
                                                              u->ge2[l - 1], n, h, w);
      UCHK(cudaGetLastError());
    }
  }
  // every layer's split-K partials, reduced in one launch on the weight-gradient stream
  if (red.n > 0) {
    k_wgrad_reduce<<<(unsigned)red_blocks, kRedEntries * kRedGroups, 0, ws>>>(red, u->wpart, u->grads);
    UCHK(cudaGetLastError());
  }
  return SC_OK;
}

// the backward pass, then the context stream waits for the weight-gradient stream (also after
// an error, so that no work of this call is left unordered with the next one)
int run_backward(sc_ctx *c, sc_unet *u) {
  const char *where = "sc_unet backward";
  const int rc = backward_body(c, u);
  cudaError_t e = cudaEventRecord(u->join, u->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sc::ctx_stream(c), u->join, 0);
  if (rc) return rc;
  UCHK(e);
  return SC_OK;
}

int refresh_bf16(sc_ctx *c, sc_unet *u, int update, float lr) {
  const char *where = "sc_unet params";
  double bc1 = 1.0, bc2 = 1.0;
  if (update) {
    bc1 = 1.0 - std::pow(0.9, (double)u->step);
    bc2 = 1.0 - std::pow(0.999, (double)u->step);
  }
  k_adam<<<u->adam_blocks, 256, 0, sc::ctx_stream(c)>>>(u->segs, u->nseg, u->params, u->grads, u->adam_m, u->adam_v,
                                                          lr, (float)bc1, (float)bc2, update);
  UCHK(cudaGetLastError());
  return SC_OK;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Self-test of the abort protocol the tensor-core kernels share.  One CTA of four warps in the
// conv kernel's roles: the producer (warp 0) has a bulk copy in flight, the MMA issuer (warp 1)
// one MMA (A = B = ones, 128 x 32 x 16, so every accumulator entry becomes 16), and then each
// role, the two epilogue warps too, waits on barrier `never`, which nothing arrives at.  Each wait
// gives up after `limit` polls and raises the abort flag; the producer then waits (bounded) for
// its copy and the issuer commits its MMA to the drain barrier and waits for it, as in
// k_conv_tma; warp 1 reads the drained accumulator back before the CTA frees its TMEM, and
// thread 0 latches the watchdog bit.  out[8]: see sc_unet_wait_selftest.
__global__ void __launch_bounds__(128) k_wait_selftest(const uint4 *src, uint32_t limit, int64_t *out,
                                                       unsigned *status) {
  __shared__ __align__(1024) uint8_t sA[128 * 16 * 2];
  __shared__ __align__(1024) uint8_t sB[32 * 16 * 2];
  __shared__ __align__(128) uint4 sC[64];
  __shared__ __align__(8) uint64_t bar[4];  // [0] copy full, [1] never, [2] drain, [3] never (epilogue)
  __shared__ uint32_t slot;
  __shared__ int abort_flag, epi_gave_up;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t one2 = 0x3F803F80u;  // two BF16 ones
  for (int i = threadIdx.x; i < (int)(sizeof(sA) / 4); i += blockDim.x) reinterpret_cast<uint32_t *>(sA)[i] = one2;
  for (int i = threadIdx.x; i < (int)(sizeof(sB) / 4); i += blockDim.x) reinterpret_cast<uint32_t *>(sB)[i] = one2;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) sc::tc::mbar_init(sc::tc::smem_addr(&bar[i]), 1);
    abort_flag = 0;
    epi_gave_up = 0;
  }
  if (warp == 1) {
    sc::tc::tmem_alloc(sc::tc::smem_addr(&slot), 32);
    sc::tc::tmem_relinquish();
  }
  sc::tc::fence_async_smem();
  sc::tc::fence_before();
  __syncthreads();
  sc::tc::fence_after();
  const uint32_t taddr = slot;
  volatile int *ab = &abort_flag;
  if (warp == 0) {
    if (lane == 0) {
      sc::tc::mbar_expect_tx(sc::tc::smem_addr(&bar[0]), sizeof(sC));
      sc::tc::bulk_load(sc::tc::smem_addr(sC), src, sizeof(sC), sc::tc::smem_addr(&bar[0]));
      const bool got = sc::tc::mbar_wait(sc::tc::smem_addr(&bar[1]), 0, limit);
      if (!got) *ab = 1;
      out[0] = got ? 0 : 1;
      out[1] = sc::tc::mbar_wait(sc::tc::smem_addr(&bar[0]), 0) ? 1 : 0;  // the copy in flight, drained
    }
    __syncwarp();
    bool same = true;
    for (int i = lane; i < 64; i += 32) {
      const uint4 a = sC[i], b = src[i];
      same &= a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
    }
    same = __all_sync(0xffffffffu, same);
    if (lane == 0) out[6] = same ? 1 : 0;
  } else if (warp == 1) {
    int drained = 0;
    if (lane == 0) {
      // K-major, no swizzle: core matrices along K 128 bytes apart, along M / N 256 bytes apart
      const uint64_t ad = sc::tc::smem_desc(sc::tc::smem_addr(sA), 128u, 256u);
      const uint64_t bd = sc::tc::smem_desc(sc::tc::smem_addr(sB), 128u, 256u);
      sc::tc::mma_bf16(taddr, ad, bd, sc::tc::idesc_bf16_f32(128, 32), 0u);
      const uint64_t t0 = global_ns();
      const bool got = sc::tc::mbar_wait_or_abort(sc::tc::smem_addr(&bar[1]), 0, ab, limit);
      out[7] = (int64_t)(global_ns() - t0);
      if (!got) *ab = 1;
      out[2] = got ? 0 : 1;
      sc::tc::mma_commit(sc::tc::smem_addr(&bar[2]));
      drained = sc::tc::mbar_wait(sc::tc::smem_addr(&bar[2]), 0) ? 1 : 0;
      out[3] = drained;
    }
    drained = __shfl_sync(0xffffffffu, drained, 0);
    sc::tc::fence_after();
    bool ok = false;
    if (drained) {
      float v[16];
      sc::tc::tmem_ld16(taddr + (32u << 16), v);  // warp 1 reads TMEM lanes 32..63
      ok = true;
      for (int j = 0; j < 16; ++j) ok &= v[j] == 16.0f;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) out[4] = ok ? 1 : 0;
  } else {
    if (lane == 0 && !sc::tc::mbar_wait(sc::tc::smem_addr(&bar[3]), 0, limit)) {
      *ab = 1;
      atomicAdd(&epi_gave_up, 1);
    }
  }
  sc::tc::fence_before();
  __syncthreads();
  if (warp == 1) sc::tc::tmem_dealloc(taddr, 32);
  if (threadIdx.x == 0) {
    out[5] = epi_gave_up;
    if (*ab) atomicOr(status, SC_STATUS_WATCHDOG);
  }
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

int sc_unet_param_count(int64_t *count) {
  if (!count) return SC_ERR_INVALID_ARG;
  Layer L[kNumLayers];
  *count = layout_params(L);
  return SC_OK;
}

int sc_unet_create(sc_ctx *c, int32_t max_batch, int32_t height, int32_t width, sc_unet **out) {
  if (!c || !out) return SC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!check_geom(max_batch, height, width))
    return fail(c, SC_ERR_INVALID_ARG, "sc_unet_create: need max_batch >= 1, height and width multiples of 8, >= 16");
  const char *where = "sc_unet_create";
  sc_unet *u = new (std::nothrow) sc_unet();
  if (!u) return fail(c, SC_ERR_OOM, "sc_unet_create: host allocation failed");
  u->max_batch = max_batch;
  u->H = height;
  u->W = width;
  for (int l = 0; l < kLevels; ++l) {
    u->hl[l] = height >> l;
    u->wl[l] = width >> l;
  }
  u->n_params = layout_params(u->L);
  int dev = sc::ctx_device(c);
  cudaError_t e = cudaDeviceGetAttribute(&u->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete u;
    return cuda_fail(c, e, where);
  }
  int64_t P[kLevels];
  for (int l = 0; l < kLevels; ++l) P[l] = (int64_t)max_batch * u->hl[l] * u->wl[l];
  // weight-gradient workspace: one region per layer (the largest split layout it can take), so
  // that all split-K reductions of a backward pass run in one launch at its end
  size_t wpart = 0;
  for (int i = 0; i < kNumLayers; ++i) {
    Layer &ly = u->L[i];
    const Wgrad g = wgrad_shape(ly);
    int lvl = 0;
    if (i < 8) lvl = i / 2;
    else if (i == kOutLayer) lvl = 0;
    else {
      const int l = 2 - (i - 8) / 3;
      lvl = ((i - 8) % 3 == 0) ? l + 1 : l;
    }
    int splits, ks;
    split_k(g.Mtiles, P[lvl], u->num_sms, &splits, &ks);
    // the TMA weight-gradient kernels: one split per CTA, up to SC_WG_MN_CTAS per SM
    splits = std::max(splits, u->num_sms * SC_WG_MN_CTAS);
    // the MN-major kernel's column layout may take more 128-row blocks than the plain one
    const int mt = ly.kind == KIND_CONV ? std::max(g.Mtiles, mn_layout(ly.cin_p, true).mtiles) : g.Mtiles;
    size_t need = (size_t)splits * mt * kTM * g.np;
    if (i == kOutLayer) need = (size_t)2 * u->num_sms * kOutParts;  // k_out_wgrad's block partials
    ly.part_off = wpart;
    ly.part_floats = need;
    wpart += (need + 63) & ~size_t(63);
  }
  const int Hv = height - 10, Wv = width - 10;
  const int lpart = max_batch * (((Wv + kSTW - 1) / kSTW) * ((Hv + kSTH - 1) / kSTH) +
                                 ((width + kSTW - 1) / kSTW) * ((height + kSTH - 1) / kSTH));
  // segments of the Adam / BF16-refresh kernel
  std::vector<Seg> segs;
  int blocks = 0;
  auto seg = [&](int64_t off, int64_t count, int kind, const Layer &ly) {
    Seg sgm{};
    sgm.off = off;
    sgm.count = (int32_t)count;
    sgm.kind = kind;
    sgm.cout = ly.cout;
    sgm.cin = ly.cin;
    sgm.cin_p = ly.cin_p;
    sgm.first_block = blocks;
    blocks += (int)((count + 255) / 256);
    segs.push_back(sgm);
  };
  for (int i = 0; i < kNumLayers; ++i) {
    seg(u->L[i].w_off, u->L[i].w_count, u->L[i].kind, u->L[i]);
    seg(u->L[i].b_off, u->L[i].cout, KIND_BIAS, u->L[i]);
  }
  // one allocation, carved twice (sizes, then pointers)
  for (int pass = 0; pass < 2; ++pass) {
    Carve cv{pass ? static_cast<char *>(u->block) : nullptr};
    const int64_t np = u->n_params;
    u->params = cv.take<float>(np);
    u->grads = cv.take<float>(np);
    u->adam_m = cv.take<float>(np);
    u->adam_v = cv.take<float>(np);
    u->segs = cv.take<Seg>(segs.size());
    for (int i = 0; i < kNumLayers; ++i) {
      u->L[i].wf = cv.take<bf16>(u->L[i].wf_elems);
      u->L[i].wd = u->L[i].wd_elems ? cv.take<bf16>(u->L[i].wd_elems) : nullptr;
      if (u->L[i].kind == KIND_UP) {
        u->L[i].wtf = cv.take<bf16>(u->L[i].wf_elems);
        u->L[i].wtd = cv.take<bf16>(u->L[i].wf_elems);
      }
      if (u->L[i].kind == KIND_CONV) {
        u->L[i].wtf = cv.take<bf16>(u->L[i].wf_elems);
        u->L[i].wtd = u->L[i].wd_elems ? cv.take<bf16>(u->L[i].wd_elems) : nullptr;
        if (conv_w_bytes(u->L[i].cin_p, u->L[i].cout) > kConvSplitBytes) {
          u->L[i].wtf2 = cv.take<bf16>(u->L[i].wf_elems);
          u->L[i].wtd2 = u->L[i].wd_elems ? cv.take<bf16>(u->L[i].wd_elems) : nullptr;
        }
      }
    }
    u->x0 = cv.take<bf16>(P[0] * kInPad);
    for (int l = 0; l < kLevels; ++l) {
      const int cl = kChans[l];
      u->a1[l] = cv.take<bf16>(P[l] * cl);
      if (l < kLevels - 1) {
        u->cat[l] = cv.take<bf16>(P[l] * 2 * cl);
        u->d1[l] = cv.take<bf16>(P[l] * cl);
        u->d2[l] = cv.take<bf16>(P[l] * cl);
        u->gd2[l] = cv.take<bf16>(P[l] * cl);
        u->gd1[l] = cv.take<bf16>(P[l] * cl);
        u->gup[l] = cv.take<bf16>(P[l] * cl);
        u->gskip[l] = cv.take<float>(P[l] * cl);
      } else {
        u->h3 = cv.take<bf16>(P[l] * cl);
      }
      if (l > 0) u->pool[l] = cv.take<bf16>(P[l] * kChans[l - 1]);
      u->ge2[l] = cv.take<bf16>(P[l] * cl);
      u->ge1[l] = cv.take<bf16>(P[l] * cl);
    }
    // the FP32 gradient of a pool output (the largest: level 1, kChans[0] channels)
    u->gpool = cv.take<float>(P[1] * kChans[0]);
    u->y = cv.take<float>(P[0] * kOutCh);
    u->gy8 = cv.take<bf16>(P[0] * kGyCh);
    for (int k = 0; k < 3; ++k) u->smap[k] = cv.take<float>((size_t)max_batch * Hv * Wv * 3);
    u->lpart = cv.take<double>(lpart);
    u->lpart_n = lpart;
    u->loss = cv.take<float>(1);
    u->wpart = cv.take<float>(wpart);
    u->wpart_floats = wpart;
    if (pass == 0) {
      u->block = sc::ctx_alloc(c, cv.off);
      if (!u->block) {
        delete u;
        return fail(c, SC_ERR_OOM, "sc_unet_create: out of device memory");
      }
      e = cudaMemsetAsync(u->block, 0, cv.off, sc::ctx_stream(c));
      if (e != cudaSuccess) {
        sc::ctx_free(c, u->block);
        delete u;
        return cuda_fail(c, e, where);
      }
    }
  }
  for (size_t i = 0, j = 0; i < (size_t)kNumLayers; ++i, j += 2) {
    segs[j].wf = u->L[i].wf;
    segs[j].wd = u->L[i].wd;
    segs[j].wtf = u->L[i].wtf;
    segs[j].wtd = u->L[i].wtd;
    segs[j].wtf2 = u->L[i].wtf2;
    segs[j].wtd2 = u->L[i].wtd2;
  }
  u->nseg = (int)segs.size();
  u->adam_blocks = blocks;
  // the segment table travels with the stream (pageable source: staged before the call returns)
  e = cudaMemcpyAsync(u->segs, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, sc::ctx_stream(c));
  if (e == cudaSuccess) e = cudaStreamSynchronize(sc::ctx_stream(c));
  if (e != cudaSuccess) {
    sc::ctx_free(c, u->block);
    delete u;
    return cuda_fail(c, e, where);
  }
  // Gaussian window of the SSIM (sigma 1.5, normalised), computed in double
  float gk[kWin];
  double gs = 0.0, gd[kWin];
  for (int i = 0; i < kWin; ++i) {
    const double d = i - 5.0;
    gd[i] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    gs += gd[i];
  }
  for (int i = 0; i < kWin; ++i) gk[i] = (float)(gd[i] / gs);
  e = cudaMemcpyToSymbol(c_gauss, gk, sizeof(gk));
  if (e == cudaSuccess) e = create_streams(u, dev);
  if (e != cudaSuccess) {
    release_streams(u);
    sc::ctx_free(c, u->block);
    delete u;
    return cuda_fail(c, e, where);
  }
  *out = u;
  return SC_OK;
}

int sc_unet_destroy(sc_ctx *c, sc_unet *u) {
  if (!c || !u) return SC_ERR_INVALID_ARG;
  release_streams(u);
  sc::ctx_free(c, u->block);
  delete u;
  return SC_OK;
}

int sc_unet_set_params(sc_ctx *c, sc_unet *u, const float *params) {
  if (!c || !u || !params) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_set_params";
  cudaStream_t s = sc::ctx_stream(c);
  const size_t bytes = (size_t)u->n_params * sizeof(float);
  UCHK(cudaMemcpyAsync(u->params, params, bytes, cudaMemcpyDeviceToDevice, s));
  UCHK(cudaMemsetAsync(u->adam_m, 0, bytes, s));
  UCHK(cudaMemsetAsync(u->adam_v, 0, bytes, s));
  u->step = 0;
  return refresh_bf16(c, u, 0, 0.0f);
}

int sc_unet_get_params(sc_ctx *c, const sc_unet *u, float *params) {
  if (!c || !u || !params) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_get_params";
  UCHK(cudaMemcpyAsync(params, u->params, (size_t)u->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                       sc::ctx_stream(c)));
  return SC_OK;
}

int sc_unet_get_grads(sc_ctx *c, const sc_unet *u, float *grads) {
  if (!c || !u || !grads) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_get_grads";
  UCHK(cudaMemcpyAsync(grads, u->grads, (size_t)u->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                       sc::ctx_stream(c)));
  return SC_OK;
}

int sc_unet_set_grads(sc_ctx *c, sc_unet *u, const float *grads) {
  if (!c || !u || !grads) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_set_grads";
  UCHK(cudaMemcpyAsync(u->grads, grads, (size_t)u->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                       sc::ctx_stream(c)));
  return SC_OK;
}

int sc_unet_forward(sc_ctx *c, sc_unet *u, const float *x, int32_t n, float *y) {
  if (!c || !u || !x || !y) return SC_ERR_INVALID_ARG;
  if (n < 1 || n > u->max_batch) return fail(c, SC_ERR_INVALID_ARG, "sc_unet_forward: n out of range");
  int rc = run_forward(c, u, x, n);
  if (rc) return rc;
  const char *where = "sc_unet_forward";
  UCHK(cudaMemcpyAsync(y, u->y, (size_t)n * u->H * u->W * kOutCh * sizeof(float), cudaMemcpyDeviceToDevice,
                       sc::ctx_stream(c)));
  return SC_OK;
}

int sc_unet_loss_grad(sc_ctx *c, sc_unet *u, const float *x, const float *target, int32_t n, float *y, float *loss) {
  if (!c || !u || !x || !target) return SC_ERR_INVALID_ARG;
  if (n < 1 || n > u->max_batch) return fail(c, SC_ERR_INVALID_ARG, "sc_unet_loss_grad: n out of range");
  const char *where = "sc_unet_loss_grad";
  int rc = run_forward(c, u, x, n);
  if (rc) return rc;
  rc = run_loss(c, u, u->y, target, n, u->H, u->W, loss ? loss : u->loss, nullptr, u->gy8, where);
  if (rc) return rc;
  rc = run_backward(c, u);
  if (rc) return rc;
  if (y)
    UCHK(cudaMemcpyAsync(y, u->y, (size_t)n * u->H * u->W * kOutCh * sizeof(float), cudaMemcpyDeviceToDevice,
                         sc::ctx_stream(c)));
  return SC_OK;
}

int sc_unet_adam(sc_ctx *c, sc_unet *u, float lr) {
  if (!c || !u || !(lr >= 0.0f)) return SC_ERR_INVALID_ARG;
  u->step += 1;
  return refresh_bf16(c, u, 1, lr);
}

int sc_unet_get_state(sc_ctx *c, const sc_unet *u, float *adam_m, float *adam_v, int64_t *step) {
  if (!c || !u) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_get_state";
  const size_t bytes = (size_t)u->n_params * sizeof(float);
  cudaStream_t s = sc::ctx_stream(c);
  if (adam_m) UCHK(cudaMemcpyAsync(adam_m, u->adam_m, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_v) UCHK(cudaMemcpyAsync(adam_v, u->adam_v, bytes, cudaMemcpyDeviceToDevice, s));
  if (step) *step = u->step;
  return SC_OK;
}

int sc_unet_set_state(sc_ctx *c, sc_unet *u, const float *params, const float *adam_m, const float *adam_v,
                      int64_t step) {
  if (!c || !u || !params || !adam_m || !adam_v || step < 0 || step > INT32_MAX)
    return fail(c, SC_ERR_INVALID_ARG, "sc_unet_set_state: null buffer or step out of range");
  const char *where = "sc_unet_set_state";
  const size_t bytes = (size_t)u->n_params * sizeof(float);
  cudaStream_t s = sc::ctx_stream(c);
  UCHK(cudaMemcpyAsync(u->params, params, bytes, cudaMemcpyDeviceToDevice, s));
  UCHK(cudaMemcpyAsync(u->adam_m, adam_m, bytes, cudaMemcpyDeviceToDevice, s));
  UCHK(cudaMemcpyAsync(u->adam_v, adam_v, bytes, cudaMemcpyDeviceToDevice, s));
  u->step = (int)step;
  return refresh_bf16(c, u, 0, 0.0f);
}

namespace {
// checkpoint file: header, then FP32 params, Adam m, Adam v (n_params each), little-endian
struct CkptHeader {
  char magic[8];       // "SCUNET1\0"
  int64_t n_params;
  int64_t step;
  int64_t chans[4];    // level widths, checked on load
};
constexpr char kCkptMagic[8] = {'S', 'C', 'U', 'N', 'E', 'T', '1', '\0'};
}  // namespace

int sc_unet_save(sc_ctx *c, const sc_unet *u, const char *path) {
  if (!c || !u || !path) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_save";
  const size_t n = (size_t)u->n_params;
  std::vector<float> host(3 * n);
  cudaStream_t s = sc::ctx_stream(c);
  UCHK(cudaMemcpyAsync(host.data(), u->params, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  UCHK(cudaMemcpyAsync(host.data() + n, u->adam_m, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  UCHK(cudaMemcpyAsync(host.data() + 2 * n, u->adam_v, n * sizeof(float), cudaMemcpyDeviceToHost, s));
  UCHK(cudaStreamSynchronize(s));
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.n_params = u->n_params;
  h.step = u->step;
  for (int l = 0; l < kLevels; ++l) h.chans[l] = kChans[l];
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(c, SC_ERR_INVALID_ARG, std::string("sc_unet_save: cannot open ") + path + " for writing");
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(host.data(), sizeof(float), 3 * n, f) == 3 * n;
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(c, SC_ERR_INVALID_ARG, std::string("sc_unet_save: write to ") + path + " failed");
  return SC_OK;
}

int sc_unet_load(sc_ctx *c, sc_unet *u, const char *path) {
  if (!c || !u || !path) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_load";
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(c, SC_ERR_INVALID_ARG, std::string("sc_unet_load: cannot open ") + path);
  CkptHeader h{};
  bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kCkptMagic, 8) == 0 &&
            h.n_params == u->n_params && h.step >= 0 && h.step <= INT32_MAX;
  for (int l = 0; ok && l < kLevels; ++l) ok = h.chans[l] == kChans[l];
  const size_t n = (size_t)u->n_params;
  std::vector<float> host;
  if (ok) {
    host.resize(3 * n);
    ok = std::fread(host.data(), sizeof(float), 3 * n, f) == 3 * n;
  }
  std::fclose(f);
  if (!ok)
    return fail(c, SC_ERR_INVALID_ARG,
                std::string("sc_unet_load: ") + path + " is not a checkpoint of this network (or is truncated)");
  cudaStream_t s = sc::ctx_stream(c);
  UCHK(cudaMemcpyAsync(u->params, host.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
  UCHK(cudaMemcpyAsync(u->adam_m, host.data() + n, n * sizeof(float), cudaMemcpyHostToDevice, s));
  UCHK(cudaMemcpyAsync(u->adam_v, host.data() + 2 * n, n * sizeof(float), cudaMemcpyHostToDevice, s));
  u->step = (int)h.step;
  const int rc = refresh_bf16(c, u, 0, 0.0f);
  if (rc) return rc;
  UCHK(cudaStreamSynchronize(s));  // the host staging buffer is released on return
  return SC_OK;
}

int sc_unet_set_loss(sc_ctx *c, sc_unet *u, int32_t kind) {
  if (!c || !u) return SC_ERR_INVALID_ARG;
  if (kind != SC_UNET_LOSS_L1_SSIM && kind != SC_UNET_LOSS_BCE && kind != SC_UNET_LOSS_L2_LINEAR)
    return fail(c, SC_ERR_INVALID_ARG, "sc_unet_set_loss: unknown loss");
  u->loss_kind = kind;
  return SC_OK;
}

int sc_unet_train_step(sc_ctx *c, sc_unet *u, const float *x, const float *target, int32_t n, float lr, float *loss) {
  int rc = sc_unet_loss_grad(c, u, x, target, n, nullptr, loss);
  if (rc) return rc;
  return sc_unet_adam(c, u, lr);
}

int sc_ssim_l1_loss(sc_ctx *c, const float *pred, const float *target, int32_t n, int32_t h, int32_t w, float *loss,
                    float *grad) {
  if (!c || !pred || !target || n < 1 || h < 11 || w < 11) return SC_ERR_INVALID_ARG;
  const char *where = "sc_ssim_l1_loss";
  // a private workspace sized for this call
  sc_unet tmp;
  const int Hv = h - 10, Wv = w - 10;
  const int lpart = n * (((Wv + kSTW - 1) / kSTW) * ((Hv + kSTH - 1) / kSTH) +
                         ((w + kSTW - 1) / kSTW) * ((h + kSTH - 1) / kSTH));
  Carve cv{nullptr};
  for (int pass = 0; pass < 2; ++pass) {
    cv.off = 0;
    for (int k = 0; k < 3; ++k) tmp.smap[k] = cv.take<float>((size_t)n * Hv * Wv * 3);
    tmp.lpart = cv.take<double>(lpart);
    tmp.lpart_n = lpart;
    if (pass == 0) {
      cv.base = static_cast<char *>(sc::ctx_alloc(c, cv.off));
      if (!cv.base) return fail(c, SC_ERR_OOM, "sc_ssim_l1_loss: out of device memory");
    }
  }
  float gk[kWin];
  double gs = 0.0, gd[kWin];
  for (int i = 0; i < kWin; ++i) {
    const double d = i - 5.0;
    gd[i] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    gs += gd[i];
  }
  for (int i = 0; i < kWin; ++i) gk[i] = (float)(gd[i] / gs);
  cudaError_t e = cudaMemcpyToSymbol(c_gauss, gk, sizeof(gk));
  int rc = e == cudaSuccess ? run_loss(c, &tmp, pred, target, n, h, w, loss, grad, nullptr, where)
                            : cuda_fail(c, e, where);
  sc::ctx_free(c, cv.base);
  tmp.block = nullptr;
  return rc;
}

static const float *frame_source(const sc_frame *f, int source) {
  switch (source) {
    case SC_UNET_SRC_RGB: return f->rgb;
    case SC_UNET_SRC_DIRECT: return f->direct;
    case SC_UNET_SRC_CAUSTIC: return f->caustic;
    default: return nullptr;
  }
}

int sc_unet_pack_frame(sc_ctx *c, const sc_frame *f, int32_t source, float *x, int32_t index) {
  if (!c || !f || !x || index < 0) return SC_ERR_INVALID_ARG;
  if (!frame_source(f, source) || !f->albedo || !f->normal_camera || !f->depth_norm || !f->mask)
    return fail(c, SC_ERR_INVALID_ARG,
                "sc_unet_pack_frame: the source estimate, albedo, normal_camera, depth_norm and mask needed");
  const char *where = "sc_unet_pack_frame";
  const int64_t P = (int64_t)f->width * f->height;
  k_pack_frame<<<(unsigned)((P + 255) / 256), 256, 0, sc::ctx_stream(c)>>>(
      reinterpret_cast<const float4 *>(frame_source(f, source)), reinterpret_cast<const float4 *>(f->albedo),
      reinterpret_cast<const float4 *>(f->normal_camera), f->depth_norm, f->mask, x + index * P * kInCh, P);
  UCHK(cudaGetLastError());
  return SC_OK;
}


int sc_unet_pack_target(sc_ctx *c, const sc_frame *f, int32_t source, float *t, int32_t index) {
  if (!c || !f || !t || index < 0 || !frame_source(f, source)) return SC_ERR_INVALID_ARG;
  const char *where = "sc_unet_pack_target";
  const int64_t P = (int64_t)f->width * f->height;
  k_pack_target<<<(unsigned)((P + 255) / 256), 256, 0, sc::ctx_stream(c)>>>(
      reinterpret_cast<const float4 *>(frame_source(f, source)), t + index * P * kOutCh, P);
  UCHK(cudaGetLastError());
  return SC_OK;
}

int sc_unet_output_rgb(sc_ctx *c, const float *y, int64_t n_px, const float *add, float *rgb) {
  if (!c || !y || !rgb || n_px < 0) return SC_ERR_INVALID_ARG;
  if (n_px == 0) return SC_OK;
  const char *where = "sc_unet_output_rgb";
  k_output_rgb<<<(unsigned)((n_px + 255) / 256), 256, 0, sc::ctx_stream(c)>>>(
      y, n_px, reinterpret_cast<const float4 *>(add), reinterpret_cast<float4 *>(rgb));
  UCHK(cudaGetLastError());
  return SC_OK;
}

static int buffer_view(const sc_unet *u, int id, int l, const void **ptr, int *dtype, int *ch, int *cs, int *co) {
  if (l < 0 || l >= kLevels) return SC_ERR_INVALID_ARG;
  const int cl = kChans[l];
  const bool dec = l < kLevels - 1;
  *dtype = 0;
  *co = 0;
  *ch = cl;
  *cs = cl;
  *ptr = nullptr;
  switch (id) {
    case SC_UNET_BUF_INPUT:
      if (l) return SC_ERR_INVALID_ARG;
      *ptr = u->x0;
      *ch = kInPad;
      *cs = kInPad;
      break;
    case SC_UNET_BUF_ENC1: *ptr = u->a1[l]; break;
    case SC_UNET_BUF_ENC2: {
      const View v = enc_out(u, l);
      *ptr = v.p;
      *cs = v.cs;
      *co = v.co;
      break;
    }
    case SC_UNET_BUF_POOL:
      if (!l) return SC_ERR_INVALID_ARG;
      *ptr = u->pool[l];
      *ch = *cs = kChans[l - 1];
      break;
    case SC_UNET_BUF_UP:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->cat[l];
      *cs = 2 * cl;
      break;
    case SC_UNET_BUF_DEC1:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->d1[l];
      break;
    case SC_UNET_BUF_DEC2:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->d2[l];
      break;
    case SC_UNET_BUF_OUT:
      if (l) return SC_ERR_INVALID_ARG;
      *ptr = u->y;
      *dtype = 1;
      *ch = *cs = kOutCh;
      break;
    case SC_UNET_BUF_GOUT:
      if (l) return SC_ERR_INVALID_ARG;
      *ptr = u->gy8;
      *ch = *cs = kGyCh;
      break;
    case SC_UNET_BUF_GDEC2:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->gd2[l];
      break;
    case SC_UNET_BUF_GDEC1:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->gd1[l];
      break;
    case SC_UNET_BUF_GUP:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->gup[l];
      break;
    case SC_UNET_BUF_GSKIP:
      if (!dec) return SC_ERR_INVALID_ARG;
      *ptr = u->gskip[l];
      *dtype = 1;
      break;
    case SC_UNET_BUF_GENC2: *ptr = u->ge2[l]; break;
    case SC_UNET_BUF_GENC1: *ptr = u->ge1[l]; break;
    default: return SC_ERR_INVALID_ARG;
  }
  return SC_OK;
}

int sc_unet_buffer(const sc_unet *u, int32_t id, int32_t level, sc_unet_buffer_info *info) {
  if (!u || !info) return SC_ERR_INVALID_ARG;
  const void *p;
  int dtype, ch, cs, co;
  int rc = buffer_view(u, id, level, &p, &dtype, &ch, &cs, &co);
  if (rc) return rc;
  info->dtype = dtype;
  info->n = u->n;
  info->h = u->hl[level];
  info->w = u->wl[level];
  info->c = ch;
  return SC_OK;
}

int sc_unet_copy_buffer(sc_ctx *c, const sc_unet *u, int32_t id, int32_t level, void *dst) {
  if (!c || !u || !dst) return SC_ERR_INVALID_ARG;
  const void *p;
  int dtype, ch, cs, co;
  int rc = buffer_view(u, id, level, &p, &dtype, &ch, &cs, &co);
  if (rc) return fail(c, rc, "sc_unet_copy_buffer: no such buffer");
  const char *where = "sc_unet_copy_buffer";
  const size_t es = dtype ? 4 : 2;
  const size_t rows = (size_t)u->n * u->hl[level] * u->wl[level];
  if (dtype) {  // FP32 tensors are [pixel][cs]
    UCHK(cudaMemcpy2DAsync(dst, ch * es, static_cast<const char *>(p) + co * es, cs * es, ch * es, rows,
                           cudaMemcpyDeviceToDevice, sc::ctx_stream(c)));
  } else {  // BF16 tensors are row-blocked
    const int64_t total = (int64_t)rows * ch;
    k_rb_to_dense<<<(unsigned)((total + 255) / 256), 256, 0, sc::ctx_stream(c)>>>(
        static_cast<const bf16 *>(p), cs, co, ch, (int64_t)u->n * u->hl[level], u->wl[level], static_cast<bf16 *>(dst));
    UCHK(cudaGetLastError());
  }
  return SC_OK;
}

int sc_unet_wait_selftest(sc_ctx *c, uint32_t poll_limit, int64_t *out_host) {
  if (!c || !out_host) return SC_ERR_INVALID_ARG;
  if (poll_limit < 1 || poll_limit > (1u << 24))
    return fail(c, SC_ERR_INVALID_ARG, "sc_unet_wait_selftest: poll_limit must be in [1, 2^24]");
  const char *where = "sc_unet_wait_selftest";
  cudaStream_t s = sc::ctx_stream(c);
  uint8_t *buf = static_cast<uint8_t *>(sc::ctx_alloc(c, 1024 + 8 * sizeof(int64_t)));
  if (!buf) return fail(c, SC_ERR_OOM, "sc_unet_wait_selftest: device allocation failed");
  int64_t *out = reinterpret_cast<int64_t *>(buf + 1024);
  int rc = SC_OK;
  cudaError_t e = cudaMemsetAsync(buf, 0x5A, 1024, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 8 * sizeof(int64_t), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 128, 0, s>>>(reinterpret_cast<const uint4 *>(buf), poll_limit, out, sc::ctx_status(c));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out, 8 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = fail(c, SC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  sc::ctx_free(c, buf);
  return rc;
}

}  // extern "C"
