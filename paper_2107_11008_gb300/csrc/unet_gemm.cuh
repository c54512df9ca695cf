// unet_gemm.cuh -- the general gathering tensor-core GEMM of the U-Net denoiser, plus the layout
// helpers, loaders and epilogue functors the TMA kernels (unet_conv.cuh, unet_wgrad_mn.cuh) share.
// It serves the contractions the TMA kernels do not: the transposed convolutions' data gradient
// and weight gradient, the weight gradients of 3x3 layers with fewer than 64 pixel tiles, and
// convolutions on rows that fit neither TMA tiling.
//
//   D[m][n] = sum_k A(m, k) * B(n, k),   m in a 128-row tile, n < N <= 256, k in a K range
//
// A and B are gathered by loader functors straight into the canonical no-swizzle K-major
// shared-memory layout (8 x 8 BF16 "core matrices"), so a convolution needs no im2col buffer:
// the 3x3 neighbourhood, zero padding, channel slices of concatenated tensors and the
// upsampling of a transposed convolution are index arithmetic in the loader.  K is consumed in
// stages of 64 held in two shared-memory buffers; while the tensor cores (tcgen05.mma,
// BF16 x BF16 -> FP32 accumulators in TMEM, issued by one thread) work on one stage, the CTA
// gathers the next, and an mbarrier armed by tcgen05.commit says when a buffer may be refilled.
// The epilogue reads the accumulators from TMEM (tcgen05.ld) 16 columns at a time and hands
// them to an epilogue functor (bias + ReLU, mask, pool routing, partial sums...).
//
// Layout: core matrices along K are kLBO = 144 bytes apart (128 bytes of data + 16 of padding),
// so the 8 threads that each store one 16-byte row of 8 different core matrices hit 8
// different bank groups; 8-row groups are kSBO = 8 * kLBO apart.
//
// BF16 activations and gradients live in HBM "row-blocked": an image row stores its groups of 8
// channels one after another, and within a group the row's pixels are consecutive 16-byte
// vectors (element (img, y, x, c) of a tensor of cs channels at
// ((img * h + y) * cs / 8 + c / 8) * w * 8 + x * 8 + c % 8).  A warp whose lanes own consecutive
// pixels then reads or writes 512 contiguous bytes per 16-byte access, and a TMA box of a
// channel group's pixels is one contiguous run instead of one 16-byte piece per pixel.
#pragma once
#include <cuda_bf16.h>

#include "device.cuh"
#include "tc.cuh"

namespace sc {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int kTM = 128;      // rows per tile (MMA M)
constexpr int kKC = 64;       // K per stage
constexpr int kThreads = 128;
constexpr uint32_t kLBO = 144;
constexpr uint32_t kSBO = 8 * kLBO;
constexpr uint32_t kStageA = (kTM / 8) * kSBO;

__host__ __device__ constexpr int pad16(int n) { return (n + 15) & ~15; }
__host__ __device__ constexpr uint32_t tmem_cols(int np) {
  return np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
}
__host__ __device__ constexpr size_t gemm_smem_bytes(int np) {
  return 2 * (size_t)kStageA + 2 * (size_t)(np / 8) * kSBO + 64;
}

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }
// element offset of channel c of pixel x in image row `row` (= img * h + y) of a row-blocked
// tensor with cs channels and rows of w pixels; c, cs multiples of 8 where 16 bytes are moved
__host__ __device__ __forceinline__ int64_t rb_off(int64_t row, int x, int c, int cs, int w) {
  return ((row * (cs >> 3) + (c >> 3)) * w + x) * 8 + (c & 7);
}
__device__ __forceinline__ uint4 ldg16(const bf16 *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint4 pack8(const float *v) {
  return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}
__device__ __forceinline__ void unpack8(const uint4 &u, float *v) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}

// one 16-byte row (8 consecutive k) of row r in k-group g of a stage buffer
__device__ __forceinline__ void st_row(uint8_t *s, int r, int g, const uint4 &v) {
  *reinterpret_cast<uint4 *>(s + (r >> 3) * kSBO + g * kLBO + (r & 7) * 16) = v;
}
// a whole core matrix: rows rg*8 .. rg*8+7 of k-group g
__device__ __forceinline__ void st_core(uint8_t *s, int rg, int g, const uint4 (&rows)[8]) {
  uint8_t *p = s + rg * kSBO + g * kLBO;
#pragma unroll
  for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(p + j * 16) = rows[j];
}

__device__ __forceinline__ uint32_t word(const uint4 &u, int i) { return i == 0 ? u.x : i == 1 ? u.y : i == 2 ? u.z : u.w; }
// pix[j] holds 8 BF16 of pixel j (element e = channel); rows[e] receives element e of pixels 0..7
__device__ __forceinline__ void transpose8(const uint4 (&pix)[8], uint4 (&rows)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint32_t sel = (e & 1) ? 0x7632u : 0x5410u;
    rows[e] = make_uint4(__byte_perm(word(pix[0], e >> 1), word(pix[1], e >> 1), sel),
                         __byte_perm(word(pix[2], e >> 1), word(pix[3], e >> 1), sel),
                         __byte_perm(word(pix[4], e >> 1), word(pix[5], e >> 1), sel),
                         __byte_perm(word(pix[6], e >> 1), word(pix[7], e >> 1), sel));
  }
}

// ---------------------------------------------------------------------------------------------
// The GEMM kernel.  Grid: (ceil(M / 128), splits); split y covers k in [y*k_split, (y+1)*k_split).
// Loaders: begin(m0, kb) once, then fill(stage, k0, kc) per stage (kc <= 64 valid k, the rest of
// the stage must be written as zeros).  Epilogue: store(row, n0, v[16], split) for row < M.
// ---------------------------------------------------------------------------------------------
template <class AL, class BL, class EP>
__global__ void __launch_bounds__(kThreads) k_gemm(AL A, BL B, EP E, int M, int N, int K, int k_split,
                                                   unsigned *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = pad16(N);
  const uint32_t stageB = (uint32_t)(np / 8) * kSBO;
  uint8_t *const sA0 = sm, *const sA1 = sm + kStageA;
  uint8_t *const sB0 = sm + 2 * kStageA, *const sB1 = sm + 2 * kStageA + stageB;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * kStageA + 2 * stageB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int m0 = blockIdx.x * kTM;
  const int kb = blockIdx.y * k_split, ke = min(K, kb + k_split);
  const uint32_t ncols = tmem_cols(np);
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(&mbar[0]), 1);
    tc::mbar_init(tc::smem_addr(&mbar[1]), 1);
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(slot), ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *slot;
  const uint32_t idesc = tc::idesc_bf16_f32(kTM, np);
  const int nchunks = ke > kb ? (ke - kb + kKC - 1) / kKC : 0;
  uint32_t phase0 = 0u, phase1 = 0u;
  bool ok = true;
  A.begin(m0, kb);
  B.begin(0, kb);
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    if (c >= 2) {  // the MMAs of chunk c-2 read this buffer
      if (!tc::mbar_wait(tc::smem_addr(&mbar[b]), b ? phase1 : phase0)) ok = false;
      if (b) phase1 ^= 1u;
      else phase0 ^= 1u;
    }
    uint8_t *const sA = b ? sA1 : sA0;
    uint8_t *const sB = b ? sB1 : sB0;
    const int k0 = kb + c * kKC;
    const int kc = min(kKC, ke - k0);
    A.fill(sA, k0, kc);
    B.fill(sB, k0, kc);
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
      for (int s = 0; s < (kc + 15) / 16; ++s)
        tc::mma_bf16(taddr, tc::smem_desc(a0 + (uint32_t)s * 2u * kLBO, kLBO, kSBO),
                     tc::smem_desc(b0 + (uint32_t)s * 2u * kLBO, kLBO, kSBO), idesc, (c > 0 || s > 0) ? 1u : 0u);
      tc::mma_commit(tc::smem_addr(&mbar[b]));
    }
  }
  if (nchunks > 0) {
    const int b = (nchunks - 1) & 1;
    if (!tc::mbar_wait(tc::smem_addr(&mbar[b]), b ? phase1 : phase0)) ok = false;
  }
  tc::fence_after();
  const int row = m0 + warp * 32 + lane;
  for (int n0 = 0; n0 < np; n0 += 16) {
    float v[16];
    tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, v);
    if (nchunks == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.0f;
    }
    if (ok && row < M) E.store(row, n0, v, (int)blockIdx.y);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
  if (!ok && tid == 0) atomicOr(status, SC_STATUS_WATCHDOG);
}

// ---------------------------------------------------------------------------------------------
// Loaders
// ---------------------------------------------------------------------------------------------

// A operand, one pixel per row (thread t owns row t of the tile): the 3x3 neighbourhood (or the
// pixel itself, ntaps == 1) of a row-blocked BF16 tensor, k = tap * cin + channel.  sign = +1 is the
// forward correlation; sign = -1 flips the taps, which is the data gradient of a 3x3 conv.
struct ANbr {
  const bf16 *src;
  int cs, co;     // channel stride of the tensor and offset of the slice
  int h, w;       // geometry (input and output have the same size)
  int cin;        // channels per tap, multiple of 8
  int ntaps;      // 9 or 1
  int sign;
  int M;
  int img, y, x, tap, c;
  bool ok;
  __device__ __forceinline__ void begin(int m0, int kb) {
    const int m = m0 + (int)threadIdx.x;
    ok = m < M;
    const int mm = ok ? m : 0;
    x = mm % w;
    const int t = mm / w;
    y = t % h;
    img = t / h;
    tap = kb / cin;
    c = kb - tap * cin;
  }
  __device__ __forceinline__ void fill(uint8_t *s, int, int kc) {
    const int r = threadIdx.x;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      uint4 v = zero4();
      if (g * 8 < kc) {
        int yy = y, xx = x;
        if (ntaps == 9) {
          const int ty = tap / 3;
          yy += sign * (ty - 1);
          xx += sign * (tap - 3 * ty - 1);
        }
        if (ok && yy >= 0 && yy < h && xx >= 0 && xx < w)
          v = ldg16(src + rb_off((int64_t)img * h + yy, xx, co + c, cs, w));
        c += 8;
        if (c == cin) {
          c = 0;
          ++tap;
        }
      }
      st_row(s, r, g, v);
    }
  }
};

// A operand of the data gradient of a 2x2 stride-2 transposed conv: row = pixel (img, y, x) of
// the low-resolution input (h x w), k = (a*2 + e) * cu + o, value = gradient of the upsampled
// tensor at (2y + a, 2x + e), channel o.
struct AUpGrad {
  const bf16 *g;
  int gcs;   // channel stride of the upsampled gradient
  int h, w;  // low-resolution geometry
  int cu;    // channels of the upsampled tensor (multiple of 8)
  int M;
  int img, y, x, ae, o;
  bool ok;
  __device__ __forceinline__ void begin(int m0, int kb) {
    const int m = m0 + (int)threadIdx.x;
    ok = m < M;
    const int mm = ok ? m : 0;
    x = mm % w;
    const int t = mm / w;
    y = t % h;
    img = t / h;
    ae = kb / cu;
    o = kb - ae * cu;
  }
  __device__ __forceinline__ void fill(uint8_t *s, int, int kc) {
    const int r = threadIdx.x;
#pragma unroll
    for (int gi = 0; gi < 8; ++gi) {
      uint4 v = zero4();
      if (gi * 8 < kc) {
        if (ok) {
          const int yy = 2 * y + (ae >> 1), xx = 2 * x + (ae & 1);
          v = ldg16(g + rb_off((int64_t)img * 2 * h + yy, xx, o, gcs, 2 * w));
        }
        o += 8;
        if (o == cu) {
          o = 0;
          ++ae;
        }
      }
      st_row(s, r, gi, v);
    }
  }
};

// B operand from a row-major BF16 matrix W[n][k] (leading dimension ldk, multiple of 8)
struct BDense {
  const bf16 *W;
  int ldk, N;
  __device__ __forceinline__ void begin(int, int) {}
  __device__ __forceinline__ void fill(uint8_t *s, int k0, int kc) {
    const int np = pad16(N);
    for (int i = threadIdx.x; i < np * 8; i += kThreads) {
      const int r = i % np, g = i / np;
      uint4 v = zero4();
      if (r < N && g * 8 < kc) v = ldg16(W + (int64_t)r * ldk + k0 + g * 8);
      st_row(s, r, g, v);
    }
  }
};

// Operand with k = pixel index (the weight gradient contracts over pixels).  Row m = tap * cin +
// channel of a pixel tensor; mode 0: tap t of ntaps (9: the 3x3 neighbourhood shifted by
// (t/3 - 1, t%3 - 1); 1: the pixel itself); mode 1: tap t = a*2 + e of a tensor of twice the
// resolution at (2y + a, 2x + e).  Rows >= `rows` are zero, except row `rows` when `ones` (the
// bias gradient rides along as a row of ones).  Each thread gathers whole 8 x 8 core matrices
// (8 pixels x 8 channels) and transposes them in registers; thread t always serves k-group t % 8.
struct TPix {
  const bf16 *src;
  int cs, co;
  int h, w;      // geometry of the pixels k runs over (n_img * h * w = K)
  int cin;       // channels per tap, multiple of 8
  int ntaps;
  int mode;      // 0 shift, 1 upsample
  int rows;      // data rows
  int ones;      // 1: row `rows` is all ones
  int R;         // rows of the stage buffer (128 for A, padded N for B)
  int m0, img, y, x;
  __device__ __forceinline__ void begin(int m0_, int kb) {
    m0 = m0_;
    const int p = kb + 8 * (int)(threadIdx.x & 7);
    x = p % w;
    const int t = p / w;
    y = t % h;
    img = t / h;
  }
  __device__ __forceinline__ void fill(uint8_t *s, int, int kc) {
    const int g = threadIdx.x & 7;
    const bool kval = g * 8 < kc;
    for (int rg = threadIdx.x >> 3; rg < R / 8; rg += kThreads / 8) {
      uint4 rv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) rv[j] = zero4();
      const int m = m0 + rg * 8;
      if (kval && m < rows) {
        const int tap = m / cin, c = m - tap * cin;
        int dy = 0, dx = 0;
        if (mode == 0 && ntaps == 9) {
          dy = tap / 3 - 1;
          dx = tap % 3 - 1;
        }
        const int sh = mode ? 2 * h : h, sw = mode ? 2 * w : w;
        uint4 pix[8];
        int yy = y, xx = x, im = img;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          int py, px;
          if (mode == 0) {
            py = yy + dy;
            px = xx + dx;
          } else {
            py = 2 * yy + (tap >> 1);
            px = 2 * xx + (tap & 1);
          }
          pix[j] = (py >= 0 && py < sh && px >= 0 && px < sw)
                       ? ldg16(src + rb_off((int64_t)im * sh + py, px, co + c, cs, sw))
                       : zero4();
          if (++xx == w) {
            xx = 0;
            if (++yy == h) {
              yy = 0;
              ++im;
            }
          }
        }
        transpose8(pix, rv);
        if (m + 8 > rows) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (m + j >= rows) rv[j] = zero4();
        }
      }
      if (kval && ones && m <= rows && rows < m + 8) {
        const uint32_t one2 = 0x3F803F80u;  // two BF16 1.0
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j == rows - m) rv[j] = make_uint4(one2, one2, one2, one2);
      }
      st_core(s, rg, g, rv);
    }
    // advance this thread's pixel by one stage (64 pixels)
    x += kKC;
    while (x >= w) {
      x -= w;
      if (++y == h) {
        y = 0;
        ++img;
      }
    }
  }
};

// ---------------------------------------------------------------------------------------------
// Epilogues (v[16] = columns n0 .. n0+15 of one row)
// ---------------------------------------------------------------------------------------------

// out = act(v + bias) in BF16 at pixel `row` (act: ReLU or identity) of a row-blocked tensor
// with rows of w pixels; N multiple of 16
struct EBiasAct {
  bf16 *out;
  int cs, co;
  const float *bias;
  int N, relu, w;
  __device__ __forceinline__ void store(int row, int n0, const float *v, int) const {
    if (n0 >= N) return;
    float t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      t[i] = v[i] + __ldg(bias + n0 + i);
      if (relu) t[i] = fmaxf(t[i], 0.0f);
    }
    const int r = row / w;
    bf16 *p = out + rb_off(r, row - r * w, co + n0, cs, w);
    *reinterpret_cast<uint4 *>(p) = pack8(t);
    *reinterpret_cast<uint4 *>(p + 8 * w) = pack8(t + 8);
  }
};

// transposed conv forward: column n = (a*2 + e) * cu + o of low-resolution pixel (img, y, x)
// lands on pixel (2y + a, 2x + e) of the output, channel o (+ bias, no activation)
struct EUpFwd {
  bf16 *out;
  int cs, co;
  const float *bias;
  int cu, h, w;  // h, w: low-resolution geometry
  __device__ __forceinline__ void store(int row, int n0, const float *v, int) const {
    if (n0 >= 4 * cu) return;
    const int ae = n0 / cu, o0 = n0 - ae * cu;
    const int x = row % w, t = row / w, y = t % h, img = t / h;
    const int yy = 2 * y + (ae >> 1), xx = 2 * x + (ae & 1);
    float u[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) u[i] = v[i] + __ldg(bias + o0 + i);
    bf16 *p = out + rb_off((int64_t)img * 2 * h + yy, xx, co + o0, cs, 2 * w);
    *reinterpret_cast<uint4 *>(p) = pack8(u);
    *reinterpret_cast<uint4 *>(p + 16 * w) = pack8(u + 8);
  }
};

// data gradient: columns n < split -> BF16 out (row-blocked, rows of w pixels), times
// (mask > 0) when a mask is given (row-blocked); columns n >= split -> FP32 out2 ([pixel][o2cs],
// unmasked).  N and split multiples of 16.
struct EGrad {
  bf16 *out;
  int ocs, oco;
  const bf16 *mask;
  int mcs, mco;
  int N, split;
  float *out2;
  int o2cs, w;
  __device__ __forceinline__ void store(int row, int n0, const float *v, int) const {
    if (n0 >= N) return;
    if (n0 >= split) {
      float4 *p = reinterpret_cast<float4 *>(out2 + (int64_t)row * o2cs + (n0 - split));
#pragma unroll
      for (int i = 0; i < 4; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
      return;
    }
    float t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
    const int r = row / w, x = row - r * w;
    if (mask) {
      float mv[16];
      const bf16 *mp = mask + rb_off(r, x, mco + n0, mcs, w);
      unpack8(ldg16(mp), mv);
      unpack8(ldg16(mp + 8 * w), mv + 8);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (!(mv[i] > 0.0f)) t[i] = 0.0f;
    }
    bf16 *p = out + rb_off(r, x, oco + n0, ocs, w);
    *reinterpret_cast<uint4 *>(p) = pack8(t);
    *reinterpret_cast<uint4 *>(p + 8 * w) = pack8(t + 8);
  }
};

// FP32 partial products of a K split: part[(split * Mpad + row) * ld + n]
struct EPartial {
  float *part;
  int ld, Mpad;
  __device__ __forceinline__ void store(int row, int n0, const float *v, int split) const {
    float4 *p = reinterpret_cast<float4 *>(part + ((int64_t)split * Mpad + row) * ld + n0);
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
};

}  // namespace unet
}  // namespace sc
