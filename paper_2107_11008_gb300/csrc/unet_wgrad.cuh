// unet_wgrad.cuh -- weight gradient of a 3x3 convolution on tcgen05 with TMA tiles (tiles of 128
// pixels: part of a row of 128k pixels, or 128 / w whole narrower rows, as in unet_conv.cuh).
//
//   gw[o][tap][c] = sum_p gz[p][o] * x[p + offset(tap)][c],   gb[o] = sum_p gz[p][o]
//
// as D[(tap, c) | ones][o] = sum over pixels.  The contraction runs over pixels, so both operands
// must have 8 consecutive pixels in each 16-byte row (K-major), while activations and gradients
// are stored with 8 consecutive channels per 16 bytes.  Per tile of 128 pixels of one row, the
// producer warp brings with TMA the 3 x 144 pixel neighbourhood of x (as the forward kernel does)
// and the 128 pixels of gz; sixteen transposer warps build each 128-row block of the A operand
// (rows (tap, c): the slab read at the tap's pixel offset, looked up in a per-CTA table of 8 x 8
// units) and the B operand (rows o) with ldmatrix.trans (8 x 8 transposes from shared memory)
// into the padded canonical layout; one thread issues the MMAs.  The accumulators of all row
// blocks (rows 9 cin + 1, 128 per block, cout columns each, 32/64/128 apart) stay in TMEM across
// the CTA's whole range of tiles; at the end the epilogue warps write them as this CTA's partial
// sums into the layer's region of the workspace, reduced in a fixed order by k_wgrad_reduce.
// Every wait is bounded.
#pragma once
#include "unet_conv.cuh"

namespace sc {
namespace unet {

constexpr uint32_t kGzTileBytes = 128 * 16;           // one group of 8 gz channels of a tile
constexpr uint32_t kTLBO = 144;                         // padded K-direction core stride
constexpr uint32_t kTSBO = 16 * kTLBO;                  // 16 pixel groups per 8-row group
constexpr uint32_t kTBlockBytes = 16 * kTSBO;           // one 128-row operand block
#ifndef SC_WG_TRANS
#define SC_WG_TRANS 16
#endif
constexpr int kWgTrans = SC_WG_TRANS;                   // transposer warps (a divisor of 16)
constexpr int kWgWarps = kWgTrans + 2;                  // + producer, MMA
constexpr int kWgThreads = 32 * kWgWarps;
constexpr int kWgMaxBlocks = 16;                        // 128-row operand blocks (512 TMEM columns / 32)
constexpr uint32_t kWgTabBytes = kWgMaxBlocks * 64 * 4;  // per (block, unit): slab offset of the unit
constexpr uint32_t kWgOnes = 0x80000001u, kWgZero = 0x80000000u;

__host__ __device__ constexpr uint32_t wg_raw_bytes(int cin, int cout, uint32_t gstride = kSlabBytes) {
  return align_up((uint32_t)(cin / 8) * gstride + (uint32_t)(cout / 8) * kGzTileBytes, 1024);
}
__host__ __device__ constexpr uint32_t wg_b_bytes(int cout) { return align_up((uint32_t)(cout / 8) * kTSBO, 1024); }
__host__ __device__ constexpr uint32_t wg_cstride(int cout) { return cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u); }
__host__ __device__ constexpr size_t wg_smem_bytes(int cin, int cout, int rstages, uint32_t gstride = kSlabBytes) {
  return (size_t)rstages * wg_raw_bytes(cin, cout, gstride) + 2 * kTBlockBytes + 2 * wg_b_bytes(cout) + 256 +
         kWgTabBytes;
}

template <bool NARROW>
__global__ void __launch_bounds__(kWgThreads, 1) k_wgrad_tma(const __grid_constant__ CUtensorMap xmap,
                                                               const __grid_constant__ CUtensorMap gmap, int cin,
                                                               int cout, int mtiles, int rstages, ConvGeo G,
                                                               float *part, unsigned *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngx = cin / 8, ngz = cout / 8;
  const int rows = 9 * cin;  // data rows; row `rows` is the ones row
  const uint32_t rawb = wg_raw_bytes(cin, cout, G.gstride), bb = wg_b_bytes(cout);
  const int h = G.h, w = G.w;
  uint8_t *sRaw = sm;
  uint8_t *sA = sm + rstages * rawb;
  uint8_t *sB = sA + 2 * kTBlockBytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + 2 * bb);
  // [0,1] raw full, [2,3] raw empty, [4,5] A full, [6,7] A empty, [8,9] B full, [10,11] B empty, [12] done
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 13);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(slot + 1);
  uint32_t *tab = reinterpret_cast<uint32_t *>(sB + 2 * bb + 256);
  const int tiles_x = NARROW ? 1 : w / 128;
  const int tiles_y = NARROW ? h / G.th : h;
  const int ntiles = G.n_img * tiles_y * tiles_x;
  const int t0 = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
  const int t1 = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);
  const int mine = t1 - t0;
  const uint32_t cstride = wg_cstride(cout);
  uint32_t cols = 32;
  while (cols < (uint32_t)mtiles * cstride) cols <<= 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(tc::smem_addr(&bar[0 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[2 + i]), kWgTrans);
      tc::mbar_init(tc::smem_addr(&bar[4 + i]), kWgTrans);
      tc::mbar_init(tc::smem_addr(&bar[6 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[8 + i]), kWgTrans);
      tc::mbar_init(tc::smem_addr(&bar[10 + i]), 1);
    }
    tc::mbar_init(tc::smem_addr(&bar[12]), 1);
    *abort_flag = 0;
  }
  // A-operand unit table (the same for every tile): unit q of 128-row block k covers operand rows
  // 128k + 8 (q / 4) .. + 7 (tap, channel group) and pixel groups 4 (q % 4) .. + 3; its entry is
  // the slab byte offset of its first ldmatrix row, or kWgOnes / kWgZero past the data rows
  for (int i = threadIdx.x; i < mtiles * 64; i += kWgThreads) {
    const int k = i >> 6, q = i & 63;
    const int r0 = 128 * k + 8 * (q >> 2), quad = q & 3;
    uint32_t e = r0 == rows ? kWgOnes : kWgZero;
    if (r0 < rows) {
      const int tap = r0 / cin, cg = (r0 - tap * cin) >> 3;
      const int dy = tap / 3, dx = tap - 3 * dy;
      e = NARROW ? (uint32_t)cg * G.gstride + (uint32_t)dx * G.slab + (uint32_t)(dy * w + 32 * quad) * 16u
                 : (uint32_t)cg * kSlabBytes + (uint32_t)(dy * kHaloW + 32 * quad + dx + kHaloLead - 1) * 16u;
    }
    tab[i] = e;
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_addr(slot), cols);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: x neighbourhood and gz tile per pixel tile ------------------------------
      int i = 0;
      for (; i < mine && !*abort_flag; ++i) {
        const int rs = i % rstages, u = i / rstages;
        if (u > 0 && !tc::mbar_wait(tc::smem_addr(&bar[2 + rs]), (u - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        const int t = t0 + i;
        const int xt = t % tiles_x, r = t / tiles_x, y = (r % tiles_y) * G.th, img = r / tiles_y;
        const uint32_t full = tc::smem_addr(&bar[0 + rs]);
        tc::mbar_expect_tx(full, (uint32_t)ngx * G.tx + (uint32_t)ngz * kGzTileBytes);
        const uint32_t dst = tc::smem_addr(sRaw + rs * rawb);
        for (int g = 0; g < ngx; ++g) {
          if (NARROW) {
            for (int dx = 0; dx < 3; ++dx)
              tc::tma_load_5d(dst + g * G.gstride + dx * G.slab, &xmap, 0, dx - 1, g, y - 1, img, full);
          } else {
            tc::tma_load_5d(dst + g * G.gstride, &xmap, 0, xt * (128 / 8) - kHaloLead / 8, g, y - 1, img, full);
          }
        }
        // gz: whole 8-pixel blocks (box (64, 128 / 8 or w / 8, 1, 1 or th, 1))
        const uint32_t gdst = dst + ngx * G.gstride;
        for (int g = 0; g < ngz; ++g)
          tc::tma_load_5d(gdst + g * kGzTileBytes, &gmap, 0, xt * (128 / 8), g, y, img, full);
      }
      for (int k = i - rstages; k < i; ++k)
        if (k >= 0) tc::mbar_wait(tc::smem_addr(&bar[0 + k % rstages]), (k / rstages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ---------------------------------------------------------------------------
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, cout);
      // descriptors advanced by start-field adds (byte offsets / 16; no carry below 2^18)
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), kTLBO, kTSBO);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sB), kTLBO, kTSBO);
      const uint32_t kstep = (2u * kTLBO) >> 4;
      // low words only (start fields); the abort flag is read only inside pending waits
      const uint32_t alo0 = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
      const uint32_t blo0 = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
      auto desc = [](uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; };
      bool ok = true;
      int m = 0;  // operand blocks consumed
      for (int i = 0; ok && i < mine; ++i) {
        const int bs = i & 1;
        if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[8 + bs]), (i >> 1) & 1, abort_flag)) ok = false;
        const uint32_t bd = blo0 + (((uint32_t)bs * bb) >> 4);
        for (int k = 0; ok && k < mtiles; ++k, ++m) {
          const int ab = m & 1;
          if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[4 + ab]), (m >> 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t ad = alo0 + (((uint32_t)ab * kTBlockBytes) >> 4);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            tc::mma_bf16(taddr + (uint32_t)k * cstride, desc(ad + (uint32_t)ks * kstep, ahi),
                         desc(bd + (uint32_t)ks * kstep, bhi), idesc, (i > 0 || ks > 0) ? 1u : 0u);
          tc::mma_commit(tc::smem_addr(&bar[6 + ab]));  // A block free
        }
        if (ok) tc::mma_commit(tc::smem_addr(&bar[10 + bs]));  // B block free
      }
      if (!ok) *abort_flag = 1;
      tc::mma_commit(tc::smem_addr(&bar[12]));  // all MMAs issued by this thread complete
    }
  } else {
    // ---- transposers (warps 2..9), then the epilogue (warps 2..5) -----------------------------
    const int tw = warp - 2;
    const int mrow = lane & 7, mat = lane >> 3;  // ldmatrix: this lane's row and matrix
    const uint32_t wofs = (uint32_t)(lane >> 2) * 16u + (uint32_t)(lane & 3) * 4u;  // store offset in a core
    const uint32_t lofs = (uint32_t)(8 * mat + mrow) * 16u;  // this lane's ldmatrix row within a unit
    const uint32_t ones = (lane >> 2) == 0 ? 0x3F803F80u : 0u;  // the ones row: row 0 of its core
    int m = 0;
    bool ok = true;
    for (int i = 0; ok && i < mine; ++i) {
      const int rs = i % rstages;
      if (!tc::mbar_wait(tc::smem_addr(&bar[0 + rs]), (i / rstages) & 1)) {
        ok = false;
        break;
      }
      const uint32_t raw = tc::smem_addr(sRaw + rs * rawb);
      const uint32_t gz = raw + ngx * G.gstride;
      // B block: rows o (cout), 128 pixels; unit q = (og, quad of pixel groups), one ldmatrix.x4 each
      const int bs = i & 1;
      if (i >= 2 && !tc::mbar_wait(tc::smem_addr(&bar[10 + bs]), ((i >> 1) - 1) & 1)) {
        ok = false;
        break;
      }
      uint8_t *bdst = sB + bs * bb;
      for (int q = tw; q < ngz * 4; q += kWgTrans) {
        const int og = q >> 2, pg = (q & 3) * 4 + mat;
        uint32_t r[4];
        tc::ldsm_x4_trans(gz + og * kGzTileBytes + (uint32_t)(8 * pg + mrow) * 16u, r[0], r[1], r[2], r[3]);
        uint8_t *c0 = bdst + og * kTSBO + (uint32_t)((q & 3) * 4) * kTLBO + wofs;
#pragma unroll
        for (int j = 0; j < 4; ++j) *reinterpret_cast<uint32_t *>(c0 + j * kTLBO) = r[j];
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar[8 + bs]));
      // A blocks: rows 128k .. 128k+127 of (tap, c) | ones | zero; 64 units (16 core rows x 4
      // quads of pixel groups) per block, 8 per warp, transposed 4 at a time
      for (int k = 0; k < mtiles; ++k, ++m) {
        const int ab = m & 1;
        if (m >= 2 && !tc::mbar_wait(tc::smem_addr(&bar[6 + ab]), ((m >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        uint8_t *adst = sA + ab * kTBlockBytes;
        const uint32_t *tk = tab + 64 * k;
#pragma unroll
        for (int b4 = 0; b4 < 64 / kWgTrans; b4 += 4) {
          uint32_t r[4][4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t te = tk[tw + kWgTrans * (b4 + e)];
            if (!(te >> 31)) {
              tc::ldsm_x4_trans(raw + te + lofs, r[e][0], r[e][1], r[e][2], r[e][3]);
            } else {
              // the ones row (bias gradient) heads the first core row after the data; the rest is zero
              const uint32_t v = te == kWgOnes ? ones : 0u;
              r[e][0] = r[e][1] = r[e][2] = r[e][3] = v;
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = tw + kWgTrans * (b4 + e);
            uint8_t *c0 = adst + (q >> 2) * kTSBO + (uint32_t)((q & 3) * 4) * kTLBO + wofs;
#pragma unroll
            for (int j = 0; j < 4; ++j) *reinterpret_cast<uint32_t *>(c0 + j * kTLBO) = r[e][j];
          }
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar[4 + ab]));
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar[2 + rs]));  // raw stage read
    }
    if (!ok) *abort_flag = 1;
    // epilogue (warps 2..5: TMEM lane quarters 2, 3, 0, 1): this CTA's partial sums of every row block
    const int qd = warp & 3;
    const bool done = tc::mbar_wait(tc::smem_addr(&bar[12]), 0);
    tc::fence_after();
    const int Mpad = mtiles * kTM;
    for (int k = 0; warp < 6 && k < mtiles; ++k)
      for (int n0 = 0; n0 < cout; n0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)k * cstride + (uint32_t)n0, v);
        if (done && !*abort_flag && mine > 0) {
          float4 *p = reinterpret_cast<float4 *>(part + ((int64_t)blockIdx.x * Mpad + 128 * k + 32 * qd + lane) * cout + n0);
#pragma unroll
          for (int j = 0; j < 4; ++j) p[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(taddr, cols);
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, SC_STATUS_WATCHDOG);
}

}  // namespace unet
}  // namespace sc
