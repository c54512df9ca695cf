// unet_wgrad_mn.cuh -- weight gradient of a 3x3 convolution on tcgen05 with MN-major operands
// that TMA delivers ready to use (tiles of 128 pixels: part of a row of 128k pixels, or 128 / w
// whole rows of w = 32 or 64 pixels).
//
//   gw[o][tap][c] = sum_p gz[p][o] * x[p + offset(tap)][c],   gb[o] = sum_p gz[p][o]
//
// as D[(tap, c) | ones][o] = sum over pixels.  The tensors hold 8 consecutive channels per 16
// bytes, which is the row of an MN-major core matrix when M (or N) is the channel and K the pixel:
// 8 consecutive pixels x 8 channels = one 128-byte core matrix.  So nothing is transposed.  One MMA
// (K = 16) reads 16 pixels, so the operand is staged per quarter of the tile (32 pixels): a ring
// slot holds one 128-row block of A as [quarter][16 pairs (tap, channel group)][32 pixels x 16
// bytes], and the pairs of an MMA are 512 bytes apart.  Each channel group's image row is one
// contiguous run of 8 w BF16 values, so a tap's pixel shift is an element offset of 8 (16 bytes)
// in a (8 w, groups, rows, images) view: one TMA copy (256 values x gb groups, zeros outside the
// image) brings a quarter of gb consecutive pairs of one tap, in rows of 512 bytes; gb = gcd(cin /
// 8, 16), so that no copy straddles two blocks.  The bias row 9 cin is a pair whose channel 0 is
// one, copied from a constant.  The gz tile arrives as one 2 KB block per group of 8 output
// channels (K-row stride 16 bytes, 128 pixels).  One thread issues the MMAs; the accumulators of
// all 128-row blocks (cout columns each, 32/64/128 apart) stay in TMEM across the CTA's contiguous
// range of tiles, and at the end the epilogue warps write them as this CTA's partial sums
// ([split][128 mtiles][cout], the layout k_wgrad_reduce sums in a fixed order).  Every wait is
// bounded.
//
// Operand extents (LBO = 128 bytes: the next 8 pixels; SBO = the next 8 channels: 512 bytes in A,
// 2 KB in gz): one MMA reads 16 pairs x 256 bytes of one quarter of its slot, and cout / 8 blocks x
// 256 bytes of its gz tile.
#pragma once
#include "unet_wgrad.cuh"

namespace sc {
namespace unet {

constexpr uint32_t kMnPair = 128 * 16;      // one (tap, channel group) pair: 128 pixels x 16 bytes
constexpr uint32_t kMnQRow = 32 * 16;       // a pair's quarter: 32 pixels x 16 bytes
constexpr uint32_t kMnQuarter = 16 * kMnQRow;  // one quarter of a slot: 16 pairs
constexpr uint32_t kMnSlot = 16 * kMnPair;  // one 128-row A block (4 quarters)
constexpr int kMnThreads = 192;             // producer, MMA issuer, 4 epilogue warps
constexpr int kMnMaxSlots = 6;

// the bias row's block: channel 0 of every pixel is one (BF16 0x3F80), the other channels zero
struct MnOnes {
  uint32_t w[kMnPair / 4];
};
__host__ __device__ constexpr MnOnes mn_ones() {
  MnOnes b{};
  for (int p = 0; p < 128; ++p) b.w[4 * p] = 0x3F80u;
  return b;
}
__device__ __align__(128) const MnOnes g_mn_ones = mn_ones();

__host__ __device__ constexpr uint32_t mn_b_bytes(int cout) { return align_up((uint32_t)(cout / 8) * kMnPair, 1024); }
__host__ __device__ constexpr size_t mn_smem_bytes(int cout, int slots) {
  return (size_t)slots * kMnSlot + 2 * mn_b_bytes(cout) + 256;
}

// xmap: the layer input as (8 w values, groups, h, images, 1), box (256, gb, 1, 1, 1); gmap: the
// output gradient, row-blocked (64, w / 8, groups, h, images), box (64, 16 or w / 8, 1, 1 or th,
// 1).  cin, cout multiples of 8, gb a divisor of both cin / 8 and 16; mtiles = ceil((9 cin + 1) /
// 128); w a multiple of 128, or 32 or 64.
template <bool NARROW>
__global__ void __launch_bounds__(kMnThreads, 1) k_wgrad_mn(const __grid_constant__ CUtensorMap xmap,
                                                              const __grid_constant__ CUtensorMap gmap, int cin,
                                                              int cout, int mtiles, int slots, int gb,
                                                              ConvGeo G, float *part, unsigned *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngx = cin / 8, ngz = cout / 8;
  const int npair = 9 * ngx;  // data blocks; block npair carries the bias row
  const uint32_t bb = mn_b_bytes(cout);
  const int h = G.h, w = G.w;
  uint8_t *sA = sm;
  uint8_t *sB = sA + slots * kMnSlot;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + 2 * bb);
  // [0, 6) A full, [6, 12) A empty, [12, 14) gz full, [14, 16) gz empty, [16] all MMAs done
  uint32_t *slotw = reinterpret_cast<uint32_t *>(bar + 17);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(slotw + 1);
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
    for (int s = 0; s < slots; ++s) {
      tc::mbar_init(tc::smem_addr(&bar[s]), 1);
      tc::mbar_init(tc::smem_addr(&bar[kMnMaxSlots + s]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(tc::smem_addr(&bar[12 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[14 + i]), 1);
    }
    tc::mbar_init(tc::smem_addr(&bar[16]), 1);
    *abort_flag = 0;
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_addr(slotw), cols);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t taddr = *slotw;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the gz tile, then the A blocks of every 128-row block, per pixel tile -----
      tc::prefetch_tmap(&xmap);
      tc::prefetch_tmap(&gmap);
      int nb = 0, na = 0;  // gz tiles and A blocks whose copies were issued
      bool stop = false;
      for (int i = 0; i < mine && !stop && !*abort_flag; ++i) {
        const int t = t0 + i;
        const int xt = t % tiles_x, r = t / tiles_x, y = (r % tiles_y) * G.th, img = r / tiles_y;
        const int bs = i & 1;
        if (i >= 2 && !tc::mbar_wait(tc::smem_addr(&bar[14 + bs]), ((i >> 1) - 1) & 1)) {
          stop = true;
          break;
        }
        const uint32_t bfull = tc::smem_addr(&bar[12 + bs]);
        tc::mbar_expect_tx(bfull, (uint32_t)ngz * kMnPair);
        const uint32_t bdst = tc::smem_addr(sB + bs * bb);
        for (int g = 0; g < ngz; ++g)
          tc::tma_load_5d(bdst + g * kMnPair, &gmap, 0, xt * (128 / 8), g, y, img, bfull);
        ++nb;
        const int x0 = NARROW ? 0 : xt * 128;
        for (int m = 0; m < mtiles; ++m) {
          const int s = na % slots, u = na / slots;
          if (u > 0 && !tc::mbar_wait(tc::smem_addr(&bar[kMnMaxSlots + s]), (u - 1) & 1)) {
            stop = true;
            break;
          }
          const int j0 = 16 * m, j1 = min(j0 + 16, npair + 1);
          const uint32_t afull = tc::smem_addr(&bar[s]);
          tc::mbar_expect_tx(afull, (uint32_t)(j1 - j0) * kMnPair);
          const uint32_t adst = tc::smem_addr(sA + s * kMnSlot);
          for (int q = 0; q < 4; ++q) {
            // the quarter's first pixel (row offset within the tile, column)
            const int p0 = 32 * q;
            const int xx = NARROW ? p0 % w : x0 + p0, yy = NARROW ? y + p0 / w : y;
            const uint32_t qd = adst + (uint32_t)q * kMnQuarter;
            for (int j = j0; j < min(j1, npair); j += gb) {
              const int tap = j / ngx, g = j - tap * ngx;
              const int dy = tap / 3, dx = tap - 3 * dy;
              tc::tma_load_5d(qd + (uint32_t)(j - j0) * kMnQRow, &xmap, 8 * (xx + dx - 1), g, yy + dy - 1, img, 0,
                              afull);
            }
            if (npair < j1) tc::bulk_load(qd + (uint32_t)(npair - j0) * kMnQRow, &g_mn_ones, kMnQRow, afull);
          }
          ++na;
        }
      }
      if (stop) *abort_flag = 1;
      // wait (bounded) for the copies still in flight before leaving: every earlier block's slot
      // was handed back by the MMA thread, so only the last `slots` A blocks and 2 gz tiles remain
      for (int k = na - slots; k < na; ++k)
        if (k >= 0) tc::mbar_wait(tc::smem_addr(&bar[k % slots]), (k / slots) & 1);
      for (int k = nb - 2; k < nb; ++k)
        if (k >= 0) tc::mbar_wait(tc::smem_addr(&bar[12 + (k & 1)]), (k >> 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ---------------------------------------------------------------------------
      const uint32_t idesc = tc::idesc_bf16_f32_mn(kTM, cout);
      // MN-major without swizzle: LBO = 128 bytes (next 8 pixels), SBO = next 8 channels (the next
      // pair of a quarter in A, the next 2 KB block in gz); descriptors advanced by start-field
      // adds of byte offsets / 16.  K step ks (16 pixels): A quarter ks / 2, half ks % 2.
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), 128u, kMnQRow);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sB), 128u, kMnPair);
      const uint32_t kstep = 256u >> 4;  // 16 pixels of gz
      const uint32_t alo0 = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
      const uint32_t blo0 = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
      auto desc = [](uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; };
      bool ok = true;
      int na = 0;
      for (int i = 0; ok && i < mine; ++i) {
        const int bs = i & 1;
        if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[12 + bs]), (i >> 1) & 1, abort_flag)) ok = false;
        const uint32_t bd = blo0 + (((uint32_t)bs * bb) >> 4);
        for (int m = 0; ok && m < mtiles; ++m, ++na) {
          const int s = na % slots;
          if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[s]), (na / slots) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t ad = alo0 + (((uint32_t)s * kMnSlot) >> 4);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            tc::mma_bf16(taddr + (uint32_t)m * cstride,
                         desc(ad + (((uint32_t)(ks >> 1) * kMnQuarter + (uint32_t)(ks & 1) * 256u) >> 4), ahi),
                         desc(bd + (uint32_t)ks * kstep, bhi), idesc, (i > 0 || ks > 0) ? 1u : 0u);
          tc::mma_commit(tc::smem_addr(&bar[kMnMaxSlots + s]));  // A slot free
        }
        if (ok) tc::mma_commit(tc::smem_addr(&bar[14 + bs]));  // gz tile free
      }
      if (!ok) *abort_flag = 1;
      tc::mma_commit(tc::smem_addr(&bar[16]));  // all MMAs issued by this thread complete
    }
  } else {
    // ---- epilogue (warps 2..5: TMEM lane quarters 2, 3, 0, 1): this CTA's partial sums ---------
    const int qd = warp & 3;
    const bool done = tc::mbar_wait(tc::smem_addr(&bar[16]), 0);
    tc::fence_after();
    const int Mpad = mtiles * kTM;
    for (int k = 0; k < mtiles; ++k)
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
