// unet_wgrad_mn.cuh -- weight gradients of the 3x3 convolutions and of the 2x2 stride-2 transposed
// convolutions on tcgen05, with MN-major operands that TMA delivers ready to use (tiles of 128
// pixels: part of a row of 128k pixels, or 128 / w whole narrower rows, as in unet_conv.cuh).
//
//   3x3:  gw[o][tap][c] = sum_p gz[p][o] * x[p + offset(tap)][c],   gb[o] = sum_p gz[p][o]
//   up:   gw[c][a][e][o] = sum_p x[p][c] * gz[(2y + a, 2x + e)][o],  gb[o] = sum over all children
//
// as D[A rows | ones][N columns] = sum over the tile's pixels (parents for the transposed conv).
// The tensors hold 8 consecutive channels per 16 bytes, which is the row of an MN-major core
// matrix when M (or N) is the channel and K the pixel: 8 consecutive pixels x 8 channels = one
// 128-byte core matrix.  So nothing is transposed.  A ring slot holds one 128-row block of A: 16
// pairs (tap, channel group), each the tile's 128 pixels shifted by the tap's offset (2 KB, pairs
// 2 KB apart).  The tensors are viewed with 8-byte elements (half a pixel) as (2 w, rows, groups,
// images): a one-pixel shift is an element offset of 2 (16 bytes), and one TMA copy (zeros outside
// the image) brings several pairs whole.  A CTA's copies are served about one after another, at a
// cost that grows slowly with their size, so few large copies matter more than anything else:
//  * columns (3x3, rows of 128k pixels, at most 48 input channels): one copy brings, for one dx and
//    gb channel groups, the three rows dy = 0..2 ((256, 3, gb) box: pairs ordered (group, dy)); a
//    block holds cpb = 16 / (3 gb) such copies (gb = 4, 2 or 1, so 12, 12 or 15 pairs; the rest
//    of the block is padding, whose accumulator rows are neither written nor read), blocks in copy
//    order k = dx * (cin / 8 / gb) + unit.  With more channels the padding costs more blocks
//    (MMAs, partials, TMEM chunks) than the fewer copies save (64 channels: 89.6 -> 98.1 us);
//  * tap-major (other 3x3 layers): pairs ordered (tap, group), one copy brings gb = gcd(cin / 8,
//    16) pairs of one tap (th rows of w pixels each), so that no copy straddles two blocks;
//  * up (the transposed conv): one tap, pairs = the input's channel groups; B is the output
//    gradient of each parent's four children, one copy per (a, e) through the parity view of the
//    child tensor (mn_layout_up; N = 4 cout columns ordered (a, e, o)).
// The bias row is a pair whose channel 0 is one, copied from a constant (the first pair after the
// data).  mn_layout() / mn_layout_up() give the block counts and the bias pair for the host, the
// kernel and the reduce.  Shared memory: the A ring, 1 KB of barriers, the two gz tiles.  One
// thread issues the MMAs; the accumulators of all 128-row blocks (N columns
// each, 32/64/128/256 apart) stay in TMEM across the CTA's contiguous range of tiles, and at the
// end the epilogue warps write them as this CTA's partial sums ([split][128 mtiles][N], the layout
// k_wgrad_reduce sums in a fixed order).  Where all blocks' accumulators do not fit in TMEM, the
// grid's y dimension splits them into chunks of `mchunk` blocks, one CTA per (tile range, chunk).
// The host runs two CTAs per SM on rows of 128k pixels where two ring slots each still fit.
// Every wait is bounded.
//
// Operand extents (LBO = 128 bytes: the next 8 pixels; SBO = 2 KB: the next 8 channels): one MMA
// (K = 16) reads 16 (or N / 8) pairs x 256 bytes from its start, which moves 256 bytes per K
// step, so every read stays inside its own 32 KB A slot or gz tile.
#pragma once
#include "unet_conv.cuh"

namespace sc {
namespace unet {

constexpr uint32_t kMnPair = 128 * 16;      // one (tap, channel group) pair: 128 pixels x 16 bytes
constexpr uint32_t kMnSlot = 16 * kMnPair;  // one 128-row A block
constexpr int kMnThreads = 192;             // producer, MMA issuer, 4 epilogue warps
constexpr int kMnMaxSlots = 6;
// TMEM columns between the accumulators of consecutive 128-row blocks (N FP32 columns each)
__host__ __device__ constexpr uint32_t wg_cstride(int n) {
  return n <= 32 ? 32u : (n <= 64 ? 64u : (n <= 128 ? 128u : 256u));
}

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

// layout of the A rows: blocks (mtiles), the bias pair, and for columns the copy shape
struct MnLayout {
  int up;      // 1: a 2x2 stride-2 transposed conv (one tap, B = the four children's gradients)
  int col;     // 1: columns (rows of 128k pixels), 0: tap-major
  int gb;      // channel groups per copy
  int nu;      // column copies per dx (cin / 8 / gb)
  int cpb;     // column copies per block
  int ncopy;   // column copies (3 nu)
  int mtiles;  // 128-row blocks
  int jones;   // the bias pair (its channel 0 is D row 8 jones)
};
__host__ __device__ inline MnLayout mn_layout(int cin, bool col) {
  MnLayout L;
  const int ng = cin / 8;
  L.up = 0;
  L.col = col ? 1 : 0;
  if (col) {
    L.gb = ng % 4 == 0 ? 4 : (ng % 2 == 0 ? 2 : 1);
    L.nu = ng / L.gb;
    L.cpb = 16 / (3 * L.gb);
    L.ncopy = 3 * L.nu;
    L.mtiles = (L.ncopy + L.cpb - 1) / L.cpb;
    L.jones = 16 * (L.mtiles - 1) + (L.ncopy - (L.mtiles - 1) * L.cpb) * 3 * L.gb;
  } else {
    int g = ng, b = 16;  // gcd(ng, 16)
    while (b) {
      const int r = g % b;
      g = b;
      b = r;
    }
    L.gb = g;
    L.nu = L.cpb = L.ncopy = 0;
    L.jones = 9 * ng;
    L.mtiles = (8 * L.jones + 1 + 127) / 128;
  }
  return L;
}

// the transposed conv: A rows c | ones (its pairs are the channel groups, 16 per copy), N = 4 cout
__host__ __device__ inline MnLayout mn_layout_up(int cin) {
  MnLayout L;
  const int ng = cin / 8;
  L.up = 1;
  L.col = 0;
  L.gb = ng < 16 ? ng : 16;
  L.nu = L.cpb = L.ncopy = 0;
  L.jones = ng;
  L.mtiles = (8 * L.jones + 1 + 127) / 128;
  return L;
}

__host__ __device__ constexpr uint32_t mn_b_bytes(int cout) { return align_up((uint32_t)(cout / 8) * kMnPair, 1024); }
// shared memory: the A ring, 1 KB of barriers, the two gz tiles
__host__ __device__ constexpr size_t mn_smem_bytes(int cout, int slots) {
  return (size_t)slots * kMnSlot + 1024 + 2 * (size_t)mn_b_bytes(cout);
}

// xmap: the layer input, gmap: its output gradient, both as (2 w, h, groups, images, 1) of 8-byte
// elements with boxes (256, 3, L.gb, 1, 1) for columns or (256 or 2 w, 1 or th, L.gb, 1, 1), and
// (256 or 2 w, 1 or th, cout / 8, 1, 1).  cin, cout multiples of 8; L = mn_layout(cin, columns)
// with columns only on rows of 128k pixels; mtiles = L.mtiles.
template <bool NARROW>
__global__ void __launch_bounds__(kMnThreads, 1) k_wgrad_mn(const __grid_constant__ CUtensorMap xmap,
                                                              const __grid_constant__ CUtensorMap gmap, int cin,
                                                              int cout, int mtiles, int mchunk, int slots,
                                                              MnLayout L, ConvGeo G, float *part,
                                                              unsigned *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngx = cin / 8, ngz = cout / 8;
  const int npair = (L.up ? 1 : 9) * ngx;  // data pairs (tap-major: pair npair carries the bias row)
  const int gb = L.gb;
  const uint32_t bb = mn_b_bytes(cout);
  const int h = G.h, w = G.w;
  uint8_t *sA = sm;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sA + slots * kMnSlot);
  uint8_t *sB = sA + slots * kMnSlot + 1024;
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
  // this CTA's 128-row blocks [mb0, mb1)
  const int mb0 = (int)blockIdx.y * mchunk, mb1 = min(mb0 + mchunk, mtiles), nmb = mb1 - mb0;
  uint32_t cols = 32;
  while (cols < (uint32_t)nmb * cstride) cols <<= 1;
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
        const int x0 = NARROW ? 0 : xt * 128;
        if (L.up) {
          // the children (2y + a, 2x + e) of the tile's parents, one copy per (a, e): N columns
          // ordered (a, e, output channel)
          const int gq = ngz / 4;
          for (int ae = 0; ae < 4; ++ae)
            tc::tma_load_5d(tc::smem_addr(sB + bs * bb) + (uint32_t)(ae * gq) * kMnPair, &gmap, 0, ae & 1, x0,
                            img * 2 * h + 2 * y + (ae >> 1), 0, bfull);
        } else {
          tc::tma_load_5d(tc::smem_addr(sB + bs * bb), &gmap, 2 * x0, y, 0, img, 0, bfull);
        }
        ++nb;
        for (int m = mb0; m < mb1; ++m) {
          const int s = na % slots, u = na / slots;
          if (u > 0 && !tc::mbar_wait(tc::smem_addr(&bar[kMnMaxSlots + s]), (u - 1) & 1)) {
            stop = true;
            break;
          }
          const uint32_t afull = tc::smem_addr(&bar[s]);
          const uint32_t adst = tc::smem_addr(sA + s * kMnSlot);
          if (L.col) {
            // columns: copies k0..k1-1 of 3 gb pairs each, then (last block) the bias pair
            const int k0 = m * L.cpb, k1 = min(k0 + L.cpb, L.ncopy);
            const bool last = m == mtiles - 1;
            tc::mbar_expect_tx(afull, ((uint32_t)(k1 - k0) * 3u * (uint32_t)gb + (last ? 1u : 0u)) * kMnPair);
            for (int k = k0; k < k1; ++k) {
              const int dx = k / L.nu, un = k - dx * L.nu;
              tc::tma_load_5d(adst + (uint32_t)((k - k0) * 3 * gb) * kMnPair, &xmap, 2 * (x0 + dx - 1), y - 1, un * gb,
                              img, 0, afull);
            }
            if (last) tc::bulk_load(adst + (uint32_t)((k1 - k0) * 3 * gb) * kMnPair, &g_mn_ones, kMnPair, afull);
            ++na;
            continue;
          }
          const int j0 = 16 * m, j1 = min(j0 + 16, npair + 1);
          tc::mbar_expect_tx(afull, (uint32_t)(j1 - j0) * kMnPair);
          for (int j = j0; j < min(j1, npair); j += gb) {
            const int tap = L.up ? 4 : j / ngx, g = L.up ? j : j - tap * ngx;  // the up conv: no shift
            const int dy = tap / 3, dx = tap - 3 * dy;
            tc::tma_load_5d(adst + (uint32_t)(j - j0) * kMnPair, &xmap, 2 * (x0 + dx - 1), y + dy - 1, g, img, 0,
                            afull);
          }
          if (npair < j1) tc::bulk_load(adst + (uint32_t)(npair - j0) * kMnPair, &g_mn_ones, kMnPair, afull);
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
      // MN-major without swizzle: LBO = 128 bytes (next 8 pixels), SBO = one pair (next 8
      // channels); descriptors advanced by start-field adds of byte offsets / 16
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), 128u, kMnPair);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sB), 128u, kMnPair);
      const uint32_t kstep = 256u >> 4;  // 16 pixels
      const uint32_t alo0 = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
      const uint32_t blo0 = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
      auto desc = [](uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; };
      bool ok = true;
      int na = 0;
      for (int i = 0; ok && i < mine; ++i) {
        const int bs = i & 1;
        if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[12 + bs]), (i >> 1) & 1, abort_flag)) ok = false;
        const uint32_t bd = blo0 + (((uint32_t)bs * bb) >> 4);
        for (int m = mb0; ok && m < mb1; ++m, ++na) {
          const int s = na % slots;
          if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[s]), (na / slots) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t ad = alo0 + (((uint32_t)s * kMnSlot) >> 4);
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            tc::mma_bf16(taddr + (uint32_t)(m - mb0) * cstride, desc(ad + (uint32_t)ks * kstep, ahi),
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
    for (int k = mb0; k < mb1; ++k) {
      // rows of a column block past its copies and its bias pair are padding: not written (the
      // reduce never reads them)
      const int pair = (32 * qd + lane) >> 3;
      const int used = L.col ? (min(L.cpb, L.ncopy - k * L.cpb) * 3 * gb + (k == mtiles - 1 ? 1 : 0)) : 16;
      for (int n0 = 0; n0 < cout; n0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(k - mb0) * cstride + (uint32_t)n0, v);
        if (done && !*abort_flag && mine > 0 && pair < used) {
          float4 *p = reinterpret_cast<float4 *>(part + ((int64_t)blockIdx.x * Mpad + 128 * k + 32 * qd + lane) * cout +
                                                 n0);
#pragma unroll
          for (int j = 0; j < 4; ++j) p[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
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
