// unet_conv.cuh -- persistent, warp-specialised 3x3 convolution (forward or data gradient) on
// tcgen05 with TMA halo tiles, for rows whose width is a multiple of 128 pixels or divides 128,
// and the same kernel in a pointwise mode (one tap: a contraction of each pixel's channels).
//
// A tile is 128 consecutive output pixels of one image row.  For each group of 8 input channels
// the producer warp loads, with one TMA tensor copy, the 3 x 144 pixel neighbourhood of the tile
// (rows y-1..y+1, columns x0-8..x0+135: whole 8-pixel blocks of the row-blocked tensor, so each
// row of the box is one contiguous 2304-byte run; outside the image the hardware fills zeros)
// into a "slab": pixel-major rows of 16 bytes.  In that slab, the 128 input pixels that tap
// (dy, dx) multiplies are consecutive 16-byte rows, so the MMA operand of every tap is the same
// slab seen from a shifted start address (8-row core matrices 128 bytes apart, k-groups one slab
// apart): nine taps, one load.  The weights of the whole layer stay resident in shared memory
// (one bulk copy per CTA, laid out in global memory exactly as the MMA reads them).  When the
// input has more channels than two A stages can hold next to the weights, a tile's channels are
// streamed in chunks of `gs` groups of 8, accumulating into the same TMEM columns.
//
// Rows narrower than 128 pixels (w = 64, 32, 16): a tile is 128 / w whole rows, and per group of
// 8 channels three TMA copies bring the (rows + 2) x w neighbourhood shifted by dx = -1, 0, +1
// (zero-filled outside the image) into three slabs whose rows are exactly w pixels long, so that
// tap (dy, dx) is again 128 consecutive 16-byte rows: slab dx read from row dy.
//
// Pointwise mode (ConvGeo.taps == 1): per group of 8 channels one TMA copy of the tile's own 128
// pixels (whole 8-pixel blocks, no halo) and a single tap; with N <= 256 output columns it serves
// the 2x2 stride-2 transposed convolution, whose columns are the four output pixels' channels.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer (one thread each), warps
// 2..5 = epilogue (TMEM -> registers -> epilogue functor).  Two shared-memory A stages and two
// TMEM accumulators let the loads of tile i+1 and the epilogue of tile i-1 overlap the MMAs of
// tile i.  The single issuing thread is the kernel's critical path, so its loop does little
// besides the MMAs: descriptors built once and advanced by 32-bit adds on their start field, the
// abort flag read only inside waits that have not completed.  Every wait is bounded; a timeout
// latches SC_STATUS_WATCHDOG and the CTA winds down.
#pragma once
#include "unet_gemm.cuh"

namespace sc {
namespace unet {

// wide-row slab: 3 rows of 144 pixels starting kHaloLead pixels left of the tile (18 blocks of 8)
constexpr int kHaloW = 144, kHaloH = 3, kHaloLead = 8;
constexpr uint32_t kSlabBytes = 6912;  // 8 channels x 3 x 144 pixels x 2 bytes (54 x 128)
constexpr uint32_t kSlabTx = 6912;
constexpr int kConvThreads = 192;

__host__ __device__ constexpr uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }
__host__ __device__ constexpr uint32_t conv_w_bytes(int cin_p, int N, int taps = 9) {
  return (uint32_t)taps * (uint32_t)cin_p * N * 2u;
}
__host__ __device__ constexpr uint32_t conv_a_bytes(int gs) { return (uint32_t)gs * kSlabBytes; }
__host__ __device__ constexpr uint32_t conv_acc_cols(int N) {
  return N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
}
// gs: groups of 8 input channels per A stage, gstride: bytes per group in a stage
__host__ __device__ constexpr size_t conv_smem_bytes(int cin_p, int N, int gs, uint32_t gstride = kSlabBytes,
                                                     int taps = 9) {
  return align_up(conv_w_bytes(cin_p, N, taps), 1024) + 2 * align_up((uint32_t)gs * gstride, 1024) + 128;
}

// Tiling of one launch: wide rows (w a multiple of 128: tiles of 128 pixels of a row, one 3 x 144
// slab per channel group) or narrow rows (128 / w rows per tile, three dx-shifted slabs).
struct ConvGeo {
  int n_img, h, w;
  int taps;          // 9 (3x3) or 1 (pointwise: the tile's own pixels, no halo)
  int narrow;        // 0 wide, 1 narrow
  int th;            // rows per tile (narrow)
  uint32_t slab;     // bytes of one dx slab (narrow)
  uint32_t gstride;  // bytes of one channel group in a stage
  uint32_t tx;       // bytes the TMA copies of one channel group deliver
  int up;            // pointwise on a transposed conv's children (the data gradient): A through the
                     // parity view, K group kg = (a, e) * ngc + child channel group
  int ngc;           // child channel groups (up only)
};
__host__ __device__ inline ConvGeo conv_geo(int n_img, int h, int w, int taps = 9) {
  ConvGeo g;
  g.n_img = n_img;
  g.h = h;
  g.w = w;
  g.taps = taps;
  g.up = 0;
  g.ngc = 0;
  g.narrow = w < 128;
  g.th = g.narrow ? 128 / w : 1;
  if (taps == 1) {  // 128 pixels x 16 bytes per channel group, whole 8-pixel blocks
    g.slab = 0u;
    g.gstride = g.tx = 128u * 16u;
    return g;
  }
  g.slab = g.narrow ? align_up((uint32_t)(g.th + 2) * w * 16u, 128) : 0u;
  g.gstride = g.narrow ? 3u * g.slab : kSlabBytes;
  g.tx = g.narrow ? 3u * (uint32_t)(g.th + 2) * w * 16u : kSlabTx;
  return g;
}

// Resident weights: wt[tap][kg][n][8] BF16 (kg = group of 8 reduction channels), i.e. for each
// (tap, kg) the N rows of 16 bytes the B operand needs.  amap: 5-D tensor map of the row-blocked
// input slice: wide rows (64 = 8 pixels x 8 channels, w / 8 pixel blocks, channel groups,
// height, images), box (64, 18, 1, 3, 1); narrow rows (8 channels, w, channel groups, height,
// images), box (8, w, 1, th + 2, 1).  Pointwise (G.taps == 1, e.g. a 2x2 stride-2 transposed
// conv, whose N columns are the four output pixels' channels): the blocked map with box
// (64, 16 or w / 8, 1, 1 or th, 1) and wt[kg][n][8].
template <class EP>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_tma(const __grid_constant__ CUtensorMap amap,
                                                              const bf16 *__restrict__ wt, int cin_p, int N, int gs,
                                                              ConvGeo G, int sign, EP E, unsigned *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ng = cin_p / 8;
  const int nchunk = ng / gs;
  const uint32_t wbytes = conv_w_bytes(cin_p, N, G.taps);
  const uint32_t astride = align_up((uint32_t)gs * G.gstride, 1024);
  const int h = G.h, w = G.w;
  uint8_t *sW = sm;
  uint8_t *sA = sm + align_up(wbytes, 1024);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sA + 2 * astride);
  // bar[0] weights full, [1,2] A full, [3,4] A empty, [5,6] accumulator full, [7,8] accumulator empty,
  // [9] drain: the MMAs still in flight when the issuer gives up (10 barriers + 2 words fit the 128
  // bytes conv_smem_bytes reserves)
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 10);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(slot + 1);
  const int tiles_x = G.narrow ? 1 : w / 128;
  const int tiles_y = G.narrow ? h / G.th : h;
  const int ntiles = G.n_img * tiles_y * tiles_x;
  const uint32_t half = conv_acc_cols(N);  // column offset of accumulator 1
  const uint32_t cols = 2 * half;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_addr(&bar[0]), 1);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(tc::smem_addr(&bar[1 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[3 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[5 + i]), 1);
      tc::mbar_init(tc::smem_addr(&bar[7 + i]), 4);
    }
    tc::mbar_init(tc::smem_addr(&bar[9]), 1);
    *abort_flag = 0;
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
      // ---- producer ------------------------------------------------------------------------
      tc::mbar_expect_tx(tc::smem_addr(&bar[0]), wbytes);
      tc::bulk_load(tc::smem_addr(sW), wt, wbytes, tc::smem_addr(&bar[0]));
      int issued = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        const int xt = t % tiles_x, r = t / tiles_x, y = (r % tiles_y) * G.th, img = r / tiles_y;
        for (int ch = 0; ch < nchunk; ++ch, ++issued) {
          const int s = issued & 1, u = issued >> 1;
          if (u > 0 && !tc::mbar_wait(tc::smem_addr(&bar[3 + s]), (u - 1) & 1)) {
            *abort_flag = 1;
            break;
          }
          if (*abort_flag) break;
          const uint32_t full = tc::smem_addr(&bar[1 + s]);
          tc::mbar_expect_tx(full, (uint32_t)gs * G.tx);
          const uint32_t dst = tc::smem_addr(sA + s * astride);
          for (int g = 0; g < gs; ++g) {
            if (G.up) {
              // the children (2y + a, 2x + e) of the tile's parents for K group (a, e, child group)
              const int kg = ch * gs + g, ae = kg / G.ngc, og = kg - ae * G.ngc;
              tc::tma_load_5d(dst + g * G.gstride, &amap, 0, ae & 1, G.narrow ? 0 : xt * 128,
                              img * 2 * h + 2 * y + (ae >> 1), og, full);
            } else if (G.taps == 1) {
              tc::tma_load_5d(dst + g * G.gstride, &amap, 0, G.narrow ? 0 : xt * (128 / 8), ch * gs + g, y, img, full);
            } else if (G.narrow) {
              for (int dx = 0; dx < 3; ++dx)
                tc::tma_load_5d(dst + g * G.gstride + dx * G.slab, &amap, 0, dx - 1, ch * gs + g, y - 1, img, full);
            } else {
              tc::tma_load_5d(dst + g * G.gstride, &amap, 0, xt * (128 / 8) - kHaloLead / 8, ch * gs + g, y - 1, img,
                              full);
            }
          }
        }
      }
      // wait (bounded) for the copies still in flight before leaving
      for (int k = issued - 2; k < issued; ++k)
        if (k >= 0) tc::mbar_wait(tc::smem_addr(&bar[1 + (k & 1)]), (k >> 1) & 1);
      tc::mbar_wait(tc::smem_addr(&bar[0]), 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer -----------------------------------------------------------------------
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, N);
      bool ok = tc::mbar_wait(tc::smem_addr(&bar[0]), 0);
      int i = 0, staged = 0;
      // Descriptors are built once and advanced by adding byte offsets / 16 to their start
      // field (every start is a multiple of 16 below 2^18, so the 14-bit field never carries):
      // A: stage base + the tap's shift in the slab + 2 groups per K step of 16;
      // B: weights of (tap, channel group) at (tap * ng + group) * N rows of 16 bytes.
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), G.gstride, 128u);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sW), (uint32_t)N * 16u, 128u);
      uint32_t toff[9];
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        if (G.taps == 1) {
          toff[tap] = 0u;
          continue;
        }
        const int ty = tap / 3, tx = tap - 3 * ty;
        const int sy = sign * (ty - 1) + 1, sx = sign * (tx - 1) + 1;  // neighbourhood row / column (0..2)
        // start of the 128 rows output pixel 0 multiplies at this tap
        toff[tap] = (G.narrow ? (uint32_t)sx * G.slab + (uint32_t)(sy * w) * 16u
                              : (uint32_t)(sy * kHaloW + sx + kHaloLead - 1) * 16u) >> 4;
      }
      const uint32_t kstep = (2u * G.gstride) >> 4, sstep = astride >> 4, tstep = (uint32_t)(ng * N);
      // only the low word (start field) of a descriptor moves: 32-bit adds, then the fixed high word
      const uint32_t alo0 = (uint32_t)adesc0, ahi = (uint32_t)(adesc0 >> 32);
      const uint32_t blo0 = (uint32_t)bdesc0, bhi = (uint32_t)(bdesc0 >> 32);
      auto desc = [](uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; };
      // the issue loop is the kernel's critical path: it checks the abort flag only inside waits
      // that have not completed yet
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++i) {
        const int a = i & 1, ua = i >> 1;  // accumulator and its use count
        if (ua > 0 && !tc::mbar_wait_or_abort(tc::smem_addr(&bar[7 + a]), (ua - 1) & 1, abort_flag)) ok = false;
        const uint32_t d = taddr + (uint32_t)a * half;
        for (int ch = 0; ok && ch < nchunk; ++ch, ++staged) {
          const int s = staged & 1, u = staged >> 1;
          if (!tc::mbar_wait_or_abort(tc::smem_addr(&bar[1 + s]), u & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t as = alo0 + (uint32_t)s * sstep;
          const uint32_t bs = blo0 + (uint32_t)(ch * gs) * (uint32_t)N;
          if (gs == 2) {  // one K step of 16 per tap
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
              if (tap >= G.taps) break;
              tc::mma_bf16(d, desc(as + toff[tap], ahi), desc(bs + (uint32_t)tap * tstep, bhi), idesc,
                           (ch > 0 || tap > 0) ? 1u : 0u);
            }
          } else {
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
              if (tap >= G.taps) break;
              const uint32_t at = as + toff[tap], bt = bs + (uint32_t)tap * tstep;
              for (int ks = 0; ks < gs / 2; ++ks)
                tc::mma_bf16(d, desc(at + (uint32_t)ks * kstep, ahi), desc(bt + 2u * (uint32_t)ks * (uint32_t)N, bhi),
                             idesc, (ch > 0 || tap > 0 || ks > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(tc::smem_addr(&bar[3 + s]));  // A stage free
        }
        if (ok) tc::mma_commit(tc::smem_addr(&bar[5 + a]));  // accumulator full
      }
      if (!ok) {
        *abort_flag = 1;
        // MMAs already issued may still be writing the accumulators: commit them to the drain
        // barrier and wait (bounded) before the CTA frees its TMEM.  On the normal path the epilogue
        // has waited for every accumulator, so nothing is in flight there.
        if (staged > 0) {
          tc::mma_commit(tc::smem_addr(&bar[9]));
          tc::mbar_wait(tc::smem_addr(&bar[9]), 0);
        }
      }
    }
  } else {
    // ---- epilogue (warps 2..5; warp w reads TMEM lanes 32 * (w % 4) ..) -------------------------
    const int q = warp & 3;
    const int r = 32 * q + lane;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int s = i & 1, u = i >> 1;
      if (!tc::mbar_wait(tc::smem_addr(&bar[5 + s]), u & 1)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after();
      const int xt = t % tiles_x, rr = t / tiles_x;
      // rr = img * tiles_y + tile row; the tile starts at pixel (img * h + y0) * w + xt * 128
      const int row = ((rr / tiles_y) * h + (rr % tiles_y) * G.th) * w + xt * 128 + r;
      for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)s * half + (uint32_t)n0, v);
        E.store(row, n0, v, 0);
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tc::smem_addr(&bar[7 + s]));
      if (*abort_flag) break;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(taddr, cols);
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, SC_STATUS_WATCHDOG);
}

}  // namespace unet
}  // namespace sc
