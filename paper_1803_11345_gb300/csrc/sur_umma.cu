// Forward 3x3 periodic convolution of the surrogate U-Net on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), BF16 operands, FP32 accumulation.  The paper has no
// counterpart (the surrogate is an extension around the solver).  Declared in include/surrogate.h
// (sur_conv3x3_tc, sur_transpose_taps, sur_check).
//
// Implicit GEMM: M = pixels, N = output channels, K = 9 taps x input channels, on 128 threads per
// CTA.  An accumulator is 128 TMEM lanes (one per pixel) x N-tile columns of FP32; the input
// channels are taken 16 at a time (one K step of the instruction per tap).  Operands sit in
// shared memory in the tensor core's no-swizzle K-major layout: 8-row x 16-byte core matrices,
// rows = pixels (A) or output channels (B), whose 8-row groups are 128 bytes apart (SBO) and whose
// two 8-channel halves ("octets") are one block apart (LBO).  A core matrix may start at any
// 16-byte row, so a shifted window of staged pixels is the same memory seen from another start:
//   * row mode (W >= 128): a tile is RT image rows x 128 columns (RT accumulators).  A is the
//     RT + 2 rows around them, each row staged with one wrapped halo column on either side, in a
//     row of 144 pixel slots whose 128 centre pixels start at slot 8 (a 128-byte boundary):
//     [octet][halo row][144 slots][8 x BF16].  The operand of tap (dy, dx) for output row r
//     starts at slot (r + dy + 1) * 144 + 8 + dx: 9 RT descriptors, no copies.  Without the
//     upsampling the rows come in by TMA (a tensor map over the NHWC input, one 128-pixel box
//     per row and octet, and 16-byte bulk copies for the two wrapped halo pixels) issued by one
//     thread, completing the stage's mbarrier by byte count.
//   * copy mode (W < 128, W a power of two dividing 128): RT accumulators of R = 128/W full rows
//     each, which a start offset cannot shift by a column across the row seams, so A holds the
//     RT R + 2 rows around them in three copies shifted by dx = -1, 0, +1 with the periodic wrap
//     applied while staging: [dx][octet][halo-tile pixel][8 x BF16]; tap (dy, dx) of accumulator r
//     starts at pixel (r R + dy + 1) * W of copy dx.
//   * B: the 9 taps' weights for the N tile, from the K-major copy [tap][N][K] (see
//     sur_transpose_taps): [octet][tap][output channel][8 x BF16], by TMA in every mode (one box
//     per octet), shared by every accumulator.
// A persistent CTA walks its tiles; every (tile, 16-channel chunk) is an item of a ring of S
// (2 to 6) shared-memory stages, filled by TMA (one lane per octet and staged row; with one N
// tile the weights of all chunks stay resident, loaded once) or, in copy mode and when
// upsampling, by four producer warps' 16-byte cp.async copies; one thread issues each item's MMAs into one of two
// accumulator sets (the epilogue of a tile overlaps the next tile's MMAs) and commits them to
// the stage's "empty" mbarrier.  Every mbarrier wait is bounded: a wait that gives up sets the
// status word read by sur_check, lets the copies and MMAs it issued finish (again bounded), frees
// the tensor memory and returns.  The epilogue reads the accumulators with tcgen05.ld (each warp
// its 32 lanes), adds the bias and an optional addend (the decoder's skip), applies ReLU, and
// stores BF16 or FP32 NHWC rows.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "../../include/surrogate.h"
#include "lbm_tma.cuh"

namespace {

using bf16 = __nv_bfloat16;
using lbmch::bulk_g2s;
using lbmch::mbar_arrive_expect_tx;
using lbmch::mbar_fence_init;
using lbmch::mbar_init;
using lbmch::mbar_try_wait;
using lbmch::smem_u32;

// Status word: set when a bounded wait of a tensor-core kernel gave up (read and cleared by
// sur_check).
__device__ int g_tc_status;

constexpr uint32_t kWaitProbes = 1u << 22;
constexpr int kTileM = 128;

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t k = 0; k < kWaitProbes; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory writes before the tensor core's reads.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[adesc] * B[bdesc] for one 128 x N x 16 step (kind::f16, BF16 in, FP32 out).
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w .. 32w + 31).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, LBO (byte distance between the
// core matrices of adjacent 8-element K groups), SBO (between adjacent 8-row M or N groups), the
// fixed version bits 46-48 = 0b001, base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

struct ConvTC {
  int H, W;             // output image
  int Hs, Ws;           // source image (H/2 x W/2 when upsampled)
  int K, N;             // input / output channels
  int rows_mode;        // 1: row mode (W >= 128), 0: copy mode
  int TW, R;            // copy mode: tile of R rows x TW = W columns; row mode: TW = 128, R = 1
  int RT;               // accumulators per tile: row mode output rows, copy mode blocks of R rows
  int tw_shift;         // log2(TW)
  int tiles_x, tiles_y; // M tiles per image along x and y
  int ntiles_n;         // N tiles
  int ntiles;           // all tiles: batch x tiles_y x tiles_x x ntiles_n
  int nchunks;          // K / 16
  int ntile;            // output channels per tile
  uint32_t ncols;       // TMEM columns allocated: two accumulator sets (double buffer)
  uint32_t acc_cols;    // TMEM column stride between accumulators of a set
  uint32_t set_cols;    // columns of one set (RT accumulators)
  uint32_t a_block, a_stage, b_block, stage_bytes;
  uint32_t tx_bytes;    // bytes one item brings in (TMA mode: the stage's expected transaction count)
  uint32_t idesc;
  int relu, out_f32, up;
  int tma;              // 1: row mode without upsampling, staged by TMA
  int wres;             // 1 (TMA mode, one N tile): all weights resident in shared memory, loaded once
  uint32_t wres_off;    // byte offset of the resident weights (after the stages)
  uint32_t w_bytes;     // bytes of the resident weights: nchunks x 18 blocks
  uint32_t bar_off;     // byte offset of the barriers
};

constexpr int kRowSlots = 144;  // pixel slots per staged row in row mode (16 bytes each)
constexpr int kRowFirst = 7;    // slot of the left halo pixel; the 128 centre pixels start at slot 8
// Warp roles of the persistent kernel: 4 producer warps (copies), 1 MMA warp (also allocates the
// tensor memory), 4 epilogue warps (one per TMEM lane quarter).
constexpr int kProducers = 128;
constexpr int kMmaWarp = 4;
constexpr int kThreadsP = 288;

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Raise the barrier's expected transaction count of its current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_role(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (uint32_t k = 0; k < kWaitProbes; ++k) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((k & 63u) == 63u && *abort) return false;
  }
  return false;
}

// Tensor-map box loads into shared memory, completing `bar` by byte count.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

struct TileCoord {
  int b, y0, x0, n0;
};
__device__ __forceinline__ TileCoord tile_coord(const ConvTC& c, int t) {
  TileCoord q;
  const int nt = t % c.ntiles_n;
  const int m = t / c.ntiles_n;
  const int per_img = c.tiles_x * c.tiles_y;
  q.b = m / per_img;
  const int rem = m - q.b * per_img;
  q.y0 = (rem / c.tiles_x) * (c.rows_mode ? c.RT : c.RT * c.R);
  q.x0 = (rem % c.tiles_x) * c.TW;
  q.n0 = nt * c.ntile;
  return q;
}

// Persistent kernel: CTA j takes tiles j, j + gridDim.x, ...; every (tile, channel chunk) is one
// item of a ring of S shared-memory stages.
template <int S>
__global__ void __launch_bounds__(kThreadsP)
k_conv3x3_tc(const bf16* __restrict__ x, const bf16* __restrict__ wt, const float* __restrict__ bias,
             const bf16* __restrict__ addend, void* __restrict__ y, const ConvTC c,
             const __grid_constant__ CUtensorMap tm_rows, const __grid_constant__ CUtensorMap tm_w) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + c.bar_off);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint64_t* wbar = done + 1;  // the resident weights have landed
  volatile int* abort = reinterpret_cast<volatile int*>(wbar + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1) + 1;
  unsigned char* const wsm = smem + c.wres_off;

  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tslot), c.ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full[k], c.tma ? 2 : kProducers);  // TMA mode: the copy warp and the halo warp
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&tfull[k], 1);
      mbar_init(&tempty[k], 128);
    }
    mbar_init(done, 1);
    mbar_init(wbar, 1);
    *abort = 0;
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  auto give_up = [&]() {
    *abort = 1;
    atomicOr(&g_tc_status, 1);
  };

  if (c.tma && tid < kProducers) {
    // ---- TMA producer: warp 0.  Lane 0 arms a stage with its byte count; one lane per (octet,
    // staged row) then issues that row's 128-pixel box and its two wrapped halo pixels, and (when
    // the weights are not resident) lanes 30 and 31 the weight boxes.  Stage i % S is full once
    // its bytes have landed.  Resident weights: every (chunk, octet) box once, on wbar.
    if (warp == 0) {
      if (c.wres) {
        if (lane == 0) mbar_arrive_expect_tx(wbar, c.w_bytes);
        __syncwarp();
        for (int j = lane; j < 2 * c.nchunks; j += 32)
          tma_load_3d(wsm + (uint32_t)j * 9 * c.b_block, &tm_w, (j >> 1) * 16 + (j & 1) * 8, 0, 0, wbar);
      }
      int i = 0;
      bool ok = true;
      const int nrow = c.RT + 2;
      for (int t = blockIdx.x; t < c.ntiles && ok; t += gridDim.x) {
        const TileCoord q = tile_coord(c, t);
        for (int ch = 0; ch < c.nchunks; ++ch, ++i) {
          const int st = i % S;
          if (i >= S && !__all_sync(0xffffffffu, wait_role(&empty[st], (uint32_t)((i / S) - 1) & 1u, abort))) {
            if (lane == 0) give_up();
            ok = false;
            break;
          }
          unsigned char* A = smem + (uint32_t)st * c.stage_bytes;
          if (lane == 0) mbar_arrive_expect_tx(&full[st], c.tx_bytes);
          __syncwarp();
          const int k0 = ch * 16;
          if (lane < 2 * nrow) {
            const int kc = lane / nrow, hr = lane - kc * nrow;
            const int yy = wrap(q.y0 + hr - 1, c.H);
            unsigned char* row = A + kc * c.a_block + hr * (kRowSlots * 16);
            tma_load_4d(row + (kRowFirst + 1) * 16, &tm_rows, k0 + kc * 8, q.x0, yy, q.b, &full[st]);
          }
          if (!c.wres && lane >= 30) {
            const int kc = lane - 30;
            tma_load_3d(A + c.a_stage + kc * 9 * c.b_block, &tm_w, k0 + kc * 8, q.n0, 0, &full[st]);
          }
        }
      }
    }
    if (warp == 1) {
      // ---- halo warp: the wrapped pixel left and right of every staged row (one 16-byte load
      // and store per lane: octet, row and side), fenced for the tensor core's reads; the stage
      // is full once these and the copy warp's bytes are in.  Per-pixel bulk copies cost as much
      // staging time as the rows' boxes.
      int i = 0;
      bool ok = true;
      const int nrow = c.RT + 2;
      for (int t = blockIdx.x; t < c.ntiles && ok; t += gridDim.x) {
        const TileCoord q = tile_coord(c, t);
        for (int ch = 0; ch < c.nchunks; ++ch, ++i) {
          const int st = i % S;
          if (i >= S && !__all_sync(0xffffffffu, wait_role(&empty[st], (uint32_t)((i / S) - 1) & 1u, abort))) {
            if (lane == 0) give_up();
            ok = false;
            break;
          }
          for (int e = lane; e < 4 * nrow; e += 32) {  // (octet, staged row, side)
            const int side = e & 1, kc = (e >> 1) / nrow, hr = (e >> 1) - kc * nrow;
            const int yy = wrap(q.y0 + hr - 1, c.H);
            const int xx = side ? wrap(q.x0 + kTileM, c.W) : wrap(q.x0 - 1, c.W);
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(
                x + (((size_t)q.b * c.H + yy) * c.W + xx) * c.K + ch * 16 + kc * 8));
            unsigned char* row = smem + (uint32_t)st * c.stage_bytes + kc * c.a_block + hr * (kRowSlots * 16);
            *reinterpret_cast<uint4*>(row + (side ? kRowFirst + 1 + kTileM : kRowFirst) * 16) = v;
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[st]);
        }
      }
    }
  } else if (tid < kProducers) {
    // ---- producers: copy item i into stage i % S; signal item i - 1 full once this thread's
    // copies of it have landed (and were fenced for the tensor core's reads).  The one-item lag
    // leaves the MMAs S - 2 items of slack before a stage is needed again.
    int i = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < c.ntiles && ok; t += gridDim.x) {
      const TileCoord q = tile_coord(c, t);
      auto src_pixel = [&](int yy, int xx) -> size_t {
        return c.up ? ((size_t)q.b * c.Hs + (yy >> 1)) * c.Ws + (xx >> 1) : ((size_t)q.b * c.H + yy) * c.W + xx;
      };
      for (int ch = 0; ch < c.nchunks; ++ch, ++i) {
        const int st = i % S;
        if (i >= S && !wait_role(&empty[st], (uint32_t)((i / S) - 1) & 1u, abort)) {
          give_up();
          ok = false;
          break;
        }
        unsigned char* A = smem + (uint32_t)st * c.stage_bytes;
        unsigned char* Bm = A + c.a_stage;
        const int k0 = ch * 16;
        if (c.rows_mode) {
          for (int kc = 0; kc < 2; ++kc)
            for (int hr = 0; hr < c.RT + 2; ++hr) {
              const int yy = wrap(q.y0 + hr - 1, c.H);
              unsigned char* dst = A + kc * c.a_block + hr * (kRowSlots * 16) + kRowFirst * 16;
              for (int j = tid; j < kTileM + 2; j += kProducers) {
                const int xx = wrap(q.x0 + j - 1, c.W);
                cp_async16(smem_u32(dst + j * 16), x + src_pixel(yy, xx) * c.K + k0 + kc * 8);
              }
            }
        } else {
          const int arows = (c.RT * c.R + 2) * c.TW;
          for (int blk = 0; blk < 6; ++blk) {  // dx * 2 + octet
            const int dx = blk >> 1, kc = blk & 1;
            for (int j = tid; j < arows; j += kProducers) {
              const int yy = wrap(q.y0 + (j >> c.tw_shift) - 1, c.H);
              const int xx = wrap(q.x0 + (j & (c.TW - 1)) + dx - 1, c.W);
              cp_async16(smem_u32(A + blk * c.a_block + j * 16), x + src_pixel(yy, xx) * c.K + k0 + kc * 8);
            }
          }
        }
        if (tid == 0) {  // the item's weights: two tensor-map boxes (one per octet) on the stage barrier
          mbar_expect_tx(&full[st], 18 * c.b_block);
          for (int kc = 0; kc < 2; ++kc) tma_load_3d(Bm + kc * 9 * c.b_block, &tm_w, k0 + kc * 8, q.n0, 0, &full[st]);
        }
        cp_async_commit();
        if (i >= 1) {
          cp_async_wait_one();
          fence_proxy_async();
          mbar_arrive(&full[(i - 1) % S]);
        }
      }
    }
    cp_async_wait_all();
    fence_proxy_async();
    if (ok && i >= 1) mbar_arrive(&full[(i - 1) % S]);
  } else if (warp == kMmaWarp) {
    // ---- MMA issuer: one thread; accumulator set kt & 1 for the kt-th tile of this CTA.
    if (lane == 0) {
      int i = 0, kt = 0;
      bool ok = true;
      if (c.wres && !wait_role(wbar, 0, abort)) {
        give_up();
        ok = false;
      }
      for (int t = blockIdx.x; t < c.ntiles && ok; t += gridDim.x, ++kt) {
        const uint32_t set = (uint32_t)(kt & 1) * c.set_cols;
        if (kt >= 2 && !wait_role(&tempty[kt & 1], (uint32_t)((kt >> 1) - 1) & 1u, abort)) {
          give_up();
          ok = false;
          break;
        }
        tc_fence_after();
        for (int ch = 0; ch < c.nchunks; ++ch, ++i) {
          const int st = i % S;
          if (!wait_role(&full[st], (uint32_t)(i / S) & 1u, abort)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(smem + (uint32_t)st * c.stage_bytes);
          const uint32_t b_base = c.wres ? smem_u32(wsm) + (uint32_t)ch * 18 * c.b_block : a_base + c.a_stage;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dxi = tap % 3;  // dxi = dx + 1
            const uint64_t bd = smem_desc(b_base + (uint32_t)tap * c.b_block, 9 * c.b_block, 128);
            const uint32_t acc = (ch > 0 || tap > 0) ? 1u : 0u;
            if (c.rows_mode) {
              for (int r = 0; r < c.RT; ++r) {
                const uint32_t start = a_base + (uint32_t)(((r + dy + 1) * kRowSlots + kRowFirst + dxi) * 16);
                tc_mma(tmem + set + (uint32_t)r * c.acc_cols, smem_desc(start, c.a_block, 128), bd, c.idesc, acc);
              }
            } else {
              for (int r = 0; r < c.RT; ++r) {  // accumulator r: image rows r R .. r R + R - 1 of the tile
                const uint32_t start =
                    a_base + (uint32_t)(dxi * 2) * c.a_block + (uint32_t)((r * c.R + dy + 1) * c.TW * 16);
                tc_mma(tmem + set + (uint32_t)r * c.acc_cols, smem_desc(start, c.a_block, 128), bd, c.idesc, acc);
              }
            }
          }
          tc_commit(smem_u32(&empty[st]));  // the stage is free once these MMAs are done
        }
        if (ok) tc_commit(smem_u32(&tfull[kt & 1]));  // the tile's accumulators are complete
      }
      // Every MMA issued has completed once this commit arrives: the tensor memory can go.
      tc_commit(smem_u32(done));
      if (!wait_bounded(done, 0)) give_up();
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31: pixel i of the tile.
    const int quarter = warp & 3;
    const int i = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    int kt = 0;
    for (int t = blockIdx.x; t < c.ntiles; t += gridDim.x, ++kt) {
      if (!wait_role(&tfull[kt & 1], (uint32_t)(kt >> 1) & 1u, abort)) {
        give_up();
        break;
      }
      tc_fence_after();
      const TileCoord q = tile_coord(c, t);
      const uint32_t set = (uint32_t)(kt & 1) * c.set_cols;
      const int nacc = c.RT;
      // 16 accumulator columns of pixel pix plus bias (bv) and addend, ReLU, stored at channel n.
      auto emit16 = [&](const uint32_t (&rr)[16], const float* bv, size_t pix, int n) {
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(rr[e]) + bv[e];
        if (addend) {
          const uint4* ap = reinterpret_cast<const uint4*>(addend + pix * c.N + n);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint4 a4 = ap[h];
            const uint32_t aw[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162*>(&aw[e]);
              v[h * 8 + 2 * e] += __bfloat162float(p2.x);
              v[h * 8 + 2 * e + 1] += __bfloat162float(p2.y);
            }
          }
        }
        if (c.relu) {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = fmaxf(v[e], 0.f);
        }
        if (c.out_f32) {
          float4* yp = reinterpret_cast<float4*>(reinterpret_cast<float*>(y) + pix * c.N + n);
#pragma unroll
          for (int h = 0; h < 4; ++h) yp[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        } else {
          uint32_t w[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            w[e] = *reinterpret_cast<const uint32_t*>(&p2);
          }
          uint4* yp = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(y) + pix * c.N + n);
          yp[0] = make_uint4(w[0], w[1], w[2], w[3]);
          yp[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      };
      // 32 columns at a time (two tensor-memory loads per wait), the block's bias read once for
      // all of the tile's accumulators: per-load waits and per-accumulator bias reads held the
      // 128^2 32 -> 64 layer at 40 us (now 29; 64-column blocks at 164 registers were no faster).
      for (int j0 = 0; j0 < c.ntile; j0 += 32) {
        const bool two = j0 + 16 < c.ntile;
        const int n = q.n0 + j0;
        float bv[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) bv[e] = (bias && (e < 16 || two)) ? __ldg(bias + n + e) : 0.f;
        for (int r = 0; r < nacc; ++r) {
          const int py = c.rows_mode ? q.y0 + r : q.y0 + r * c.R + (i >> c.tw_shift);
          const int px = c.rows_mode ? q.x0 + i : q.x0 + (i & (c.TW - 1));
          const size_t pix = ((size_t)q.b * c.H + py) * c.W + px;
          const uint32_t ta = lane_base + set + (uint32_t)r * c.acc_cols + (uint32_t)j0;
          uint32_t r0[16], r1[16];
          tc_ld16(ta, r0);
          if (two) tc_ld16(ta + 16, r1);
          tc_wait_ld();
          emit16(r0, bv, pix, n);
          if (two) emit16(r1, bv + 16, pix, n + 16);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[kt & 1]);  // this set may take the next tile's MMAs
    }
  }
  // The resident weights' copies have landed before the CTA's shared memory is released (at once
  // unless a wait gave up before they did).
  if (c.wres && tid == 0) wait_bounded(wbar, 0);
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) tmem_dealloc(tmem, c.ncols);
}

// w[tap][k][n] -> wt[tap][n][k].
__global__ void k_transpose_taps(const bf16* __restrict__ w, bf16* __restrict__ wt, int K, int N) {
  const size_t total = (size_t)9 * K * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int tap = (int)(e / ((size_t)K * N));
    const int r = (int)(e - (size_t)tap * K * N);
    const int k = r / N, n = r - (r / N) * N;
    wt[((size_t)tap * N + n) * K + k] = w[e];
  }
}

constexpr int kMaxSmem = 227 * 1024;
constexpr int kMaxStages = 6;

// The tile geometry and shared-memory plan for a layer, or false if the kernel cannot serve it.
// *stages: stages of the ring (2 to 4, as many as fit).
bool plan(int batch, int H, int W, int K, int N, bool up, ConvTC* c, size_t* smem, int* stages) {
  if (batch < 1 || H < 1 || W < 1 || K < 16 || K % 16 || N < 16 || N % 16) return false;
  if (up && (H % 2 || W % 2)) return false;
  const int ntile = N > 128 ? 128 : N;
  if (N % ntile) return false;
  c->H = H;
  c->W = W;
  c->Hs = up ? H / 2 : H;
  c->Ws = up ? W / 2 : W;
  c->K = K;
  c->N = N;
  c->ntile = ntile;
  c->ntiles_n = N / ntile;
  c->nchunks = K / 16;
  c->b_block = (uint32_t)(ntile * 16);
  const uint32_t ncols1 = ntile <= 32 ? 32u : (ntile <= 64 ? 64u : 128u);
  if (W >= kTileM) {
    if (W % kTileM) return false;
    c->rows_mode = 1;
    c->TW = kTileM;
    c->R = 1;
    c->tw_shift = 7;
    // output rows per tile: the most of 8, 4, 2, 1 dividing H whose two accumulator sets fit the
    // 512 TMEM columns (8 for up to 32 output channels: each staged row then serves more outputs;
    // batch 16, 256^2 32 -> 32: 56 us against 67 at 4 rows)
    int RT = 8;
    while (RT > 1 && (H % RT || (uint32_t)RT * ncols1 > 256u)) RT >>= 1;
    c->RT = RT;
    c->a_block = (uint32_t)((RT + 2) * kRowSlots * 16);
    c->a_stage = 2 * c->a_block;
    c->tx_bytes = (uint32_t)(2 * (RT + 2) * kTileM * 16);  // TMA mode: the boxes (halo pixels by loads)
  } else {
    if (kTileM % W || (W & (W - 1))) return false;
    c->rows_mode = 0;
    c->TW = W;
    c->R = kTileM / W;
    if (H % c->R) return false;
    int sh = 0;
    while ((1 << sh) < W) ++sh;
    c->tw_shift = sh;
    // accumulators per tile (RT of R rows each, sharing every staged weight chunk): the most of 4,
    // 2, 1 that divides the image's row blocks and whose two sets fit the 512 TMEM columns
    int RT = 4;
    auto fits2 = [&](int rt) {  // two stages of the three shifted copies and the weights
      return 2 * (6 * (size_t)((rt * c->R + 2) * W * 16) + 18 * (size_t)c->b_block) + 256 <= (size_t)kMaxSmem;
    };
    while (RT > 1 && ((H / c->R) % RT || (uint32_t)RT * ncols1 > 256u || !fits2(RT))) RT >>= 1;
    c->RT = RT;
    c->a_block = (uint32_t)((RT * c->R + 2) * W * 16);
    c->a_stage = 6 * c->a_block;
    c->tx_bytes = c->a_stage;
  }
  c->tma = c->rows_mode && !up;
  c->acc_cols = ncols1;
  c->set_cols = (uint32_t)c->RT * ncols1;
  c->ncols = 2 * c->set_cols;
  c->tiles_x = W / c->TW;
  c->tiles_y = H / (c->rows_mode ? c->RT : c->RT * c->R);
  const long long nt = (long long)batch * c->tiles_x * c->tiles_y * c->ntiles_n;
  if (nt > 0x7FFFFFFFll) return false;
  c->ntiles = (int)nt;
  // Resident weights (TMA mode with one N tile, where they and two stages fit): the stages carry
  // the input rows only.
  const size_t tail = (2 * kMaxStages + 6) * sizeof(uint64_t) + 16;  // barriers, abort flag, TMEM slot
  c->w_bytes = (uint32_t)(c->nchunks * 18 * c->b_block);
  c->wres = c->tma && c->ntiles_n == 1 && (size_t)c->w_bytes + 2 * (size_t)c->a_stage + tail <= (size_t)kMaxSmem;
  // Tensor-map copies land on 128-byte boundaries: the weight boxes follow the A operand of a
  // stage and every stage starts where the previous one ends.
  if (c->a_stage % 128 || c->b_block % 128) return false;
  c->stage_bytes = c->wres ? c->a_stage : c->a_stage + 18 * c->b_block;
  if (!c->wres) c->tx_bytes += 18 * c->b_block;
  // Instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
  // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  c->idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ntile >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
  c->up = up;
  const size_t wb = c->wres ? c->w_bytes : 0;
  int st = kMaxStages;
  while (st > 2 && (size_t)st * c->stage_bytes + wb + tail > (size_t)kMaxSmem) --st;
  *stages = st;
  c->wres_off = (uint32_t)((size_t)st * c->stage_bytes);
  c->bar_off = (uint32_t)((size_t)st * c->stage_bytes + wb);
  *smem = (size_t)st * c->stage_bytes + wb + tail;
  // Descriptor start addresses are 14-bit multiples of 16 bytes: every operand must lie in the
  // first 256 KB of shared memory, which the 227 KB limit ensures.
  return *smem <= (size_t)kMaxSmem && c->ncols <= 512u;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor maps of TMA mode: the NHWC input (channels, x, y, image) with a box of 8 channels x 128
// pixels x 1 row, and the K-major weights (channels, output channels, taps) with a box of 8
// channels x N tile x 9 taps.  BF16, no swizzle, no interleave; rows and weights stay in bounds,
// so the fill mode never applies.
bool make_maps(const ConvTC& c, int batch, const void* x, const void* wt, CUtensorMap* rows, CUtensorMap* w) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  if (c.tma) {
    const cuuint64_t xd[4] = {(cuuint64_t)c.K, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)batch};
    const cuuint64_t xs[3] = {(cuuint64_t)c.K * 2, (cuuint64_t)c.W * c.K * 2, (cuuint64_t)c.H * c.W * c.K * 2};
    const cuuint32_t xb[4] = {8, (cuuint32_t)kTileM, 1, 1};
    if (enc(rows, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), xd, xs, xb, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  const cuuint64_t wd[3] = {(cuuint64_t)c.K, (cuuint64_t)c.N, 9};
  const cuuint64_t ws[2] = {(cuuint64_t)c.K * 2, (cuuint64_t)c.N * c.K * 2};
  const cuuint32_t wb[3] = {8, (cuuint32_t)c.ntile, 9};
  return enc(w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(wt), wd, ws, wb, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S>
int launch_s(const ConvTC& c, size_t smem, int batch, const void* x, const void* wt, const float* bias,
             const void* addend, void* y, cudaStream_t s) {
  CUtensorMap tm_rows, tm_w;
  std::memset(&tm_rows, 0, sizeof(tm_rows));
  std::memset(&tm_w, 0, sizeof(tm_w));
  if (!make_maps(c, batch, x, wt, &tm_rows, &tm_w)) return SUR_ERR_CUDA;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(k_conv3x3_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess)
      return SUR_ERR_CUDA;
    configured = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3x3_tc<S>, kThreadsP, smem) != cudaSuccess)
    return SUR_ERR_CUDA;
  // At most 512 TMEM columns per SM: keep resident CTAs x columns within it.
  const int max_ctas = (int)(512u / c.ncols);
  if (per_sm > max_ctas) {
    smem = (size_t)(kMaxSmem / max_ctas) & ~(size_t)1023;
    per_sm = max_ctas;
  }
  if (per_sm < 1) return SUR_ERR_PARAM;
  const long long want = (long long)(sms > 0 ? sms : 148) * per_sm;
  const int grid = (int)(c.ntiles < want ? c.ntiles : want);
  k_conv3x3_tc<S><<<grid, kThreadsP, smem, s>>>((const bf16*)x, (const bf16*)wt, bias, (const bf16*)addend, y, c,
                                                 tm_rows, tm_w);
  return cudaGetLastError() == cudaSuccess ? SUR_OK : SUR_ERR_CUDA;
}

int launch(const void* x, const void* wt, const float* bias, const void* addend, void* y, int batch, int H, int W,
           int K, int N, int relu, int out_f32, int up, cudaStream_t s) {
  ConvTC c;
  size_t smem = 0;
  int stages = 0;
  if (!plan(batch, H, W, K, N, up != 0, &c, &smem, &stages)) return SUR_ERR_PARAM;
  c.relu = relu;
  c.out_f32 = out_f32;
  if (stages == 6) return launch_s<6>(c, smem, batch, x, wt, bias, addend, y, s);
  if (stages == 5) return launch_s<5>(c, smem, batch, x, wt, bias, addend, y, s);
  if (stages == 4) return launch_s<4>(c, smem, batch, x, wt, bias, addend, y, s);
  if (stages == 3) return launch_s<3>(c, smem, batch, x, wt, bias, addend, y, s);
  return launch_s<2>(c, smem, batch, x, wt, bias, addend, y, s);
}

}  // namespace

extern "C" {

int sur_conv3x3_tc(const void* x, const void* wt, const float* bias, const void* addend, void* y, int batch, int H,
                   int W, int K, int N, int relu, int out_f32, int upsampled, void* stream) {
  if (!x || !wt || !y) return SUR_ERR_PARAM;
  if (((uintptr_t)x | (uintptr_t)wt | (uintptr_t)y | (uintptr_t)addend) % 16) return SUR_ERR_PARAM;
  if (addend && out_f32) return SUR_ERR_PARAM;
  if ((long long)batch * H * W > (1ll << 30)) return SUR_ERR_PARAM;
  return launch(x, wt, bias, addend, y, batch, H, W, K, N, relu, out_f32, upsampled, (cudaStream_t)stream);
}

int sur_conv3x3_tc_supported(int batch, int H, int W, int K, int N, int upsampled) {
  ConvTC c;
  size_t smem = 0;
  int stages = 0;
  return plan(batch, H, W, K, N, upsampled != 0, &c, &smem, &stages) ? 1 : 0;
}

int sur_transpose_taps(const void* w, void* wt, int K, int N, void* stream) {
  if (!w || !wt || K < 1 || N < 1) return SUR_ERR_PARAM;
  const size_t total = (size_t)9 * K * N;
  const int blocks = (int)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256);
  k_transpose_taps<<<blocks, 256, 0, (cudaStream_t)stream>>>((const bf16*)w, (bf16*)wt, K, N);
  return cudaGetLastError() == cudaSuccess ? SUR_OK : SUR_ERR_CUDA;
}

int sur_check(void* stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SUR_ERR_CUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return SUR_ERR_CUDA;
  if (!v) return SUR_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int)) != cudaSuccess) return SUR_ERR_CUDA;
  return SUR_ERR_TIMEOUT;
}

}  // extern "C"
