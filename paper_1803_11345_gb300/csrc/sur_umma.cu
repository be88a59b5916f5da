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
//   * row mode (W >= 128): a CTA owns RT image rows x 128 columns (RT accumulators).  A is the
//     RT + 2 rows around them, each row staged with one wrapped halo column on either side
//     (130 pixels): [octet][halo row][130 pixels][8 x BF16].  The operand of tap (dy, dx) for
//     output row r starts at pixel (r + dy + 1) * 130 + dx + 1: 9 RT descriptors, no copies.
//   * copy mode (W < 128, W a power of two dividing 128): one accumulator of R = 128/W full rows,
//     which a start offset cannot shift by a column across the row seams, so A holds the R + 2
//     rows around them in three copies shifted by dx = -1, 0, +1 with the periodic wrap applied
//     while staging: [dx][octet][halo-tile pixel][8 x BF16]; tap (dy, dx) starts at pixel
//     (dy + 1) * W of copy dx.
//   * B: the 9 taps' weights for the N tile, from the K-major copy [tap][N][K] (see
//     sur_transpose_taps): [tap][octet][output channel][8 x BF16], shared by every accumulator.
// Stages are filled by 16-byte cp.async copies (double-buffered when there is more than one
// channel chunk); one thread issues the chunk's MMAs and commits them to an mbarrier, whose
// completion frees the stage.  Every mbarrier wait is bounded: a wait that gives up sets the
// status word read by sur_check, lets the copies and MMAs it issued finish (again bounded), frees
// the tensor memory and returns.  The epilogue reads the accumulators with tcgen05.ld (each warp
// its 32 lanes), adds the bias and an optional addend (the decoder's skip), applies ReLU, and
// stores BF16 or FP32 NHWC rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/surrogate.h"
#include "lbm_tma.cuh"

namespace {

using bf16 = __nv_bfloat16;
using lbmch::mbar_fence_init;
using lbmch::mbar_init;
using lbmch::mbar_try_wait;
using lbmch::smem_u32;

// Status word: set when a bounded wait of a tensor-core kernel gave up (read and cleared by
// sur_check).
__device__ int g_tc_status;

constexpr uint32_t kWaitProbes = 1u << 22;
constexpr int kThreads = 128;
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
  int RT;               // row mode: output rows (accumulators) per CTA; copy mode: 1
  int tw_shift;         // log2(TW)
  int tiles_x, tiles_y; // tiles per image along x and y
  int nchunks, stages;  // K / 16; staging buffers (1 or 2)
  int ntile;            // output channels per CTA
  uint32_t ncols;       // TMEM columns allocated (accumulators x N tile, a power of two >= 32)
  uint32_t acc_cols;    // TMEM column stride between accumulators
  uint32_t a_block, a_stage, b_block, stage_bytes;
  uint32_t idesc;
  int relu, out_f32, up;
};

constexpr int kHaloW = kTileM + 2;  // staged pixels per halo row in row mode

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void __launch_bounds__(kThreads)
k_conv3x3_tc(const bf16* __restrict__ x, const bf16* __restrict__ wt, const float* __restrict__ bias,
             const bf16* __restrict__ addend, void* __restrict__ y, const ConvTC c) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per_img = c.tiles_x * c.tiles_y;
  const int b = blockIdx.x / per_img;
  const int rem = blockIdx.x - b * per_img;
  const int rows_per_tile = c.rows_mode ? c.RT : c.R;
  const int y0 = (rem / c.tiles_x) * rows_per_tile, x0 = (rem % c.tiles_x) * c.TW;
  const int n0 = blockIdx.y * c.ntile;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + c.stages * c.stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  if (warp == 0) {
    tmem_alloc(smem_u32(tslot), c.ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto src_pixel = [&](int yy, int xx) -> size_t {
    return c.up ? ((size_t)b * c.Hs + (yy >> 1)) * c.Ws + (xx >> 1) : ((size_t)b * c.H + yy) * c.W + xx;
  };
  auto load_chunk = [&](int ch, int st) {
    unsigned char* A = smem + (uint32_t)st * c.stage_bytes;
    unsigned char* Bm = A + c.a_stage;
    const int k0 = ch * 16;
    if (c.rows_mode) {
      const int hrows = c.RT + 2;
      for (int kc = 0; kc < 2; ++kc)
        for (int hr = 0; hr < hrows; ++hr) {
          const int yy = wrap(y0 + hr - 1, c.H);
          unsigned char* dst = A + kc * c.a_block + hr * (kHaloW * 16);
          for (int j = tid; j < kHaloW; j += kThreads) {
            const int xx = wrap(x0 + j - 1, c.W);
            cp_async16(smem_u32(dst + j * 16), x + src_pixel(yy, xx) * c.K + k0 + kc * 8);
          }
        }
    } else {
      const int arows = (c.R + 2) * c.TW;
      for (int blk = 0; blk < 6; ++blk) {  // dx * 2 + octet
        const int dx = blk >> 1, kc = blk & 1;
        for (int j = tid; j < arows; j += kThreads) {
          const int yy = wrap(y0 + (j >> c.tw_shift) - 1, c.H);
          const int xx = wrap(x0 + (j & (c.TW - 1)) + dx - 1, c.W);
          cp_async16(smem_u32(A + blk * c.a_block + j * 16), x + src_pixel(yy, xx) * c.K + k0 + kc * 8);
        }
      }
    }
    for (int q = tid; q < 18 * c.ntile; q += kThreads) {
      const int blk = q / c.ntile;  // tap * 2 + octet
      const int n = q - blk * c.ntile;
      const int tap = blk >> 1, kc = blk & 1;
      cp_async16(smem_u32(Bm + blk * c.b_block + n * 16), wt + ((size_t)tap * c.N + n0 + n) * c.K + k0 + kc * 8);
    }
    cp_async_commit();
  };

  // ok is the same in every thread: each bounded wait is followed by a block-wide AND.
  bool ok = true;
  int committed = -1;  // last chunk whose MMAs were committed
  load_chunk(0, 0);
  for (int ch = 0; ch < c.nchunks; ++ch) {
    const int st = c.stages == 2 ? (ch & 1) : 0;
    const bool prefetch = c.stages == 2 && ch + 1 < c.nchunks;
    if (prefetch && ch >= 1) {
      // the MMAs of chunk ch - 1 read the stage chunk ch + 1 goes to: wait for them first
      ok = __syncthreads_and(wait_bounded(&mbar[(ch + 1) & 1], (uint32_t)((ch - 1) >> 1) & 1u));
      if (!ok) break;
    }
    if (prefetch) {
      load_chunk(ch + 1, (ch + 1) & 1);
      cp_async_wait_one();  // this thread's copies of chunk ch have landed
    } else {
      cp_async_wait_all();
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_u32(smem + (uint32_t)st * c.stage_bytes);
      const uint32_t b_base = a_base + c.a_stage;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dxi = tap % 3;  // dxi = dx + 1
        const uint64_t bd = smem_desc(b_base + (uint32_t)(tap * 2) * c.b_block, c.b_block, 128);
        if (c.rows_mode) {
          for (int r = 0; r < c.RT; ++r) {
            const uint32_t start = a_base + (uint32_t)(((r + dy + 1) * kHaloW + dxi) * 16);
            tc_mma(tmem + (uint32_t)r * c.acc_cols, smem_desc(start, c.a_block, 128), bd, c.idesc,
                   (ch > 0 || tap > 0) ? 1u : 0u);
          }
        } else {
          const uint32_t start = a_base + (uint32_t)(dxi * 2) * c.a_block + (uint32_t)((dy + 1) * c.TW * 16);
          tc_mma(tmem, smem_desc(start, c.a_block, 128), bd, c.idesc, (ch > 0 || tap > 0) ? 1u : 0u);
        }
      }
      tc_commit(smem_u32(&mbar[st]));
    }
    committed = ch;
    if (c.stages == 1 && ch + 1 < c.nchunks) {
      ok = __syncthreads_and(wait_bounded(&mbar[0], (uint32_t)ch & 1u));
      if (!ok) break;
      load_chunk(ch + 1, 0);
    }
  }
  // Completion of the last commit covers every MMA issued before it.
  const int sl = committed < 0 ? 0 : (c.stages == 2 ? (committed & 1) : 0);
  const uint32_t ph = c.stages == 2 ? ((uint32_t)(committed >> 1) & 1u) : ((uint32_t)committed & 1u);
  if (ok) ok = __syncthreads_and(wait_bounded(&mbar[sl], ph));
  if (!ok) {
    // A wait gave up: record it, let this CTA's copies and MMAs finish (bounded), free the
    // tensor memory and return without writing the output.
    if (tid == 0) atomicOr(&g_tc_status, 1);
    cp_async_wait_all();
    if (committed >= 0) wait_bounded(&mbar[sl], ph);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, c.ncols);
    return;
  }
  tc_fence_after();

  // Epilogue: this thread's pixel is TMEM lane i = 32 warp + lane of each accumulator.
  const int i = warp * 32 + lane;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  const int nacc = c.rows_mode ? c.RT : 1;
  for (int r = 0; r < nacc; ++r) {
    const int py = c.rows_mode ? y0 + r : y0 + (i >> c.tw_shift);
    const int px = c.rows_mode ? x0 + i : x0 + (i & (c.TW - 1));
    const size_t pix = ((size_t)b * c.H + py) * c.W + px;
    for (int j0 = 0; j0 < c.ntile; j0 += 16) {
      uint32_t rr[16];
      tc_ld16(lane_base + (uint32_t)r * c.acc_cols + (uint32_t)j0, rr);
      tc_wait_ld();
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(rr[q]) + (bias ? bias[n0 + j0 + q] : 0.f);
      if (addend) {
        const uint4* ap = reinterpret_cast<const uint4*>(addend + pix * c.N + n0 + j0);
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
        for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q], 0.f);
      }
      if (c.out_f32) {
        float4* yp = reinterpret_cast<float4*>(reinterpret_cast<float*>(y) + pix * c.N + n0 + j0);
#pragma unroll
        for (int h = 0; h < 4; ++h) yp[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
      } else {
        uint32_t w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
          w[e] = *reinterpret_cast<const uint32_t*>(&p2);
        }
        uint4* yp = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(y) + pix * c.N + n0 + j0);
        yp[0] = make_uint4(w[0], w[1], w[2], w[3]);
        yp[1] = make_uint4(w[4], w[5], w[6], w[7]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, c.ncols);
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

// The tile geometry and shared-memory plan for a layer, or false if the kernel cannot serve it.
bool plan(int batch, int H, int W, int K, int N, bool up, ConvTC* c, size_t* smem) {
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
  c->nchunks = K / 16;
  c->stages = c->nchunks > 1 ? 2 : 1;
  c->b_block = (uint32_t)(ntile * 16);
  const uint32_t ncols1 = ntile <= 32 ? 32u : (ntile <= 64 ? 64u : 128u);
  if (W >= kTileM) {
    if (W % kTileM) return false;
    c->rows_mode = 1;
    c->TW = kTileM;
    c->R = 1;
    c->tw_shift = 7;
    // output rows per CTA: the most of 4, 2, 1 dividing H whose accumulators fit 256 TMEM columns
    int RT = 4;
    while (RT > 1 && (H % RT || (uint32_t)RT * ncols1 > 256u)) RT >>= 1;
    c->RT = RT;
    c->acc_cols = ncols1;
    c->ncols = (uint32_t)RT * ncols1;
    c->a_block = (uint32_t)((RT + 2) * kHaloW * 16);
    c->a_stage = 2 * c->a_block;
  } else {
    if (kTileM % W || (W & (W - 1))) return false;
    c->rows_mode = 0;
    c->TW = W;
    c->R = kTileM / W;
    if (H % c->R) return false;
    int sh = 0;
    while ((1 << sh) < W) ++sh;
    c->tw_shift = sh;
    c->RT = 1;
    c->acc_cols = ncols1;
    c->ncols = ncols1;
    c->a_block = (uint32_t)((c->R + 2) * W * 16);
    c->a_stage = 6 * c->a_block;
  }
  c->tiles_x = W / c->TW;
  c->tiles_y = H / (c->rows_mode ? c->RT : c->R);
  c->stage_bytes = c->a_stage + 18 * c->b_block;
  // Instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
  // both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  c->idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ntile >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
  c->up = up;
  *smem = (size_t)c->stages * c->stage_bytes + 2 * sizeof(uint64_t) + 16;
  // Descriptor start addresses are 14-bit multiples of 16 bytes: every operand must lie in the
  // first 256 KB of shared memory, which the 227 KB limit ensures.
  return *smem <= (size_t)kMaxSmem;
}

int launch(const void* x, const void* wt, const float* bias, const void* addend, void* y, int batch, int H, int W,
           int K, int N, int relu, int out_f32, int up, cudaStream_t s) {
  ConvTC c;
  size_t smem = 0;
  if (!plan(batch, H, W, K, N, up != 0, &c, &smem)) return SUR_ERR_PARAM;
  c.relu = relu;
  c.out_f32 = out_f32;
  const long long tiles = (long long)batch * c.tiles_x * c.tiles_y;
  if (tiles > 0x7FFFFFFFll) return SUR_ERR_PARAM;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e != cudaSuccess) return SUR_ERR_CUDA;
    configured = true;
  }
  // At most 512 TMEM columns per SM: keep resident CTAs x columns within it (an allocation beyond
  // it would wait for another CTA to free its columns), by asking for more shared memory if needed.
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3x3_tc, kThreads, smem) != cudaSuccess)
    return SUR_ERR_CUDA;
  const int max_ctas = (int)(512 / c.ncols);
  if (per_sm > max_ctas) smem = (size_t)(kMaxSmem / max_ctas) & ~(size_t)1023;
  dim3 grid((unsigned)tiles, (unsigned)(N / c.ntile));
  k_conv3x3_tc<<<grid, kThreads, smem, s>>>((const bf16*)x, (const bf16*)wt, bias, (const bf16*)addend, y, c);
  return cudaGetLastError() == cudaSuccess ? SUR_OK : SUR_ERR_CUDA;
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
  return plan(batch, H, W, K, N, upsampled != 0, &c, &smem) ? 1 : 0;
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
