// Kernels of the learned surrogate (a small convolutional U-Net that advances (phi, ux, uy) by
// many lattice Boltzmann steps at once).  The paper has no counterpart; the solver stays the
// judge and fallback.  Activations are NHWC (pixels x channels) BF16 on periodic H x W images;
// 3x3 convolutions are implicit GEMMs on the BF16 tensor cores with FP32 accumulation
// (mma.sync m16n8k16); everything else is element-wise.  Declared in include/surrogate.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/surrogate.h"

namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------------------------
// Warp-level BF16 MMA, 16x8x16, FP32 accumulate.  Fragment layout (PTX ISA, mma.m16n8k16):
// g = lane / 4, t = lane % 4;  A (16x16, row major): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..],
// a2 = A[g][2t+8..], a3 = A[g+8][2t+8..];  B (16x8, k x n): b0 = B[2t..2t+1][g],
// b1 = B[2t+8..2t+9][g];  C (16x8): c0,c1 = C[g][2t..2t+1], c2,c3 = C[g+8][2t..2t+1].
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Pixel p = (b*H + y)*W + x shifted by (dy, dx) with periodic wrap.
__device__ __forceinline__ int shift_pixel(int p, int H, int W, int dy, int dx) {
  const int x = p % W;
  const int by = p / W;
  const int y = by % H;
  const int b = by / H;
  int yy = y + dy, xx = x + dx;
  yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
  xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
  return (b * H + yy) * W + xx;
}

// The same shift on the fine H x W image, returned as the index of the coarse (H/2 x W/2) pixel
// that the 2x nearest upsampling copies there.
__device__ __forceinline__ int shift_pixel_up(int p, int H, int W, int dy, int dx) {
  const int x = p % W;
  const int by = p / W;
  const int y = by % H;
  const int b = by / H;
  int yy = y + dy, xx = x + dx;
  yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
  xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
  return (b * (H >> 1) + (yy >> 1)) * (W >> 1) + (xx >> 1);
}

// ---------------------------------------------------------------------------------------------
// Implicit-GEMM 3x3 periodic convolution:
//   Y[p][n] = sum_tap sum_k X[p + sgn*off(tap)][k] * Wt(tap, k, n)  (+ bias[n], ReLU)
// forward:       X = input (K = Cin),  Wt(tap,k,n) = Wgt[tap][k][n] (n = Cout), sgn = +1
// backward data: X = dY (K = Cout),    Wt(tap,k,n) = Wgt[tap][n][k] (n = Cin),  sgn = -1
// Requires K % 16 == 0 and N % 16 == 0.  The kernel (k_conv3x3_halo, below) stages a spatial
// block with its halo once per 16 input channels and runs all nine taps from shared memory.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// Halo-tile form of the same convolution.  A CTA owns a TH x TW block of output pixels of one
// image (TH * TW <= 256) and TN <= 64 output channels.  Each stage brings 16 input channels of
// the block plus its one-pixel periodic halo, (TH + 2) x (TW + 2) pixels, and the weights of all
// nine taps for them into shared memory; the nine taps then read shifted windows of the same
// halo tile (each lane of ldmatrix gives its own row address, so a shift is an address offset).
// Compared with staging one tap at a time, every input value crosses from L2 once per stage
// instead of nine times and a stage carries nine times the tensor work to hide the next stage's
// loads behind.  8 warps, each 32 pixels x TN channels; stages double-buffered by cp.async.
struct HaloGeom {
  int TW, TH;      // output block: TW columns x TH rows
  int tiles_x;     // blocks per image row band
  int tiles_img;   // blocks per image
  int HP;          // halo pixels (TH + 2) * (TW + 2)
};

template <int TN, bool TRANSW, bool OUT_F32, bool UPX>
__global__ void __launch_bounds__(256, 2)
k_conv3x3_halo(const bf16* __restrict__ X, const bf16* __restrict__ Wg, const float* __restrict__ bias,
               void* __restrict__ Y, const HaloGeom hg, int H, int W, int K, int N, int sgn, int relu,
               const bf16* __restrict__ addend) {
  constexpr int KC = 16, AST = KC + 8;           // channels per stage; padded halo rows (48 B)
  constexpr int NT = TN / 8;                     // n8 tiles per warp
  constexpr int BR = TRANSW ? TN : KC;           // per tap: B[k][n] (forward) or B[n][k] (transposed)
  constexpr int BC = (TRANSW ? KC : TN) + 8;
  constexpr int ACH = 4;                         // halo chunks (16 B) per thread per stage: 2 HP <= 1024
  extern __shared__ __align__(16) unsigned char conv_smem[];
  const int HP = hg.HP, TW = hg.TW, TH = hg.TH, HW = TW + 2;
  bf16* sAbase = reinterpret_cast<bf16*>(conv_smem);                      // [2][HP][AST]
  bf16* sBbase = sAbase + 2 * (size_t)HP * AST;                           // [2][9][BR][BC]
  auto sA = [&](int buf, int h) -> bf16* { return sAbase + ((size_t)buf * HP + h) * AST; };
  auto sB = [&](int buf, int tap, int r) -> bf16* { return sBbase + (((size_t)buf * 9 + tap) * BR + r) * BC; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int img = blockIdx.x / hg.tiles_img, tin = blockIdx.x % hg.tiles_img;
  const int ty0 = (tin / hg.tiles_x) * TH, tx0 = (tin % hg.tiles_x) * TW;
  const int n0 = blockIdx.y * TN;
  const int nst = K / KC;

  // Global source pixel of each halo chunk this thread copies (the same every stage).
  int aps[ACH];
#pragma unroll
  for (int j = 0; j < ACH; ++j) {
    const int c = tid + j * 256;
    const int h = c >> 1;
    aps[j] = -1;
    if (h < HP) {
      const int hy = h / HW, hx = h - hy * HW;
      int yy = ty0 - 1 + hy, xx = tx0 - 1 + hx;
      yy = ((yy % H) + H) % H;
      xx = ((xx % W) + W) % W;
      aps[j] = UPX ? (img * (H >> 1) + (yy >> 1)) * (W >> 1) + (xx >> 1) : (img * H + yy) * W + xx;
    }
  }
  auto load_stage = [&](int st, int buf) {
    const int k0 = st * KC;
#pragma unroll
    for (int j = 0; j < ACH; ++j) {
      const int c = tid + j * 256;
      if (aps[j] >= 0) cp_async16(sA(buf, c >> 1) + (c & 1) * 8, X + (size_t)aps[j] * K + k0 + (c & 1) * 8, true);
    }
    if (!TRANSW) {
      for (int c = tid; c < 9 * KC * TN / 8; c += 256) {
        const int tap = c / (KC * TN / 8), r = c % (KC * TN / 8);
        const int kk = r / (TN / 8), c8 = (r % (TN / 8)) * 8;
        cp_async16(sB(buf, tap, kk) + c8, Wg + ((size_t)tap * K + k0 + kk) * N + n0 + c8, true);
      }
    } else {
      for (int c = tid; c < 9 * TN * KC / 8; c += 256) {
        const int tap = c / (TN * KC / 8), r = c % (TN * KC / 8);
        const int nn = r / (KC / 8), part = (r % (KC / 8)) * 8;
        cp_async16(sB(buf, tap, nn) + part, Wg + ((size_t)tap * N + n0 + nn) * K + k0 + part, true);
      }
    }
  };

  // The halo row of this lane's ldmatrix row for each m16 tile (tap (0, 0)); rows of pixels past
  // the block point at a valid row and are never stored.
  int hrow[2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int q = warp * 32 + mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
    const int i = q / TW, jx = q - i * TW;
    hrow[mt] = (q < TH * TW) ? (i + 1) * HW + jx + 1 : HW + 1;
  }

  float acc[2][NT][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][b][q] = 0.f;

  load_stage(0, 0);
  cp_async_commit();
  for (int st = 0; st < nst; ++st) {
    const int buf = st & 1;
    if (st + 1 < nst) {
      load_stage(st + 1, buf ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int shift = sgn * ((tap / 3 - 1) * HW + (tap % 3 - 1));
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) ldsm_x4(a[mt], sA(buf, hrow[mt] + shift) + 8 * (lane >> 4));
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        uint32_t b[4];
        if (!TRANSW) ldsm_x4_t(b, sB(buf, tap, (lane & 7) + 8 * ((lane >> 3) & 1)) + np * 16 + 8 * (lane >> 4));
        else ldsm_x4(b, sB(buf, tap, np * 16 + (lane & 7) + 8 * (lane >> 4)) + 8 * ((lane >> 3) & 1));
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma16816(acc[mt][2 * np], a[mt], b);
          mma16816(acc[mt][2 * np + 1], a[mt], b + 2);
        }
      }
    }
    __syncthreads();  // the buffer is refilled by the next stage's loads
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int q = warp * 32 + mt * 16 + g + hh * 8;
      if (q >= TH * TW) continue;
      const int i = q / TW, jx = q - i * TW;
      const int yy = ty0 + i, xx = tx0 + jx;
      if (yy >= H || xx >= W) continue;
      const size_t p = ((size_t)img * H + yy) * W + xx;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int n = n0 + nt * 8 + 2 * t;
        float v0 = acc[mt][nt][hh * 2], v1 = acc[mt][nt][hh * 2 + 1];
        if (bias) {
          v0 += bias[n];
          v1 += bias[n + 1];
        }
        if (addend) {
          const float2 av = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(addend + p * N + n));
          v0 += av.x;
          v1 += av.y;
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (OUT_F32) {
          float* y = static_cast<float*>(Y) + p * N + n;
          y[0] = v0;
          y[1] = v1;
        } else {
          bf16* y = static_cast<bf16*>(Y) + p * N + n;
          *reinterpret_cast<__nv_bfloat162*>(y) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
}

// Weight gradient: dW[tap][ci][co] += sum_p X[p + off(tap)][ci] * dY[p][co]; a GEMM with
// M = Cin, N = Cout and K = pixels, split over pixel chunks (FP32 atomics into dW).
// CTA: TCI input channels (one warp per 16) x TCO output channels for one tap and one chunk.
constexpr int WCHUNK = 1024;
constexpr int TK = 16;  // pixels per K slice

template <int TCI, int TCO>
__global__ void __launch_bounds__(TCI * 2)
k_conv3x3_wgrad(const bf16* __restrict__ X, const bf16* __restrict__ dY, float* __restrict__ dW, int npix,
                int H, int W, int Cin, int Cout, int up) {
  constexpr int NTH = TCI * 2;  // TCI/16 warps
  constexpr int NT = TCO / 8;
  __shared__ __align__(16) bf16 sA[TCI][TK + 8];  // [ci][pixel]
  __shared__ __align__(16) bf16 sB[TK][TCO + 8];  // [pixel][co]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.z % 9;
  const int chunk = blockIdx.z / 9;
  const int c0 = blockIdx.x * TCI, o0 = blockIdx.y * TCO;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  const int pbeg = chunk * WCHUNK, pend = min(npix, pbeg + WCHUNK);
  for (int pk = pbeg; pk < pend; pk += TK) {
    // A: TCI ci x 16 pixels (transposed gather of X rows), 16-byte chunks of 8 ci.
    for (int c = tid; c < TK * TCI / 8; c += NTH) {
      const int pp = c % TK, cg = (c / TK) * 8;
      const int p = pk + pp;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (p < pend) {
        const int ps = up ? shift_pixel_up(p, H, W, dy, dx) : shift_pixel(p, H, W, dy, dx);
        v = *reinterpret_cast<const uint4*>(X + (size_t)ps * Cin + c0 + cg);
      }
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) sA[cg + q][pp] = e[q];
    }
    // B: 16 pixels x TCO co.
    for (int c = tid; c < TK * TCO / 8; c += NTH) {
      const int pp = c / (TCO / 8), c8 = (c % (TCO / 8)) * 8;
      const int p = pk + pp;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (p < pend) v = *reinterpret_cast<const uint4*>(dY + (size_t)p * Cout + o0 + c8);
      *reinterpret_cast<uint4*>(&sB[pp][c8]) = v;
    }
    __syncthreads();
    uint32_t a[4];
    const int r0 = warp * 16;
    a[0] = pack2(sA[r0 + g][2 * t], sA[r0 + g][2 * t + 1]);
    a[1] = pack2(sA[r0 + g + 8][2 * t], sA[r0 + g + 8][2 * t + 1]);
    a[2] = pack2(sA[r0 + g][2 * t + 8], sA[r0 + g][2 * t + 9]);
    a[3] = pack2(sA[r0 + g + 8][2 * t + 8], sA[r0 + g + 8][2 * t + 9]);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      uint32_t b[2];
      b[0] = pack2(sB[2 * t][j * 8 + g], sB[2 * t + 1][j * 8 + g]);
      b[1] = pack2(sB[2 * t + 8][j * 8 + g], sB[2 * t + 9][j * 8 + g]);
      mma16816(acc[j], a, b);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int ci = c0 + warp * 16 + g + hh * 8;
      const int co = o0 + j * 8 + 2 * t;
      float* d = dW + ((size_t)tap * Cin + ci) * Cout + co;
      atomicAdd(d, acc[j][hh * 2]);
      atomicAdd(d + 1, acc[j][hh * 2 + 1]);
    }
}

// ---------------------------------------------------------------------------------------------
// Element-wise pieces.

__global__ void k_relu_bwd(const bf16* __restrict__ y, const bf16* __restrict__ dy, bf16* __restrict__ dx,
                           size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dx[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

// bias gradient: db[c] += sum_p dy[p][c]
__global__ void k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, int npix, int C) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int p = blockIdx.x; p < npix; p += gridDim.x) s += __bfloat162float(dy[(size_t)p * C + c]);
  atomicAdd(db + c, s);
}

// 2x2 average pooling, NHWC: out (B, H/2, W/2, C)
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int H, int W, int C) {
  const size_t n = (size_t)B * (H / 2) * (W / 2) * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C;
    size_t r = i / C;
    const int xo = r % (W / 2);
    r /= (W / 2);
    const int yo = r % (H / 2);
    const int b = r / (H / 2);
    const size_t base = (((size_t)b * H + 2 * yo) * W + 2 * xo) * C + c;
    const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + C]) +
                    __bfloat162float(x[base + (size_t)W * C]) + __bfloat162float(x[base + (size_t)W * C + C]);
    y[i] = __float2bfloat16(0.25f * s);
  }
}

// backward of 2x2 average pooling: dx[fine] = dy[coarse] / 4
__global__ void k_pool2_bwd(const bf16* __restrict__ dy, bf16* __restrict__ dx, int B, int H, int W, int C) {
  const size_t n = (size_t)B * H * W * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C;
    size_t r = i / C;
    const int x = r % W;
    r /= W;
    const int y = r % H;
    const int b = r / H;
    const size_t j = (((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c;
    dx[i] = __float2bfloat16(0.25f * __bfloat162float(dy[j]));
  }
}

// nearest 2x upsampling: y (B, 2H, 2W, C) from x (B, H, W, C)
__global__ void k_up2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int H, int W, int C) {
  const size_t n = (size_t)B * 2 * H * 2 * W * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C;
    size_t r = i / C;
    const int xf = r % (2 * W);
    r /= (2 * W);
    const int yf = r % (2 * H);
    const int b = r / (2 * H);
    y[i] = x[(((size_t)b * H + yf / 2) * W + xf / 2) * C + c];
  }
}

// backward of nearest 2x upsampling: dx[coarse] = sum of the four fine gradients
__global__ void k_up2_bwd(const bf16* __restrict__ dy, bf16* __restrict__ dx, int B, int H, int W, int C) {
  const size_t n = (size_t)B * H * W * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C;
    size_t r = i / C;
    const int x = r % W;
    r /= W;
    const int y = r % H;
    const int b = r / H;
    const size_t base = (((size_t)b * 2 * H + 2 * y) * 2 * W + 2 * x) * C + c;
    const size_t W2C = (size_t)2 * W * C;
    const float s = __bfloat162float(dy[base]) + __bfloat162float(dy[base + C]) + __bfloat162float(dy[base + W2C]) +
                    __bfloat162float(dy[base + W2C + C]);
    dx[i] = __float2bfloat16(s);
  }
}

// y = a + b (BF16)
__global__ void k_add(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// Conservative update from the network output (C channels, first four used):
//   phi' = phi - [Jx(x,y) - Jx(x-1,y) + Jy(x,y) - Jy(x,y-1)],  u' = u + du
// with (Jx, Jy, dux, duy) = out[.., 0..3] and (phi, ux, uy) = base[.., 0..2] (the FP32 state).  The
// discrete divergence telescopes on the periodic image, so sum phi' = sum phi up to FP32 rounding.
__global__ void k_flux_update(const float* __restrict__ out, const float* __restrict__ base, float* __restrict__ pred,
                              int B, int H, int W, int C) {
  const int n = B * H * W;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int x = p % W, y = (p / W) % H, b = p / (W * H);
    const int xm = x == 0 ? W - 1 : x - 1, ym = y == 0 ? H - 1 : y - 1;
    const size_t pw = (size_t)(b * H + y) * W + xm, ps = (size_t)(b * H + ym) * W + x;
    const float div = (out[(size_t)p * C] - out[pw * C]) + (out[(size_t)p * C + 1] - out[ps * C + 1]);
    pred[(size_t)p * 3 + 0] = base[(size_t)p * 3 + 0] - div;
    pred[(size_t)p * 3 + 1] = base[(size_t)p * 3 + 1] + out[(size_t)p * C + 2];
    pred[(size_t)p * 3 + 2] = base[(size_t)p * 3 + 2] + out[(size_t)p * C + 3];
  }
}

// Its gradient: dout = d(pred)/d(out)^T dpred (BF16, unused channels 0).
__global__ void k_flux_update_bwd(const float* __restrict__ dpred, bf16* __restrict__ dout, int B, int H, int W,
                                  int C) {
  const int n = B * H * W;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int x = p % W, y = (p / W) % H, b = p / (W * H);
    const int xp = x == W - 1 ? 0 : x + 1, yp = y == H - 1 ? 0 : y + 1;
    const size_t pe = (size_t)(b * H + y) * W + xp, pn = (size_t)(b * H + yp) * W + x;
    const float dphi = dpred[(size_t)p * 3];
    dout[(size_t)p * C + 0] = __float2bfloat16(dpred[pe * 3] - dphi);  // d/dJx(p): -dphi(p) + dphi(p+x)
    dout[(size_t)p * C + 1] = __float2bfloat16(dpred[pn * 3] - dphi);
    dout[(size_t)p * C + 2] = __float2bfloat16(dpred[(size_t)p * 3 + 1]);
    dout[(size_t)p * C + 3] = __float2bfloat16(dpred[(size_t)p * 3 + 2]);
    for (int c = 4; c < C; ++c) dout[(size_t)p * C + c] = __float2bfloat16(0.f);
  }
}

// Mean squared error over npix x 3: *loss += mean((pred - target)^2), dpred = dL/dpred.
__global__ void k_mse3(const float* __restrict__ pred, const float* __restrict__ target, float* __restrict__ dpred,
                       float* __restrict__ loss, size_t n, float inv_count) {
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float e = pred[i] - target[i];
    s += e * e;
    if (dpred) dpred[i] = 2.f * e * inv_count;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// Loss on the first `used` of C channels: pred = x_in + out (residual), L = mean (pred - target)^2
// over pixels x used channels; dout = 2 (pred - target) / count (BF16), loss summed in FP32.
__global__ void k_mse(const float* __restrict__ out, const bf16* __restrict__ xin, const float* __restrict__ target,
                      bf16* __restrict__ dout, float* __restrict__ loss, int npix, int C, int used, float inv_count) {
  float s = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    for (int c = 0; c < C; ++c) {
      float d = 0.f;
      if (c < used) {
        const float pred = __bfloat162float(xin[(size_t)p * C + c]) + out[(size_t)p * C + c];
        const float e = pred - target[(size_t)p * used + c];
        s += e * e;
        d = 2.f * e * inv_count;
      }
      dout[(size_t)p * C + c] = __float2bfloat16(d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// Adam (Kingma & Ba 2015) on FP32 master weights, refreshing their BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wb, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

__global__ void k_cast_bf16(const float* __restrict__ x, bf16* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Solver state (npix x 3 FP32: phi, ux, uy) -> network input x (npix x C BF16: phi, s ux, s uy,
// then zeros) and base (npix x 3 FP32: phi, s ux, s uy), s the velocity scale of the network.
__global__ void k_pack_state(const float* __restrict__ st, bf16* __restrict__ x, float* __restrict__ base,
                             size_t npix, int C, float s) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npix; p += (size_t)gridDim.x * blockDim.x) {
    const float v[3] = {st[p * 3], s * st[p * 3 + 1], s * st[p * 3 + 2]};
    for (int c = 0; c < 3; ++c) base[p * 3 + c] = v[c];
    for (int c = 0; c < C; ++c) x[p * C + c] = __float2bfloat16(c < 3 ? v[c] : 0.f);
  }
}

// Network prediction (npix x 3: phi, s ux, s uy) -> solver state (phi, ux, uy).
__global__ void k_unpack_state(const float* __restrict__ pred, float* __restrict__ st, size_t npix, float inv_s) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npix; p += (size_t)gridDim.x * blockDim.x) {
    st[p * 3] = pred[p * 3];
    st[p * 3 + 1] = pred[p * 3 + 1] * inv_s;
    st[p * 3 + 2] = pred[p * 3 + 2] * inv_s;
  }
}

// Per image b of a batch, in FP64 and in a fixed order (one block per image, fixed per-thread
// strides, fixed tree): sums[b] = sum_p a[p][0] (b2 == NULL), or the sum of (a[p][0] - b2[p][0])^2.
constexpr int kSumThreads = 512;
__global__ void __launch_bounds__(kSumThreads)
k_channel0_sums(const float* __restrict__ a, const float* __restrict__ b2, int npix, int C, double* __restrict__ sums) {
  __shared__ double sh[kSumThreads];
  const size_t off = (size_t)blockIdx.x * npix;
  double acc = 0.0;
  for (int p = threadIdx.x; p < npix; p += kSumThreads) {
    const double v = (double)a[(off + p) * C];
    if (b2) {
      const double d = v - (double)b2[(off + p) * C];
      acc += d * d;
    } else {
      acc += v;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

int check(cudaError_t e) { return e == cudaSuccess ? SUR_OK : SUR_ERR_CUDA; }

int tile_n(int N) { return N % 64 == 0 ? 64 : (N % 32 == 0 ? 32 : (N % 16 == 0 ? 16 : 0)); }

// Output block of the halo-tile convolution: up to 64 columns wide and 256 pixels, with its halo
// tile at most 512 pixels (the kernel's per-thread chunk count) and no taller than the image.
HaloGeom halo_geom(int H, int W) {
  HaloGeom g;
  g.TW = W < 64 ? W : 64;
  int th = 256 / g.TW;
  const int cap = 512 / (g.TW + 2) - 2;
  if (th > cap) th = cap;
  if (th > H) th = H;
  g.TH = th < 1 ? 1 : th;
  g.tiles_x = (W + g.TW - 1) / g.TW;
  g.tiles_img = g.tiles_x * ((H + g.TH - 1) / g.TH);
  g.HP = (g.TH + 2) * (g.TW + 2);
  return g;
}

template <int TN, bool TRANSW>
constexpr size_t halo_smem_max() {
  return (2 * 512 * 24 + 2 * 9 * (size_t)(TRANSW ? TN : 16) * ((TRANSW ? 16 : TN) + 8)) * sizeof(bf16);
}

template <int TN, bool TRANSW, bool OUT_F32, bool UPX>
int halo_launch(int batch, const HaloGeom& hg, cudaStream_t s, const bf16* X, const bf16* Wg, const float* bias,
                void* y, int H, int W, int K, int N, int sgn, int relu, const bf16* addend) {
  auto kern = k_conv3x3_halo<TN, TRANSW, OUT_F32, UPX>;
  static bool configured = false;  // per instantiation, once per process
  if (!configured) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)halo_smem_max<TN, TRANSW>()) !=
        cudaSuccess)
      return SUR_ERR_CUDA;
    configured = true;
  }
  const size_t smem =
      (2 * (size_t)hg.HP * 24 + 2 * 9 * (size_t)(TRANSW ? TN : 16) * ((TRANSW ? 16 : TN) + 8)) * sizeof(bf16);
  dim3 grd((unsigned)(batch * hg.tiles_img), (unsigned)(N / TN));
  kern<<<grd, 256, smem, s>>>(X, Wg, bias, y, hg, H, W, K, N, sgn, relu, addend);
  return check(cudaGetLastError());
}

// Channel tile of the halo-tile convolution: 64, 32 or 16 dividing N, halved while the grid
// would not give every SM a CTA.
int halo_tile_n(long long blocks, int N) {
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess || sms < 1)
    sms = 1;
  int tn = N % 64 == 0 ? 64 : (N % 32 == 0 ? 32 : 16);
  while (tn > 16 && blocks * (N / tn) < sms) tn /= 2;
  return tn;
}

template <int TCI, int TCO>
void wgrad_launch(dim3 grd, cudaStream_t s, const bf16* x, const bf16* dy, float* dw, int npix, int H, int W, int Cin,
                  int Cout, int up) {
  k_conv3x3_wgrad<TCI, TCO><<<grd, TCI * 2, 0, s>>>(x, dy, dw, npix, H, W, Cin, Cout, up);
}

}  // namespace

extern "C" {

int sur_conv3x3(const void* x, const void* w, const float* bias, void* y, int batch, int H, int W, int K, int N,
                int transposed_weights, int sgn, int relu, int out_f32, void* stream) {
  if (!x || !w || !y || batch < 1 || H < 1 || W < 1 || K % 16 || K < 16 || N % 16 || N < 16 ||
      (sgn != 1 && sgn != -1))
    return SUR_ERR_PARAM;
  if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)y) % 16) return SUR_ERR_PARAM;
  const long long npix = (long long)batch * H * W;
  if (npix > (1ll << 30)) return SUR_ERR_PARAM;
  const HaloGeom hg = halo_geom(H, W);
  const int tn = halo_tile_n((long long)batch * hg.tiles_img, N);
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* X = (const bf16*)x;
  const bf16* Wg = (const bf16*)w;
#define SUR_HALO(TN_)                                                                                          \
  if (tn == TN_) {                                                                                             \
    if (!transposed_weights && !out_f32)                                                                       \
      return halo_launch<TN_, false, false, false>(batch, hg, s, X, Wg, bias, y, H, W, K, N, sgn, relu, nullptr); \
    if (!transposed_weights)                                                                                   \
      return halo_launch<TN_, false, true, false>(batch, hg, s, X, Wg, bias, y, H, W, K, N, sgn, relu, nullptr);  \
    if (!out_f32)                                                                                              \
      return halo_launch<TN_, true, false, false>(batch, hg, s, X, Wg, bias, y, H, W, K, N, sgn, relu, nullptr);  \
    return halo_launch<TN_, true, true, false>(batch, hg, s, X, Wg, bias, y, H, W, K, N, sgn, relu, nullptr);     \
  }
  SUR_HALO(64) SUR_HALO(32) SUR_HALO(16)
#undef SUR_HALO
  return SUR_ERR_PARAM;
}

static int wgrad_impl(const void* x, const void* dy, float* dw, int batch, int H, int W, int Cin, int Cout, int up,
                      void* stream) {
  const int tci = tile_n(Cin), tco = tile_n(Cout);
  if (!x || !dy || !dw || batch < 1 || H < 1 || W < 1 || !tci || !tco) return SUR_ERR_PARAM;
  if (up && (H % 2 || W % 2)) return SUR_ERR_PARAM;
  if (((uintptr_t)x | (uintptr_t)dy) % 16) return SUR_ERR_PARAM;
  const long long npix = (long long)batch * H * W;
  const long long chunks = (npix + WCHUNK - 1) / WCHUNK;
  if (chunks * 9 > 65535) return SUR_ERR_PARAM;
  dim3 grd(Cin / tci, Cout / tco, (unsigned)(chunks * 9));
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* X = (const bf16*)x;
  const bf16* D = (const bf16*)dy;
#define SUR_WG(A, B) \
  if (tci == A && tco == B) wgrad_launch<A, B>(grd, s, X, D, dw, (int)npix, H, W, Cin, Cout, up);
  SUR_WG(16, 16) SUR_WG(16, 32) SUR_WG(16, 64) SUR_WG(32, 16) SUR_WG(32, 32) SUR_WG(32, 64) SUR_WG(64, 16)
  SUR_WG(64, 32) SUR_WG(64, 64)
#undef SUR_WG
  return check(cudaGetLastError());
}

int sur_conv3x3_wgrad(const void* x, const void* dy, float* dw, int batch, int H, int W, int Cin, int Cout,
                      void* stream) {
  return wgrad_impl(x, dy, dw, batch, H, W, Cin, Cout, 0, stream);
}

int sur_conv3x3_wgrad_up(const void* xc, const void* dy, float* dw, int batch, int H, int W, int Cin, int Cout,
                         void* stream) {
  return wgrad_impl(xc, dy, dw, batch, H, W, Cin, Cout, 1, stream);
}

int sur_conv3x3_up_add(const void* xc, const void* w, const float* bias, const void* addend, void* y, int batch,
                       int H, int W, int K, int N, void* stream) {
  if (!xc || !w || !y || batch < 1 || H < 2 || W < 2 || H % 2 || W % 2 || K % 16 || K < 16 || N % 16 || N < 16)
    return SUR_ERR_PARAM;
  if (((uintptr_t)xc | (uintptr_t)w | (uintptr_t)y | (uintptr_t)addend) % 16) return SUR_ERR_PARAM;
  const long long npix = (long long)batch * H * W;
  if (npix > (1ll << 30)) return SUR_ERR_PARAM;
  const HaloGeom hg = halo_geom(H, W);
  const int tn = halo_tile_n((long long)batch * hg.tiles_img, N);
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* X = (const bf16*)xc;
  const bf16* Wg = (const bf16*)w;
  const bf16* A = (const bf16*)addend;
  if (tn == 64) return halo_launch<64, false, false, true>(batch, hg, s, X, Wg, bias, y, H, W, K, N, 1, 0, A);
  if (tn == 32) return halo_launch<32, false, false, true>(batch, hg, s, X, Wg, bias, y, H, W, K, N, 1, 0, A);
  if (tn == 16) return halo_launch<16, false, false, true>(batch, hg, s, X, Wg, bias, y, H, W, K, N, 1, 0, A);
  return SUR_ERR_PARAM;
}

int sur_relu_bwd(const void* y, const void* dy, void* dx, size_t n, void* stream) {
  k_relu_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)y, (const bf16*)dy, (bf16*)dx, n);
  return check(cudaGetLastError());
}

int sur_bias_grad(const void* dy, float* db, int npix, int C, void* stream) {
  dim3 grd(256, (C + 63) / 64);
  k_bias_grad<<<grd, 64, 0, (cudaStream_t)stream>>>((const bf16*)dy, db, npix, C);
  return check(cudaGetLastError());
}

int sur_pool2(const void* x, void* y, int batch, int H, int W, int C, void* stream) {
  if (H % 2 || W % 2) return SUR_ERR_PARAM;
  k_pool2<<<grid_for((size_t)batch * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y,
                                                                                      batch, H, W, C);
  return check(cudaGetLastError());
}

int sur_pool2_bwd(const void* dy, void* dx, int batch, int H, int W, int C, void* stream) {
  if (H % 2 || W % 2) return SUR_ERR_PARAM;
  k_pool2_bwd<<<grid_for((size_t)batch * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, (bf16*)dx,
                                                                                      batch, H, W, C);
  return check(cudaGetLastError());
}

int sur_up2(const void* x, void* y, int batch, int H, int W, int C, void* stream) {
  k_up2<<<grid_for((size_t)batch * 4 * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, batch,
                                                                                    H, W, C);
  return check(cudaGetLastError());
}

int sur_up2_bwd(const void* dy, void* dx, int batch, int H, int W, int C, void* stream) {
  k_up2_bwd<<<grid_for((size_t)batch * H * W * C), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, (bf16*)dx,
                                                                                    batch, H, W, C);
  return check(cudaGetLastError());
}

int sur_add(const void* a, const void* b, void* y, size_t n, void* stream) {
  k_add<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)a, (const bf16*)b, (bf16*)y, n);
  return check(cudaGetLastError());
}

int sur_mse(const float* out, const void* xin, const float* target, void* dout, float* loss, int npix, int C,
            int used, void* stream) {
  if (used < 1 || used > C) return SUR_ERR_PARAM;
  const float inv = 1.0f / ((float)npix * used);
  k_mse<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(out, (const bf16*)xin, target, (bf16*)dout, loss, npix, C,
                                                          used, inv);
  return check(cudaGetLastError());
}

int sur_adam(float* w, const float* grad, float* m, float* v, void* wb, size_t n, float lr, float b1, float b2,
             float eps, int step, void* stream) {
  if (step < 1) return SUR_ERR_PARAM;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, grad, m, v, (bf16*)wb, n, lr, b1, b2, eps, c1, c2);
  return check(cudaGetLastError());
}

int sur_flux_update(const float* out, const float* base, float* pred, int batch, int H, int W, int C, void* stream) {
  if (C < 4 || C % 16) return SUR_ERR_PARAM;
  k_flux_update<<<grid_for((size_t)batch * H * W), 256, 0, (cudaStream_t)stream>>>(out, base, pred, batch, H, W, C);
  return check(cudaGetLastError());
}

int sur_flux_update_bwd(const float* dpred, void* dout, int batch, int H, int W, int C, void* stream) {
  if (C < 4 || C % 16) return SUR_ERR_PARAM;
  k_flux_update_bwd<<<grid_for((size_t)batch * H * W), 256, 0, (cudaStream_t)stream>>>(dpred, (bf16*)dout, batch, H,
                                                                                       W, C);
  return check(cudaGetLastError());
}

int sur_mse3(const float* pred, const float* target, float* dpred, float* loss, size_t n, void* stream) {
  if (n == 0) return SUR_ERR_PARAM;
  k_mse3<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(pred, target, dpred, loss, n, 1.0f / (float)n);
  return check(cudaGetLastError());
}

int sur_zero(void* p, size_t bytes, void* stream) {
  return check(cudaMemsetAsync(p, 0, bytes, (cudaStream_t)stream));
}

int sur_cast_bf16(const float* x, void* y, size_t n, void* stream) {
  k_cast_bf16<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, (bf16*)y, n);
  return check(cudaGetLastError());
}

int sur_pack_state(const float* state, void* x, float* base, size_t npix, int C, float u_scale, void* stream) {
  if (!state || !x || !base || C < 3) return SUR_ERR_PARAM;
  k_pack_state<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(state, (bf16*)x, base, npix, C, u_scale);
  return check(cudaGetLastError());
}

int sur_unpack_state(const float* pred, float* state, size_t npix, float u_scale, void* stream) {
  if (!pred || !state || !(u_scale != 0.f)) return SUR_ERR_PARAM;
  k_unpack_state<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(pred, state, npix, 1.f / u_scale);
  return check(cudaGetLastError());
}

int sur_phi_sums(const float* state, int batch, int npix, int C, double* sums, void* stream) {
  if (!state || !sums || batch < 1 || npix < 1 || C < 1) return SUR_ERR_PARAM;
  k_channel0_sums<<<batch, kSumThreads, 0, (cudaStream_t)stream>>>(state, nullptr, npix, C, sums);
  return check(cudaGetLastError());
}

int sur_phi_sq_diff(const float* a, const float* b, int batch, int npix, int C, double* sums, void* stream) {
  if (!a || !b || !sums || batch < 1 || npix < 1 || C < 1) return SUR_ERR_PARAM;
  k_channel0_sums<<<batch, kSumThreads, 0, (cudaStream_t)stream>>>(a, b, npix, C, sums);
  return check(cudaGetLastError());
}

}  // extern "C"
