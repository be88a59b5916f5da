// Device code shared by the two paired 16-bit step kernels (lbm_pair.cu: loads in registers;
// lbm_pair_tma.cu: rows staged in shared memory by the bulk-copy engine): a node pair's packed
// 16-bit words, their decode into packed FP32 (lbm_f2.cuh), and the encode, closures and stores
// of a collided pair.
#pragma once
#include "lbm_device.cuh"
#include "lbm_f2.cuh"
#include "lbm_internal.h"

namespace lbmch {

// Pulled populations of one set for a node pair, as stored: the eight moving directions as
// packed 16-bit pairs (low half = node x, high half = node x+1), the rest population as FP32.
struct RawPair {
  uint32_t w[8];
  float r0a, r0b;
};

// The same pull while its loads are in flight: for a direction with c_x != 0 the pair straddles
// two aligned words, kept apart (w: the word at x, e: the word at x - 2 or x + 2) until finish()
// combines them, one band later, so that no instruction waits on the loads in the meantime.
struct RawPairLoad {
  uint32_t w[8];
  uint32_t e[6];
  float r0a, r0b;
};

// Index among the six c_x != 0 directions (1, 3, 5, 6, 7, 8), or -1.
__host__ __device__ constexpr int side_index(int i) {
  return i == 1 ? 0 : i == 3 ? 1 : i == 5 ? 2 : i == 6 ? 3 : i == 7 ? 4 : i == 8 ? 5 : -1;
}

__device__ __forceinline__ void finish(const RawPairLoad& l, RawPair& o) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (lat_cx(i) == 0) o.w[i - 1] = l.w[i - 1];
    else if (lat_cx(i) == 1) o.w[i - 1] = __byte_perm(l.e[side_index(i)], l.w[i - 1], 0x5432);
    else o.w[i - 1] = __byte_perm(l.w[i - 1], l.e[side_index(i)], 0x5432);
  }
  o.r0a = l.r0a;
  o.r0b = l.r0b;
}

// Two floats converted to FP16 toward zero and packed (low half = lo).
__device__ __forceinline__ uint32_t cvt_rz_pair(float lo, float hi) {
  uint32_t d;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ uint32_t ld_word(const char* __restrict__ b, unsigned byte_off) {
  return __ldg(reinterpret_cast<const unsigned int*>(b + byte_off));
}
__device__ __forceinline__ void st_word(char* __restrict__ b, unsigned byte_off, uint32_t v) {
  *reinterpret_cast<unsigned int*>(b + byte_off) = v;
}

// s += (float)h for a 16-bit pattern h by one mixed-precision add: the conversion is exact, so the
// sum is the one converting first and adding in FP32 gives.
template <int PREC> __device__ __forceinline__ void mix_add(float& s, unsigned short h) {
  if constexpr (PREC == 2) asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(s) : "h"(h));
  else asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(s) : "h"(h));
}

// Both lanes onto the grid of step 2^-24 (k = kGridF) or 2^-23 (k = kGridG) by the one-node
// kernel's snap (PopHalf), in packed instructions.
__device__ __forceinline__ F2 grid_snap2(F2 v, float k) { return f2_sub(f2_add(v, F2(k)), F2(k)); }

// Two floats rounded to the storage type and packed (low half = first), and back.  packf / packg
// encode a node pair's f deviations / g values as PopHalf::encf / encg do for one node.
template <int PREC> struct Pack;
template <> struct Pack<2> {
  using H = __half;
  __device__ __forceinline__ static uint32_t pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ __forceinline__ static uint32_t packf(F2 v) { return pack(v.v.x, v.v.y); }
  __device__ __forceinline__ static uint32_t packg(F2 v) {
    const F2 s = grid_snap2(v, kGridG);
    return pack(s.v.x, s.v.y);
  }
  __device__ __forceinline__ static float2 unpack(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  }
};
template <> struct Pack<3> {
  using H = __nv_bfloat16;
  __device__ __forceinline__ static uint32_t pack(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ __forceinline__ static uint32_t packf(F2 v) {
    const F2 s = grid_snap2(v, kGridF);
    return pack(s.v.x, s.v.y);
  }
  __device__ __forceinline__ static uint32_t packg(F2 v) {
    const F2 s = grid_snap2(v, kGridG);
    return pack(s.v.x, s.v.y);
  }
  __device__ __forceinline__ static float2 unpack(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
  }
};

// The pulled populations of the pair decoded (lane .x node x, lane .y node x+1); f stays in the
// stored form, deviations from w_i, which is the form the collision takes.
template <int PREC>
__device__ __forceinline__ void unpack_pair(const RawPair& rp, F2 out[9]) {
  out[0] = F2(rp.r0a, rp.r0b);
#pragma unroll
  for (int i = 1; i < 9; ++i) out[i] = F2(Pack<PREC>::unpack(rp.w[i - 1]));
}

template <int PREC>
__device__ __forceinline__ F2 phi_pair(const RawPair& rp) {
  F2 v[9];
  unpack_pair<PREC>(rp, v);
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// Store a collided node pair (x, x+1) at element e (= row * pitch + x) of the output state:
// direction i of both nodes rounds into one 32-bit word per set; the rest populations are the
// closures (Eq. 10) of the rounded values, summed in direction order, so that the stored pair
// sums to the collision's rho and phi exactly.  key: 0 rounds to nearest, else the step's key for
// stochastic rounding (each node draws the stream the one-node kernel draws for it).
template <int PREC>
__device__ __forceinline__ void store_pair(char* __restrict__ dst, Plane32 pl, unsigned e, const F2 f[9],
                                           const F2 g[9], F2 drho, F2 phi, uint32_t key) {
  using P = Pop<PREC>;
  F2 sf(0.0f), sg(0.0f);
  auto put = [&](int i, uint32_t wf, uint32_t wg) {
    st_word(dst, ((unsigned)(i - 1) * pl.n + e) * 2u, wf);
    st_word(dst, ((unsigned)(7 + i) * pl.n + e) * 2u, wg);
    mix_add<PREC>(sf.v.x, (unsigned short)(wf & 0xFFFFu));
    mix_add<PREC>(sf.v.y, (unsigned short)(wf >> 16));
    mix_add<PREC>(sg.v.x, (unsigned short)(wg & 0xFFFFu));
    mix_add<PREC>(sg.v.y, (unsigned short)(wg >> 16));
  };
  if (!key) {  // one uniform branch: the round-to-nearest loop carries no stochastic code
#pragma unroll
    for (int i = 1; i < 9; ++i) put(i, Pack<PREC>::packf(f[i]), Pack<PREC>::packg(g[i]));
  } else {
    using H = typename Pack<PREC>::H;
    uint32_t ra = sr_start(e, key), rb = sr_start(e + 1u, key);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      if (i > 1) {
        ra = sr_next(ra);
        rb = sr_next(rb);
      }
      using SF = SRound<H, -24>;
      using SG = SRound<H, -23>;
      if constexpr (PREC == 3) {  // BF16: the two high halves of the rounded FP32 patterns
        put(i, __byte_perm(SF::bits(f[i].v.x, ra & 0xFFFFu), SF::bits(f[i].v.y, rb & 0xFFFFu), 0x7632),
            __byte_perm(SG::bits(g[i].v.x, ra >> 16), SG::bits(g[i].v.y, rb >> 16), 0x7632));
      } else {  // FP16: both nodes converted toward zero and packed by one instruction
        put(i, cvt_rz_pair(SF::pre(f[i].v.x, ra & 0xFFFFu), SF::pre(f[i].v.y, rb & 0xFFFFu)),
            cvt_rz_pair(SG::pre(g[i].v.x, ra >> 16), SG::pre(g[i].v.y, rb >> 16)));
      }
    }
  }
  const F2 f0 = drho - sf, g0 = phi - sg;
  *reinterpret_cast<float2*>(dst + ((unsigned)P::kRestFirst * pl.n + e) * 4u) = f0.v;
  *reinterpret_cast<float2*>(dst + ((unsigned)(P::kRestFirst + 1) * pl.n + e) * 4u) = g0.v;
}

}  // namespace lbmch
