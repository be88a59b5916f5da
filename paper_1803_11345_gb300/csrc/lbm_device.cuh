// Device-side building blocks of the fused step: lattice constants, population storage
// policies, streaming by pull with moving-wall bounce-back, the isotropic stencils and both
// collisions of the hybrid central-moment / BGK scheme (arXiv:1803.11345).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_internal.h"

namespace lbmch {

// D2Q9 velocities in the paper's order: c_x = [0,1,0,-1,0,1,-1,-1,1], c_y = [0,0,1,0,-1,1,1,-1,-1]
// (lattice paragraph before Eq. 4).  Written as functions so that unrolled loops fold them.
__host__ __device__ constexpr int lat_cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int lat_cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// Direction with c_opp = -c_i.
__host__ __device__ constexpr int lat_opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
// Weights w_0 = 4/9, w_1..4 = 1/9, w_5..8 = 1/36 (paragraph after Eq. 14), as an exact rational
// numerator over 36.
__host__ __device__ constexpr int lat_w36(int i) { return i == 0 ? 16 : (i <= 4 ? 4 : 1); }

// ---------------------------------------------------------------------------------------------
// Storage policies.  A population buffer holds 18 planes (f_0..f_8, g_0..g_8) of `plane`
// elements; node (x, y) sits at y * pitch + x inside each plane.
//
// Every accessor takes the plane stride either as a 64-bit element count (any lattice) or as a
// Plane32: the same count for buffers under 4 GiB, where every byte offset inside the buffer fits
// in 32 bits, so an address is one 32-bit multiply-add plus one add to the base instead of 64-bit
// multiplies (the step kernel is partly instruction-bound).
struct Plane32 {
  unsigned n;  // elements per plane
};

// Element idx of the plane that starts `first` planes of element type E into the buffer.
template <class E>
__device__ __forceinline__ const E* plane_elem(const char* b, long long pl, int first, int idx) {
  return reinterpret_cast<const E*>(b) + first * pl + idx;
}
template <class E>
__device__ __forceinline__ const E* plane_elem(const char* b, Plane32 pl, int first, int idx) {
  return reinterpret_cast<const E*>(b + ((unsigned)first * pl.n + (unsigned)idx) * (unsigned)sizeof(E));
}
template <class E, class PL>
__device__ __forceinline__ E* plane_elem(char* b, PL pl, int first, int idx) {
  return const_cast<E*>(plane_elem<E>(static_cast<const char*>(b), pl, first, idx));
}

template <int PREC> struct Pop;

// Lattice weight w_i in the arithmetic type, and in FP64 for the FP64 views of the state.
template <class C> __host__ __device__ constexpr C lat_w(int i) { return C(lat_w36(i)) / C(36); }

// How the storage policies below present f: every accessor for f gives and takes the deviation
// d_i = f_i - w_i from the rest state (rho = 1, v = 0), the form the collision computes in, so
// that no quantity of order one is added to the small departures from rest that carry the flow.
// g is presented as stored.  ldf_full / stf_full give and take f_i itself, in FP64, for the
// FP64 views of the state (fields, checkpoints).

// FP64 / FP32: plain values, plane p at element offset p * plane.  The f planes hold f_i itself
// (FP64: checkpoints round-trip bit for bit) or its deviation d_i (FP32, DEV: the rounding unit
// of a stored value is then that of d_i, ~1e-3 to 1e-2, instead of that of w_i).
template <class T, bool DEV> struct PopDense {
  using C = T;
  static constexpr size_t kBytesPerElem = 18 * sizeof(T);
  // stored f value <-> deviation
  __device__ __forceinline__ static C fdec(int i, C v) { return DEV ? v : v - lat_w<C>(i); }
  __device__ __forceinline__ static C fenc(int i, C d) { return DEV ? d : d + lat_w<C>(i); }
  template <class PL> __device__ __forceinline__ static C ld(const char* b, PL pl, int p, int idx) {
    return __ldg(plane_elem<T>(b, pl, p, idx));
  }
  template <class PL> __device__ __forceinline__ static void st(char* b, PL pl, int p, int idx, C v) {
    *plane_elem<T>(b, pl, p, idx) = v;
  }
  template <class PL> __device__ __forceinline__ static C ldf(const char* b, PL pl, int i, int idx) {
    return fdec(i, ld(b, pl, i, idx));
  }
  template <class PL> __device__ __forceinline__ static C ldg(const char* b, PL pl, int i, int idx) {
    return ld(b, pl, 9 + i, idx);
  }
  template <class PL> __device__ __forceinline__ static void stf(char* b, PL pl, int i, int idx, C d) {
    st(b, pl, i, idx, fenc(i, d));
  }
  template <class PL> __device__ __forceinline__ static void stg(char* b, PL pl, int i, int idx, C v) {
    st(b, pl, 9 + i, idx, v);
  }
  template <class PL> __device__ __forceinline__ static double ldf_full(const char* b, PL pl, int i, int idx) {
    return DEV ? (double)ld(b, pl, i, idx) + lat_w<double>(i) : (double)ld(b, pl, i, idx);
  }
  template <class PL> __device__ __forceinline__ static void stf_full(char* b, PL pl, int i, int idx, double v) {
    st(b, pl, i, idx, DEV ? (T)(v - lat_w<double>(i)) : (T)v);
  }
  // f: deviations; drho, phi: the node's density deviation and order parameter (used by the
  // 16-bit closures only).
  template <class PL>
  __device__ __forceinline__ static void store_node(char* b, PL pl, int idx, const C f[9], const C g[9], C /*drho*/,
                                                    C /*phi*/, uint32_t /*sr_key: 16-bit storage only*/ = 0) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      stf(b, pl, i, idx, f[i]);
      stg(b, pl, i, idx, g[i]);
    }
  }
  // The moving-wall term of a bounced link, and the closures' inputs: as computed (the 16-bit
  // policies put them on a grid).
  __device__ __forceinline__ static C wall_term(C t, bool /*is_g*/) { return t; }
  __device__ __forceinline__ static C grid_f(C v) { return v; }
  __device__ __forceinline__ static C grid_g(C v) { return v; }
  // Raw access: the stored bits, decoded only where used (keeps loads in flight).
  using R = T;
  template <class PL> __device__ __forceinline__ static R rawf(const char* b, PL pl, int i, int idx) {
    return ld(b, pl, i, idx);
  }
  template <class PL> __device__ __forceinline__ static R rawg(const char* b, PL pl, int i, int idx) {
    return ld(b, pl, 9 + i, idx);
  }
  __device__ __forceinline__ static C decf(int i, R r) { return fdec(i, r); }
  __device__ __forceinline__ static C decg(int, R r) { return r; }
  __device__ __forceinline__ static R keep(C v) { return v; }   // an already-decoded value
  __device__ __forceinline__ static C kept(R r) { return r; }
};
template <> struct Pop<0> : PopDense<double, false> {};
template <> struct Pop<1> : PopDense<float, true> {};

// 16-bit storage: 16 planes of 16-bit floats hold the moving populations, d_i = f_i - w_i for
// i = 1..8 at plane i-1 and g_i (rest value 0) at plane 7+i; then two FP32 planes hold the rest
// populations d_0 = f_0 - 4/9 and g_0, stored as closures so that every node's stored
// populations sum to its rho and phi (see store_node).  Arithmetic is FP32.
template <class H> struct Cvt;
template <> struct Cvt<__half> {
  __device__ __forceinline__ static float to(__half h) { return __half2float(h); }
  __device__ __forceinline__ static __half from(float v) { return __float2half_rn(v); }
};
template <> struct Cvt<__nv_bfloat16> {
  __device__ __forceinline__ static float to(__nv_bfloat16 h) { return __bfloat162float(h); }
  __device__ __forceinline__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

// Stochastic rounding of the 16-bit storage (an option; round-to-nearest is the default).
// Rounding to nearest leaves an error that is a fixed function of the value, so on a smooth
// field the errors of neighbouring nodes are alike and add up (in a slow shear the stored
// deviations quantise the viscous stress); rounding up with probability equal to the fraction of
// a unit that is dropped makes every stored value unbiased, and the errors average out.
//
// Random bits: a counter-based stream per node and step.  A 32-bit key for the step (host) and
// the node index go through the MurmurHash3 32-bit finaliser (A. Appleby); a Weyl sequence (adding
// the 32-bit golden-ratio constant) then gives one word per moving direction i = 1..8, drawn in
// order: its low half rounds f_i, its high half g_i.  Each field is uniform over nodes and steps,
// which is what makes every rounding unbiased.
__device__ __forceinline__ uint32_t sr_mix(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t sr_next(uint32_t x) { return x + 0x9e3779b9u; }
// First word of node idx at the step whose key is `key` (direction 1); sr_next gives the next.
__device__ __forceinline__ uint32_t sr_start(unsigned idx, uint32_t key) { return sr_mix(idx * 0x9e3779b9u ^ key); }

// Exact conservation under 16-bit storage.  The collision conserves rho and phi, and the rest
// populations are stored (FP32) as closures of the rounded moving ones, so a node's stored values
// sum to its rho and phi -- but only as exactly as FP32 forms those sums.  They are exact when
// every value involved lies on one fixed binary grid and no partial sum leaves the range in which
// FP32 holds that grid exactly: f deviations on multiples of 2^-24 with partial sums below 1 in
// magnitude, g values on multiples of 2^-23 with partial sums below 2 (|phi| stays near 1).  Every
// FP16 value is a multiple of 2^-24 (its smallest subnormal), and every FP16 or BF16 value of
// magnitude 2^-13 (FP16) / 2^-16 (BF16) or more is a multiple of 2^-23; values below that are first
// put on the grid, by an addition and a subtraction of a constant whose unit in the last place is
// the grid step (the sum is rounded at that step, the subtraction is exact), or by the same
// addition rounded toward zero for stochastic rounding; that holds while the value is below 1/4
// (f) or 1/2 (g) in magnitude, as every moving population and moving-wall term of a flow the
// scheme resolves is.  Values of order one (the rest populations of an initial or restored state)
// are scaled, rounded to an integer and scaled back instead.  Stored values and the moving-wall
// terms then sit on the grid, every sum of the step is exact, and the FP64 totals of
// lbm_conservation (exact sums of grid values) stay the same, bit for bit, from step to step.
constexpr float kGridF = 0.75f;  // unit in the last place 2^-24: the f grid (for |v| < 1/4)
constexpr float kGridG = 1.5f;   // unit in the last place 2^-23: the g grid (for |v| < 1/2)
__device__ __forceinline__ float grid_snap(float v, float k) { return __fsub_rn(__fadd_rn(v, k), k); }
// v rounded to the nearest multiple of 2^-S for any |v| < 2^(24 - S) (the scalings are exact).
template <int S> __device__ __forceinline__ float grid_round(float v) {
  constexpr float up = (float)(1u << S), down = 1.0f / (float)(1u << S);
  return rintf(v * up) * down;
}
// |v| cut toward zero onto the grid of step 2^q, given k = 2^(q + 23) (0.5: the f grid, 1: the g
// grid; exact for |v| < k), sign kept.
__device__ __forceinline__ float grid_trunc(float v, float k) { return copysignf(__fsub_rn(__fadd_rz(fabsf(v), k), k), v); }

// v rounded to the 16-bit type with 16 random bits r (a fraction r / 2^16 of the type's unit at
// v): the fraction is added to |v| and the result cut toward zero, so v rounds away from zero with
// probability equal to the dropped fraction of a unit.  The unit is 2^(e-10) (FP16) or 2^(e-7)
// (BF16) for an exponent e, but never below the grid step 2^Q of the set (Q = -24 for f, -23 for
// g, see above), which for small values is also the step of the cut; the FMA adds exactly up to
// the FP32 rounding of the sum (2^-13 of a unit at most).  (Rounding BF16 by an integer add to the
// FP32 pattern and snapping the rare results below its grid step to the nearest grid value is
// cheaper, but that snap is a rounding to nearest and brought back the bias this mode removes:
// measured 8.1e-3 instead of 4.8e-3 on a sheared droplet against the FP64 oracle.)
template <class H, int Q> struct SRound;
template <int Q> struct SRound<__half, Q> {
  __device__ __forceinline__ static float pre(float v, uint32_t r) {
    const int ef = (int)((__float_as_uint(v) >> 23) & 0xFFu);
    const float u = __uint_as_float((uint32_t)max(ef - 26, Q + 111) << 23);  // unit * 2^-16
    const float rf = __uint_as_float(0x4B000000u | r) - 8388608.0f;          // r as a float, exactly
    const float p = fmaf(copysignf(u, v), rf, v);
    // FP16's subnormal step 2^-24 is the f grid; g's coarser grid needs its own cut first (the
    // conversion toward zero then cuts again on FP16's grid, which contains it).
    return Q == -24 ? p : grid_trunc(p, 1.0f);
  }
  __device__ __forceinline__ static __half round(float v, uint32_t r) { return __float2half_rz(pre(v, r)); }
};
template <int Q> struct SRound<__nv_bfloat16, Q> {
  // The pre-rounded value cut onto the grid; its high half is then the value cut toward zero.
  __device__ __forceinline__ static uint32_t bits(float v, uint32_t r) {
    const int ef = (int)((__float_as_uint(v) >> 23) & 0xFFu);
    const float u = __uint_as_float((uint32_t)max(ef - 23, Q + 111) << 23);  // unit * 2^-16
    const float rf = __uint_as_float(0x4B000000u | r) - 8388608.0f;
    const float p = fmaf(copysignf(u, v), rf, v);
    return __float_as_uint(grid_trunc(p, Q == -24 ? 0.5f : 1.0f));
  }
  __device__ __forceinline__ static __nv_bfloat16 round(float v, uint32_t r) {
    return __ushort_as_bfloat16((unsigned short)(bits(v, r) >> 16));
  }
};

template <class H> struct PopHalf {
  using C = float;
  static constexpr bool kFP16 = std::is_same<H, __half>::value;
  static constexpr size_t kBytesPerElem = 16 * sizeof(H) + 2 * sizeof(float);
  // The two FP32 rest planes follow the 16 half planes: 16 * sizeof(H) / 4 float planes in.
  static constexpr int kRestFirst = 16 * (int)sizeof(H) / (int)sizeof(float);
  // Values onto the grids of the f and g sets (exact conservation, see above): grid_f / grid_g
  // for any value the state holds (|v| < 1 for f deviations, < 2 for g), the cheaper snaps for
  // the small moving populations and wall terms of the step.
  __device__ __forceinline__ static float grid_f(float v) { return grid_round<24>(v); }
  __device__ __forceinline__ static float grid_g(float v) { return grid_round<23>(v); }
  __device__ __forceinline__ static float snap_f(float v) { return grid_snap(v, kGridF); }
  __device__ __forceinline__ static float snap_g(float v) { return grid_snap(v, kGridG); }
  // Moving populations rounded to nearest, on the grid: FP16 f needs no snap (FP16 values are
  // multiples of 2^-24); the others are snapped first (a second rounding of the snapped value can
  // differ from a single rounding only when the snap lands exactly halfway between two 16-bit
  // values).
  __device__ __forceinline__ static H encf(float d) { return Cvt<H>::from(kFP16 ? d : snap_f(d)); }
  __device__ __forceinline__ static H encg(float v) { return Cvt<H>::from(snap_g(v)); }
  // The moving-wall term of a bounced link, on the set's grid.
  __device__ __forceinline__ static float wall_term(float t, bool is_g) { return is_g ? snap_g(t) : snap_f(t); }
  template <class PL> __device__ __forceinline__ static const float* rest(const char* b, PL pl, int set, int idx) {
    return plane_elem<float>(b, pl, kRestFirst + set, idx);
  }
  template <class PL> __device__ __forceinline__ static float* rest(char* b, PL pl, int set, int idx) {
    return plane_elem<float>(b, pl, kRestFirst + set, idx);
  }
  template <class PL> __device__ __forceinline__ static const H* half(const char* b, PL pl, int p, int idx) {
    return plane_elem<H>(b, pl, p, idx);
  }
  template <class PL> __device__ __forceinline__ static H* half(char* b, PL pl, int p, int idx) {
    return plane_elem<H>(b, pl, p, idx);
  }
  template <class PL> __device__ __forceinline__ static C ldf(const char* b, PL pl, int i, int idx) {
    if (i == 0) return __ldg(rest(b, pl, 0, idx));
    return Cvt<H>::to(__ldg(half(b, pl, i - 1, idx)));
  }
  template <class PL> __device__ __forceinline__ static C ldg(const char* b, PL pl, int i, int idx) {
    if (i == 0) return __ldg(rest(b, pl, 1, idx));
    return Cvt<H>::to(__ldg(half(b, pl, 7 + i, idx)));
  }
  // Single values (checkpoint restore, of any size), put on the grids.
  template <class PL> __device__ __forceinline__ static void stf(char* b, PL pl, int i, int idx, C d) {
    if (i == 0) *rest(b, pl, 0, idx) = grid_f(d);
    else *half(b, pl, i - 1, idx) = Cvt<H>::from(grid_f(d));
  }
  template <class PL> __device__ __forceinline__ static void stg(char* b, PL pl, int i, int idx, C v) {
    if (i == 0) *rest(b, pl, 1, idx) = grid_g(v);
    else *half(b, pl, 7 + i, idx) = Cvt<H>::from(grid_g(v));
  }
  template <class PL> __device__ __forceinline__ static double ldf_full(const char* b, PL pl, int i, int idx) {
    return (double)ldf(b, pl, i, idx) + lat_w<double>(i);
  }
  template <class PL> __device__ __forceinline__ static void stf_full(char* b, PL pl, int i, int idx, double v) {
    stf(b, pl, i, idx, (float)(v - lat_w<double>(i)));
  }
  // Store one node with the rest populations as closures (Eq. 10: f_0 = rho - sum_{i>0} f_i,
  // g_0 = phi - sum_{i>0} g_i) of the ROUNDED moving populations, so that the stored values sum
  // to the node's rho and phi (the collision conserves both; the caller passes them, on the
  // grids): 16-bit rounding then redistributes among directions but does not create or destroy
  // mass or order parameter.  In deviations (sum_i w_i = 1): d_0 = (rho - 1) - sum_{i>0} d_i.
  // sr_key: 0 rounds to nearest; otherwise the step's key for stochastic rounding.
  template <class PL>
  __device__ __forceinline__ static void store_node(char* b, PL pl, int idx, const C f[9], const C g[9], float drho,
                                                    float phi, uint32_t sr_key = 0) {
    float sf = 0.0f, sg = 0.0f;
    auto put = [&](int i, H hf, H hg) {
      *half(b, pl, i - 1, idx) = hf;
      *half(b, pl, 7 + i, idx) = hg;
      sf += Cvt<H>::to(hf);
      sg += Cvt<H>::to(hg);
    };
    if (!sr_key) {  // one uniform branch: the round-to-nearest loop carries no stochastic code
#pragma unroll
      for (int i = 1; i < 9; ++i) put(i, encf(f[i]), encg(g[i]));
    } else {
      uint32_t w = sr_start((unsigned)idx, sr_key);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        if (i > 1) w = sr_next(w);
        put(i, SRound<H, -24>::round(f[i], w & 0xFFFFu), SRound<H, -23>::round(g[i], w >> 16));
      }
    }
    *rest(b, pl, 0, idx) = rest_f(drho, sf);
    *rest(b, pl, 1, idx) = phi - sg;
  }
  // The f rest closure from rho - 1 and the sum of the rounded moving deviations.
  __device__ __forceinline__ static float rest_f(float drho, float sum_dev) { return drho - sum_dev; }
  // Raw access: 32-bit words holding either the FP32 rest value (i = 0) or the 16-bit pattern of
  // a moving population, decoded only where used so that loads stay in flight.
  using R = uint32_t;
  template <class PL> __device__ __forceinline__ static R rawf(const char* b, PL pl, int i, int idx) {
    if (i == 0) return __float_as_uint(__ldg(rest(b, pl, 0, idx)));
    return (R)__ldg(reinterpret_cast<const unsigned short*>(half(b, pl, i - 1, idx)));
  }
  template <class PL> __device__ __forceinline__ static R rawg(const char* b, PL pl, int i, int idx) {
    if (i == 0) return __float_as_uint(__ldg(rest(b, pl, 1, idx)));
    return (R)__ldg(reinterpret_cast<const unsigned short*>(half(b, pl, 7 + i, idx)));
  }
  __device__ __forceinline__ static float h2f(R r) {
    H h;
    *reinterpret_cast<unsigned short*>(&h) = (unsigned short)r;
    return Cvt<H>::to(h);
  }
  __device__ __forceinline__ static C decf(int i, R r) { return i == 0 ? __uint_as_float(r) : h2f(r); }
  __device__ __forceinline__ static C decg(int i, R r) { return i == 0 ? __uint_as_float(r) : h2f(r); }
  __device__ __forceinline__ static R keep(C v) { return __float_as_uint(v); }
  __device__ __forceinline__ static C kept(R r) { return __uint_as_float(r); }
};
template <> struct Pop<2> : PopHalf<__half> {};
template <> struct Pop<3> : PopHalf<__nv_bfloat16> {};

// ---------------------------------------------------------------------------------------------
// Lattice geometry and physical parameters as passed to the kernels.

struct Geometry {
  int nx, ny, pitch;
  long long plane;  // elements per plane (pitch * ny)
  int walls;        // 0 periodic, 1 bounce-back walls at y = -1/2 and y = ny - 1/2
};

template <class C> struct Phys {
  C omega_l, omega_g, tau_l, tau_g;  // f relaxation of phase l (phi=+1) and g (phi=-1)
  C omega3, omega_phi;
  C gamma, a, Gamma;
  C u_top, u_bottom;      // wall x-velocities
  C wet_bottom, wet_top;  // wall gradients of phi along the outward normal (Eq. 18); ghost rows
  C force_x, force_y;     // body force per unit volume
  int visc;               // 0 omega-linear (paper), 1 tau-linear
  int k8_printed;         // 0 projected k8, 1 printed k8
  int bgk;                // 0 central moments (paper), 1 BGK baseline
  int force_mode;         // 0 uniform, 1 on phase l only: F (1 + phi)/2
  int forced;             // force_x or force_y non-zero
  uint32_t sr_key;        // 16-bit storage: 0 rounds to nearest, else this step's stochastic-rounding key
  int rounding;           // lbm_rounding (a batch derives sr_key from seed and its step counter)
  uint32_t seed;          // stochastic-rounding seed
};

// Physics in the kernel's arithmetic type from the validated host parameters.
template <class C> inline Phys<C> make_phys(const HostPhys& h) {
  Phys<C> p;
  p.omega_l = (C)h.omega_l;
  p.omega_g = (C)h.omega_g;
  p.tau_l = (C)h.tau_l;
  p.tau_g = (C)h.tau_g;
  p.omega3 = (C)h.omega3;
  p.omega_phi = (C)h.omega_phi;
  p.gamma = (C)h.gamma;
  p.a = (C)h.a;
  p.Gamma = (C)h.Gamma;
  p.u_top = (C)h.u_top;
  p.u_bottom = (C)h.u_bottom;
  p.wet_bottom = (C)h.wet_bottom;
  p.wet_top = (C)h.wet_top;
  p.force_x = (C)h.force_x;
  p.force_y = (C)h.force_y;
  p.visc = h.visc;
  p.k8_printed = h.k8_printed;
  p.bgk = h.bgk;
  p.force_mode = h.force_mode;
  p.forced = h.force_x != 0.0 || h.force_y != 0.0;
  p.sr_key = h.sr_key;
  p.rounding = h.rounding;
  p.seed = h.seed;
  return p;
}

// Body force at a node of order parameter phi.
template <class C>
__device__ __forceinline__ void body_force(const Phys<C>& ph, C phi, C& Fx, C& Fy) {
  const C w = ph.force_mode ? C(0.5) * (phi + C(1)) : C(1);
  Fx = ph.force_x * w;
  Fy = ph.force_y * w;
}

// ---------------------------------------------------------------------------------------------
// Streaming, Eqs. 4-5, in pull form: the population of direction i at node (x, y) and time t is
// the post-collision value of node (x - c_xi, y - c_yi) at t - 1.  x is periodic; y periodic or
// walled.  A link whose source lies beyond a wall is the bounced-back population of the node
// itself, opposite direction, plus the moving-wall term 6 w_i s c_xi u_w, where s is the node's
// own density (for f) or order parameter (for g) at t - 1.
template <int PREC, bool IS_G, class PL = long long>
__device__ __forceinline__ void pull(const char* __restrict__ src, const Geometry& geo,
                                     typename Pop<PREC>::C u_top, typename Pop<PREC>::C u_bot,
                                     int x, int y, typename Pop<PREC>::C out[9], PL pl = PL()) {
  using P = Pop<PREC>;
  using C = typename P::C;
  if constexpr (std::is_same<PL, long long>::value) pl = geo.plane;
  auto LD = [&](int i, int idx) -> C { return IS_G ? P::ldg(src, pl, i, idx) : P::ldf(src, pl, i, idx); };
  const int xm = (x == 0) ? geo.nx - 1 : x - 1;
  const int xp = (x == geo.nx - 1) ? 0 : x + 1;
  const int r0 = y * geo.pitch;
  const bool bot = geo.walls && y == 0;
  const bool top = geo.walls && y == geo.ny - 1;
  if (!bot && !top) {
    const int ym = (y == 0) ? geo.ny - 1 : y - 1;
    const int yp = (y == geo.ny - 1) ? 0 : y + 1;
    const int rm = ym * geo.pitch, rp = yp * geo.pitch;
    out[0] = LD(0, r0 + x);
    out[1] = LD(1, r0 + xm);
    out[2] = LD(2, rm + x);
    out[3] = LD(3, r0 + xp);
    out[4] = LD(4, rp + x);
    out[5] = LD(5, rm + xm);
    out[6] = LD(6, rm + xp);
    out[7] = LD(7, rp + xp);
    out[8] = LD(8, rp + xm);
    return;
  }
  // Wall row: the node's own nine post-collision values give s (rho for f, phi for g) and the
  // reflected links.  f values are deviations from w_i; w_i is the same for a link and its
  // reflection, so the links move as deviations and only s needs the rest density 1.
  C own[9];
  C s = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    own[i] = LD(i, r0 + x);
    s += own[i];
  }
  if (!IS_G) s += C(1);
  out[0] = own[0];
  out[1] = LD(1, r0 + xm);
  out[3] = LD(3, r0 + xp);
  const C k6 = C(6) * s / C(36);
  if (bot) {  // directions 2, 5, 6 come from below the wall at y = -1/2
    const int rp = (y + 1) * geo.pitch;
    out[2] = own[4];
    out[5] = own[7] + P::wall_term(k6 * u_bot, IS_G);   // 6 w_5 s c_x5 u_w, w_5 = 1/36, c_x5 = +1
    out[6] = own[8] - P::wall_term(k6 * u_bot, IS_G);   // c_x6 = -1
    out[4] = LD(4, rp + x);
    out[7] = LD(7, rp + xp);
    out[8] = LD(8, rp + xm);
  } else {    // directions 4, 7, 8 come from above the wall at y = ny - 1/2
    const int rm = (y - 1) * geo.pitch;
    out[4] = own[2];
    out[7] = own[5] - P::wall_term(k6 * u_top, IS_G);   // c_x7 = -1
    out[8] = own[6] + P::wall_term(k6 * u_top, IS_G);   // c_x8 = +1
    out[2] = LD(2, rm + x);
    out[5] = LD(5, rm + xm);
    out[6] = LD(6, rm + xp);
  }
}

// Raw variant of pull(): for rows away from walls the nine values are the stored bits, left
// undecoded (returns false); wall rows need arithmetic, so they are pulled decoded and kept as
// such (returns true).  unpack() turns either form into values.
template <int PREC, bool IS_G, class PL = long long>
__device__ __forceinline__ bool pull_raw(const char* __restrict__ src, const Geometry& geo,
                                         typename Pop<PREC>::C u_top, typename Pop<PREC>::C u_bot,
                                         int x, int y, typename Pop<PREC>::R out[9], PL pl = PL()) {
  using P = Pop<PREC>;
  using C = typename P::C;
  if (geo.walls && (y == 0 || y == geo.ny - 1)) {
    C v[9];
    pull<PREC, IS_G, PL>(src, geo, u_top, u_bot, x, y, v, pl);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = P::keep(v[i]);
    return true;
  }
  if constexpr (std::is_same<PL, long long>::value) pl = geo.plane;
  auto LD = [&](int i, int idx) { return IS_G ? P::rawg(src, pl, i, idx) : P::rawf(src, pl, i, idx); };
  const int xm = (x == 0) ? geo.nx - 1 : x - 1;
  const int xp = (x == geo.nx - 1) ? 0 : x + 1;
  const int ym = (y == 0) ? geo.ny - 1 : y - 1;
  const int yp = (y == geo.ny - 1) ? 0 : y + 1;
  const int r0 = y * geo.pitch, rm = ym * geo.pitch, rp = yp * geo.pitch;
  out[0] = LD(0, r0 + x);
  out[1] = LD(1, r0 + xm);
  out[2] = LD(2, rm + x);
  out[3] = LD(3, r0 + xp);
  out[4] = LD(4, rp + x);
  out[5] = LD(5, rm + xm);
  out[6] = LD(6, rm + xp);
  out[7] = LD(7, rp + xp);
  out[8] = LD(8, rp + xm);
  return false;
}

template <int PREC, bool IS_G>
__device__ __forceinline__ void unpack(const typename Pop<PREC>::R raw[9], bool decoded,
                                       typename Pop<PREC>::C out[9]) {
  using P = Pop<PREC>;
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = decoded ? P::kept(raw[i]) : (IS_G ? P::decg(i, raw[i]) : P::decf(i, raw[i]));
}

// c_i . (vx, vy) for lattice direction i, without multiplying by the velocity set's 0 and +-1
// components (for finite inputs the same value as the two products and the sum).
template <class C>
__device__ __forceinline__ C lat_dot(int i, C vx, C vy) {
  const int cx = lat_cx(i), cy = lat_cy(i);
  if (cx == 0) return cy > 0 ? vy : -vy;
  if (cy == 0) return cx > 0 ? vx : -vx;
  if (cx == cy) return cx > 0 ? vx + vy : -(vx + vy);
  return cx > 0 ? vx - vy : vy - vx;
}

// 1 / x for the collision's two runtime reciprocals (1/rho and the relaxation frequency).
template <class C>
__device__ __forceinline__ C recip(C x) {
  return C(1) / x;
}

// ---------------------------------------------------------------------------------------------
// Collision of one node.  Inputs: pulled f as deviations d_i = f_i - w_i from the rest state,
// pulled g; phi = sum g; the Eq. 12 stencils dx, dy, lap of phi.  Outputs overwrite f (again as
// deviations) and g with the post-collision values.  Returns rho - 1.
//
// Every moment of f is carried minus its value at rest (rho = 1, u = 0): rho = 1 + drho, the raw
// second moments m20 = m02 = 1/3 + M, m22 = 1/9 + R22, the central moments k3 = 2/3 + K3 and
// k8 = 1/9 + K8, the pressure p~ = 1/3 + Pt.  The rest values cancel from Eq. 17 and from the
// inverse transform, so they never enter the arithmetic and no rounding at the scale of w_i
// (order 0.1) touches the departures from rest (order u ~ 1e-2 and below) that carry the flow.
template <class C>
__device__ __forceinline__ C collide(const Phys<C>& ph, C f[9], C g[9], C phi, C dx, C dy, C lap) {
  const C cs2 = C(1) / C(3);
  // Macroscopic moments (paragraph after Eq. 14); sum_i w_i c_i = 0, so j needs no rest value.
  const C drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const C rho = C(1) + drho;
  const C jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const C jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const C inv_rho = recip(rho);
  // Body force (Guo's scheme): the velocity carries half the force, u = (j + F/2)/rho.
  C Fx = C(0), Fy = C(0);
  if (ph.forced) body_force(ph, phi, Fx, Fy);
  const C ux = ph.forced ? (jx + C(0.5) * Fx) * inv_rho : jx * inv_rho;
  const C uy = ph.forced ? (jy + C(0.5) * Fy) * inv_rho : jy * inv_rho;
  const C ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
  // Chemical potential (free-energy paragraph); the non-ideal part q = p~ - rho c_s^2 of the
  // pressure (Eqs. 13, 14), and Pt = p~ - 1/3.
  const C phi2 = phi * phi;
  const C mu = ph.a * (phi2 * phi - phi) - ph.gamma * lap;
  const C q = ph.a * phi2 * (C(0.75) * phi2 - C(0.5)) - ph.gamma * phi * lap;
  const C Pt = drho * cs2 + q;
  // Relaxation frequency of f for this phi (paragraph after Eq. 14).
  C om;
  if (ph.visc == 0) om = ph.omega_g + C(0.5) * (phi + C(1)) * (ph.omega_l - ph.omega_g);
  else om = recip(ph.tau_g + C(0.5) * (phi + C(1)) * (ph.tau_l - ph.tau_g));

  if (!ph.bgk) {
    // Pre-collision central moments k3, k4, k5 (Eq. 15 basis, k = T^T f) from the raw second
    // moments: kappa_20 = m_20 - rho ux^2, kappa_02 = m_02 - rho uy^2, kappa_11 = m_11 - rho ux uy.
    const C corners = (f[5] + f[6]) + (f[7] + f[8]);
    const C M20 = (f[1] + f[3]) + corners;  // m_20 - 1/3
    const C M02 = (f[2] + f[4]) + corners;  // m_02 - 1/3
    const C m11 = (f[5] - f[6]) + (f[7] - f[8]);
    C k20 = M20 - rho * ux2, k02 = M02 - rho * uy2, k11 = m11 - rho * uxy;  // kappa_20 - 1/3, ...
    if (ph.forced) {
      // with the half-force velocity the first central moments are -F/2 before the collision:
      // kappa_20 = m_20 - 2 ux kappa_10 - rho ux^2 and so on
      k20 += ux * Fx;
      k02 += uy * Fy;
      k11 += C(0.5) * (ux * Fy + uy * Fx);
    }
    const C K3 = k20 + k02, k4 = k20 - k02, k5 = k11;  // K3 = k3 - 2/3
    // Equilibrium central moments (the k_eq list and Eq. 16): k3e = 2 p~; in k6e, k7e and k8e
    // the ideal parts rho c_s^2 of p~ cancel against the rho c_s^2 terms, leaving q.
    const C K3e = C(2) * Pt;
    const C k4e = ph.gamma * (dx * dx - dy * dy);
    const C k5e = ph.gamma * dx * dy;
    const C k6e = -C(0.5) * uy * k4e - C(2) * ux * k5e - rho * uy * ux2 - q * uy;
    const C k7e = C(0.5) * ux * k4e - C(2) * uy * k5e - rho * ux * uy2 - q * ux;
    const C grad_term = ph.k8_printed ? lap : (dx * dx + dy * dy);
    const C K8e = Pt * cs2 + q * (ux2 + uy2) + C(3) * rho * ux2 * uy2 - C(0.5) * cs2 * ph.gamma * grad_term +
                  C(0.5) * k4e * (uy2 - ux2) + C(4) * uxy * k5e;  // k8e - 1/9
    // Eq. 17 with omega_4 = omega_5 = omega_rho, omega_3 free, omega_6..8 = 1.
    const C K3s = K3 + ph.omega3 * (K3e - K3);
    const C k4s = k4 + om * (k4e - k4);
    const C k5s = k5 + om * (k5e - k5);
    // Force: central moments of Guo's source, (T^T S)_j; zero for j = 0, 3, 4, 5, F for j = 1, 2,
    // and for j = 6..8 (omega = 1, so half of each is added):
    C k6s = k6e, k7s = k7e, K8s = K8e;
    if (ph.forced) {
      k6s += C(0.5) * (Fy * cs2 - C(2) * Fx * uxy - Fy * ux2);
      k7s += C(0.5) * (Fx * cs2 - Fx * uy2 - C(2) * Fy * uxy);
      K8s += C(2) * uxy * (Fx * uy + Fy * ux);
    }
    // f* = (T^T)^-1 k*, k* = [rho, F_x/2, F_y/2, k3*, k4*, k5*, k6*, k7*, k8*] (the paper's
    // [rho, 0, 0, ...] without a force): central -> raw moments by the binomial shift
    // c = cbar + u, then the D2Q9 raw-moment inversion.  A20 = a20 - 1/3, R20 = r20 - 1/3,
    // R22 = r22 - 1/9; a20, a02 themselves only multiply velocities.
    const C A20 = C(0.5) * (K3s + k4s), A02 = C(0.5) * (K3s - k4s), a11 = k5s;
    const C a20 = A20 + cs2, a02 = A02 + cs2;
    C R20 = A20 + rho * ux2;
    C R02 = A02 + rho * uy2;
    C r11 = a11 + rho * uxy;
    C r21 = k6s + C(2) * ux * a11 + uy * a20 + rho * ux2 * uy;
    C r12 = k7s + C(2) * uy * a11 + ux * a02 + rho * ux * uy2;
    C R22 = K8s + C(2) * (uy * k6s + ux * k7s) + uy2 * a20 + ux2 * a02 + C(4) * uxy * a11 + rho * ux2 * uy2;
    C r10 = jx, r01 = jy;
    if (ph.forced) {
      const C q1 = C(0.5) * Fx, q2 = C(0.5) * Fy;  // k*_1, k*_2
      r10 = jx + Fx;                               // rho ux + k*_1
      r01 = jy + Fy;
      R20 += C(2) * ux * q1;
      R02 += C(2) * uy * q2;
      r11 += ux * q2 + uy * q1;
      r21 += ux2 * q2 + C(2) * uxy * q1;
      r12 += uy2 * q1 + C(2) * uxy * q2;
      R22 += C(2) * uxy * (uy * q1 + ux * q2);
    }
    // Deviations: f0 = rho - r20 - r02 + r22 (w_0 = 4/9 = 1 - 2/3 + 1/9), f1 = (r20 - r22)/2 +
    // (r10 - r12)/2 (w_1 = 1/9 = (1/3 - 1/9)/2), f5 = (r22 + r11 + r21 + r12)/4 (w_5 = 1/36), ...
    f[0] = drho - R20 - R02 + R22;
    const C hx = C(0.5) * (R20 - R22), hy = C(0.5) * (R02 - R22);
    const C qx = C(0.5) * (r10 - r12), qy = C(0.5) * (r01 - r21);
    f[1] = hx + qx;
    f[3] = hx - qx;
    f[2] = hy + qy;
    f[4] = hy - qy;
    const C s22 = C(0.25) * R22, s11 = C(0.25) * r11, s21 = C(0.25) * r21, s12 = C(0.25) * r12;
    f[5] = s22 + s11 + s21 + s12;
    f[6] = s22 - s11 + s21 - s12;
    f[7] = s22 + s11 - s21 - s12;
    f[8] = s22 - s11 - s21 + s12;
  } else {
    // Double-BGK baseline, Eq. 6 with f_eq from Eqs. 8, 10, 11; 3 p~ = 1 + 3 Pt, so
    // f_eq,i - w_i = w_i (3 Pt + rho (...)) + the gradient terms, and f_eq,0 - w_0 = drho - sum.
    const C uu = ux2 + uy2;
    const C gxx = ph.gamma * dx * dx, gyy = ph.gamma * dy * dy, gxy = ph.gamma * dx * dy;
    C sum = C(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const C w = C(lat_w36(i)) / C(36);
      const C cu = lat_dot<C>(i, ux, uy);
      // Eq. 11 weights (w^yy_4 = +1/3): axis i: w^xx = 1/3 on x-links, -1/6 on y-links; diagonals -1/24.
      C wxx, wyy, wxy;
      if (i <= 4) {
        const bool xl = lat_cx(i) != 0;
        wxx = xl ? C(1) / C(3) : -C(1) / C(6);
        wyy = xl ? -C(1) / C(6) : C(1) / C(3);
        wxy = C(0);
      } else {
        wxx = -C(1) / C(24);
        wyy = -C(1) / C(24);
        wxy = C(0.25 * lat_cx(i) * lat_cy(i));
      }
      const C deq = w * (C(3) * Pt + rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu)) +
                    (wxx * gxx + wyy * gyy + wxy * gxy);
      sum += deq;
      f[i] = f[i] + om * (deq - f[i]);
      if (ph.forced) {
        // Guo's source S_i = w_i [3 (c_i - u) . F + 9 (c_i . u)(c_i . F)], weighted 1 - omega/2
        const C cF = lat_dot<C>(i, Fx, Fy);
        f[i] += (C(1) - C(0.5) * om) * w * (C(3) * (cF - (ux * Fx + uy * Fy)) + C(9) * cu * cF);
      }
    }
    const C deq0 = drho - sum;
    f[0] = f[0] + om * (deq0 - f[0]);
    if (ph.forced) f[0] += (C(1) - C(0.5) * om) * (C(4) / C(9)) * (-C(3) * (ux * Fx + uy * Fy));
  }

  // g: BGK towards g_eq (Eqs. 7, 9, 10).  The rest population's departure from equilibrium is
  // g0eq - g0 = (phi - sum_{i>0} geq_i) - g0 = -sum_{i>0} (geq_i - g_i) (phi = sum g), so g0 is
  // updated by that small increment: g0, of the order of phi, then takes one rounding per step
  // instead of the roundings of phi and of the closure at its own scale (FP32: ulp(1) ~ 1e-7).
  {
    const C uu = ux2 + uy2;
    const C gmu = ph.Gamma * mu;
    C dsum = C(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const C w = C(lat_w36(i)) / C(36);
      const C cu = lat_dot<C>(i, ux, uy);
      const C geq = w * (gmu + phi * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu));
      const C d = geq - g[i];
      dsum += d;
      g[i] = g[i] + ph.omega_phi * d;
    }
    g[0] = g[0] - ph.omega_phi * dsum;
  }
  return drho;
}

// Isotropic stencils of Eq. 12 from the 3x3 neighbourhood of phi.  Index convention:
// s[dy+1][dx+1] = phi(x + dx, y + dy).
template <class C>
__device__ __forceinline__ void stencils(const C s[3][3], C& dx, C& dy, C& lap) {
  const C E = s[1][2], W = s[1][0], N = s[2][1], S = s[0][1];
  const C NE = s[2][2], NW = s[2][0], SW = s[0][0], SE = s[0][2];
  dx = (E - W) * (C(1) / C(3)) + ((NE - SW) + (SE - NW)) * (C(1) / C(12));
  dy = (N - S) * (C(1) / C(3)) + ((NE - SW) + (NW - SE)) * (C(1) / C(12));
  lap = (C(4) * ((E + W) + (N + S)) + ((NE + SW) + (NW + SE)) - C(20) * s[1][1]) * (C(1) / C(6));
}

}  // namespace lbmch
