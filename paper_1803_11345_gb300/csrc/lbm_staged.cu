// Staged variant of the fused step: whole rows of all 18 population planes are streamed
// into shared-memory rings by the bulk-copy (TMA) engine, and every pull (Eqs. 4-5), the
// phi sums and the Eq. 12 stencils read shared memory.
//
// CTA = BX columns x BY thread rows, marching down `rows` lattice rows in bands of BY, in the
// same order as the generic kernel (lbm_kernels.cu):
//   step Y:  wait for the rows of this step -> phi of rows Y+BY .. Y+2BY-1 from staged g (kept
//            in registers for the next step) -> f of rows Y .. Y+BY-1 from staged f ->
//            __syncthreads -> thread 0 issues the bulk copies of the rows needed one step
//            later into the slots just freed -> collision of rows Y .. Y+BY-1 -> stores.
// Staged row v of a set (f or g) holds, for each of its 9 planes, columns
// [x0 - H, x0 + BX + H) with H = 16 bytes / element size, so every copy is 16-byte aligned;
// the halo chunks wrap around periodically.  This needs nx to be a multiple of H; other widths
// use the generic kernel.
#include <algorithm>
#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_tma.cuh"

namespace lbmch {

// Layout of a staged row and of the state in global memory, per storage precision.
template <int PREC> struct Stage {
  using P = Pop<PREC>;
  using C = typename P::C;
  static constexpr bool kHalf = PREC >= 2;
  static constexpr int kEs = PREC == 0 ? 8 : (PREC == 1 ? 4 : 2);  // bytes of a packed population
  static constexpr int H = 16 / kEs;                                   // halo columns per side
  // Element size of population p of either set (16-bit storage keeps p = 0 in FP32).
  __host__ __device__ static constexpr int es(bool g, int p) { return (kHalf && p == 0) ? 4 : kEs; }
  // Byte offset of plane p inside a staged row of W columns (16-bit: the FP32 rest plane first).
  __host__ __device__ static constexpr int soff(bool g, int p, int W) {
    return !kHalf ? p * W * kEs : (p == 0 ? 0 : W * 4 + (p - 1) * W * 2);
  }
  __host__ __device__ static constexpr int row_bytes(bool g, int W) { return soff(g, 8, W) + W * es(g, 8); }
  // Global byte offset of element idx of population p of set g (layout of Pop<PREC>).
  __device__ __forceinline__ static long long goff(bool g, int p, long long pl, long long idx) {
    if (!kHalf) return ((g ? 9 : 0) + p) * pl * kEs + idx * kEs;
    if (p == 0) return 16 * pl * 2 + (g ? pl * 4 : 0) + idx * 4;
    return ((g ? 7 : -1) + p) * pl * 2 + idx * 2;
  }
  // Output staging: plane q = 0..17 (f_0..f_8, g_0..g_8), n elements each, packed in order.
  __host__ __device__ static constexpr int oes(int q) { return q < 9 ? es(false, q) : es(true, q - 9); }
  __host__ __device__ static constexpr int ooff(int q, int n) { return q == 0 ? 0 : ooff(q - 1, n) + n * oes(q - 1); }
  // Population value from a staged row (a points at the element); f as its deviation from w_p,
  // as Pop<PREC> presents it.
  __device__ __forceinline__ static C sld(const char* a, bool g, int p) {
    if constexpr (!kHalf) {
      const C v = *reinterpret_cast<const C*>(a);
      return g ? v : P::fdec(p, v);
    } else {
      if (p == 0) return *reinterpret_cast<const float*>(a);
      using Hf = typename std::conditional<PREC == 2, __half, __nv_bfloat16>::type;
      return Cvt<Hf>::to(*reinterpret_cast<const Hf*>(a));
    }
  }
  // Store the post-collision populations of one node (element e of every output plane of n
  // elements) into the staging buffer, with the same encoding as Pop<PREC>::store_node.
  __device__ __forceinline__ static void store_node(char* ob, int n, int e, const C f[9], const C g[9], C drho,
                                                    C phi) {
    if constexpr (!kHalf) {
#pragma unroll
      for (int q = 0; q < 18; ++q) reinterpret_cast<C*>(ob + ooff(q, n))[e] = q < 9 ? P::fenc(q, f[q]) : g[q - 9];
    } else {
      using Hf = typename std::conditional<PREC == 2, __half, __nv_bfloat16>::type;
      float sf = 0.0f, sg = 0.0f;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const Hf hf = PopHalf<Hf>::encf(f[i]);
        const Hf hg = PopHalf<Hf>::encg(g[i]);
        reinterpret_cast<Hf*>(ob + ooff(i, n))[e] = hf;
        reinterpret_cast<Hf*>(ob + ooff(9 + i, n))[e] = hg;
        sf += Cvt<Hf>::to(hf);
        sg += Cvt<Hf>::to(hg);
      }
      reinterpret_cast<float*>(ob + ooff(0, n))[e] = PopHalf<Hf>::rest_f(drho, sf);
      reinterpret_cast<float*>(ob + ooff(9, n))[e] = phi - sg;
    }
  }
};

template <int BY, int D> struct Ring {
  static constexpr int R = (D + 1) * BY + 2;  // rows per ring (f and g alike)
};

template <int PREC, int BX, int BY, int D>
size_t staged_smem_bytes() {
  using S = Stage<PREC>;
  using C = typename S::C;
  constexpr int W = BX + 2 * S::H;
  constexpr int R = Ring<BY, D>::R;
  size_t b = (size_t)R * S::row_bytes(true, W) + (size_t)R * S::row_bytes(false, W);
  b += (size_t)S::ooff(18, BX * BY);
  b += (size_t)(3 * BY + 1) * (BX + 2) * sizeof(C);
  b = (b + 15) / 16 * 16;
  b += 2 * R * sizeof(uint64_t) + 16;
  return b;
}

// Probes before a wait is declared stuck (each probe suspends for a short hardware window):
// far beyond any legitimate copy latency, short enough to return control in well under a second.
// The waits of the main loop take their limit from the launch (lbm_set_wait_limit; this one by
// default, 0 = give up without probing); the prologue's waits and those that drain the copies
// still in flight after an abort always take this one, so that no copy can land in shared memory
// after the CTA has returned.
constexpr uint32_t kWaitProbes = 1u << 22;

template <int PREC, int BX, int BY, int D>
__global__ void __launch_bounds__(BX * BY)
k_step_staged(const char* __restrict__ src, char* __restrict__ dst, const Geometry geo,
              const Phys<typename Pop<PREC>::C> ph, const int rows, int* __restrict__ flag,
              const uint32_t wait_limit) {
  using S = Stage<PREC>;
  using P = Pop<PREC>;
  using C = typename S::C;
  constexpr int H = S::H;
  constexpr int W = BX + 2 * H;
  constexpr int R = Ring<BY, D>::R;
  constexpr int RBG = S::row_bytes(true, W);
  constexpr int RBF = S::row_bytes(false, W);
  constexpr int NOUT = BX * BY;    // elements per output plane
  constexpr int PHR = 3 * BY + 1;  // phi ring rows (same argument as the generic kernel)
  constexpr int PHW = BX + 2;
  constexpr int NW = BX * BY / 32;

  extern __shared__ __align__(128) char smem[];
  char* gring = smem;
  char* fring = gring + R * RBG;
  char* obuf = fring + R * RBF;
  C* sphi = reinterpret_cast<C*>(obuf + S::ooff(18, NOUT));
  size_t boff = (size_t)R * RBG + (size_t)R * RBF + S::ooff(18, NOUT) + sizeof(C) * PHR * PHW;
  boff = (boff + 15) / 16 * 16;
  uint64_t* gbar = reinterpret_cast<uint64_t*>(smem + boff);
  uint64_t* fbar = gbar + R;
  int* abort_flag = reinterpret_cast<int*>(fbar + R);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const int warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * BX;
  const int y0 = blockIdx.y * rows;
  const int y1 = min(y0 + rows, geo.ny);
  const int xv = min(BX, geo.nx - x0);
  const bool colv = tx < xv;
  const int gvb = y0 - 2, fvb = y0 - 1;  // first staged g / f row
  const int g_last = y1 + 1, f_last = y1;
  const bool interior = x0 > 0 && x0 + xv < geo.nx;
  const int xl = (x0 == 0) ? geo.nx - H : x0 - H;
  const int xr = (x0 + xv == geo.nx) ? 0 : x0 + xv;

  if (tid == 0) {
    for (int k = 0; k < R; ++k) {
      mbar_init(&gbar[k], 1);
      mbar_init(&fbar[k], 1);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  auto phys_row = [&](int v) -> int {
    if (v < 0) return geo.walls ? 0 : v + geo.ny;
    if (v >= geo.ny) return geo.walls ? geo.ny - 1 : v - geo.ny;
    return v;
  };
  // Ghost rows beyond a wall hold the adjacent row's phi plus the wall gradient (Eq. 18); both
  // gradients are 0 on periodic lattices.
  auto ghost = [&](int v) -> C {
    if (!geo.walls) return C(0);
    return v < 0 ? ph.wet_bottom : (v >= geo.ny ? ph.wet_top : C(0));
  };

  // Staging of row v of set g (true) or f (false) by one warp: lane 0 arms the slot's barrier
  // with the byte count, then one lane per (plane, segment) issues its copy.
  auto issue_row_warp = [&](bool g, int v) {
    const int k = v - (g ? gvb : fvb);
    char* drow = g ? gring + (k % R) * RBG : fring + (k % R) * RBF;
    uint64_t* bar = g ? &gbar[k % R] : &fbar[k % R];
    const long long rowidx = (long long)phys_row(v) * geo.pitch;
    if (lane == 0) {
      uint32_t total = 0;
#pragma unroll
      for (int p = 0; p < 9; ++p) total += (uint32_t)((xv + 2 * H) * S::es(g, p));
      mbar_arrive_expect_tx(bar, total);
    }
    __syncwarp();
    if (interior) {
      if (lane < 9) {
        const int p = lane, e = S::es(g, p);
        bulk_g2s(drow + S::soff(g, p, W), src + S::goff(g, p, geo.plane, rowidx + x0 - H),
                 (uint32_t)((xv + 2 * H) * e), bar);
      }
    } else if (lane < 27) {
      const int p = lane / 3, seg = lane - 3 * p, e = S::es(g, p);
      char* d = drow + S::soff(g, p, W);
      if (seg == 0) bulk_g2s(d, src + S::goff(g, p, geo.plane, rowidx + xl), (uint32_t)(H * e), bar);
      else if (seg == 1) bulk_g2s(d + H * e, src + S::goff(g, p, geo.plane, rowidx + x0), (uint32_t)(xv * e), bar);
      else bulk_g2s(d + (H + xv) * e, src + S::goff(g, p, geo.plane, rowidx + xr), (uint32_t)(H * e), bar);
    }
  };
  // All threads call this with the same arguments; rows are dealt out to warps.
  int g_next = gvb, f_next = fvb;
  auto issue_upto = [&](int g_target, int f_target) {
    const int ng = max(0, min(g_target, g_last) - g_next + 1);
    const int nf = max(0, min(f_target, f_last) - f_next + 1);
    for (int k = warp; k < ng + nf; k += NW) {
      if (k < ng) issue_row_warp(true, g_next + k);
      else issue_row_warp(false, f_next + (k - ng));
    }
    g_next += ng;
    f_next += nf;
  };
  bool stuck = false;
  auto wait_row = [&](bool g, int v, uint32_t limit) {
    const int k = v - (g ? gvb : fvb);
    uint64_t* bar = g ? &gbar[k % R] : &fbar[k % R];
    if (!mbar_wait_bounded(bar, (uint32_t)((k / R) & 1), limit)) stuck = true;
  };

  // Pointers to the staged rows v-1, v, v+1 of a set, for the node at virtual row v (a wall
  // mirror row stands for its physical twin) and column byte offset.
  struct Rows3 {
    const char* lo;
    const char* mid;
    const char* hi;
    int y;  // physical row of the node
  };
  auto rows3 = [&](bool g, int v, int cbytes) -> Rows3 {
    if (geo.walls) v = v < 0 ? 0 : (v >= geo.ny ? geo.ny - 1 : v);
    const int k = v - (g ? gvb : fvb);
    const int sm = k % R;
    const int sl = sm == 0 ? R - 1 : sm - 1;
    const int sh = sm == R - 1 ? 0 : sm + 1;
    const char* base = (g ? gring : fring) + cbytes;
    const int rb = g ? RBG : RBF;
    Rows3 r3;
    r3.lo = base + sl * rb;
    r3.mid = base + sm * rb;
    r3.hi = base + sh * rb;
    r3.y = phys_row(v);
    return r3;
  };
  // Pull (Eqs. 4-5) from staged rows, same rule as pull() in lbm_device.cuh; c0 = the node's
  // column offset is folded into the row pointers, so every access has a constant offset.
  auto pull_s = [&](bool g, const Rows3& q, C out[9]) {
    auto L = [&](const char* row, int p, int dc) -> C {
      return S::sld(row + S::soff(g, p, W) + dc * S::es(g, p), g, p);
    };
    const bool bot = geo.walls && q.y == 0;
    const bool top = geo.walls && q.y == geo.ny - 1;
    if (!bot && !top) {
      out[0] = L(q.mid, 0, 0);
      out[1] = L(q.mid, 1, -1);
      out[2] = L(q.lo, 2, 0);
      out[3] = L(q.mid, 3, 1);
      out[4] = L(q.hi, 4, 0);
      out[5] = L(q.lo, 5, -1);
      out[6] = L(q.lo, 6, 1);
      out[7] = L(q.hi, 7, 1);
      out[8] = L(q.hi, 8, -1);
      return;
    }
    C own[9];
    C s = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      own[i] = L(q.mid, i, 0);
      s += own[i];
    }
    if (!g) s += C(1);  // f values are deviations from w_i: rho = 1 + their sum
    out[0] = own[0];
    out[1] = L(q.mid, 1, -1);
    out[3] = L(q.mid, 3, 1);
    const C k6 = C(6) * s / C(36);
    if (bot) {
      out[2] = own[4];
      out[5] = own[7] + P::wall_term(k6 * ph.u_bottom, g);
      out[6] = own[8] - P::wall_term(k6 * ph.u_bottom, g);
      out[4] = L(q.hi, 4, 0);
      out[7] = L(q.hi, 7, 1);
      out[8] = L(q.hi, 8, -1);
    } else {
      out[4] = own[2];
      out[7] = own[5] - P::wall_term(k6 * ph.u_top, g);
      out[8] = own[6] + P::wall_term(k6 * ph.u_top, g);
      out[2] = L(q.lo, 2, 0);
      out[5] = L(q.lo, 5, -1);
      out[6] = L(q.lo, 6, 1);
    }
  };
  auto sum9 = [](const C v[9]) -> C {
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
  };
  constexpr int kEsC = S::kEs;  // column stride of every staged plane but the 16-bit g_0 one
  static_assert(S::kHalf || kEsC == (int)sizeof(C), "staged element size");
  // phi of virtual row v for this thread's column (and the halo columns for tx == 0 / BX-1).
  // The column offset differs between the 16-bit g_0 plane (4 bytes) and the others; fold the
  // column into the pointer per plane inside sld instead for that case.
  // 16-bit staging: planes have two element sizes (the FP32 rest plane and 16-bit others), so
  // each access carries its own column offset.
  auto pull_explicit = [&](bool g, int v, int c, C out[9]) {
    const Rows3 q = rows3(g, v, 0);
    const bool bot = geo.walls && q.y == 0;
    const bool top = geo.walls && q.y == geo.ny - 1;
    auto L = [&](const char* row, int p, int dc) -> C {
      return S::sld(row + S::soff(g, p, W) + (c + dc) * S::es(g, p), g, p);
    };
    if (!bot && !top) {
      out[0] = L(q.mid, 0, 0);
      out[1] = L(q.mid, 1, -1);
      out[2] = L(q.lo, 2, 0);
      out[3] = L(q.mid, 3, 1);
      out[4] = L(q.hi, 4, 0);
      out[5] = L(q.lo, 5, -1);
      out[6] = L(q.lo, 6, 1);
      out[7] = L(q.hi, 7, 1);
      out[8] = L(q.hi, 8, -1);
      return;
    }
    C own[9];
    C s = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      own[i] = L(q.mid, i, 0);
      s += own[i];
    }
    if (!g) s += C(1);  // f values are deviations from w_i: rho = 1 + their sum
    out[0] = own[0];
    out[1] = L(q.mid, 1, -1);
    out[3] = L(q.mid, 3, 1);
    const C k6 = C(6) * s / C(36);
    if (bot) {
      out[2] = own[4];
      out[5] = own[7] + P::wall_term(k6 * ph.u_bottom, g);
      out[6] = own[8] - P::wall_term(k6 * ph.u_bottom, g);
      out[4] = L(q.hi, 4, 0);
      out[7] = L(q.hi, 7, 1);
      out[8] = L(q.hi, 8, -1);
    } else {
      out[4] = own[2];
      out[7] = own[5] - P::wall_term(k6 * ph.u_top, g);
      out[8] = own[6] + P::wall_term(k6 * ph.u_top, g);
      out[2] = L(q.lo, 2, 0);
      out[5] = L(q.lo, 5, -1);
      out[6] = L(q.lo, 6, 1);
    }
  };
  // phi of virtual row v for this thread's column (and the halo columns for tx == 0 / BX-1).
  auto phi_row = [&](int v, C gkeep[9]) {
    const int sl = (v - (y0 - 1)) % PHR;
    auto pull_col = [&](int c, C out[9]) {
      if constexpr (S::kHalf) pull_explicit(true, v, c, out);
      else pull_s(true, rows3(true, v, c * kEsC), out);
    };
    C gt[9];
    const C gh = ghost(v);
    if (colv) {
      pull_col(tx + H, gkeep);
      sphi[sl * PHW + tx + 1] = sum9(gkeep) + gh;
    }
    if (tx == 0) {
      pull_col(H - 1, gt);
      sphi[sl * PHW + 0] = sum9(gt) + gh;
    }
    if (tx == BX - 1) {
      pull_col(H + xv, gt);
      sphi[sl * PHW + xv + 1] = sum9(gt) + gh;
    }
  };
  // f of the node (column tx) at virtual row r.
  auto pull_f = [&](int r, C out[9]) {
    if constexpr (S::kHalf) pull_explicit(false, r, tx + H, out);
    else pull_s(false, rows3(false, r, (tx + H) * kEsC), out);
  };

  // Threads that write the output planes of a band back with bulk stores: (plane q, row j).
  const bool storer = tid < 18 * BY;
  const int st_q = tid % 18, st_j = tid / 18;

  // Prologue: stage the first rows, then phi of rows y0-1 .. y0+BY-1.
  issue_upto(gvb + R - 1, fvb + R - 1);
  for (int v = gvb; v <= min(y0 + BY, g_last); ++v) wait_row(true, v, kWaitProbes);
  C gcur[9], gnxt[9];
  {
    const int r = y0 + ty;
    if (r <= y1) phi_row(r, gcur);
    if (ty == 0) {
      C gt[9];
      phi_row(y0 - 1, gt);
    }
  }
  // The prologue rows and the first step's rows span 2BY+3 > R rows: refill once the prologue
  // has read its rows (everything below g row y0+BY-1 is free).
  __syncthreads();
  issue_upto(y0 + BY - 1 + R - 1, fvb + R - 1);

  for (int Y = y0; Y < y1; Y += BY) {
    // rows of this step: g [Y+BY-1, Y+2BY] for phi, f [Y-1, Y+BY] for the pulls
    for (int v = max(Y + BY + 1, gvb); v <= min(Y + 2 * BY, g_last); ++v) wait_row(true, v, wait_limit);
    for (int v = (Y == y0 ? fvb : Y + 1); v <= min(Y + BY, f_last); ++v) wait_row(false, v, wait_limit);
    const int rn = Y + BY + ty;
    if (rn <= y1) phi_row(rn, gnxt);
    const int r = Y + ty;
    const bool act = colv && r < y1;
    C f[9];
    if (act) pull_f(r, f);
    if (stuck) atomicExch(abort_flag, 1);
    if (storer) bulk_wait_read_all();  // last band's stores are done reading the staging buffer
    __syncthreads();
    if (*abort_flag) {
      if (tid == 0) atomicOr(flag, kFlagTimeout);
      // Let the copies already issued land before the CTA's shared memory is released.
      if (tid == 0) {
        for (int v = max(gvb, g_next - R); v < g_next; ++v) wait_row(true, v, kWaitProbes);
        for (int v = max(fvb, f_next - R); v < f_next; ++v) wait_row(false, v, kWaitProbes);
      }
      if (storer) bulk_wait_all();
      return;
    }
    // Everything staged below g row Y+2BY-1 and f row Y+BY-1 has been read: refill.
    issue_upto(Y + 2 * BY - 1 + R - 1, Y + BY - 1 + R - 1);
    if (act) {
      C s[3][3];
      const int sm = (r - 1 - (y0 - 1)) % PHR;
      const int s0 = sm + 1 == PHR ? 0 : sm + 1;
      const int sp = s0 + 1 == PHR ? 0 : s0 + 1;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        s[0][d] = sphi[sm * PHW + tx + d];
        s[1][d] = sphi[s0 * PHW + tx + d];
        s[2][d] = sphi[sp * PHW + tx + d];
      }
      C dxp, dyp, lap;
      stencils<C>(s, dxp, dyp, lap);
      const C phi = s[1][1];
      const C drho = collide<C>(ph, f, gcur, phi, dxp, dyp, lap);
      if (!(isfinite(drho) && isfinite(phi))) atomicOr(flag, kFlagNonfinite);
      S::store_node(obuf, NOUT, ty * BX + tx, f, gcur, drho, phi);
      fence_proxy_async_smem();
    }
    __syncthreads();
    if (storer) {
      const int rs = Y + st_j;
      if (rs < y1) {
        const int e = S::oes(st_q);
        const bool g = st_q >= 9;
        const int p = g ? st_q - 9 : st_q;
        bulk_s2g(dst + S::goff(g, p, geo.plane, (long long)rs * geo.pitch + x0),
                 obuf + S::ooff(st_q, NOUT) + st_j * BX * e, (uint32_t)(xv * e));
      }
      bulk_commit();
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) gcur[i] = gnxt[i];
  }
  if (storer) bulk_wait_all();
}

// -------------------------------------------------------------------------------------------
// Host side.

namespace {

template <int PREC> Phys<typename Pop<PREC>::C> phys_of(const HostPhys& h) {
  return make_phys<typename Pop<PREC>::C>(h);
}

template <int PREC, int BX, int BY, int D>
cudaError_t staged_launch(const HostGeometry& g, const HostPhys& p, int rows, const char* src, char* dst,
                          int* flag, cudaStream_t s) {
  const size_t smem = staged_smem_bytes<PREC, BX, BY, D>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_staged<PREC, BX, BY, D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  Geometry geo;
  geo.nx = g.nx;
  geo.ny = g.ny;
  geo.pitch = g.pitch;
  geo.plane = g.plane;
  geo.walls = g.walls;
  dim3 blk(BX, BY);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + rows - 1) / rows);
  const uint32_t limit = p.wait_probes < 0 ? kWaitProbes : (uint32_t)p.wait_probes;
  k_step_staged<PREC, BX, BY, D><<<grd, blk, smem, s>>>(src, dst, geo, phys_of<PREC>(p), rows, flag, limit);
  return cudaGetLastError();
}

template <int PREC, int BX, int BY, int D>
int staged_occupancy() {
  const size_t smem = staged_smem_bytes<PREC, BX, BY, D>();
  cudaFuncSetAttribute(k_step_staged<PREC, BX, BY, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_staged<PREC, BX, BY, D>, BX * BY, smem);
  return nb;
}

#define LBM_STAGED_TILES(X) X(32, 4, 1) X(32, 8, 1) X(64, 2, 1) X(64, 4, 1) X(64, 4, 2) X(128, 2, 1) X(128, 1, 2)

template <int PREC>
cudaError_t staged_prec(const HostGeometry& g, const HostPhys& p, const StepTile& t, const char* src,
                        char* dst, int* flag, cudaStream_t s) {
#define LBM_CASE(X, Y, Z) \
  if (t.bx == X && t.by == Y && t.depth == Z) return staged_launch<PREC, X, Y, Z>(g, p, t.rows, src, dst, flag, s);
  LBM_STAGED_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template <int PREC>
int staged_occ_prec(const StepTile& t) {
#define LBM_CASE(X, Y, Z) \
  if (t.bx == X && t.by == Y && t.depth == Z) return staged_occupancy<PREC, X, Y, Z>();
  LBM_STAGED_TILES(LBM_CASE)
#undef LBM_CASE
  return 0;
}

}  // namespace

int staged_halo(int prec) { return prec == 0 ? 2 : (prec == 1 ? 4 : 8); }

bool staged_supported(int prec, const HostGeometry& g, const StepTile& t) {
  if (g.nx % staged_halo(prec) != 0) return false;
#define LBM_CASE(X, Y, Z) \
  if (t.bx == X && t.by == Y && t.depth == Z) return true;
  LBM_STAGED_TILES(LBM_CASE)
#undef LBM_CASE
  return false;
}

int staged_blocks_per_sm(int prec, const StepTile& t) {
  switch (prec) {
    case 0: return staged_occ_prec<0>(t);
    case 1: return staged_occ_prec<1>(t);
    case 2: return staged_occ_prec<2>(t);
    case 3: return staged_occ_prec<3>(t);
  }
  return 0;
}

cudaError_t launch_step_staged(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                               const char* src, char* dst, int* flag, cudaStream_t s) {
  switch (prec) {
    case 0: return staged_prec<0>(g, p, t, src, dst, flag, s);
    case 1: return staged_prec<1>(g, p, t, src, dst, flag, s);
    case 2: return staged_prec<2>(g, p, t, src, dst, flag, s);
    case 3: return staged_prec<3>(g, p, t, src, dst, flag, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbmch
