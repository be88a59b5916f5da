// Fused step for 16-bit population storage with two neighbouring nodes per thread.
//
// The 16-bit step is bound by instruction issue, not by memory: a node moves only 80 bytes but
// costs as many address computations, loads, stores and loop steps as an FP32 node.  Here a
// thread owns the node pair (x, x+1), x even, so that
//   * a population the pair pulls from straight above or below (c_x = 0) is one aligned 32-bit
//     word holding both 16-bit values;
//   * a population arriving from the left (c_x = +1) is the high half of the word at x-2 and the
//     low half of the word at x (one byte permute), from the right (c_x = -1) the high half of
//     the word at x and the low half of the word at x+2;
//   * the rest populations f_0, g_0 (FP32) are one 64-bit load;
//   * the results of the two nodes are stored as 32-bit words (64-bit for the rest
//     populations), rounded two at a time;
// and every address is formed once for two nodes.  The two nodes' arithmetic runs in the packed
// FP32 instructions (lbm_f2.cuh): a 16-bit word of one direction decodes to the register pair
// (node x, node x+1), the collision and stencils are the one-node kernel's functions instantiated
// on that pair, and the encoded pair is again one word.  Decode, encode and closures round as
// the one-node kernel does; the collision may place its FMAs differently (see F2Prod).  With walls the kernel
// collides the interior rows only (it forms phi on the wall rows with the bounce-back pull) and
// k_step_edge, the one-node tile code, steps the two wall rows in a second launch.
// Requirements: nx even (pairs never straddle the periodic seam), population copy under 4 GiB.
#include "lbm_device.cuh"
#include "lbm_f2.cuh"
#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_step.cuh"

namespace lbmch {

namespace {

// Eqs. 4-5 in pull form for the pair (x, x+1) at row y of a periodic lattice: direction i comes
// from row y - c_yi and columns x - c_xi, x + 1 - c_xi.  xm2 / xp2 are the even columns x - 2 and
// x + 2 with periodic wrap; ym / yp the rows above and below with wrap.
template <int PREC, bool IS_G>
__device__ __forceinline__ void pull_pair(const char* __restrict__ src, Plane32 pl, int pitch, int x, int xm2,
                                          int xp2, int y, int ym, int yp, RawPairLoad& o) {
  using P = Pop<PREC>;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const unsigned p = IS_G ? 7 + i : i - 1;  // half plane of direction i
    const int row = lat_cy(i) == 1 ? ym : (lat_cy(i) == -1 ? yp : y);
    const unsigned rbase = (p * pl.n + (unsigned)(row * pitch)) * 2u;
    o.w[i - 1] = ld_word(src, rbase + 2u * (unsigned)x);
    if (lat_cx(i) == 1) o.e[side_index(i)] = ld_word(src, rbase + 2u * (unsigned)xm2);
    if (lat_cx(i) == -1) o.e[side_index(i)] = ld_word(src, rbase + 2u * (unsigned)xp2);
  }
  const unsigned rest = ((unsigned)(P::kRestFirst + (IS_G ? 1 : 0)) * pl.n + (unsigned)(y * pitch + x)) * 4u;
  const float2 r0 = __ldg(reinterpret_cast<const float2*>(src + rest));
  o.r0a = r0.x;
  o.r0b = r0.y;
}

// One tile: node pairs x0 + 2 tx (BX pairs, 2 BX columns, clipped to nx) and rows
// [y0, y0 + rows) (clipped to ny), by one CTA of BX x BY threads marching down BY rows at a time.
// Same software pipeline and phi ring as the one-node kernel (see step_tile).
template <int PREC, int BX, int BY, bool WALLS>
__device__ __forceinline__ void step_pair_tile(const char* __restrict__ src, char* __restrict__ dst,
                                               const Geometry& geo, const Phys<F2>& ph, const int x0,
                                               const int y0, const int rows, int* __restrict__ flag,
                                               float (*sphi)[2 * BX + 2], const Plane32 pl) {
  using P = Pop<PREC>;
  using R = typename P::R;
  constexpr int RING = 3 * BY + 1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = geo.nx, ny = geo.ny, pitch = geo.pitch;
  const float u_top = ph.u_top.v.x, u_bottom = ph.u_bottom.v.x;
  const int y1 = min(y0 + rows, ny);
  const int xv = min(2 * BX, nx - x0);  // valid columns of this strip (even)
  const int x = x0 + 2 * tx;
  const bool colv = 2 * tx < xv;
  const int xm2 = (x == 0) ? nx - 2 : x - 2;
  const int xp2 = (x + 2 >= nx) ? 0 : x + 2;
  // Halo phi, the nodes left and right of the strip.  With walls, threads tx == 0 and tx == BX-1
  // pull the halo node with the one-node code (bounce-back on the wall rows).  On periodic
  // lattices the pair's own loads serve: the node left of the strip (x0 - 1, thread 0) takes six
  // of its nine g values from words thread 0 loads anyway (c_x = +1: low halves of the words at
  // x - 2; c_x = -1: low halves of the words at x), the node right of it (thread of the last
  // pair) the high halves of its words at x and x + 2; the rest population and the two c_x = 0
  // directions are three extra loads.
  const bool halo = WALLS && (tx == 0 || tx == BX - 1);
  const bool hL = !WALLS && tx == 0;
  const bool hR = !WALLS && colv && 2 * tx + 2 == xv;
  const int hx = (tx == 0) ? ((x0 == 0) ? nx - 1 : x0 - 1) : ((x0 + xv == nx) ? 0 : x0 + xv);
  const int hcol = (tx == 0) ? 0 : xv + 1;

  auto wrap = [&](int r) -> int {  // periodic wrap; with walls, ghost rows map to the wall rows
    if constexpr (WALLS) return r < 0 ? 0 : (r >= ny ? ny - 1 : r);
    return r < 0 ? r + ny : (r >= ny ? r - ny : r);
  };
  auto slot = [&](int r) -> int { return (int)((unsigned)(r - (y0 - 1)) % (unsigned)RING); };
  auto pull_g2 = [&](int r, RawPairLoad& o) {
    const int y = wrap(r);
    pull_pair<PREC, true>(src, pl, pitch, x, xm2, xp2, y, y == 0 ? ny - 1 : y - 1, y == ny - 1 ? 0 : y + 1, o);
  };
  auto pull_f2 = [&](int r, RawPairLoad& o) {
    pull_pair<PREC, false>(src, pl, pitch, x, xm2, xp2, r, r == 0 ? ny - 1 : r - 1, r == ny - 1 ? 0 : r + 1, o);
  };
  // A row whose pulls cross a wall (walled lattices: y = 0 and y = ny - 1).  Ghost rows beyond a
  // wall (y = -1, ny) are read only by the wall rows' stencils, which this kernel does not use.
  auto wall_row = [&](int r) -> bool { return WALLS && (r == 0 || r == ny - 1); };
  auto pull_h = [&](int r, R out[9]) -> bool {
    return pull_raw<PREC, true, Plane32>(src, geo, u_top, u_bottom, hx, wrap(r), out, pl);
  };
  auto phi_h = [&](const R raw[9], bool dec) -> float {
    float v[9];
    unpack<PREC, true>(raw, dec, v);
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
  };
  auto put_phi = [&](int r, const RawPair& g) {
    float* row = sphi[slot(r)];
    if constexpr (WALLS) if (wall_row(r)) {  // bounce-back pull, node by node
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float v[9];
        pull<PREC, true, Plane32>(src, geo, u_top, u_bottom, x + k, r, v, pl);
        row[2 * tx + 1 + k] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
      }
      return;
    }
    const F2 p = phi_pair<PREC>(g);
    row[2 * tx + 1] = p.v.x;
    row[2 * tx + 2] = p.v.y;
  };
  bool hBd = false;

  RawPair gA, gB, fA;
  RawPairLoad gC, fB;  // in flight
  R hB[9];
  uint32_t eL0 = 0, eL2 = 0, eL4 = 0, eR0 = 0, eR2 = 0, eR4 = 0;  // the halo nodes' extra loads
  auto own_ld = [&](int r, int col, uint32_t& e0, uint32_t& e2, uint32_t& e4) {
    const int y = wrap(r);
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    e0 = __float_as_uint(__ldg(reinterpret_cast<const float*>(
        src + ((unsigned)(P::kRestFirst + 1) * pl.n + (unsigned)(y * pitch + col)) * 4u)));
    e2 = __ldg(reinterpret_cast<const unsigned short*>(src + (9u * pl.n + (unsigned)(ym * pitch + col)) * 2u));
    e4 = __ldg(reinterpret_cast<const unsigned short*>(src + (11u * pl.n + (unsigned)(yp * pitch + col)) * 2u));
  };
  auto own_put = [&](int r, const RawPairLoad& l, uint32_t e0, uint32_t e2, uint32_t e4, bool right) {
    float v[9];
    v[0] = __uint_as_float(e0);
    v[2] = P::h2f(e2);
    v[4] = P::h2f(e4);
    if (!right) {
      v[1] = P::h2f(l.e[side_index(1)]);
      v[5] = P::h2f(l.e[side_index(5)]);
      v[8] = P::h2f(l.e[side_index(8)]);
      v[3] = P::h2f(l.w[2]);
      v[6] = P::h2f(l.w[5]);
      v[7] = P::h2f(l.w[6]);
    } else {
      v[1] = P::h2f(l.w[0] >> 16);
      v[5] = P::h2f(l.w[4] >> 16);
      v[8] = P::h2f(l.w[7] >> 16);
      v[3] = P::h2f(l.e[side_index(3)] >> 16);
      v[6] = P::h2f(l.e[side_index(6)] >> 16);
      v[7] = P::h2f(l.e[side_index(7)] >> 16);
    }
    sphi[slot(r)][right ? xv + 1 : 0] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
  };
  auto own_now = [&](int r) {  // pipeline start: loads and sums at once, from the g words in gC
    if (hL) {
      own_ld(r, xm2 + 1, eL0, eL2, eL4);
      own_put(r, gC, eL0, eL2, eL4, false);
    }
    if (hR) {
      own_ld(r, xp2, eR0, eR2, eR4);
      own_put(r, gC, eR0, eR2, eR4, true);
    }
  };
  {
    const int r = y0 + ty;
    if (r <= y1) {
      if (colv) {
        pull_g2(r, gC);
        finish(gC, gA);
        put_phi(r, gA);
        own_now(r);
      }
      if (halo) {
        hBd = pull_h(r, hB);
        sphi[slot(r)][hcol] = phi_h(hB, hBd);
      }
    }
    if (ty == 0) {
      if (colv) {
        RawPair gt;
        pull_g2(y0 - 1, gC);
        finish(gC, gt);
        put_phi(y0 - 1, gt);
        own_now(y0 - 1);
      }
      if (halo) {
        R ht[9];
        const bool d = pull_h(y0 - 1, ht);
        sphi[slot(y0 - 1)][hcol] = phi_h(ht, d);
      }
    }
    const int rb = y0 + BY + ty;
    if (rb <= y1) {
      if (colv) {
        pull_g2(rb, gC);
        finish(gC, gB);
        own_now(rb);
      }
      if (halo) hBd = pull_h(rb, hB);
    }
    if (colv && r < y1) {
      pull_f2(r, fB);
      finish(fB, fA);
    }
  }

  for (int Y = y0; Y < y1; Y += BY) {
    const int r = Y + ty;            // collided now
    const int rb = Y + BY + ty;      // phi formed now
    const int rc = Y + 2 * BY + ty;  // g issued now
    const bool act = colv && r < y1 && !wall_row(r);
    if (rc <= y1 && colv) pull_g2(rc, gC);
    if (rc <= y1) {
      if (hL) own_ld(rc, xm2 + 1, eL0, eL2, eL4);
      if (hR) own_ld(rc, xp2, eR0, eR2, eR4);
    }
    if (rb < y1 && colv) pull_f2(rb, fB);
    if (rb <= y1) {
      if (colv) put_phi(rb, gB);
      if (halo) sphi[slot(rb)][hcol] = phi_h(hB, hBd);
    }
    if (rc <= y1 && halo) hBd = pull_h(rc, hB);
    __syncthreads();
    if (act) {
      // phi of columns x-1 .. x+2 on rows r-1, r, r+1, two aligned float2 per row; stencil
      // entry s[dy+1][dx+1] holds (node x, node x+1).
      const int rs[3] = {slot(r - 1), slot(r), slot(r + 1)};
      F2 s[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float2 lo = *reinterpret_cast<const float2*>(&sphi[rs[d]][2 * tx]);
        const float2 hi = *reinterpret_cast<const float2*>(&sphi[rs[d]][2 * tx + 2]);
        s[d][0] = F2(lo);
        s[d][1] = F2(lo.y, hi.x);
        s[d][2] = F2(hi);
      }
      F2 dxp, dyp, lap;
      stencils<F2>(s, dxp, dyp, lap);
      const F2 phi = s[1][1];
      F2 f[9], g[9];
      unpack_pair<PREC>(fA, f);
      unpack_pair<PREC>(gA, g);
      const F2 drho = collide<F2>(ph, f, g, phi, dxp, dyp, lap);
      if (!(isfinite(drho.v.x) && isfinite(drho.v.y) && isfinite(phi.v.x) && isfinite(phi.v.y))) atomicOr(flag, kFlagNonfinite);
      store_pair<PREC>(dst, pl, (unsigned)(r * pitch + x), f, g, drho, phi, ph.sr_key);
    }
    gA = gB;
    finish(gC, gB);  // the loads issued at the top of this band have had the band to arrive
    if (rc <= y1) {  // the halo phi of row rc, into a ring slot no stencil reads this band
      if (hL) own_put(rc, gC, eL0, eL2, eL4, false);
      if (hR) own_put(rc, gC, eR0, eR2, eR4, true);
    }
    finish(fB, fA);
  }
}

// Residency target: 3 CTAs of 128 threads per SM (12 warps); the walled variant, which also pulls
// the wall rows' bounce-back populations, 2 (it spills at the 3-CTA register cap).  WALLS:
// compiled separately so that the periodic kernel carries no wall code.
template <int PREC, int BX, int BY, bool WALLS>
__global__ void __launch_bounds__(BX * BY, WALLS ? 2 : 3)
k_step_pair(const char* __restrict__ src, char* __restrict__ dst, const Geometry geo, const Phys<F2> ph,
            const int rows, int* __restrict__ flag) {
  __shared__ __align__(16) float sphi[3 * BY + 1][2 * BX + 2];
  step_pair_tile<PREC, BX, BY, WALLS>(src, dst, geo, ph, blockIdx.x * 2 * BX, blockIdx.y * rows, rows, flag, sphi,
                               Plane32{(unsigned)geo.plane});
}

// Batched paired step: a persistent grid deals out a work list of 256-column tiles drawn from
// many periodic 16-bit lattices (lbm_batch.cu), each stepped by the tile code above with its
// member's geometry and physics, so a member's state is the one k_step_pair<PREC, 128, 1> gives
// the single lattice.  The step counter and the stochastic-rounding key follow k_step_batch.
__device__ __forceinline__ Phys<F2> widen(const Phys<float>& p) {
  Phys<F2> q;
  q.omega_l = F2(p.omega_l);
  q.omega_g = F2(p.omega_g);
  q.tau_l = F2(p.tau_l);
  q.tau_g = F2(p.tau_g);
  q.omega3 = F2(p.omega3);
  q.omega_phi = F2(p.omega_phi);
  q.gamma = F2(p.gamma);
  q.a = F2(p.a);
  q.Gamma = F2(p.Gamma);
  q.u_top = F2(p.u_top);
  q.u_bottom = F2(p.u_bottom);
  q.wet_bottom = F2(p.wet_bottom);
  q.wet_top = F2(p.wet_top);
  q.force_x = F2(p.force_x);
  q.force_y = F2(p.force_y);
  q.visc = p.visc;
  q.k8_printed = p.k8_printed;
  q.bgk = p.bgk;
  q.force_mode = p.force_mode;
  q.forced = p.forced;
  q.sr_key = p.sr_key;
  q.rounding = p.rounding;
  q.seed = p.seed;
  return q;
}

template <int PREC>
__global__ void __launch_bounds__(128, 3)
k_step_pair_batch(const BatchItem* __restrict__ items, const int nitems, const BatchMember* __restrict__ members,
                  const Phys<float>* __restrict__ phys, const int parity, int* __restrict__ flags,
                  long long* __restrict__ tcount) {
  __shared__ __align__(16) float sphi[4][2 * 128 + 2];
  const long long t = tcount[parity];
  if (blockIdx.x == 0 && threadIdx.x == 0) tcount[1 - parity] = t + 1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem w = items[it];
    const BatchMember m = members[w.member];
    Phys<F2> ph = widen(phys[w.member]);
    if (ph.rounding) ph.sr_key = sr_step_key(ph.seed, t);  // the key a single lattice uses at step t
    Geometry geo;
    geo.nx = m.nx;
    geo.ny = m.ny;
    geo.pitch = m.pitch;
    geo.plane = m.plane;
    geo.walls = m.walls;
    step_pair_tile<PREC, 128, 1, false>(parity ? m.buf1 : m.buf0, parity ? m.buf0 : m.buf1, geo, ph, w.x0, w.y0,
                                        w.rows, flags + w.member, sphi, Plane32{(unsigned)geo.plane});
    __syncthreads();  // the phi ring is reused by the next item
  }
}

// Compiled tiles: 128-thread CTAs (3 per SM); 256-thread shapes spill at the register cap of
// 2 CTAs per SM and were 1.5x slower.
#define LBM_PAIR_TILES(X) X(64, 2) X(128, 1)

template <int PREC, int BX, int BY>
cudaError_t pair_bxby(const HostGeometry& g, const HostPhys& p, int rows, const char* src, char* dst, int* flag,
                      cudaStream_t s) {
  dim3 grd((g.nx + 2 * BX - 1) / (2 * BX), (g.ny + rows - 1) / rows);
  const Geometry geo = to_geo(g);
  const Phys<F2> ph2 = make_phys<F2>(p);
  if (!g.walls) {
    k_step_pair<PREC, BX, BY, false><<<grd, dim3(BX, BY), 0, s>>>(src, dst, geo, ph2, rows, flag);
  } else {
    k_step_pair<PREC, BX, BY, true><<<grd, dim3(BX, BY), 0, s>>>(src, dst, geo, ph2, rows, flag);
    const Phys<float> ph = make_phys<float>(p);
    // the two wall rows: one-node tile code, one row each
    constexpr int EX = 256;
    k_step_edge<PREC, EX><<<dim3((g.nx + EX - 1) / EX, 2), EX, 0, s>>>(src, dst, geo, ph, flag);
  }
  return cudaGetLastError();
}

template <int PREC>
cudaError_t pair_prec(const HostGeometry& g, const HostPhys& p, const StepTile& t, const char* src, char* dst,
                      int* flag, cudaStream_t s) {
#define LBM_CASE(X, Y) \
  if (t.bx == X && t.by == Y) return pair_bxby<PREC, X, Y>(g, p, t.rows, src, dst, flag, s);
  LBM_PAIR_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template <int PREC>
int pair_occ(int bx, int by, bool walls) {
  int nb = 0;
#define LBM_CASE(X, Y)                                                                                         \
  if (bx == X && by == Y)                                                                                      \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                                             \
        &nb, walls ? k_step_pair<PREC, X, Y, true> : k_step_pair<PREC, X, Y, false>, X * Y, 0);
  LBM_PAIR_TILES(LBM_CASE)
#undef LBM_CASE
  return nb;
}

}  // namespace

cudaError_t launch_step_pair_batch(int prec, const BatchItem* items, int nitems, const BatchMember* members,
                                  const void* phys, int parity, int* flags, long long* tcount, int grid,
                                  cudaStream_t s) {
  const Phys<float>* ph = static_cast<const Phys<float>*>(phys);
  if (prec == 2) k_step_pair_batch<2><<<grid, 128, 0, s>>>(items, nitems, members, ph, parity, flags, tcount);
  else if (prec == 3) k_step_pair_batch<3><<<grid, 128, 0, s>>>(items, nitems, members, ph, parity, flags, tcount);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int pair_batch_blocks_per_sm(int prec) {
  int nb = 0;
  if (prec == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_pair_batch<2>, 128, 0);
  if (prec == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_pair_batch<3>, 128, 0);
  return nb > 0 ? nb : 1;
}

bool pair_supported(int prec, const HostGeometry& g, int bx, int by) {
  if ((prec != 2 && prec != 3) || g.nx % 2 || !offsets_fit_32(prec, g.plane)) return false;
#define LBM_CASE(X, Y) \
  if (bx == X && by == Y) return true;
  LBM_PAIR_TILES(LBM_CASE)
#undef LBM_CASE
  return false;
}

int pair_blocks_per_sm(int prec, const StepTile& t, bool walls) {
  return prec == 2 ? pair_occ<2>(t.bx, t.by, walls) : (prec == 3 ? pair_occ<3>(t.bx, t.by, walls) : 0);
}

cudaError_t launch_step_pair(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t, const char* src,
                             char* dst, int* flag, cudaStream_t s) {
  if (prec == 2) return pair_prec<2>(g, p, t, src, dst, flag, s);
  if (prec == 3) return pair_prec<3>(g, p, t, src, dst, flag, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbmch
