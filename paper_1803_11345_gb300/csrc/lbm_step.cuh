// The fused step kernel and the batched variant as templates, shared by the translation units
// that instantiate them: lbm_kernels.cu (population buffers under 4 GiB, 32-bit plane offsets)
// and lbm_step64.cu (larger buffers, 64-bit offsets), compiled in parallel.
//
// k_step is the whole time step in one launch: every CTA owns a strip of BX columns and
// `rows` lattice rows and marches down it BY rows at a time.  For each block of rows it
//   (1) pulls g (Eq. 5) for the NEXT block of rows, sums phi = sum g and stores phi in a
//       shared-memory ring of rows that also holds one halo column on each side;
//   (2) pulls f (Eq. 4) for the current rows;
//   (3) after one __syncthreads, reads the 3x3 phi neighbourhood from the ring for the Eq. 12
//       stencils and runs both collisions on the g values it pulled one iteration earlier;
//   (4) writes f*, g* to the other population buffer.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbmch {

// Compiled tile shapes.
#define LBM_TILES(X) X(32, 4) X(32, 8) X(64, 2) X(64, 4) X(128, 1) X(128, 2) X(256, 1)

inline Geometry to_geo(const HostGeometry& h) {
  Geometry g;
  g.nx = h.nx;
  g.ny = h.ny;
  g.pitch = h.pitch;
  g.plane = h.plane;
  g.walls = h.walls;
  return g;
}

// -------------------------------------------------------------------------------------------
// Fused step.

// One tile of the step: columns [x0, x0+BX) (clipped to nx) and rows [y0, y0+rows) (clipped to
// ny) of one lattice, by one CTA of BX x BY threads.  sphi is the CTA's phi ring.
template <int PREC, int BX, int BY, class PL>
__device__ __forceinline__ void step_tile(const char* __restrict__ src, char* __restrict__ dst,
                                          const Geometry& geo, const Phys<typename Pop<PREC>::C>& ph,
                                          const int x0, const int y0, const int rows, int* __restrict__ flag,
                                          typename Pop<PREC>::C (*sphi)[BX + 2], const PL pl) {
  using P = Pop<PREC>;
  using C = typename P::C;
  constexpr int RING = 3 * BY + 1;  // rows kept: see the ring argument below

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int y1 = min(y0 + rows, geo.ny);
  const int xv = min(BX, geo.nx - x0);  // valid columns of this strip
  const int x = x0 + tx;
  const bool colv = tx < xv;
  // Threads tx == 0 and tx == BX-1 also own the left / right halo column of the strip.
  const bool halo = tx == 0 || tx == BX - 1;
  const int hx = (tx == 0) ? ((x0 == 0) ? geo.nx - 1 : x0 - 1) : ((x0 + xv == geo.nx) ? 0 : x0 + xv);
  const int hcol = (tx == 0) ? 0 : xv + 1;

  // Virtual row r in [y0 - 1, y1] -> physical row (periodic wrap, or with walls the adjacent
  // row, whose phi plus the wall gradient is the ghost value: phi(x, -1) = phi(x, 0) +
  // wet_bottom, phi(x, ny) = phi(x, ny - 1) + wet_top; both gradients are 0 when periodic).
  auto phys_row = [&](int r) -> int {
    if (r < 0) return geo.walls ? 0 : r + geo.ny;
    if (r >= geo.ny) return geo.walls ? geo.ny - 1 : r - geo.ny;
    return r;
  };
  auto ghost = [&](int r) -> C {
    if (!geo.walls) return C(0);
    return r < 0 ? ph.wet_bottom : (r >= geo.ny ? ph.wet_top : C(0));
  };
  auto slot = [&](int r) -> int { return (int)((unsigned)(r - (y0 - 1)) % (unsigned)RING); };  // r >= y0 - 1
  auto sum9 = [](const C v[9]) -> C {
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
  };
  using R = typename P::R;
  auto pull_g = [&](int xx, int r, R out[9]) -> bool {
    return pull_raw<PREC, true, PL>(src, geo, ph.u_top, ph.u_bottom, xx, phys_row(r), out, pl);
  };
  auto pull_f = [&](int r, R out[9]) -> bool {
    return pull_raw<PREC, false, PL>(src, geo, ph.u_top, ph.u_bottom, x, r, out, pl);
  };
  auto phi_of = [&](const R raw[9], bool dec) -> C {
    C v[9];
    unpack<PREC, true>(raw, dec, v);
    return sum9(v);
  };

  // Software pipeline: at the band of rows Y .. Y+BY-1 a thread (row Y+ty) holds
  //   gA: g pulled for its row Y+ty (collided now), loaded two bands ago;
  //   gB: g pulled for row Y+BY+ty (its phi is formed now), loaded one band ago;
  //   gC: g for row Y+2BY+ty, issued now;
  //   fA: f pulled for row Y+ty, loaded one band ago;  fB: f for row Y+BY+ty, issued now;
  //   hB: g of its halo node (if any) for row Y+BY+ty, loaded one band ago, then reissued
  //       for row Y+2BY+ty.
  // The registers hold the stored bits; values are decoded only where used, so every load has a
  // whole band of work to arrive.  The *d flags mark wall rows, which are pulled decoded.
  R gA[9], gB[9], gC[9], fA[9], fB[9], hB[9];
  bool gAd = false, gBd = false, gCd = false, fAd = false, fBd = false, hBd = false;
  {
    // Prologue: phi of rows y0-1 (halo, thread row 0) and y0+ty, loaded and used at once.
    const int r = y0 + ty;
    if (r <= y1) {
      if (colv) {
        gAd = pull_g(x, r, gA);
        sphi[slot(r)][tx + 1] = phi_of(gA, gAd) + ghost(r);
      }
      if (halo) {
        hBd = pull_g(hx, r, hB);
        sphi[slot(r)][hcol] = phi_of(hB, hBd) + ghost(r);
      }
    }
    if (ty == 0) {
      R gt[9];
      if (colv) {
        const bool d = pull_g(x, y0 - 1, gt);
        sphi[slot(y0 - 1)][tx + 1] = phi_of(gt, d) + ghost(y0 - 1);
      }
      if (halo) {
        const bool d = pull_g(hx, y0 - 1, gt);
        sphi[slot(y0 - 1)][hcol] = phi_of(gt, d) + ghost(y0 - 1);
      }
    }
    const int rb = y0 + BY + ty;
    if (rb <= y1) {
      if (colv) gBd = pull_g(x, rb, gB);
      if (halo) hBd = pull_g(hx, rb, hB);
    }
    if (colv && r < y1) fAd = pull_f(r, fA);
  }

  // Ring argument: iteration j writes rows [Y+BY, Y+2BY) and reads rows [Y-1, Y+BY]; iteration
  // j-1 read [Y-BY-1, Y].  A thread may still be reading iteration j-1's rows while another
  // writes iteration j's, so those two ranges (3BY+1 rows) must map to distinct slots: RING =
  // 3BY+1.  Iteration j+1's writes cannot meet iteration j-1's reads (one barrier apart).
  for (int Y = y0; Y < y1; Y += BY) {
    const int r = Y + ty;            // collided now
    const int rb = Y + BY + ty;      // phi formed now
    const int rc = Y + 2 * BY + ty;  // g issued now
    const bool act = colv && r < y1;
    if (rc <= y1 && colv) gCd = pull_g(x, rc, gC);
    if (rb < y1 && colv) fBd = pull_f(rb, fB);
    if (rb <= y1) {
      if (colv) sphi[slot(rb)][tx + 1] = phi_of(gB, gBd) + ghost(rb);
      if (halo) sphi[slot(rb)][hcol] = phi_of(hB, hBd) + ghost(rb);
    }
    if (rc <= y1 && halo) hBd = pull_g(hx, rc, hB);
    __syncthreads();
    if (act) {
      C s[3][3];
      const int sm = slot(r - 1), s0 = slot(r), sp = slot(r + 1);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        s[0][d] = sphi[sm][tx + d];
        s[1][d] = sphi[s0][tx + d];
        s[2][d] = sphi[sp][tx + d];
      }
      C dxp, dyp, lap;
      stencils<C>(s, dxp, dyp, lap);
      const C phi = s[1][1];
      C f[9], g[9];
      unpack<PREC, false>(fA, fAd, f);
      unpack<PREC, true>(gA, gAd, g);
      const C drho = collide<C>(ph, f, g, phi, dxp, dyp, lap);
      if (!(isfinite(drho) && isfinite(phi))) atomicOr(flag, kFlagNonfinite);
      P::store_node(dst, pl, r * geo.pitch + x, f, g, drho, phi, ph.sr_key);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      gA[i] = gB[i];
      gB[i] = gC[i];
      fA[i] = fB[i];
    }
    gAd = gBd;
    gBd = gCd;
    fAd = fBd;
  }
}

// OFF32: the population buffer is under 4 GiB, so plane offsets are formed in 32 bits.
template <int PREC, int BX, int BY, bool OFF32>
__global__ void __launch_bounds__(BX * BY)
k_step(const char* __restrict__ src, char* __restrict__ dst, const Geometry geo,
       const Phys<typename Pop<PREC>::C> ph, const int rows, int* __restrict__ flag) {
  using C = typename Pop<PREC>::C;
  __shared__ C sphi[3 * BY + 1][BX + 2];
  if constexpr (OFF32)
    step_tile<PREC, BX, BY>(src, dst, geo, ph, blockIdx.x * BX, blockIdx.y * rows, rows, flag, sphi,
                            Plane32{(unsigned)geo.plane});
  else
    step_tile<PREC, BX, BY>(src, dst, geo, ph, blockIdx.x * BX, blockIdx.y * rows, rows, flag, sphi, geo.plane);
}

// The two wall rows (y = 0 and y = ny - 1) of a walled lattice, one row each for blockIdx.y = 0
// and 1: the rows another kernel (the paired 16-bit step) leaves out.
template <int PREC, int BX>
__global__ void __launch_bounds__(BX)
k_step_edge(const char* __restrict__ src, char* __restrict__ dst, const Geometry geo,
            const Phys<typename Pop<PREC>::C> ph, int* __restrict__ flag) {
  using C = typename Pop<PREC>::C;
  __shared__ C sphi[4][BX + 2];
  step_tile<PREC, BX, 1>(src, dst, geo, ph, blockIdx.x * BX, blockIdx.y ? geo.ny - 1 : 0, 1, flag, sphi,
                         Plane32{(unsigned)geo.plane});
}

// -------------------------------------------------------------------------------------------
// Batched step: a persistent grid walks a list of tiles drawn from many independent lattices.

template <int PREC, int BX, int BY, bool OFF32>
__global__ void __launch_bounds__(BX * BY)
k_step_batch(const BatchItem* __restrict__ items, const int nitems, const BatchMember* __restrict__ members,
             const Phys<typename Pop<PREC>::C>* __restrict__ phys, const int parity, int* __restrict__ flags,
             long long* __restrict__ tcount) {
  using C = typename Pop<PREC>::C;
  __shared__ C sphi[3 * BY + 1][BX + 2];
  // The batch's time step: read from the slot of this parity; the successor goes to the other
  // slot, which only the next launch reads (a captured graph replays these launches unchanged).
  const long long t = tcount[parity];
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) tcount[1 - parity] = t + 1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem w = items[it];
    const BatchMember m = members[w.member];
    Phys<C> ph = phys[w.member];
    if (ph.rounding) ph.sr_key = sr_step_key(ph.seed, t);  // the key a single lattice uses at step t
    Geometry geo;
    geo.nx = m.nx;
    geo.ny = m.ny;
    geo.pitch = m.pitch;
    geo.plane = m.plane;
    geo.walls = m.walls;
    const char* src = parity ? m.buf1 : m.buf0;
    char* dst = parity ? m.buf0 : m.buf1;
    if constexpr (OFF32)
      step_tile<PREC, BX, BY>(src, dst, geo, ph, w.x0, w.y0, w.rows, flags + w.member, sphi,
                              Plane32{(unsigned)geo.plane});
    else
      step_tile<PREC, BX, BY>(src, dst, geo, ph, w.x0, w.y0, w.rows, flags + w.member, sphi, geo.plane);
    __syncthreads();  // the phi ring is reused by the next item
  }
}


template <int PREC, int BX, int BY, bool OFF32>
cudaError_t launch_k_step(const HostGeometry& g, const HostPhys& p, int rows, const char* src, char* dst,
                          int* flag, cudaStream_t s) {
  using C = typename Pop<PREC>::C;
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + rows - 1) / rows);
  k_step<PREC, BX, BY, OFF32><<<grd, dim3(BX, BY), 0, s>>>(src, dst, to_geo(g), make_phys<C>(p), rows, flag);
  return cudaGetLastError();
}

template <int PREC, int BX, int BY, bool OFF32>
cudaError_t launch_k_step_batch(const BatchItem* items, int nitems, const BatchMember* members, const void* phys,
                                int parity, int* flags, long long* tcount, int grid, cudaStream_t s) {
  using C = typename Pop<PREC>::C;
  k_step_batch<PREC, BX, BY, OFF32><<<grid, dim3(BX, BY), 0, s>>>(items, nitems, members,
                                                                   static_cast<const Phys<C>*>(phys), parity, flags,
                                                                   tcount);
  return cudaGetLastError();
}

// The 64-bit-offset instantiations (lbm_step64.cu): one tile shape (BX, BY) of LBM_TILES.
cudaError_t launch_step64(int prec, int bx, int by, const HostGeometry& g, const HostPhys& p, int rows,
                          const char* src, char* dst, int* flag, cudaStream_t s);
cudaError_t launch_step_batch64(int prec, int bx, int by, const BatchItem* items, int nitems,
                                const BatchMember* members, const void* phys, int parity, int* flags,
                                long long* tcount, int grid, cudaStream_t s);

}  // namespace lbmch
