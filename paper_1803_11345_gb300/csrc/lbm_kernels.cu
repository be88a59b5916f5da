// Kernels of the hybrid central-moment / BGK lattice Boltzmann scheme for the coupled
// Cahn-Hilliard--Navier-Stokes equations (arXiv:1803.11345), for sm_103a: the host launchers of
// the fused step (kernel templates in lbm_step.cuh; this file instantiates the 32-bit-offset
// variants), initialisation, fields, FP64 reductions and checkpoint planes.
// Populations live in two buffers (A -> B, then B -> A); the state between launches is the
// post-collision populations.
#include <algorithm>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbmch {

namespace {

template <class C> Phys<C> to_phys(const HostPhys& h) { return make_phys<C>(h); }


}  // namespace

// -------------------------------------------------------------------------------------------
// Initial state: populations = equilibria of Eqs. 8-10 built from the initial fields, then one
// collision at t = 0.  fields = [phi | ux | uy | rho], each nx*ny FP64, dense rows.

template <int PREC>
__global__ void k_init(const double* __restrict__ fields, char* __restrict__ dst, const Geometry geo,
                       const Phys<typename Pop<PREC>::C> ph) {
  using P = Pop<PREC>;
  using C = typename P::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const long long N = (long long)geo.nx * geo.ny;
  const double* phi0 = fields;
  const double* ux0 = fields + N;
  const double* uy0 = fields + 2 * N;
  const double* rho0 = fields + 3 * N;
  C s[3][3];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      int xx = x + dx;
      xx = xx < 0 ? xx + geo.nx : (xx >= geo.nx ? xx - geo.nx : xx);
      int yy = y + dy;
      C ghost = C(0);  // wall gradient added to the ghost rows (Eq. 18)
      if (geo.walls) {
        ghost = yy < 0 ? ph.wet_bottom : (yy >= geo.ny ? ph.wet_top : C(0));
        yy = yy < 0 ? 0 : (yy >= geo.ny ? geo.ny - 1 : yy);
      } else {
        yy = yy < 0 ? yy + geo.ny : (yy >= geo.ny ? yy - geo.ny : yy);
      }
      s[dy + 1][dx + 1] = (C)phi0[(long long)yy * geo.nx + xx] + ghost;
    }
  C gx, gy, lap;
  stencils<C>(s, gx, gy, lap);
  const long long n = (long long)y * geo.nx + x;
  // f is formed as deviations f_i - w_i (the form the collision and the storage take): with
  // 3 p~ = 1 + 3 Pt, f_eq,i - w_i = w_i (3 Pt + rho poly_i) + the Eq. 11 gradient terms.
  const C phi = s[1][1], ux = (C)ux0[n], uy = (C)uy0[n];
  const C drho = (C)(rho0[n] - 1.0), rho = C(1) + drho;
  const C cs2 = C(1) / C(3);
  const C phi2 = phi * phi;
  const C mu = ph.a * (phi2 * phi - phi) - ph.gamma * lap;
  const C Pt = drho * cs2 + (ph.a * phi2 * (C(0.75) * phi2 - C(0.5)) - ph.gamma * phi * lap);
  const C uu = ux * ux + uy * uy;
  C f[9], g[9];
  C sf = C(0), sg = C(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const C w = C(lat_w36(i)) / C(36);
    const C cu = C(lat_cx(i)) * ux + C(lat_cy(i)) * uy;
    const C poly = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
    C wxx, wyy, wxy;
    if (i <= 4) {
      const bool xl = lat_cx(i) != 0;
      wxx = xl ? C(1) / C(3) : -C(1) / C(6);
      wyy = xl ? -C(1) / C(6) : C(1) / C(3);
      wxy = C(0);
    } else {
      wxx = -C(1) / C(24);
      wyy = -C(1) / C(24);
      wxy = C(0.25) * C(lat_cx(i) * lat_cy(i));
    }
    f[i] = w * (C(3) * Pt + rho * poly) + ph.gamma * (wxx * gx * gx + wyy * gy * gy + wxy * gx * gy);
    g[i] = w * (ph.Gamma * mu + phi * poly);
    sf += f[i];
    sg += g[i];
  }
  f[0] = drho - sf;
  g[0] = phi - sg;
  const C drho_c = collide<C>(ph, f, g, phi, gx, gy, lap);
  // rho - 1 and phi of the initial state on the storage's grids (16-bit storage; see PopHalf):
  // the closures then give stored values whose sums every later step keeps exactly.
  P::store_node(dst, geo.plane, y * geo.pitch + x, f, g, P::grid_f(drho_c), P::grid_g(phi));
}

// -------------------------------------------------------------------------------------------
// Macroscopic fields of the stored state: out = [rho | ux | uy | phi], dense FP64.  The stored
// populations are post-collision, so sum f c = rho u + F/2 with u the velocity of that collision;
// u = (sum f c - F/2)/rho is reported (F = force_x, force_y, weighted by (1 + phi)/2 in mode 1).

template <int PREC>
__global__ void k_fields(const char* __restrict__ src, const Geometry geo, const double fx, const double fy,
                         const int fmode, double* __restrict__ out) {
  using P = Pop<PREC>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const int idx = y * geo.pitch + x;
  double drho = 0, jx = 0, jy = 0, phi = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double di = (double)P::ldf(src, geo.plane, i, idx);  // f_i - w_i
    drho += di;
    jx += di * lat_cx(i);
    jy += di * lat_cy(i);
    phi += (double)P::ldg(src, geo.plane, i, idx);
  }
  const double rho = 1.0 + drho;
  const long long N = (long long)geo.nx * geo.ny;
  const long long n = (long long)y * geo.nx + x;
  const double wf = fmode ? 0.5 * (1.0 + phi) : 1.0;
  out[n] = rho;
  out[N + n] = (jx - 0.5 * fx * wf) / rho;
  out[2 * N + n] = (jy - 0.5 * fy * wf) / rho;
  out[3 * N + n] = phi;
}

// -------------------------------------------------------------------------------------------
// Deterministic FP64 reduction: fixed grid, fixed per-thread order, fixed tree.

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

template <int PREC>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_partials(const char* __restrict__ src, const Geometry geo, double* __restrict__ partials) {
  using P = Pop<PREC>;
  __shared__ double sh[4][kRedThreads];
  double acc[4] = {0, 0, 0, 0};
  const long long N = (long long)geo.nx * geo.ny;
  for (long long n = (long long)blockIdx.x * kRedThreads + threadIdx.x; n < N;
       n += (long long)gridDim.x * kRedThreads) {
    const int y = (int)(n / geo.nx), x = (int)(n - (long long)y * geo.nx);
    const int idx = y * geo.pitch + x;
    double drho = 0, jx = 0, jy = 0, phi = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double di = (double)P::ldf(src, geo.plane, i, idx);  // f_i - w_i
      drho += di;
      jx += di * lat_cx(i);
      jy += di * lat_cy(i);
      phi += (double)P::ldg(src, geo.plane, i, idx);
    }
    acc[0] += phi;
    acc[1] += 1.0 + drho;
    acc[2] += jx;
    acc[3] += jy;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads)
k_reduce_final(const double* __restrict__ partials, int nparts, double* __restrict__ out4) {
  __shared__ double sh[4][kRedThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nparts; b += kRedThreads)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += partials[b * 4 + q];
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out4[threadIdx.x] = sh[threadIdx.x][0];
}

// -------------------------------------------------------------------------------------------
// One population plane between the state and a dense FP64 array.

template <int PREC>
__global__ void k_plane_get(const char* __restrict__ src, const Geometry geo, int p, double* __restrict__ out) {
  using P = Pop<PREC>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const int idx = y * geo.pitch + x;
  const double v = p < 9 ? P::ldf_full(src, geo.plane, p, idx) : (double)P::ldg(src, geo.plane, p - 9, idx);
  out[(long long)y * geo.nx + x] = v;
}

template <int PREC>
__global__ void k_plane_set(char* __restrict__ dst, const Geometry geo, int p, const double* __restrict__ in) {
  using P = Pop<PREC>;
  using C = typename P::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const int idx = y * geo.pitch + x;
  const double v = in[(long long)y * geo.nx + x];
  if (p < 9) P::stf_full(dst, geo.plane, p, idx, v);
  else P::stg(dst, geo.plane, p - 9, idx, (C)v);
}

// -------------------------------------------------------------------------------------------
// Host launchers.

bool offsets_fit_32(int prec, long long plane) { return pop_buffer_bytes(prec, plane) < (size_t(1) << 32); }

size_t pop_buffer_bytes(int prec, long long plane) {
  switch (prec) {
    case 0: return (size_t)plane * Pop<0>::kBytesPerElem;
    case 1: return (size_t)plane * Pop<1>::kBytesPerElem;
    case 2: return (size_t)plane * Pop<2>::kBytesPerElem;
    case 3: return (size_t)plane * Pop<3>::kBytesPerElem;
  }
  return 0;
}

namespace {

dim3 node_grid(const HostGeometry& g, dim3 blk) {
  return dim3((g.nx + blk.x - 1) / blk.x, (g.ny + blk.y - 1) / blk.y);
}


template <int PREC, int BX, int BY>
cudaError_t step_bxby(const HostGeometry& g, const HostPhys& p, int rows, bool wide, const char* src, char* dst,
                      int* flag, cudaStream_t s) {
  if (!wide && offsets_fit_32(PREC, g.plane)) return launch_k_step<PREC, BX, BY, true>(g, p, rows, src, dst, flag, s);
  return launch_step64(PREC, BX, BY, g, p, rows, src, dst, flag, s);
}

template <int PREC>
cudaError_t step_prec(const HostGeometry& g, const HostPhys& p, const StepTile& t, const char* src,
                      char* dst, int* flag, cudaStream_t s) {
#define LBM_CASE(X, Y) \
  if (t.bx == X && t.by == Y) return step_bxby<PREC, X, Y>(g, p, t.rows, t.wide != 0, src, dst, flag, s);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template <int PREC>
int occupancy(int bx, int by) {
  int nb = 0;
#define LBM_CASE(X, Y) \
  if (bx == X && by == Y) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<PREC, X, Y, true>, X * Y, 0);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return nb;
}

}  // namespace

bool tile_supported(int prec, int bx, int by) {
  (void)prec;
#define LBM_CASE(X, Y) \
  if (bx == X && by == Y) return true;
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return false;
}

StepTile default_tile(int prec, const HostGeometry& g, int device) {
  // Measured on GB300: FP32 / FP64, the software-pipelined generic kernel with one row of 256
  // threads per CTA; 16-bit storage on lattices of 4 M nodes or more, the paired kernel with
  // 128 x 1 threads (256 columns) where the lattice allows it (1.3x the generic kernel at 4096^2;
  // on small lattices each CTA gets few rows and the pipeline start-up dominates: at 1024 x 512
  // the generic kernel is faster).  Grids sized to one wave.
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (sms <= 0) sms = 152;
  StepTile t;
  t.staged = 0;
  t.depth = 1;
  if (pair_supported(prec, g, 128, 1) && (long long)g.nx * g.ny >= (1ll << 22)) {
    t.bx = 128;
    t.by = 1;
    t.pair = 1;
    t.rows = default_rows(g, t, sms * std::max(1, pair_blocks_per_sm(prec, t, g.walls != 0)));
    return t;
  }
  t.bx = 256;
  t.by = 1;
  t.rows = rows_for_wave(g, t, sms * generic_blocks_per_sm(prec, t));
  return t;
}

int generic_blocks_per_sm(int prec, const StepTile& t) {
  int per_sm = 0;
  switch (prec) {
    case 0: per_sm = occupancy<0>(t.bx, t.by); break;
    case 1: per_sm = occupancy<1>(t.bx, t.by); break;
    case 2: per_sm = occupancy<2>(t.bx, t.by); break;
    case 3: per_sm = occupancy<3>(t.bx, t.by); break;
  }
  return per_sm > 0 ? per_sm : 1;
}

int rows_for_wave(const HostGeometry& g, const StepTile& t, int ctas) {
  // One full wave: gx * gy ~ ctas CTAs, rows a multiple of BY.
  const int cols = t.pair ? 2 * t.bx : t.bx;  // a paired tile covers two columns per thread
  const int gx = (g.nx + cols - 1) / cols;
  int gy = std::max(1, ctas / gx);
  int rows = (g.ny + gy - 1) / gy;
  rows = ((rows + t.by - 1) / t.by) * t.by;
  return std::max(rows, t.by);
}

int default_rows(const HostGeometry& g, const StepTile& t, int ctas_per_wave) {
  const int rows = rows_for_wave(g, t, ctas_per_wave);
  // The one-node kernels, and the walled paired kernel (2 CTAs per SM): one wave of long CTAs
  // measured fastest (walled 4096 x 2048 FP16: 108 rows 48.8k MLUPS, 36 rows 47.0k).
  if (!t.pair || g.walls) return rows;
  // The periodic paired kernel holds 3 CTAs per SM, and one wave ends with a long uneven tail: up
  // to 4 waves while a CTA keeps at least 32 rows (4096^2 FP16: 36 rows, 57.2k MLUPS against 55.3k
  // for one wave of 147 rows; 16 rows was slower again).
  const int waves = std::min(4, std::max(1, rows / 32));
  return waves > 1 ? rows_for_wave(g, t, ctas_per_wave * waves) : rows;
}

cudaError_t launch_init(int prec, const HostGeometry& g, const HostPhys& p, const double* fields,
                        char* dst, cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd = node_grid(g, blk);
  switch (prec) {
    case 0: k_init<0><<<grd, blk, 0, s>>>(fields, dst, to_geo(g), to_phys<double>(p)); break;
    case 1: k_init<1><<<grd, blk, 0, s>>>(fields, dst, to_geo(g), to_phys<float>(p)); break;
    case 2: k_init<2><<<grd, blk, 0, s>>>(fields, dst, to_geo(g), to_phys<float>(p)); break;
    case 3: k_init<3><<<grd, blk, 0, s>>>(fields, dst, to_geo(g), to_phys<float>(p)); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                        const char* src, char* dst, int* flag, cudaStream_t s) {
  if (t.staged && t.pair) return launch_step_pair_tma(prec, g, p, t, src, dst, flag, s);
  if (t.staged) return launch_step_staged(prec, g, p, t, src, dst, flag, s);
  if (t.pair) return launch_step_pair(prec, g, p, t, src, dst, flag, s);
  switch (prec) {
    case 0: return step_prec<0>(g, p, t, src, dst, flag, s);
    case 1: return step_prec<1>(g, p, t, src, dst, flag, s);
    case 2: return step_prec<2>(g, p, t, src, dst, flag, s);
    case 3: return step_prec<3>(g, p, t, src, dst, flag, s);
  }
  return cudaErrorInvalidValue;
}

size_t phys_bytes(int prec) { return prec == 0 ? sizeof(Phys<double>) : sizeof(Phys<float>); }

cudaError_t upload_phys(int prec, const HostPhys* host, int count, void* dev, cudaStream_t s) {
  if (prec == 0) {
    Phys<double>* tmp = new Phys<double>[count];
    for (int i = 0; i < count; ++i) tmp[i] = to_phys<double>(host[i]);
    cudaError_t e = cudaMemcpyAsync(dev, tmp, sizeof(Phys<double>) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] tmp;
    return e;
  }
  Phys<float>* tmp = new Phys<float>[count];
  for (int i = 0; i < count; ++i) tmp[i] = to_phys<float>(host[i]);
  cudaError_t e = cudaMemcpyAsync(dev, tmp, sizeof(Phys<float>) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete[] tmp;
  return e;
}

namespace {

template <int PREC, int BX, int BY>
cudaError_t batch_bxby(const BatchItem* items, int nitems, const BatchMember* members, const void* phys,
                       int parity, int* flags, long long* tcount, int grid, bool off32, cudaStream_t s) {
  if (off32)
    return launch_k_step_batch<PREC, BX, BY, true>(items, nitems, members, phys, parity, flags, tcount, grid, s);
  return launch_step_batch64(PREC, BX, BY, items, nitems, members, phys, parity, flags, tcount, grid, s);
}

template <int PREC>
cudaError_t batch_prec(const StepTile& t, const BatchItem* items, int nitems, const BatchMember* members,
                       const void* phys, int parity, int* flags, long long* tcount, int grid, bool off32,
                       cudaStream_t s) {
#define LBM_CASE(X, Y)                                                                                   \
  if (t.bx == X && t.by == Y)                                                                            \
    return batch_bxby<PREC, X, Y>(items, nitems, members, phys, parity, flags, tcount, grid, off32, s);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template <int PREC>
int batch_occ(int bx, int by) {
  int nb = 0;
#define LBM_CASE(X, Y) \
  if (bx == X && by == Y) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_batch<PREC, X, Y, true>, X * Y, 0);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return nb;
}

}  // namespace

cudaError_t launch_step_batch(int prec, const StepTile& t, const BatchItem* items, int nitems,
                              const BatchMember* members, const void* phys, int parity, int* flags,
                              long long* tcount, int grid, bool off32, cudaStream_t s) {
  if (t.pair) return launch_step_pair_batch(prec, items, nitems, members, phys, parity, flags, tcount, grid, s);
  switch (prec) {
    case 0: return batch_prec<0>(t, items, nitems, members, phys, parity, flags, tcount, grid, off32, s);
    case 1: return batch_prec<1>(t, items, nitems, members, phys, parity, flags, tcount, grid, off32, s);
    case 2: return batch_prec<2>(t, items, nitems, members, phys, parity, flags, tcount, grid, off32, s);
    case 3: return batch_prec<3>(t, items, nitems, members, phys, parity, flags, tcount, grid, off32, s);
  }
  return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int prec, const StepTile& t) {
  if (t.pair) return pair_batch_blocks_per_sm(prec);
  int nb = 0;
  switch (prec) {
    case 0: nb = batch_occ<0>(t.bx, t.by); break;
    case 1: nb = batch_occ<1>(t.bx, t.by); break;
    case 2: nb = batch_occ<2>(t.bx, t.by); break;
    case 3: nb = batch_occ<3>(t.bx, t.by); break;
  }
  return nb > 0 ? nb : 1;
}

cudaError_t launch_fields(int prec, const HostGeometry& g, const HostPhys& p, const char* src, double* out,
                          cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd = node_grid(g, blk);
  switch (prec) {
    case 0: k_fields<0><<<grd, blk, 0, s>>>(src, to_geo(g), p.force_x, p.force_y, p.force_mode, out); break;
    case 1: k_fields<1><<<grd, blk, 0, s>>>(src, to_geo(g), p.force_x, p.force_y, p.force_mode, out); break;
    case 2: k_fields<2><<<grd, blk, 0, s>>>(src, to_geo(g), p.force_x, p.force_y, p.force_mode, out); break;
    case 3: k_fields<3><<<grd, blk, 0, s>>>(src, to_geo(g), p.force_x, p.force_y, p.force_mode, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_fill(double* __restrict__ p, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s) {
  const int nb = (int)std::min<long long>(4096, (n + 255) / 256);
  k_fill<<<std::max(nb, 1), 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

// Interleaved FP32 node state (phi, ux, uy per node, nx*ny nodes) <-> the dense FP64 field
// layout of k_init ([phi | ux | uy | rho], rho = 1) and of k_fields ([rho | ux | uy | phi]).
__global__ void k_state_to_fields(const float* __restrict__ st, long long n, double* __restrict__ fields) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    fields[i] = (double)st[3 * i];
    fields[n + i] = (double)st[3 * i + 1];
    fields[2 * n + i] = (double)st[3 * i + 2];
    fields[3 * n + i] = 1.0;
  }
}
__global__ void k_fields_to_state(const double* __restrict__ fields, long long n, float* __restrict__ st) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    st[3 * i] = (float)fields[3 * n + i];
    st[3 * i + 1] = (float)fields[n + i];
    st[3 * i + 2] = (float)fields[2 * n + i];
  }
}

cudaError_t launch_state_to_fields(const float* st, long long n, double* fields, cudaStream_t s) {
  const int nb = (int)std::min<long long>(4096, (n + 255) / 256);
  k_state_to_fields<<<std::max(nb, 1), 256, 0, s>>>(st, n, fields);
  return cudaGetLastError();
}
cudaError_t launch_fields_to_state(const double* fields, long long n, float* st, cudaStream_t s) {
  const int nb = (int)std::min<long long>(4096, (n + 255) / 256);
  k_fields_to_state<<<std::max(nb, 1), 256, 0, s>>>(fields, n, st);
  return cudaGetLastError();
}

size_t reduce_partials_bytes() { return sizeof(double) * 4 * kRedBlocks; }

cudaError_t launch_reduce(int prec, const HostGeometry& g, const char* src, double* partials,
                          double* out4, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny;
  int nb = (int)std::min<long long>(kRedBlocks, (N + kRedThreads - 1) / kRedThreads);
  nb = std::max(nb, 1);
  switch (prec) {
    case 0: k_reduce_partials<0><<<nb, kRedThreads, 0, s>>>(src, to_geo(g), partials); break;
    case 1: k_reduce_partials<1><<<nb, kRedThreads, 0, s>>>(src, to_geo(g), partials); break;
    case 2: k_reduce_partials<2><<<nb, kRedThreads, 0, s>>>(src, to_geo(g), partials); break;
    case 3: k_reduce_partials<3><<<nb, kRedThreads, 0, s>>>(src, to_geo(g), partials); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kRedThreads, 0, s>>>(partials, nb, out4);
  return cudaGetLastError();
}

cudaError_t launch_plane_get(int prec, const HostGeometry& g, const char* src, int p, double* out,
                             cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd = node_grid(g, blk);
  switch (prec) {
    case 0: k_plane_get<0><<<grd, blk, 0, s>>>(src, to_geo(g), p, out); break;
    case 1: k_plane_get<1><<<grd, blk, 0, s>>>(src, to_geo(g), p, out); break;
    case 2: k_plane_get<2><<<grd, blk, 0, s>>>(src, to_geo(g), p, out); break;
    case 3: k_plane_get<3><<<grd, blk, 0, s>>>(src, to_geo(g), p, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_plane_set(int prec, const HostGeometry& g, char* dst, int p, const double* in,
                             cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd = node_grid(g, blk);
  switch (prec) {
    case 0: k_plane_set<0><<<grd, blk, 0, s>>>(dst, to_geo(g), p, in); break;
    case 1: k_plane_set<1><<<grd, blk, 0, s>>>(dst, to_geo(g), p, in); break;
    case 2: k_plane_set<2><<<grd, blk, 0, s>>>(dst, to_geo(g), p, in); break;
    case 3: k_plane_set<3><<<grd, blk, 0, s>>>(dst, to_geo(g), p, in); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbmch
