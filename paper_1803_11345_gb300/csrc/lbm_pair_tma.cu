// Paired 16-bit step with the population rows staged in shared memory by the bulk-copy (TMA)
// engine.
//
// The register-pipelined paired kernel (lbm_pair.cu) keeps two row-bands of loaded words in
// flight in registers, which holds it at about 160 registers and 12 warps per SM, and with so few
// warps its packed arithmetic waits on fixed-latency dependencies.  Here every population row a
// CTA pulls from is copied into shared memory by cp.async.bulk (one copy per plane and row, issued
// by one warp and completed on an mbarrier), so no load is in flight in registers, every pull is a
// shared load at a constant offset from a row base, and the kernel fits 4 CTAs of 128 threads per
// SM.  The arithmetic is the paired kernel's: the same pair words, decode, collision, closures and
// stores (lbm_pair.cuh), so the two kernels give the same fields.
//
// CTA = 128 threads = 128 node pairs = a strip of 256 columns, marching down `rows` rows.  A
// staged row v of a set (f or g) holds, for each of the 8 moving directions, the 16-bit values of
// columns [x0 - 8, x0 + 264) and, for the FP32 rest plane, columns [x0 - 4, x0 + 260): the halos
// make every copy 16-byte aligned, and they wrap around periodically.  Rings of RG = 4 + D g rows
// and RF = 3 + D f rows; step Y:
//   wait for g row Y+2 and f row Y+1 -> phi of row Y+1 from g rows Y..Y+2 (and of the two halo
//   nodes) into the phi ring -> __syncthreads -> warp 0 issues g row Y+2+D, warp 1 f row Y+1+D,
//   into the slots this band freed -> collision of row Y: f and g pulled from rows Y-1..Y+1,
//   Eq. 12 stencils from the phi ring -> stores straight to global memory.
// Every wait is bounded; a wait that runs out sets kFlagTimeout, the CTA lets the copies it issued
// land, and returns.
// Requirements: periodic lattice, nx a multiple of 8, population copy under 4 GiB.
#include "lbm_pair.cuh"
#include "lbm_step.cuh"
#include "lbm_tma.cuh"

namespace lbmch {

namespace {

constexpr int kPT = 128;                            // threads (node pairs) per CTA
constexpr int kCols = 2 * kPT;                      // columns per strip
constexpr int kH16 = 8, kH32 = 4;                   // halo columns per side: 16-bit, FP32 planes
constexpr int kHalfRow = (kCols + 2 * kH16) * 2;    // bytes of one staged 16-bit plane row
constexpr int kRestOff = 8 * kHalfRow;              // the FP32 rest plane follows the 8 others
constexpr int kRowBytes = kRestOff + (kCols + 2 * kH32) * 4;
constexpr int kPhiW = kCols + 2;                    // phi ring row: the strip and its two halo nodes
static_assert(kHalfRow % 16 == 0 && kRowBytes % 16 == 0 && (4 * kPhiW * 4) % 16 == 0, "staging alignment");

// Probes before a wait is declared stuck (each probe suspends for a short hardware window): far
// beyond any legitimate copy latency, short enough to return control in well under a second.  The
// main loop's waits take their limit from the launch (lbm_set_wait_limit); the prologue and the
// drain after an abort use this one.
constexpr uint32_t kPairWaitProbes = 1u << 22;

template <int D> struct TmaRing {
  static constexpr int RG = 4 + D, RF = 3 + D;
  static constexpr size_t kPhiOff = (size_t)(RG + RF) * kRowBytes;
  static constexpr size_t kBarOff = kPhiOff + 4 * kPhiW * sizeof(float);
  static constexpr size_t kBytes = kBarOff + (RG + RF) * sizeof(uint64_t) + 16;
};

template <int PREC, int D>
__global__ void __launch_bounds__(kPT, 4)
k_step_pair_tma(const char* __restrict__ src, char* __restrict__ dst, const Geometry geo, const Phys<F2> ph,
                const int rows, int* __restrict__ flag, const uint32_t wait_limit) {
  using P = Pop<PREC>;
  using Ring = TmaRing<D>;
  constexpr int RG = Ring::RG, RF = Ring::RF;
  extern __shared__ __align__(128) char smem[];
  char* const gring = smem;
  char* const fring = smem + RG * kRowBytes;
  float(*const sphi)[kPhiW] = reinterpret_cast<float(*)[kPhiW]>(smem + Ring::kPhiOff);
  uint64_t* const gbar = reinterpret_cast<uint64_t*>(smem + Ring::kBarOff);
  uint64_t* const fbar = gbar + RG;
  int* const abort_flag = reinterpret_cast<int*>(fbar + RF);

  const int tx = threadIdx.x, lane = tx & 31, warp = tx >> 5;
  const int nx = geo.nx, ny = geo.ny, pitch = geo.pitch;
  const Plane32 pl{(unsigned)geo.plane};
  const int x0 = blockIdx.x * kCols;
  const int y0 = blockIdx.y * rows;
  const int y1 = min(y0 + rows, ny);
  const int xv = min(kCols, nx - x0);  // columns of this strip, a multiple of 8
  const int x = x0 + 2 * tx;
  const bool colv = 2 * tx < xv;
  const bool last_pair = colv && 2 * tx + 2 == xv;  // this thread also forms the right halo node
  const bool interior = x0 >= kH16 && x0 + xv + kH16 <= nx;
  const int gfirst = y0 - 2, ffirst = y0 - 1;  // first staged row of each set
  const int glast = y1 + 1, flast = y1;

  if (tx == 0) {
    for (int k = 0; k < RG; ++k) mbar_init(&gbar[k], 1);
    for (int k = 0; k < RF; ++k) mbar_init(&fbar[k], 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  auto wrap_row = [&](int v) { return v < 0 ? v + ny : (v >= ny ? v - ny : v); };

  // Stage row v of set g (true) or f, by one whole warp: lane 0 arms the slot's barrier with the
  // byte count, then one lane per plane (three per plane at the lattice's left and right edges,
  // where a halo wraps around) issues its copy.
  auto issue = [&](bool g, int v) {
    const int k = v - (g ? gfirst : ffirst);
    const int slot = k % (g ? RG : RF);
    char* const drow = (g ? gring : fring) + slot * kRowBytes;
    uint64_t* const bar = g ? &gbar[slot] : &fbar[slot];
    const size_t row = (size_t)wrap_row(v) * (size_t)pitch;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(8 * (xv + 2 * kH16) * 2 + (xv + 2 * kH32) * 4));
    __syncwarp();
    // Element 0 of the row in staged plane q: 0..7 the moving directions 1..8, 8 the rest plane.
    auto plane_row = [&](int q) -> const char* {
      return q < 8 ? src + ((size_t)((g ? 8 : 0) + q) * pl.n + row) * 2
                   : src + ((size_t)(P::kRestFirst + (g ? 1 : 0)) * pl.n + row) * 4;
    };
    if (interior) {
      if (lane < 9) {
        const int q = lane;
        if (q < 8)
          bulk_g2s(drow + q * kHalfRow, plane_row(q) + (size_t)(x0 - kH16) * 2, (uint32_t)((xv + 2 * kH16) * 2), bar);
        else
          bulk_g2s(drow + kRestOff, plane_row(8) + (size_t)(x0 - kH32) * 4, (uint32_t)((xv + 2 * kH32) * 4), bar);
      }
    } else if (lane < 27) {
      const int q = lane / 3, seg = lane - 3 * q;
      const int es = q < 8 ? 2 : 4, H = q < 8 ? kH16 : kH32;
      char* const d = drow + q * kHalfRow;
      const char* const ps = plane_row(q);
      if (seg == 0) bulk_g2s(d, ps + (size_t)(x0 == 0 ? nx - H : x0 - H) * es, (uint32_t)(H * es), bar);
      else if (seg == 1) bulk_g2s(d + H * es, ps + (size_t)x0 * es, (uint32_t)(xv * es), bar);
      else bulk_g2s(d + (H + xv) * es, ps + (size_t)(x0 + xv == nx ? 0 : x0 + xv) * es, (uint32_t)(H * es), bar);
    }
  };
  bool stuck = false;
  auto wait_row = [&](bool g, int v, uint32_t limit) {
    const int k = v - (g ? gfirst : ffirst);
    const int R = g ? RG : RF;
    if (!mbar_wait_bounded(g ? &gbar[k % R] : &fbar[k % R], (uint32_t)((k / R) & 1), limit)) stuck = true;
  };
  // Staged rows v-1, v, v+1 of a set (v at least one row past the set's first).
  struct Rows3 {
    const char* lo;
    const char* mid;
    const char* hi;
  };
  auto rows3 = [&](bool g, int v) -> Rows3 {
    const int R = g ? RG : RF;
    const int sm = (v - (g ? gfirst : ffirst)) % R;
    const int sl = sm == 0 ? R - 1 : sm - 1, sh = sm == R - 1 ? 0 : sm + 1;
    const char* const b = g ? gring : fring;
    return Rows3{b + sl * kRowBytes, b + sm * kRowBytes, b + sh * kRowBytes};
  };
  // Eqs. 4-5 for the pair (x, x+1) at node row v from the staged rows: direction i from row
  // v - c_yi and columns x - c_xi, x + 1 - c_xi, as the words of lbm_pair.cuh (the thread's word
  // sits at byte 4 tx + 16 of a staged 16-bit plane row).
  auto pull_s = [&](bool g, int v, RawPair& o) {
    const Rows3 q = rows3(g, v);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const char* const r = lat_cy(i) == 1 ? q.lo : (lat_cy(i) == -1 ? q.hi : q.mid);
      const char* const pw = r + (i - 1) * kHalfRow + 4 * tx + 2 * kH16;
      const uint32_t w = *reinterpret_cast<const uint32_t*>(pw);
      if (lat_cx(i) == 0) o.w[i - 1] = w;
      else if (lat_cx(i) == 1) o.w[i - 1] = __byte_perm(*reinterpret_cast<const uint32_t*>(pw - 4), w, 0x5432);
      else o.w[i - 1] = __byte_perm(w, *reinterpret_cast<const uint32_t*>(pw + 4), 0x5432);
    }
    const float2 r0 = *reinterpret_cast<const float2*>(q.mid + kRestOff + 8 * tx + 4 * kH32);
    o.r0a = r0.x;
    o.r0b = r0.y;
  };
  // phi of one halo node (staged 16-bit column c16, FP32 column c32) at node row v, summed in the
  // one-node kernel's order.
  auto halo_phi = [&](int v, int c16, int c32) -> float {
    const Rows3 q = rows3(true, v);
    float s[9];
    s[0] = *reinterpret_cast<const float*>(q.mid + kRestOff + c32 * 4);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const char* const r = lat_cy(i) == 1 ? q.lo : (lat_cy(i) == -1 ? q.hi : q.mid);
      s[i] = P::h2f(*reinterpret_cast<const unsigned short*>(r + (i - 1) * kHalfRow + (c16 - lat_cx(i)) * 2));
    }
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8];
  };
  auto ring_row = [&](int v) { return (v - (y0 - 1)) & 3; };  // phi ring slot of node row v >= y0 - 1
  auto put_phi = [&](int v) {
    float* const prow = sphi[ring_row(v)];
    if (colv) {
      RawPair gp;
      pull_s(true, v, gp);
      const F2 p = phi_pair<PREC>(gp);
      prow[2 * tx + 1] = p.v.x;
      prow[2 * tx + 2] = p.v.y;
    }
    if (tx == 0) prow[0] = halo_phi(v, kH16 - 1, kH32 - 1);
    if (last_pair) prow[xv + 1] = halo_phi(v, kH16 + xv, kH32 + xv);
  };
  // After a wait ran out: let every copy this CTA issued land (the latest issue of each slot)
  // before its shared memory is released, and report the timeout.
  int g_next = gfirst, f_next = ffirst;
  auto abort_cta = [&]() {
    if (tx == 0) {
      atomicOr(flag, kFlagTimeout);
      for (int v = max(gfirst, g_next - RG); v < g_next; ++v) wait_row(true, v, kPairWaitProbes);
      for (int v = max(ffirst, f_next - RF); v < f_next; ++v) wait_row(false, v, kPairWaitProbes);
    }
  };

  // Prologue: the first RG g rows and RF f rows (dealt out to the warps), then phi of rows y0-1, y0.
  {
    const int ng = min(gfirst + RG - 1, glast) - gfirst + 1;
    const int nf = min(ffirst + RF - 1, flast) - ffirst + 1;
    for (int k = warp; k < ng + nf; k += kPT / 32) {
      if (k < ng) issue(true, gfirst + k);
      else issue(false, ffirst + (k - ng));
    }
    g_next += ng;
    f_next += nf;
    for (int v = gfirst; v <= y0 + 1; ++v) wait_row(true, v, kPairWaitProbes);
    for (int v = ffirst; v <= y0; ++v) wait_row(false, v, kPairWaitProbes);
    if (stuck) atomicExch(abort_flag, 1);
    __syncthreads();
    if (*abort_flag) {
      abort_cta();
      return;
    }
    put_phi(y0 - 1);
    put_phi(y0);
  }

  for (int Y = y0; Y < y1; ++Y) {
    wait_row(true, Y + 2, wait_limit);  // Y + 2 <= y1 + 1 = glast
    put_phi(Y + 1);
    wait_row(false, Y + 1, wait_limit);  // Y + 1 <= y1 = flast
    if (stuck) atomicExch(abort_flag, 1);
    __syncthreads();
    if (*abort_flag) {
      abort_cta();
      return;
    }
    // Rows at or below Y - 2 are no longer read: refill their slots.
    if (g_next <= min(Y + 2 + D, glast)) {
      if (warp == 0) issue(true, g_next);
      ++g_next;
    }
    if (f_next <= min(Y + 1 + D, flast)) {
      if (warp == 1) issue(false, f_next);
      ++f_next;
    }
    if (colv) {
      const int rs[3] = {ring_row(Y - 1), ring_row(Y), ring_row(Y + 1)};
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
      RawPair fr, gr;
      pull_s(false, Y, fr);
      pull_s(true, Y, gr);
      F2 f[9], g[9];
      unpack_pair<PREC>(fr, f);
      unpack_pair<PREC>(gr, g);
      const F2 drho = collide<F2>(ph, f, g, phi, dxp, dyp, lap);
      if (!(isfinite(drho.v.x) && isfinite(drho.v.y) && isfinite(phi.v.x) && isfinite(phi.v.y)))
        atomicOr(flag, kFlagNonfinite);
      store_pair<PREC>(dst, pl, (unsigned)(Y * pitch + x), f, g, drho, phi, ph.sr_key);
    }
  }
}

template <int PREC, int D>
cudaError_t tma_launch(const HostGeometry& g, const HostPhys& p, int rows, const char* src, char* dst, int* flag,
                       cudaStream_t s) {
  const size_t smem = TmaRing<D>::kBytes;
  static bool configured = false;
  if (!configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_step_pair_tma<PREC, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const dim3 grd((g.nx + kCols - 1) / kCols, (g.ny + rows - 1) / rows);
  const uint32_t limit = p.wait_probes < 0 ? kPairWaitProbes : (uint32_t)p.wait_probes;
  k_step_pair_tma<PREC, D><<<grd, kPT, smem, s>>>(src, dst, to_geo(g), make_phys<F2>(p), rows, flag, limit);
  return cudaGetLastError();
}

template <int PREC, int D>
int tma_occupancy() {
  const size_t smem = TmaRing<D>::kBytes;
  cudaFuncSetAttribute(k_step_pair_tma<PREC, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_pair_tma<PREC, D>, kPT, smem);
  return nb;
}

}  // namespace

bool pair_tma_supported(int prec, const HostGeometry& g, int depth) {
  return (prec == 2 || prec == 3) && !g.walls && g.nx % 8 == 0 && g.ny >= 3 && (depth == 1 || depth == 2) &&
         offsets_fit_32(prec, g.plane);
}

int pair_tma_blocks_per_sm(int prec, int depth) {
  if (prec == 2) return depth == 2 ? tma_occupancy<2, 2>() : tma_occupancy<2, 1>();
  if (prec == 3) return depth == 2 ? tma_occupancy<3, 2>() : tma_occupancy<3, 1>();
  return 0;
}

cudaError_t launch_step_pair_tma(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                                 const char* src, char* dst, int* flag, cudaStream_t s) {
  if (prec == 2) return t.depth == 2 ? tma_launch<2, 2>(g, p, t.rows, src, dst, flag, s)
                                     : tma_launch<2, 1>(g, p, t.rows, src, dst, flag, s);
  if (prec == 3) return t.depth == 2 ? tma_launch<3, 2>(g, p, t.rows, src, dst, flag, s)
                                     : tma_launch<3, 1>(g, p, t.rows, src, dst, flag, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbmch
