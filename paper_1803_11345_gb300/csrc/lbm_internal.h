// Host-side interface between the C ABI (lbm_capi.cu) and the kernels (lbm_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

struct lbm_params;  // include/lbm.h

namespace lbmch {

struct HostGeometry {
  int nx, ny, pitch;
  long long plane;
  int walls;
};

struct HostPhys {
  double omega_l, omega_g, tau_l, tau_g, omega3, omega_phi, gamma, a, Gamma, u_top, u_bottom;
  double wet_bottom, wet_top, force_x, force_y;
  int visc, k8_printed, bgk, force_mode;
  int rounding = 0;      // lbm_rounding
  uint32_t seed = 0;     // stochastic-rounding seed
  uint32_t sr_key = 0;   // per launch: 0 rounds to nearest, else the step's stochastic-rounding key
  int wait_probes = -1;  // staged kernel: probes before a bulk-copy wait gives up (< 0: the default)
};

// Key of the stochastic-rounding stream for time step t: the 32-bit finaliser of MurmurHash3
// (A. Appleby) over the seed and both halves of t; never 0 (0 means round to nearest).  The same
// function on the host (single lattices) and on the device (batches, whose captured graphs derive
// the key from a step counter in device memory), so a batch member draws a lattice's stream.
__host__ __device__ inline uint32_t sr_fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__host__ __device__ inline uint32_t sr_step_key(uint32_t seed, long long t) {
  const uint32_t k = sr_fmix32(sr_fmix32(seed ^ 0x5bd1e995u) + (uint32_t)t) ^
                     sr_fmix32((uint32_t)((unsigned long long)t >> 32));
  return k ? k : 1u;
}

// Bits of a lattice's device status word: a node produced a non-finite rho or phi; a bounded
// device-side wait gave up (the step that set it is incomplete).
constexpr int kFlagNonfinite = 1;
constexpr int kFlagTimeout = 2;

// Tile of the fused step: BX columns x BY rows of threads, `rows` lattice rows per CTA.
// staged = 1 selects the bulk-copy staged kernel (lbm_staged.cu) with `depth` bands of
// prefetch; staged = 0 the generic kernel (lbm_kernels.cu).
struct StepTile {
  int bx, by, rows;
  int staged, depth;
  int wide = 0;  // generic kernel with 64-bit plane offsets even when the buffer is under 4 GiB
  int pair = 0;  // 16-bit storage, two nodes per thread (lbm_pair.cu); columns per CTA = 2 bx
                 // (with staged = 1: the bulk-copy staged paired kernel, lbm_pair_tma.cu)
};

// Batched stepping: one member lattice (two population copies) and one unit of work (a tile of
// one member).  Plain structs shared by host and device code.
struct BatchMember {
  int nx, ny, pitch, walls;
  long long plane;
  char* buf0;
  char* buf1;
};
struct BatchItem {
  int member, x0, y0, rows;
};

// Upload per-member physics in the kernel's arithmetic type; `dev` must hold
// count * phys_bytes(prec) bytes.
size_t phys_bytes(int prec);
cudaError_t upload_phys(int prec, const HostPhys* host, int count, void* dev, cudaStream_t s);
// One time step of every member: items[] dealt round-robin to `grid` resident CTAs.  parity 0:
// state in buf0 -> buf1; parity 1: buf1 -> buf0.  flags[m] collects member m's non-finite flag.
// off32: every member's population buffer is under 4 GiB (32-bit plane offsets).
// tcount[2]: the batch's time step, tcount[parity] current; each launch writes its successor into
// tcount[1 - parity] (the stochastic-rounding key of a member is derived from it on the device).
cudaError_t launch_step_batch(int prec, const StepTile& t, const BatchItem* items, int nitems,
                              const BatchMember* members, const void* phys, int parity, int* flags,
                              long long* tcount, int grid, bool off32, cudaStream_t s);
int batch_blocks_per_sm(int prec, const StepTile& t);

// Parameter validation shared by the single-lattice and batched entry points (message or NULL),
// and the bytes of one population copy (256-aligned, large enough to stage four FP64 fields and
// the reduction partials).
const char* validate_params(const ::lbm_params* p, HostGeometry* g, HostPhys* ph);
size_t copy_bytes(int prec, const HostGeometry& g);

// Message returned by lbm_last_error(NULL) on the calling thread.
void set_thread_error(const char* msg);

// Interleaved FP32 node state (phi, ux, uy) of n nodes <-> dense FP64 fields: to the k_init layout
// [phi | ux | uy | rho = 1], from the k_fields layout [rho | ux | uy | phi].
cudaError_t launch_state_to_fields(const float* st, long long n, double* fields, cudaStream_t s);
cudaError_t launch_fields_to_state(const double* fields, long long n, float* st, cudaStream_t s);

// Fill n doubles with v.
cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s);

// The paired 16-bit step (lbm_pair.cu): whether tile bx x by can serve the lattice (16-bit
// storage, nx even, buffer under 4 GiB), resident CTAs per SM, and the launch.
bool pair_supported(int prec, const HostGeometry& g, int bx, int by);
// The paired 16-bit kernel with its rows staged by the bulk-copy engine (lbm_pair_tma.cu): 128
// pairs per CTA, ring depth 1 or 2; periodic lattices with nx a multiple of 8.
// The batched paired kernel (lbm_pair.cu): 128 x 1 threads, 256-column items of periodic 16-bit
// members, every member's buffer under 4 GiB; phys holds Phys<float> per member.
cudaError_t launch_step_pair_batch(int prec, const BatchItem* items, int nitems, const BatchMember* members,
                                  const void* phys, int parity, int* flags, long long* tcount, int grid,
                                  cudaStream_t s);
int pair_batch_blocks_per_sm(int prec);
bool pair_tma_supported(int prec, const HostGeometry& g, int depth);
int pair_tma_blocks_per_sm(int prec, int depth);
cudaError_t launch_step_pair_tma(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                                 const char* src, char* dst, int* flag, cudaStream_t s);
int pair_blocks_per_sm(int prec, const StepTile& t, bool walls);
cudaError_t launch_step_pair(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t, const char* src,
                             char* dst, int* flag, cudaStream_t s);

// Bytes of one population buffer (18 planes) for a storage precision.
size_t pop_buffer_bytes(int prec, long long plane);
// Every byte offset inside one population buffer fits in 32 bits (the step kernel then forms
// plane offsets in 32-bit arithmetic).
bool offsets_fit_32(int prec, long long plane);

// Launchers; each returns the cudaError_t of the launch.
cudaError_t launch_init(int prec, const HostGeometry& g, const HostPhys& p, const double* fields,
                        char* dst, cudaStream_t s);
cudaError_t launch_step(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                        const char* src, char* dst, int* flag, cudaStream_t s);
cudaError_t launch_fields(int prec, const HostGeometry& g, const HostPhys& p, const char* src, double* out,
                          cudaStream_t s);
// Deterministic FP64 totals [sum phi, sum rho, sum jx, sum jy] into out4 (device), using
// `partials` (device, >= reduce_partials_bytes()) as scratch.
size_t reduce_partials_bytes();
cudaError_t launch_reduce(int prec, const HostGeometry& g, const char* src, double* partials,
                          double* out4, cudaStream_t s);
// One plane (0..8 f, 9..17 g) between the state and a dense FP64 array of nx*ny.
cudaError_t launch_plane_get(int prec, const HostGeometry& g, const char* src, int p, double* out,
                             cudaStream_t s);
cudaError_t launch_plane_set(int prec, const HostGeometry& g, char* dst, int p, const double* in,
                             cudaStream_t s);

// Staged kernel: halo width (columns) per precision, whether a lattice/tile can use it, its
// resident CTAs per SM, and its launcher.
int staged_halo(int prec);
bool staged_supported(int prec, const HostGeometry& g, const StepTile& t);
int staged_blocks_per_sm(int prec, const StepTile& t);
cudaError_t launch_step_staged(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                               const char* src, char* dst, int* flag, cudaStream_t s);

// Default tile for a precision and lattice, sized so the grid fills the GPU in one wave (the paired kernel: a few waves).
StepTile default_tile(int prec, const HostGeometry& g, int device);
// Resident CTAs per SM of the generic kernel for a tile.
int generic_blocks_per_sm(int prec, const StepTile& t);
// Rows per CTA so that the grid is about `ctas` CTAs (one wave).
int rows_for_wave(const HostGeometry& g, const StepTile& t, int ctas);
// Default rows per CTA for a tile, given the CTAs of one wave: one wave for the one-node kernels,
// up to 4 waves of at least 32 rows for the paired kernel on periodic lattices.
int default_rows(const HostGeometry& g, const StepTile& t, int ctas_per_wave);
// Whether a tile shape has a compiled kernel.
bool tile_supported(int prec, int bx, int by);

}  // namespace lbmch
