// Host-side interface between the C ABI (lbm_capi.cu) and the kernels (lbm_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace lbmch {

struct HostGeometry {
  int nx, ny, pitch;
  long long plane;
  int walls;
};

struct HostPhys {
  double omega_l, omega_g, tau_l, tau_g, omega3, omega_phi, gamma, a, Gamma, u_top, u_bottom;
  int visc, k8_printed, bgk;
};

// Tile of the fused step: BX columns x BY rows of threads, `rows` lattice rows per CTA.
// staged = 1 selects the bulk-copy staged kernel (lbm_staged.cu) with `depth` bands of
// prefetch; staged = 0 the generic kernel (lbm_kernels.cu).
struct StepTile {
  int bx, by, rows;
  int staged, depth;
};

// Message returned by lbm_last_error(NULL) on the calling thread.
void set_thread_error(const char* msg);

// Fill n doubles with v.
cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t s);

// Bytes of one population buffer (18 planes) for a storage precision.
size_t pop_buffer_bytes(int prec, long long plane);

// Launchers; each returns the cudaError_t of the launch.
cudaError_t launch_init(int prec, const HostGeometry& g, const HostPhys& p, const double* fields,
                        char* dst, cudaStream_t s);
cudaError_t launch_step(int prec, const HostGeometry& g, const HostPhys& p, const StepTile& t,
                        const char* src, char* dst, int* flag, cudaStream_t s);
cudaError_t launch_fields(int prec, const HostGeometry& g, const char* src, double* out,
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

// Default tile for a precision and lattice, sized so the grid fills the GPU in one wave.
StepTile default_tile(int prec, const HostGeometry& g, int device);
// Resident CTAs per SM of the generic kernel for a tile.
int generic_blocks_per_sm(int prec, const StepTile& t);
// Rows per CTA so that the grid is about `ctas` CTAs (one wave).
int rows_for_wave(const HostGeometry& g, const StepTile& t, int ctas);
// Whether a tile shape has a compiled kernel.
bool tile_supported(int prec, int bx, int by);

}  // namespace lbmch
