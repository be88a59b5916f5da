// Conservation totals without any device allocation (declared in include/lbm.h).
//
// The reduction kernels of lbm_conservation need scratch for their per-block partial sums; that
// entry point takes it from the lattice's spare population copy.  This one serves callers that
// hold a population state in device memory they manage themselves and may not allocate (an
// arena owned by a host framework, a process under a fixed device-memory budget, a checkpoint
// restored into a preallocated slab): its scratch is the file-scope array below, reserved once
// when the library is loaded and kept by every GPU that loads it until the process exits.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// Partials of at most kMaxBlocks reduction blocks (4 doubles each) followed by the 4 totals.
constexpr int kMaxBlocks = 1024;
constexpr int kScratchDoubles = 4 * kMaxBlocks + 4;
static __device__ __align__(256) double g_totals_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

int fail(int code, const char* msg) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "lbm_totals_noalloc: %s", msg);
  lbmch::set_thread_error(buf);
  return code;
}

}  // namespace

extern "C" {

int lbm_totals_noalloc(const void* state, int nx, int ny, int prec, double* totals, void* stream) {
  lbmch::set_thread_error("");
  if (!state || !totals) return fail(LBM_ERR_PARAM, "state and totals are required");
  if (nx < 3 || ny < 3) return fail(LBM_ERR_PARAM, "nx and ny must be >= 3");
  if (prec < LBM_FP64 || prec > LBM_BF16S) return fail(LBM_ERR_PARAM, "prec must be an lbm_precision");
  const long long pitch = ((long long)nx + 31) / 32 * 32;
  if (pitch * (long long)ny > INT_MAX)
    return fail(LBM_ERR_PARAM, "lattice larger than the library's maximum (pitch * ny must fit in int32)");
  if (((uintptr_t)state) % 16 != 0) return fail(LBM_ERR_PARAM, "state must be 16-byte aligned");
  if (lbmch::reduce_partials_bytes() > sizeof(double) * 4 * kMaxBlocks)
    return fail(LBM_ERR_PARAM, "reduction needs more partials than the static scratch holds");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_PARAM, "device ordinal beyond 63");
  double* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the device address of the array.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_totals_scratch);
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }

  lbmch::HostGeometry g;
  g.nx = nx;
  g.ny = ny;
  g.pitch = (int)pitch;
  g.plane = pitch * ny;
  g.walls = 0;
  cudaStream_t s = (cudaStream_t)stream;
  // Every block writes its own partials before the final pass reads them, so nothing in the
  // array has to start at zero.
  e = lbmch::launch_reduce(prec, g, (const char*)state, scratch, scratch + 4 * kMaxBlocks, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(totals, scratch + 4 * kMaxBlocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"
