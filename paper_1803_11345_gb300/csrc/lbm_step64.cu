// Instantiations of the fused step for population buffers of 4 GiB or more (64-bit plane
// offsets); lbm_kernels.cu holds the 32-bit-offset variants used below that size.  A separate
// translation unit so that the two sets compile in parallel.
#include "lbm_step.cuh"

namespace lbmch {

namespace {

template <int PREC>
cudaError_t step64_prec(int bx, int by, const HostGeometry& g, const HostPhys& p, int rows, const char* src,
                        char* dst, int* flag, cudaStream_t s) {
#define LBM_CASE(X, Y) \
  if (bx == X && by == Y) return launch_k_step<PREC, X, Y, false>(g, p, rows, src, dst, flag, s);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

template <int PREC>
cudaError_t batch64_prec(int bx, int by, const BatchItem* items, int nitems, const BatchMember* members,
                         const void* phys, int parity, int* flags, long long* tcount, int grid, cudaStream_t s) {
#define LBM_CASE(X, Y)           \
  if (bx == X && by == Y)        \
    return launch_k_step_batch<PREC, X, Y, false>(items, nitems, members, phys, parity, flags, tcount, grid, s);
  LBM_TILES(LBM_CASE)
#undef LBM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step64(int prec, int bx, int by, const HostGeometry& g, const HostPhys& p, int rows,
                          const char* src, char* dst, int* flag, cudaStream_t s) {
  switch (prec) {
    case 0: return step64_prec<0>(bx, by, g, p, rows, src, dst, flag, s);
    case 1: return step64_prec<1>(bx, by, g, p, rows, src, dst, flag, s);
    case 2: return step64_prec<2>(bx, by, g, p, rows, src, dst, flag, s);
    case 3: return step64_prec<3>(bx, by, g, p, rows, src, dst, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_batch64(int prec, int bx, int by, const BatchItem* items, int nitems,
                                const BatchMember* members, const void* phys, int parity, int* flags,
                                long long* tcount, int grid, cudaStream_t s) {
  switch (prec) {
    case 0: return batch64_prec<0>(bx, by, items, nitems, members, phys, parity, flags, tcount, grid, s);
    case 1: return batch64_prec<1>(bx, by, items, nitems, members, phys, parity, flags, tcount, grid, s);
    case 2: return batch64_prec<2>(bx, by, items, nitems, members, phys, parity, flags, tcount, grid, s);
    case 3: return batch64_prec<3>(bx, by, items, nitems, members, phys, parity, flags, tcount, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbmch
