// Instantiations of the device Newton corrector (rates, fused assembly and
// solve per iteration) for E = 1..8 rows per lane.
#include "warp_kernel.cuh"

namespace camp {

template <int E>
static cudaError_t launch_e(const WarpArgs &a, int wpb, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = ensure_max_smem((const void *)newton_bicgstab_kernel<E>);
  if (e != cudaSuccess) return e;
  newton_bicgstab_kernel<E><<<grid, wpb * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int E>
static cudaError_t occ_e(int wpb, size_t smem, int *blocks) {
  cudaError_t e = ensure_max_smem((const void *)newton_bicgstab_kernel<E>);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, newton_bicgstab_kernel<E>,
                                                       wpb * 32, smem);
}

cudaError_t launch_newton(int E, const WarpArgs &a, int wpb, int grid, size_t smem,
                            cudaStream_t st) {
  switch (E) {
    case 1: return launch_e<1>(a, wpb, grid, smem, st);
    case 2: return launch_e<2>(a, wpb, grid, smem, st);
    case 3: return launch_e<3>(a, wpb, grid, smem, st);
    case 4: return launch_e<4>(a, wpb, grid, smem, st);
    case 5: return launch_e<5>(a, wpb, grid, smem, st);
    case 6: return launch_e<6>(a, wpb, grid, smem, st);
    case 7: return launch_e<7>(a, wpb, grid, smem, st);
    case 8: return launch_e<8>(a, wpb, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t newton_occupancy(int E, int wpb, size_t smem, int *blocks) {
  switch (E) {
    case 1: return occ_e<1>(wpb, smem, blocks);
    case 2: return occ_e<2>(wpb, smem, blocks);
    case 3: return occ_e<3>(wpb, smem, blocks);
    case 4: return occ_e<4>(wpb, smem, blocks);
    case 5: return occ_e<5>(wpb, smem, blocks);
    case 6: return occ_e<6>(wpb, smem, blocks);
    case 7: return occ_e<7>(wpb, smem, blocks);
    case 8: return occ_e<8>(wpb, smem, blocks);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace camp
