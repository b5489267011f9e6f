// Per-E launch and occupancy entry points of the warp-packed kernel, defined
// in the instantiation units and dispatched from solver.cu.
#pragma once
#include "camp_internal.h"

#define CAMP_WARP_DEFINE(E)                                                     \
  cudaError_t launch_warp_##E(const WarpArgs &a, int wpb, int grid,             \
                              size_t smem, cudaStream_t st) {                   \
    cudaError_t e = ensure_max_smem((const void *)warp_bicgstab_kernel<E>);     \
    if (e != cudaSuccess) return e;                                             \
    warp_bicgstab_kernel<E><<<grid, wpb * 32, smem, st>>>(a);                   \
    return cudaGetLastError();                                                  \
  }                                                                             \
  cudaError_t occ_warp_##E(int wpb, size_t smem, int *blocks) {                 \
    cudaError_t e = ensure_max_smem((const void *)warp_bicgstab_kernel<E>);     \
    if (e != cudaSuccess) return e;                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
        blocks, warp_bicgstab_kernel<E>, wpb * 32, smem);                       \
  }
