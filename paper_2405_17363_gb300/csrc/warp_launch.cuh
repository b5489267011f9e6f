// Per-E launch and occupancy entry points of the warp-packed kernels
// (plain solve, fused assembly, Newton), defined in the instantiation units and
// dispatched from solver.cu.
#pragma once
#include "camp_internal.h"

// One launch and one occupancy function of a kernel template instance:
// launch_<name>_<E> and occ_<name>_<E>.
#define CAMP_KERNEL_DEFINE(name, kernel, E)                                     \
  cudaError_t launch_##name##_##E(const WarpArgs &a, int wpb, int grid,         \
                                  size_t smem, cudaStream_t st) {               \
    cudaError_t e = ensure_max_smem((const void *)kernel<E>);                   \
    if (e != cudaSuccess) return e;                                             \
    if (a.ord_ws) { /* in-launch ordering: every CTA resident */                \
      void *args[] = {(void *)&a};                                              \
      return cudaLaunchCooperativeKernel((const void *)kernel<E>, dim3(grid),   \
                                         dim3(wpb * 32), args, smem, st);       \
    }                                                                           \
    kernel<E><<<grid, wpb * 32, smem, st>>>(a);                                 \
    return cudaGetLastError();                                                  \
  }                                                                             \
  cudaError_t occ_##name##_##E(int wpb, size_t smem, int *blocks) {             \
    cudaError_t e = ensure_max_smem((const void *)kernel<E>);                   \
    if (e != cudaSuccess) return e;                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
        blocks, kernel<E>, wpb * 32, smem);                                     \
  }
// The plain solve launches cooperatively when it orders its cells itself
// (a.ord_ws set): its grid barriers need every CTA resident.
#define CAMP_WARP_DEFINE(E)                                                     \
  cudaError_t launch_warp_##E(const WarpArgs &a, int wpb, int grid,             \
                              size_t smem, cudaStream_t st) {                   \
    cudaError_t e = ensure_max_smem((const void *)warp_bicgstab_kernel<E>);     \
    if (e != cudaSuccess) return e;                                             \
    if (a.ord_ws) {                                                             \
      void *args[] = {(void *)&a};                                              \
      return cudaLaunchCooperativeKernel((const void *)warp_bicgstab_kernel<E>, \
                                         dim3(grid), dim3(wpb * 32), args,      \
                                         smem, st);                             \
    }                                                                           \
    warp_bicgstab_kernel<E><<<grid, wpb * 32, smem, st>>>(a);                   \
    return cudaGetLastError();                                                  \
  }                                                                             \
  cudaError_t occ_warp_##E(int wpb, size_t smem, int *blocks) {                 \
    cudaError_t e = ensure_max_smem((const void *)warp_bicgstab_kernel<E>);     \
    if (e != cudaSuccess) return e;                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
        blocks, warp_bicgstab_kernel<E>, wpb * 32, smem);                       \
  }
