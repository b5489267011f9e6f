#pragma once
#include "camp_internal.h"
#define CAMP_MIXED_DEFINE(E)                                                    \
  cudaError_t launch_mixed_##E(const MixedArgs &a, int wpb, int grid,           \
                               size_t smem, cudaStream_t st) {                  \
    cudaError_t e = ensure_max_smem((const void *)mixed_refine_kernel<E>);      \
    if (e != cudaSuccess) return e;                                             \
    if (a.ord_ws) {                                                             \
      void *args[] = {(void *)&a};                                              \
      return cudaLaunchCooperativeKernel((const void *)mixed_refine_kernel<E>,  \
                                         dim3(grid), dim3(wpb * 32), args,      \
                                         smem, st);                             \
    }                                                                           \
    mixed_refine_kernel<E><<<grid, wpb * 32, smem, st>>>(a);                    \
    return cudaGetLastError();                                                  \
  }                                                                             \
  cudaError_t occ_mixed_##E(int wpb, size_t smem, int *blocks) {                \
    cudaError_t e = ensure_max_smem((const void *)mixed_refine_kernel<E>);      \
    if (e != cudaSuccess) return e;                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
        blocks, mixed_refine_kernel<E>, wpb * 32, smem);                        \
  }
