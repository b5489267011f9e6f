// Instantiations of the persistent batch kernel (E rows per lane in
// {3, 4, 5, 6, 8}; A staged in shared memory or read through L1).
#include "warp_kernel.cuh"

namespace camp {

template <int E, bool S>
static cudaError_t prep(int wpb, size_t smem, int *blocks) {
  cudaError_t e = ensure_max_smem((const void *)batch_bicgstab_kernel<E, S>);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks, batch_bicgstab_kernel<E, S>, wpb * 32, smem);
}

const void *batch_kernel(int E, bool s) {
  switch (E) {
    case 3: return s ? (const void *)batch_bicgstab_kernel<3, true> : (const void *)batch_bicgstab_kernel<3, false>;
    case 4: return s ? (const void *)batch_bicgstab_kernel<4, true> : (const void *)batch_bicgstab_kernel<4, false>;
    case 5: return s ? (const void *)batch_bicgstab_kernel<5, true> : (const void *)batch_bicgstab_kernel<5, false>;
    case 6: return s ? (const void *)batch_bicgstab_kernel<6, true> : (const void *)batch_bicgstab_kernel<6, false>;
    case 8: return s ? (const void *)batch_bicgstab_kernel<8, true> : (const void *)batch_bicgstab_kernel<8, false>;
    default: return nullptr;
  }
}

cudaError_t batch_prepare(int E, bool s, int wpb, size_t smem, int *blocks) {
  switch (E) {
    case 3: return s ? prep<3, true>(wpb, smem, blocks) : prep<3, false>(wpb, smem, blocks);
    case 4: return s ? prep<4, true>(wpb, smem, blocks) : prep<4, false>(wpb, smem, blocks);
    case 5: return s ? prep<5, true>(wpb, smem, blocks) : prep<5, false>(wpb, smem, blocks);
    case 6: return s ? prep<6, true>(wpb, smem, blocks) : prep<6, false>(wpb, smem, blocks);
    case 8: return s ? prep<8, true>(wpb, smem, blocks) : prep<8, false>(wpb, smem, blocks);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace camp
