// Instantiations of the fused assembly + solve kernel
// for E = 1 2 3 4 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_KERNEL_DEFINE(assemble, assemble_bicgstab_kernel, 1)
CAMP_KERNEL_DEFINE(assemble, assemble_bicgstab_kernel, 2)
CAMP_KERNEL_DEFINE(assemble, assemble_bicgstab_kernel, 3)
CAMP_KERNEL_DEFINE(assemble, assemble_bicgstab_kernel, 4)
}  // namespace camp
