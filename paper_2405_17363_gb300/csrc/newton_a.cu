// Instantiations of the device Newton corrector (rates, fused assembly and solve per iteration)
// for E = 1 2 3 4 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 1)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 2)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 3)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 4)
}  // namespace camp
