// Instantiations of the device Newton corrector (rates, fused assembly and solve per iteration)
// for E = 5 6 7 8 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 5)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 6)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 7)
CAMP_KERNEL_DEFINE(newton, newton_bicgstab_kernel, 8)
}  // namespace camp
