// Instantiations of the warp-packed kernel for E = 9 10 11 12 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_WARP_DEFINE(9)
CAMP_WARP_DEFINE(10)
CAMP_WARP_DEFINE(11)
CAMP_WARP_DEFINE(12)
}  // namespace camp
