// Instantiations of the warp-packed kernel for E = 1 2 3 4 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_WARP_DEFINE(1)
CAMP_WARP_DEFINE(2)
CAMP_WARP_DEFINE(3)
CAMP_WARP_DEFINE(4)
}  // namespace camp
