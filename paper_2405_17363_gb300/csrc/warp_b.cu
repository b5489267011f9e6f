// Instantiations of the warp-packed kernel for E = 5 6 7 8 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_WARP_DEFINE(5)
CAMP_WARP_DEFINE(6)
CAMP_WARP_DEFINE(7)
CAMP_WARP_DEFINE(8)
}  // namespace camp
