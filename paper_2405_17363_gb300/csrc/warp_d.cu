// Instantiations of the warp-packed kernel for E = 13 14 15 16 rows per lane.
#include "warp_kernel.cuh"
#include "warp_launch.cuh"
namespace camp {
CAMP_WARP_DEFINE(13)
CAMP_WARP_DEFINE(14)
CAMP_WARP_DEFINE(15)
CAMP_WARP_DEFINE(16)
}  // namespace camp
