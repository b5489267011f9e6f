// Instantiations of the FP32-inner refinement kernel for E = 1 2 3 4 5 6 7 8 rows per lane.
#include "mixed_kernel.cuh"
#include "mixed_launch.cuh"
namespace camp {
CAMP_MIXED_DEFINE(1)
CAMP_MIXED_DEFINE(2)
CAMP_MIXED_DEFINE(3)
CAMP_MIXED_DEFINE(4)
CAMP_MIXED_DEFINE(5)
CAMP_MIXED_DEFINE(6)
CAMP_MIXED_DEFINE(7)
CAMP_MIXED_DEFINE(8)
}  // namespace camp
