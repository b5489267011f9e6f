// Instantiations of the FP32-inner refinement kernel for E = 9 10 11 12 13 14 15 16 rows per lane.
#include "mixed_kernel.cuh"
#include "mixed_launch.cuh"
namespace camp {
CAMP_MIXED_DEFINE(9)
CAMP_MIXED_DEFINE(10)
CAMP_MIXED_DEFINE(11)
CAMP_MIXED_DEFINE(12)
CAMP_MIXED_DEFINE(13)
CAMP_MIXED_DEFINE(14)
CAMP_MIXED_DEFINE(15)
CAMP_MIXED_DEFINE(16)
}  // namespace camp
