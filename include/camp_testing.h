/*
 * camp_testing.h -- test hooks of libcampsolve.  Not for production use:
 * they exist so that tests can drive the rare paths of an ordered solve on
 * any GPU without faulting or hanging it.  The paper has no counterpart.
 */
#ifndef CAMP_TESTING_H
#define CAMP_TESTING_H

#include "camp_solver.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * ordering_wait_cycles: the limit (SM clock cycles) of every bounded wait of
 * the handle's in-launch ordering (the grid barrier and the per-group waits
 * for order entries); 0 restores the default of 2^31 cycles (about a
 * second).  A limit of a few cycles makes the waits run out, so a test can
 * check that the launch reports it (CAMP_CELL_INVALID,
 * camp_solver_get_fault) and that the next solve is correct.
 * refuse_cooperative != 0: every cooperative launch of the handle is treated
 * as refused (cudaErrorCooperativeLaunchTooLarge, as on a GPU that offers
 * fewer SMs than the occupancy query counts), so the solve takes its fallback
 * (the separate ordering pass).  Host settings only; nothing is enqueued.
 * CAMP_EINVAL for a null handle or a negative limit.
 */
camp_status camp_solver_set_test_hooks(camp_solver_t h, long long ordering_wait_cycles,
                                       int refuse_cooperative);

#ifdef __cplusplus
}
#endif

#endif /* CAMP_TESTING_H */
