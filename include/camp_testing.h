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

/*
 * Single-cell tickets of the plain warp-packed solve at 16 lanes per cell:
 * the launch may solve some cells one per warp on all 32 lanes (the end of a
 * large batch, where a lone warp's latency decides the launch's length, and
 * small batches), on a split schedule that keeps every operation of the pair
 * solve, so the results are bit for bit those of the pair solve.  pairs < 0:
 * the library's automatic choice (the default); 0: none; k > 0: the last k
 * pair tickets of every such launch become 2k single-cell tickets (at most
 * all of them).  Host setting only; nothing is enqueued.  CAMP_EINVAL for a
 * null handle.
 */
camp_status camp_solver_set_single_tail(camp_solver_t h, int pairs);

/*
 * The split schedule behind single-cell tickets (host only, no GPU), for a
 * pattern as camp_solver_create takes it: one cell on 32 lanes, lane v and
 * lane v + 16 taking the rows of lane v of the 16-lane schedule
 * (camp_schedule_build with lanes_per_cell 16), divided at a row boundary,
 * every row's slots in the same order.  Layout and arguments as
 * camp_schedule_build, with 32 lanes: words (may be NULL to query
 * slots_per_lane) receives slots_per_lane * 32 slots [slot][lane], two uint32
 * per slot (entry or 0xFFFFFFFF, then the slot word).  CAMP_EUNSUPPORTED
 * when the pattern's 16-lane schedule would use more than 5 rows per lane.
 */
camp_status camp_schedule_build_split(int n, int nnz, const int *row_ptr,
                                      const int *col_idx, unsigned *words,
                                      int capacity_slots, int *slots_per_lane);

#ifdef __cplusplus
}
#endif

#endif /* CAMP_TESTING_H */
