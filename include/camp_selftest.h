/*
 * camp_selftest.h -- self-test entry point of libcampsolve.
 *
 * Runs one numerical building block of the warp-packed kernels element-wise
 * on caller data (DEVICE pointers in [n], out [n], enqueued on `stream`), so
 * tests can compare it with exact references computed on the host:
 *   op 0: out = 1/in, Newton-Raphson from an FP32 seed, two steps (the Jacobi
 *         reciprocals; at most one rounding error on normal results);
 *   op 1: the same with one step (the iteration scalars; relative error about
 *         2^-44);
 *   op 2: out = the FP32 rounding of in (to nearest, ties to even) widened
 *         back, both on the integer pipe;
 *   op 3: out = the sum of in over each aligned group of `lanes` consecutive
 *         elements (the integer-pipe segment sum: every term aligned to the
 *         group's largest exponent with 5 guard bits, summed exactly, rounded
 *         once);
 *   op 4: the same sum by the FP64 shuffle tree;
 *   op 5: the op-3 sum with its reductions done by full-warp redux.sync
 *         (bit-identical to op 3 by construction);
 *   op 6: FP64 rate probe: each of n threads runs four independent chains
 *         of `lanes` dependent FMAs from in[i] and writes their sum to
 *         out[i] (4 * n * lanes DFMAs to time; lanes in [1, 2^20]).
 * For ops 3 to 5, n must be a multiple of 32 and lanes a power of two in
 * [1, 32].  Returns CAMP_EINVAL for bad arguments, CAMP_ECUDA if the launch
 * fails.  The paper has no counterpart: this is test support.
 */
#ifndef CAMP_SELFTEST_H
#define CAMP_SELFTEST_H
#include "camp_solver.h"
#ifdef __cplusplus
extern "C" {
#endif
camp_status camp_selftest(int op, int n, const double *in, double *out,
                          int lanes, void *stream);
#ifdef __cplusplus
}
#endif
#endif
