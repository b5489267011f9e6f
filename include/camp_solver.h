/*
 * camp_solver.h -- C ABI of the batched Jacobi-preconditioned BiCGSTAB solver
 * for the per-cell Newton systems of a stiff chemistry ODE step.
 *
 * Operation (the paper, Sec. 2.2 and Sec. 3.1): every grid cell c carries one
 * sparse linear system A_c x_c = b_c, A_c = I - gamma_c J_c, the matrix of the
 * Newton iteration inside the BDF step; all cells share one CSR sparsity
 * pattern and are independent of each other.  Each cell is solved on its own
 * inside one thread block or one warp, with its own convergence test and no
 * communication between cells (the paper's Block-cells strategy, Sec. 3.1 and
 * Sec. 3.2).  The iteration is BiCGSTAB with the Jacobi preconditioner
 * M = diag(A) applied on the right (the paper's "BCG" solver, Sec. 3.1; the
 * preconditioner is the one the paper leaves to future work, Sec. 5.2).
 *
 * Conventions shared by every entry point
 *  - Layout.  A_vals is cell-major [cells x nnz] in the order of the pattern
 *    given to camp_solver_create (row-major CSR, columns sorted); b, x and the
 *    adjoint vectors are [cells x n]; per-cell outputs are [cells].  All
 *    arrays are contiguous, FP64 unless stated, int32 for counts.
 *  - Ownership.  Array arguments are device pointers owned by the caller
 *    (except camp_solver_solve_host, which takes host pointers).  The solver
 *    handle owns only its device copies of the pattern, the transposed
 *    pattern, the SpMV schedules, its staging buffers and the cell-ordering
 *    workspace.
 *  - Streams.  Work is enqueued on the stream set with camp_solver_set_stream
 *    (default: the legacy default stream) and returns without waiting.  The
 *    solves of one handle share its device work queue and ordering state:
 *    calls on one handle must not overlap on the GPU or come from two host
 *    threads at once (keep them on one stream and one thread, or use one
 *    handle per stream); different handles are independent.
 *  - Errors.  A negative camp_status means nothing was enqueued (argument or
 *    pattern error) or the CUDA runtime reported an error; camp_last_error()
 *    gives a message.  Non-convergence of a cell is NOT an error: it shows in
 *    that cell's iters/resid/status and the call returns CAMP_OK.
 *  - Per-cell result.  x solves the cell to ||b - A x||_2 <= tol ||b||_2
 *    (status CAMP_CELL_CONVERGED) unless maxit iterations run out
 *    (CAMP_CELL_MAXIT), BiCGSTAB breaks down twice in a row
 *    (CAMP_CELL_BREAKDOWN) or a non-finite value appears
 *    (CAMP_CELL_NONFINITE).  resid_out is the true relative residual
 *    ||b - A x||_2 / ||b||_2 of the returned x; iters_out counts products
 *    v = A p^ (one per BiCGSTAB iteration, half-step exits included).
 *    b == 0 gives x = 0, 0 iterations, resid 0.
 */
#ifndef CAMP_SOLVER_H
#define CAMP_SOLVER_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct camp_solver *camp_solver_t;
typedef struct camp_batch *camp_batch_t;

typedef enum {
  CAMP_OK = 0,
  CAMP_EINVAL = -1,      /* bad argument (null pointer, size, tol, maxit) */
  CAMP_ECUDA = -2,       /* CUDA runtime error; see camp_last_error() */
  CAMP_ENOMEM = -3,      /* device or host allocation failed */
  CAMP_EPATTERN = -4,    /* invalid CSR pattern */
  CAMP_EUNSUPPORTED = -5 /* size outside what the kernels support */
} camp_status;

enum {
  CAMP_CELL_CONVERGED = 0,
  CAMP_CELL_MAXIT = 1,
  CAMP_CELL_BREAKDOWN = 2,
  CAMP_CELL_NONFINITE = 3,
  /* the launch that solved this cell was ordered in-launch and one of its
   * bounded waits ran out (camp_solver_set_ordering): x and iters are not
   * valid, resid is NaN; solve again */
  CAMP_CELL_INVALID = 4
};

/* flags for camp_solver_solve_ex */
enum {
  CAMP_TRANSPOSE = 1, /* solve A^T x = b (through the transposed pattern) */
  CAMP_X0_GIVEN = 2   /* x holds the initial guess on entry (default x0 = 0) */
};

/* arrangements (camp_solver_set_arrangement); see the Sec. 3.2 configurations */
enum {
  CAMP_ARR_AUTO = 0,  /* library choice (tuned table or heuristic) */
  CAMP_ARR_WARP = 1,  /* 32/lanes_per_cell cells per warp, one warp per group */
  CAMP_ARR_BLOCK = 2, /* cells_per_block cells per CTA, one thread per row */
  CAMP_ARR_BLOCK_COUPLED = 3 /* as BLOCK, but the CTA's cells form one system */
};

/*
 * Create a solver for one sparsity pattern (the pattern shared by all cells,
 * Sec. 3.1).  row_ptr [n+1] and col_idx [nnz] are HOST arrays, copied.
 * Requirements: 1 <= n <= 1024, n <= nnz <= 65535, row_ptr[0] = 0,
 * row_ptr[n] = nnz, nondecreasing; columns in [0, n) strictly increasing
 * within a row; every diagonal entry present.  Otherwise CAMP_EPATTERN (or
 * CAMP_EINVAL for null pointers / sizes).  Allocates device memory on the
 * current device.
 */
camp_status camp_solver_create(camp_solver_t *out, int n, int nnz,
                               const int *row_ptr, const int *col_idx);

/* Free the handle and its device memory (synchronises its stream first). */
camp_status camp_solver_destroy(camp_solver_t h);

/* Stream for subsequent calls: a cudaStream_t passed as void* (NULL = legacy
 * default stream). */
camp_status camp_solver_set_stream(camp_solver_t h, void *stream);

/*
 * Override the thread arrangement (Sec. 3.2, Table GPU1).
 *   CAMP_ARR_WARP : lanes_per_cell in {1,2,4,8,16,32} lanes solve one cell,
 *                   32/lanes_per_cell cells share a warp; warps_per_block
 *                   warps per CTA (0 = library default).
 *                   lanes_per_cell = 32 is "warp per cell".
 *   CAMP_ARR_BLOCK: cells_per_block cells per CTA with one thread per row
 *                   (cells_per_block = 1 is the paper's Block-cells(1)).
 *   CAMP_ARR_BLOCK_COUPLED: the paper's Block-cells(k) semantics (Sec. 3.2):
 *                   the cells of a CTA share the BiCGSTAB scalars and one
 *                   convergence test, i.e. they are solved as one
 *                   block-diagonal system; tol applies to the block's
 *                   combined residual ||b - A x|| / ||b||, and iters, resid
 *                   and status are the block's, written to each of its
 *                   cells.  Cells are grouped in index order, cells_per_block
 *                   per CTA (the last CTA takes the remainder).
 *   CAMP_ARR_AUTO : library choice.
 * With 16 lanes per cell (the automatic choice for 33 to 80 species), a
 * launch whose pairs would keep at most a quarter of the GPU's resident warps
 * busy solves each cell alone on a warp instead, on a split of the 16-lane
 * layout that performs the same operations in the same order: the results
 * are bit for bit those of the pair solve, and a small batch finishes about
 * a fifth sooner.
 * Unused arguments are ignored.  Returns CAMP_EINVAL for unsupported values.
 */
camp_status camp_solver_set_arrangement(camp_solver_t h, int arrangement,
                                        int lanes_per_cell, int cells_per_block,
                                        int warps_per_block);

/*
 * Cell ordering for the warp arrangement (Sec. 3.2: the cells that share a
 * warp run in lockstep, so pairing cells of similar difficulty wastes fewer
 * lanes).  The difficulty estimate of a cell is the largest departure of a
 * diagonal entry from one, max_i |A_ii - 1| (for A = I - gamma J: gamma
 * times the largest loss rate), binned on half octaves; cells are paired
 * and handed to warps hardest first, and an ordered launch gives every warp
 * of its first wave one group from each difficulty stratum so that every SM
 * gets a mix.  Results are bitwise identical in every mode (a cell's solve
 * does not depend on its neighbours).
 *   0: index order.
 *   1 (default): the solve launch orders the cells itself (a cooperative
 *      launch: every CTA classifies a share of the cells, one grid barrier,
 *      then each warp waits for its group's order entries).  The estimate
 *      reads the whole diagonal on the handle's first ordered solve and every
 *      64th; in between only the (up to 8) rows where it peaked, picked on
 *      the host from the counts of that full read (copied back without
 *      blocking).  Device scratch: 8 bytes per cell plus 4 per row.
 *      Solves on other streams (camp_solver_solve_host's chunks) use index
 *      order; launches whose warp regions cannot lend the ordering 2,576
 *      bytes of shared memory, or whose cooperative launch the GPU refuses
 *      (fewer SMs available than its occupancy query counts), use mode 2.  Under stream capture the
 *      last picked rows are used as they are (allocate first: run one solve
 *      before capturing).  Every wait of the launch is bounded (about a
 *      second).  If one runs out, the same launch marks every cell of the
 *      call CAMP_CELL_INVALID (when status_out is given) with resid NaN,
 *      and leaves the handle's ordering state clean, so the next call runs
 *      normally; camp_solver_get_fault reports it without synchronising.
 *   2: a separate classify and scatter pass (a memset and two small
 *      launches before the solve; about 5 bytes of scratch per cell).
 * The fused launches (camp_solver_assemble_solve, camp_solver_newton_solve)
 * have no matrix before a cell is assembled: in modes 1 and 2 they order
 * inside the launch, as mode 1 does, by |gamma[c]| on the same half-octave
 * classes (gamma scales every off-identity entry of A = I - gamma J), with
 * the same bounded waits, time-out report and scratch (8 bytes per cell); a
 * refused cooperative launch runs them in index order.
 */
camp_status camp_solver_set_ordering(camp_solver_t h, int ordering);

/*
 * Whether a bounded wait of an in-launch ordering (ordering mode 1 of the
 * plain FP64 solve and the FP32-inner refinement; modes 1 and 2 of the fused
 * assembly and Newton launches) ran out in any launch of
 * this handle since the previous query: *ordering_timed_out = 1 (and the
 * report is cleared) or 0.  Reads a host-mapped word the GPU sets; it does
 * not synchronise, so it covers only launches that have completed (call it
 * after the stream has been synchronised, as one does before reading the
 * results).  The cells of such a launch carry CAMP_CELL_INVALID.
 * CAMP_EINVAL for a null argument.
 */
camp_status camp_solver_get_fault(camp_solver_t h, int *ordering_timed_out);

/*
 * Solve all cells: A_vals [cells x nnz], b [cells x n] in; x [cells x n],
 * iters_out [cells] (int32), resid_out [cells] out.  Device pointers.
 * tol > 0, maxit >= 1, cells >= 0 (0 enqueues nothing).
 * The solve of each cell follows Sec. 3.1 (one cell per block/warp, no
 * inter-cell communication, convergence decided on the device).
 */
camp_status camp_solver_solve(camp_solver_t h, int cells, const double *A_vals,
                              const double *b, double *x, double tol,
                              int maxit, int *iters_out, double *resid_out);

/*
 * As camp_solver_solve, plus: status_out [cells] (int32, may be NULL) and
 * flags (CAMP_TRANSPOSE, CAMP_X0_GIVEN).  With CAMP_TRANSPOSE the same
 * A_vals (forward pattern order) are used and A^T x = b is solved; this is
 * the adjoint solve of the gradient below.
 */
camp_status camp_solver_solve_ex(camp_solver_t h, int cells,
                                 const double *A_vals, const double *b,
                                 double *x, double tol, int maxit,
                                 int *iters_out, double *resid_out,
                                 int *status_out, int flags);

/*
 * Gradient of a loss L with respect to the matrix values, given the adjoint
 * lambda = A^{-T} dL/dx and the solution x:
 *   gA[c, k] = -lambda[c, row(k)] * x[c, col(k)]   for every pattern entry k.
 * lambda, x [cells x n] and gA [cells x nnz] are device pointers.
 * (dL/db = lambda needs no kernel.)
 */
camp_status camp_solver_grad_A(camp_solver_t h, int cells,
                               const double *lambda, const double *x,
                               double *gA);

/*
 * End-to-end solve from HOST memory: copies b and then A_vals to the device
 * (A in chunks of shrinking size), solves each chunk while the next one is
 * copied, and returns after every result is in host memory.  When x,
 * iters_out, resid_out (and status_out) are device-addressable host memory
 * (page-locked/mapped), the kernels write them in place; otherwise results
 * are staged on the device and copied back per chunk.  Host arrays should be
 * page-locked for full speed (pageable memory works but the copies are
 * synchronous).  status_out may be NULL.  Device staging buffers are owned by
 * the handle and grow on demand.  The call synchronizes with its own copy
 * and solve streams only.
 */
camp_status camp_solver_solve_host(camp_solver_t h, int cells,
                                   const double *A_vals, const double *b,
                                   double *x, double tol, int maxit,
                                   int *iters_out, double *resid_out,
                                   int *status_out);

/*
 * Mixed precision (iterative refinement): FP64 outer sweeps r = b - A x,
 * stop when ||r|| <= tol ||b||, else an FP32 BiCGSTAB solve of A d = r/||r||
 * (FP32 copy of A, FP32 Jacobi) to relative tolerance tol_inner or maxit_inner
 * iterations, then x += ||r|| d in FP64; at most max_sweeps sweeps (status
 * CAMP_CELL_MAXIT after that).  iters_out = total FP32 inner iterations,
 * sweeps_out [cells] (int32, may be NULL) = outer sweeps that ran an inner
 * solve; resid_out = final FP64 true relative residual.  Device pointers.
 * The handle's cell ordering (camp_solver_set_ordering) applies when several
 * cells share a warp (at most 48 species with the automatic arrangement);
 * results do not depend on it.
 */
camp_status camp_solver_solve_mixed(camp_solver_t h, int cells,
                                    const double *A_vals, const double *b,
                                    double *x, double tol, int max_sweeps,
                                    double tol_inner, int maxit_inner,
                                    int *iters_out, int *sweeps_out,
                                    double *resid_out, int *status_out);

/*
 * Uneven batching: one persistent launch solves the cells of up to 8
 * mechanisms (patterns of different sizes) together.  Each warp takes work
 * items -- one group of 32/lanes cells of one mechanism -- from a device
 * queue head (an atomic counter, reset by the same CUDA graph that launches
 * the kernel) until the queue is empty; mechanisms with more species are
 * queued first.  The solve of every cell is the one of camp_solver_solve.
 * mechs [nmech] are existing solver handles (not owned; they must outlive the
 * batch).  Allocates the 4-byte queue head on the device.
 */
camp_status camp_batch_create(camp_batch_t *out, int nmech,
                              const camp_solver_t *mechs);
camp_status camp_batch_destroy(camp_batch_t b);
camp_status camp_batch_set_stream(camp_batch_t b, void *stream);

/*
 * Launch configuration of the batch (the autotuner's knobs; 0 = automatic):
 * rows_per_lane in {3, 4, 5, 6, 8} fixes the lanes per cell of every
 * mechanism (fewest lanes with at most that many rows per lane), so the cells
 * per warp; warps_per_block in [1, 8]; stage_A_in_smem = 1 copies each cell's
 * matrix values to shared memory, 0 reads them through L1.
 */
camp_status camp_batch_set_config(camp_batch_t b, int rows_per_lane,
                                  int warps_per_block, int stage_A_in_smem);

/*
 * Cell ordering of the batch (the cells that share a warp run in lockstep):
 * 1 (default) hands each mechanism's cells to warps hardest first, by the
 * same difficulty estimate and classes as camp_solver_set_ordering (a
 * classify and a scatter launch over all mechanisms, part of the batch's
 * graph; device scratch of 5 bytes per cell plus 512 bytes per mechanism);
 * 0 keeps index order.  Results are bitwise the same either way.
 * CAMP_EINVAL for other values.
 */
camp_status camp_batch_set_ordering(camp_batch_t b, int ordering);

/*
 * Solve cells[m] cells of every mechanism m in one launch (captured once in a
 * CUDA graph and replayed; a change of launch shape re-captures it).  The
 * arrays are HOST arrays [nmech] of DEVICE pointers with the layouts of
 * camp_solver_solve; status_out may be NULL (or hold NULL entries).
 * Asynchronous on the batch's stream.
 */
camp_status camp_batch_solve(camp_batch_t b, const int *cells,
                             const double *const *A_vals,
                             const double *const *bvec, double *const *x,
                             double tol, int maxit, int *const *iters_out,
                             double *const *resid_out, int *const *status_out);

/*
 * Solve without allocating device memory (the paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc -- for example a
 * host model whose device memory all comes from its own pool, or a time loop
 * that must not allocate once it runs).  It needs no solver handle: the
 * pattern (row_ptr [n+1], col_idx [nnz]) is a HOST array as for
 * camp_solver_create, the other arrays are DEVICE pointers with the layouts
 * and meaning of camp_solver_solve_ex (status_out may be NULL), and the solve
 * of every cell is that of camp_solver_solve with the automatic arrangement.
 * The SpMV schedule and the diagonal positions, which a handle keeps in
 * device memory of its own, are staged instead into one static device array
 * of 256 KiB inside the library, which every GPU that loads the library holds
 * until the process exits; a pattern whose schedule and diagonal positions do
 * not fit returns CAMP_EUNSUPPORTED before any work is enqueued, as does
 * n > 512.  No cudaMalloc, cudaFree or other allocating routine is called.
 *  - The first call on a device performs a one-time set-up with that device
 *    current (it looks up the device address of the static array); make that
 *    first call before any stream capture.
 *  - Every call shares the one static array and overwrites it (it keeps the
 *    last call's schedule; nothing in it needs to start at zero).  Calls whose
 *    work overlaps on the GPU -- on different streams, or from different host
 *    threads -- race on it: order them on one stream.
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream): four host-to-device copies from host buffers inside the
 *    library (the diagonal slots, the first padding slot of every lane, the
 *    slot of every entry and the slot words), then the kernel.  The copies
 *    read pageable host memory, so a call may wait on the host until earlier
 *    work on the stream has finished.
 *  - While `stream` is capturing a CUDA graph the call returns
 *    CAMP_EUNSUPPORTED and enqueues nothing: a captured copy would read the
 *    library's host buffers when the graph is replayed, after later calls
 *    may have overwritten them.
 *  - The set-up's device address is kept until the process exits: after a
 *    cudaDeviceReset of a device, do not call this entry point on it again.
 */
camp_status camp_solve_noalloc(int n, int nnz, const int *row_ptr,
                               const int *col_idx, int cells,
                               const double *A_vals, const double *b,
                               double *x, double tol, int maxit,
                               int *iters_out, double *resid_out,
                               int *status_out, void *stream);

/*
 * Inspect the static SpMV schedule the warp-packed kernels use for a pattern
 * (host only, no GPU needed).  The rows are assigned whole to lanes_per_cell
 * lanes by longest-first bin packing; each lane runs slots_per_lane slots.
 * words (host, may be NULL to query slots_per_lane only) receives
 * slots_per_lane * lanes_per_cell slots laid out [slot][lane], two uint32 per
 * slot: word0 = the entry k (pattern order) whose value the slot multiplies,
 * or 0xFFFFFFFF for a padding slot; word1 = column (bits 0-10) | row
 * (bits 11-21) | 1 << 31 on the last entry of a row (store the running sum to
 * that row).  Padding slots contribute zero.  The kernels stage each cell's
 * matrix values in this slot order.  capacity_slots is the number of slots
 * words can hold.  Pattern requirements as for camp_solver_create.
 */
camp_status camp_schedule_build(int n, int nnz, const int *row_ptr,
                                const int *col_idx, int lanes_per_cell,
                                unsigned *words, int capacity_slots,
                                int *slots_per_lane);

/*
 * Fused Jacobian assembly.  The matrix of each cell is the Newton matrix of
 * the BDF step, A = I - gamma J, J the Jacobian of the species rates
 * f_i = sum_j (dy_i/dt)_j of the mechanism (Sec. 2.2).  For a mass-action
 * mechanism the kernel can build A for every cell in shared memory from the
 * cell's concentrations instead of reading A_vals from HBM.
 *
 * camp_solver_set_mechanism attaches R reactions (HOST arrays [R]): reaction
 * r consumes reactant_a[r] and, when reactant_b[r] >= 0, reactant_b[r], and
 * produces product[r], at rate rate_k[r] y_a (first order, reactant_b = -1)
 * or rate_k[r] y_a y_b (second order); rate constants are shared by all
 * cells.  Every Jacobian entry the reactions create must be in the handle's
 * pattern (else CAMP_EPATTERN).  Replaces any earlier mechanism.
 *
 * camp_solver_assemble_solve then solves, for every cell,
 * (I - gamma[c] J(conc[c])) x = b[c] exactly as camp_solver_solve_ex would
 * with those matrix values: conc [cells x n], gamma [cells], b, x [cells x n],
 * iters_out, resid_out, status_out (may be NULL) [cells], device pointers.
 * At most 8 rows per lane of the warp arrangement (n <= 256).  Cells are
 * ordered by |gamma| inside the launch (camp_solver_set_ordering); after a
 * time-out of that ordering every cell carries resid NaN and (status_out
 * given) CAMP_CELL_INVALID.
 */
camp_status camp_solver_set_mechanism(camp_solver_t h, int R,
                                      const int *reactant_a,
                                      const int *reactant_b,
                                      const int *product,
                                      const double *rate_k);
camp_status camp_solver_assemble_solve(camp_solver_t h, int cells,
                                       const double *conc, const double *gamma,
                                       const double *b, double *x, double tol,
                                       int maxit, int *iters_out,
                                       double *resid_out, int *status_out);

/*
 * Device Newton corrector of one implicit (BDF) step per cell.  The systems
 * the paper solves are the Newton systems of CVODE's BDF step (Sec. 2.2,
 * A = I - gamma J); moving the loop around them onto the GPU is its future
 * work (Sec. 6).  For every cell c this solves G(y) = y - gamma[c] f(y) -
 * a_hist[c] = 0, f the mass-action rates of the mechanism set by
 * camp_solver_set_mechanism, by Newton's method from the initial guess in y:
 * each iteration evaluates f(y), assembles A = I - gamma[c] J(y) in shared
 * memory, solves A d = -G(y) with the Jacobi-BiCGSTAB of camp_solver_solve_ex
 * (lin_tol, lin_maxit, zero initial guess) and sets y += d; it stops when
 * ||d||_2 <= newton_tol ||y||_2 (||d||_2 <= newton_tol when y = 0), after
 * max_newton iterations, or when a linear solve does not converge.  One
 * kernel launch runs every iteration of every cell.
 *
 * a_hist, y [cells x n] row-major, gamma [cells]; y is read as the initial
 * guess and replaced by the last iterate.  newton_iters_out (iterations run),
 * lin_iters_out (BiCGSTAB iterations summed), upd_out (last ||d|| / ||y||),
 * resid_out (relative residual of the last linear solve) [cells] are
 * required; status_out [cells] may be NULL: 0 converged, 1 iterations
 * exhausted, 2 linear solve failed (y keeps the iterate before it),
 * 3 non-finite; CAMP_CELL_INVALID (with resid NaN) on every cell after a
 * time-out of the in-launch ordering by |gamma| (camp_solver_set_ordering).
 * All device pointers, written on the handle's stream.
 * CAMP_EINVAL for a non-positive or non-finite tolerance, max_newton < 0 or
 * lin_maxit < 1; CAMP_EUNSUPPORTED beyond 8 rows per lane (n <= 256).
 */
camp_status camp_solver_newton_solve(camp_solver_t h, int cells,
                                     const double *a_hist, const double *gamma,
                                     double *y, double newton_tol, int max_newton,
                                     double lin_tol, int lin_maxit,
                                     int *newton_iters_out, int *lin_iters_out,
                                     double *upd_out, double *resid_out,
                                     int *status_out);

/* Thread-local message describing the last error (never NULL). */
const char *camp_last_error(void);

/* Library version string. */
const char *camp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CAMP_SOLVER_H */
