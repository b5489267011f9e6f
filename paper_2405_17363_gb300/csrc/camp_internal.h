// Internal declarations shared by the host layer and the kernel translation
// units of the batched BiCGSTAB library.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "camp_solver.h"

namespace camp {

// SpMV schedule slot (see build_schedule in solver.cu), laid out
// [slot j][lane-in-cell sl] so a cell's lanes read consecutive words:
//   col (bits 0-10) | row (bits 11-21) | end (bit 31): the slot multiplies the
//   gathered vector's entry col; on the last slot of a row (end) the running
//   sum is stored to row.  Alongside, src[j][sl] is the entry of the cell's
//   A row (pattern order) that slot uses, or -1 for padding: each cell's A is
//   staged in slot order, so lanes read consecutive shared-memory words.
typedef unsigned int SchedWord;
constexpr unsigned kSlotEnd = 0x80000000u;
// Bytes the plain launches reserve at the start of dynamic shared memory for
// nsch schedule words (rounded to 16); the host sizes the allocation and the
// kernels place their per-warp regions with this one function.
__host__ __device__ inline size_t sched_smem_bytes(int nsch) {
  return (((size_t)nsch * sizeof(SchedWord)) + 15) & ~(size_t)15;
}

// Arguments of the warp-packed kernel: Lc lanes per cell, k = 32/Lc cells per
// warp ("segments"), E rows per lane (template), one group of k consecutive
// cells per warp at a time.
struct WarpArgs {
  int cells, n, nnz;
  int Lc, log2Lc, k;       // lanes per cell, log2, cells per warp
  int L;                   // schedule slots per lane
  int segA, segV;          // shared-memory doubles per cell: A block, one vector
  int segStride;           // doubles from one cell's block to the next (bank-spread)
  int ngroups;             // ceil(cells / k)
  const double *A, *b;     // [cells x nnz], [cells x n]
  double *x;               // [cells x n]
  int *iters;              // [cells]
  double *resid;           // [cells]
  int *status;             // [cells] or null
  const SchedWord *sched;  // [L x Lc] slot words
  const int *src;          // [L x Lc] A entry of each slot (transposed view: permuted), -1 pad
  const int *dst;          // [nnz] slot of each A entry (pattern order): inverse of src
  const int *padfrom;      // [Lc] first padding slot of each lane
  const int *dslot;        // [n] slot of each row's diagonal entry
  // Single-cell tickets (the plain launch at 16 lanes per cell): tickets t <
  // single_from solve the pair at positions 2t, 2t+1; tickets t >= single_from
  // solve the one cell at position 2 * single_from + (t - single_from) with
  // all 32 lanes, bit for bit as its pair would (split schedule below: each
  // 16-lane lane's rows divided between lanes v and v + 16, every row's
  // entries in the same order).  No single tickets when sched2 is null or
  // single_from >= ngroups.
  int single_from;
  int L2;                  // slots per lane of the split schedule
  const SchedWord *sched2; // [L2 x 32]
  const int *dst2;         // [nnz] split slot of each A entry
  const int *padfrom2;     // [32] first padding slot of each lane
  const int *dslot2;       // [n] split slot of each row's diagonal entry
  double tol;
  int maxit;
  int x0_given;
  // Optional dynamic queue for the plain launch: [0] next group, [1] warps
  // finished.  The last warp to finish resets both to zero, so the pair is
  // ready for the next launch in stream order.  Null: static assignment.
  unsigned int *queue;
  // Optional cell order: group g's segment s solves cell order[g*k + s]
  // (cells sorted by an estimate of their iteration count), or null.  With
  // an order, each SM should get a mix of hard and easy groups in the first
  // wave.  ord_stride 0: every warp first solves group w*B + b (b its CTA
  // of B, w its warp in the CTA; b reversed for odd w), so each CTA, hence
  // each SM, takes one group from every stratum of B groups; the queue's
  // tickets then take groups ord_wave + t (ord_wave = all warps of the grid)
  // in order.  ord_stride > 0 (fewer groups than warps): ticket t takes
  // group (t * ord_stride) mod ord_wave (ord_wave = ngroups, ord_stride
  // coprime with it), so tickets taken together get mixed difficulty.
  const int *order;
  int ord_wave, ord_stride;
  // In-launch difficulty ordering (plain solve only; ord_ws null: off).  The
  // launch is cooperative: every CTA first classifies a contiguous share of
  // the cells by the largest |A_ii - 1| over the diagonal entries at pattern
  // positions ord_rows[0 .. ord_nrows) (the whole diagonal, or the rows where
  // the estimate peaked before), then, through two grid barriers, writes the
  // hardest-first order to ord_out (= order) before any warp solves.
  // ord_ws: kOrdWords ints (class totals, the barrier counter, the
  // time-out flag), zero on entry and cleared by the launch's last warp;
  // ord_cls: [cells] class | rank << 6 words; ord_hits (or null): per
  // sampled row, the CTAs whose hardest cell peaked there; ord_err: a
  // host-mapped word set to 1 (and left set for the host to read) when a
  // bounded wait ran out; ord_wait: the limit of every wait, in SM clock
  // cycles.  After a time-out the launch's last warp marks every cell of the
  // launch CAMP_CELL_INVALID (resid NaN) and clears the order entries.
  int *ord_out;
  int *ord_ws;
  int *ord_cls;
  const int *ord_rows;
  int ord_nrows;
  unsigned *ord_hits;
  int *ord_err;
  long long ord_wait;
  // Fused assembly (assemble_bicgstab_kernel only): the cell's matrix is
  // built in shared memory as A = I - gamma J(conc) instead of read from A.
  // Lane sl runs tcount terms p: J[slot (tmeta >> 11) * Lc + sl] +=
  // tval * (conc[(tmeta & 0x7ff) - 1] or 1 when that field is 0); arrays
  // are laid out [p][lane], padding terms add zero.
  const double *conc;      // [cells x n]
  const double *gamma;     // [cells]
  const double *tval;      // [tcount x Lc] sign * rate constant
  const int *tmeta;        // [tcount x Lc] species + 1 | slot row << 11
  int tcount;
  // Newton corrector (newton_bicgstab_kernel only): lane sl accumulates
  // f[row sl + e*Lc] += rval * y[a] * (y[b] or 1) over its rcount terms,
  // rmeta = (a + 1) | (b + 1) << 11 | e << 22 ([p][lane]); the history term
  // is read from b, y (in: initial guess, out: solution) from x, the linear
  // tolerance and iteration cap from tol and maxit.
  const double *rval;
  const int *rmeta;
  int rcount;
  double newton_tol;
  int max_newton;
  int *newton_iters;       // [cells]
  double *upd;             // [cells] final ||d|| / ||y||
};

// Persistent launch over up to kMaxMech mechanisms: mechanism m owns work
// items [item_begin[m], item_begin[m+1]) (one item = one group of
// 32/m[m].Lc cells); counter is the queue head (reset to 0 before launch).
constexpr int kMaxMech = 8;
struct BatchArgs {
  int nmech;
  int total_items;
  int item_begin[kMaxMech + 1];
  int warp_doubles;            // shared-memory doubles per warp
  unsigned int *counter;
  WarpArgs m[kMaxMech];        // schedules in global memory
};

// Arguments of the block kernel (the paper's Block-cells(k) arrangement):
// cpb cells per CTA, one thread per row, rows of cell j at threads [j*n, j*n+n).
struct BlockArgs {
  int cells, n, nnz, cpb;
  const double *A, *b;
  double *x;
  int *iters;
  double *resid;
  int *status;
  const int *a_perm;
  const int *diag;
  const int *row_ptr, *col_idx;  // the view's CSR
  double tol;
  int maxit;
  int x0_given;
  int coupled;  // 1: the block's cells form one system (shared scalars, one test)
};

// per-cell grad kernel arguments
struct GradArgs {
  int cells, n, nnz;
  const int *row_of;   // [nnz] row index of entry k
  const int *col_idx;  // [nnz]
  const double *lambda, *x;
  double *gA;
};

// Launchers (each returns the launch error, cudaSuccess on success).
// plain solve; a cooperative launch when a.ord_ws is set (grid must then be
// co-resident: at most SMs x the occupancy of the launch shape)
cudaError_t launch_warp(int E, const WarpArgs &a, int warps_per_block,
                        int grid, size_t smem, cudaStream_t st);
cudaError_t warp_set_smem(int E, size_t smem);
cudaError_t warp_occupancy(int E, int warps_per_block, size_t smem, int *blocks);
// persistent batch kernel: E in {3,4,5,6,8}, A staged in shared memory or not
const void *batch_kernel(int E, bool a_smem);
cudaError_t batch_prepare(int E, bool a_smem, int warps_per_block, size_t smem,
                          int *blocks_per_sm);
cudaError_t launch_block(const BlockArgs &a, int threads, size_t smem,
                         cudaStream_t st);
cudaError_t block_set_smem(size_t smem);
// fused-assembly solve, E in 1..8
cudaError_t launch_assemble(int E, const WarpArgs &a, int warps_per_block,
                            int grid, size_t smem, cudaStream_t st);
cudaError_t assemble_occupancy(int E, int warps_per_block, size_t smem, int *blocks);
// device Newton corrector around the fused assembly + solve, E in 1..8
cudaError_t launch_newton(int E, const WarpArgs &a, int warps_per_block,
                          int grid, size_t smem, cudaStream_t st);
cudaError_t newton_occupancy(int E, int warps_per_block, size_t smem, int *blocks);
cudaError_t launch_grad(const GradArgs &a, cudaStream_t st);
// Difficulty ordering: cells binned by decreasing max_i |A_ii - 1| (half
// octaves), written to *order (inside the caller's scratch of
// difficulty_scratch_bytes(cells) bytes).
size_t difficulty_scratch_bytes(int cells);
cudaError_t launch_difficulty_order(const double *A, int cells, int n, int nnz,
                                    const int *diag, void *scratch, int **order,
                                    cudaStream_t st);

// Difficulty ordering of a persistent multi-mechanism batch (order.cu): one
// classify and one scatter launch over the concatenated cells of all
// mechanisms (cell_begin: offsets, cell_begin[nmech] = total); counts holds
// per mechanism kOrdClasses totals then kOrdClasses cursors (zero on entry);
// order + cell_begin[m] receives mechanism m's cells, hardest class first.
struct BatchOrderArgs {
  int nmech;
  const double *A[kMaxMech];
  const int *diag[kMaxMech];
  int n[kMaxMech], nnz[kMaxMech];
  int cell_begin[kMaxMech + 1];
  unsigned char *cls;
  int *counts;
  int *order;
};
const void *batch_classify_kernel_fn();  // __global__ (const BatchOrderArgs)
const void *batch_scatter_kernel_fn();   // __global__ (const BatchOrderArgs), 1 thread per cell

constexpr int kMaxE = 16;  // rows per lane supported by the warp kernel

// Difficulty classes of the ordering (half octaves of max_i |A_ii - 1|) and
// the in-launch ordering's workspace: class totals, one barrier counter
// (word kOrdClasses) and one time-out flag (word kOrdFlag).
constexpr int kOrdClasses = 64;
constexpr int kOrdFlag = kOrdClasses + 1;
constexpr int kOrdWords = kOrdClasses + 2;
// Default limit of the in-launch ordering's waits (SM clock cycles, about a
// second at 2 GHz; a legitimate wait is microseconds).
constexpr long long kOrdWaitCycles = 1ll << 31;
// Cells one CTA classifies per pass of the in-launch ordering, and the
// shared-memory bytes that ordering borrows from the CTA's warp regions
// before they are used: histogram, class bases, the CTA's hardest key, and
// one 64-bit (estimate, row) key per cell of a pass.
constexpr int kOrdPiece = 256;
constexpr size_t kOrdKeyOffset = (2 * kOrdClasses + 4) * sizeof(int);
constexpr size_t kOrdSmemBytes = kOrdKeyOffset + kOrdPiece * sizeof(unsigned long long);
// Rows the ordering samples once it has seen where the estimate peaks, and
// how often (in ordered solves) it reads the whole diagonal again to re-pick.
constexpr int kOrdSample = 8;
constexpr unsigned kOrdRecalibrate = 64;
constexpr int kOrdBatch = 8;  // diagonal loads a thread keeps in flight

// Raise a kernel's dynamic shared-memory limit to the device maximum once per
// (kernel, device): setting the attribute on every launch serialises
// otherwise-concurrent work on some drivers.
cudaError_t ensure_max_smem(const void *kernel);
// Vectors of n (padded) doubles per cell in the warp kernel's shared memory
// for E rows per lane: the gathered vector and the two products; up to
// kRegVecMaxE rows per lane the shadow residual and the Jacobi reciprocals
// stay in registers (freeing shared memory for more resident warps), beyond
// it they take two more vectors.  The Newton launch adds one vector.
constexpr int kRegVecMaxE = 5;
__host__ __device__ constexpr int warp_vectors(int E) { return E <= kRegVecMaxE ? 3 : 5; }

}  // namespace camp

namespace camp {
// Arguments of the FP32-inner / FP64-outer refinement kernel (warp-packed
// layout as WarpArgs).
struct MixedArgs {
  int cells, n, nnz;
  int Lc, log2Lc, k, L;
  int segA, segV;
  int ngroups;
  const double *A, *b;
  double *x;
  int *iters;     // total inner FP32 iterations
  int *sweeps;    // outer sweeps (or null)
  double *resid;  // final FP64 true relative residual
  int *status;    // or null
  const SchedWord *sched;
  const int *src;
  const int *dst;
  const int *padfrom;
  const int *dslot;
  double tol;
  int max_sweeps;
  float tol_in;
  int maxit_in;
  int a64_smem;   // 1: FP64 A staged in shared memory; 0: read through L1 from A
  // dynamic group queue and difficulty ordering, as in WarpArgs
  unsigned int *queue;
  const int *order;
  int ord_wave, ord_stride;
  int *ord_out;
  int *ord_ws;
  int *ord_cls;
  const int *ord_rows;
  int ord_nrows;
  unsigned *ord_hits;
  int *ord_err;
  long long ord_wait;
};
// a cooperative launch when a.ord_ws is set (grid at most SMs x occupancy)
cudaError_t launch_mixed(int E, const MixedArgs &a, int warps_per_block,
                         int grid, size_t smem, cudaStream_t st);
cudaError_t mixed_occupancy(int E, int warps_per_block, size_t smem, int *blocks);
}  // namespace camp
