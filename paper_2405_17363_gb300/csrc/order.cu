// Difficulty ordering of the cells for the warp-packed solve.  The cells that
// share a warp run in lockstep until the last one converges, so pairing cells
// of similar iteration counts wastes fewer lanes, and solving the hardest
// first shortens the end of the launch (the last groups are the short ones).
// The estimate is the largest departure of a diagonal entry from one,
// max_i |A_ii - 1|: for the step matrix I - gamma J it is gamma times the
// largest loss rate, the stiffness of the cell's step.  Only the diagonal is
// read (the sectors it touches stay in L2 for the solve).  Cells are binned
// on half octaves of the estimate (hardest bin first) by a counting sort:
// one launch classifies and counts, one scatters; the order inside a bin is
// arbitrary, since a cell's result does not depend on where it is solved.
#include "warp_common.cuh"

namespace camp {
namespace {

constexpr int kClasses = kOrdClasses;

__global__ void classify_kernel(const double *__restrict__ A, int cells, int n, int nnz,
                                const int *__restrict__ diag, unsigned char *__restrict__ cls,
                                int *__restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < cells; c += warps) {
    const double *Ac = A + (size_t)c * nnz;
    unsigned worst = 0;  // high word of max |A_ii - 1| (non-negative: ordered as integers)
    for (int i = lane; i < n; i += 32) {
      const unsigned hi = diag_departure_hi(__ldg(Ac + __ldg(diag + i)));
      worst = hi > worst ? hi : worst;
    }
    worst = __reduce_max_sync(kFull, worst);
    if (lane == 0) {
      const int k = difficulty_class(worst);
      cls[c] = (unsigned char)k;
      atomicAdd(counts + k, 1);
    }
  }
}

// counts[0..kClasses) per-class totals, counts[kClasses..) running cursors
__global__ void scatter_kernel(const unsigned char *__restrict__ cls, int cells,
                               int *__restrict__ counts, int *__restrict__ order) {
  __shared__ int start[kClasses];
  if (threadIdx.x < 32) {
    // exclusive prefix of the class totals, two classes per lane
    const int l = threadIdx.x;
    const int a = counts[2 * l], b = counts[2 * l + 1];
    int s = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, s, o);
      if (l >= o) s += t;
    }
    start[2 * l] = s - a - b;
    start[2 * l + 1] = s - b;
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cells) {
    const int k = cls[c];
    order[start[k] + atomicAdd(counts + kClasses + k, 1)] = c;
  }
}

// The same two steps for the persistent multi-mechanism batch, all
// mechanisms in one launch each: cell i of the concatenated cell space
// belongs to mechanism m with cell_begin[m] <= i < cell_begin[m + 1]; every
// mechanism has its own class totals and cursors (counts + m * 2 kClasses)
// and its own order (order + cell_begin[m], cell indices within m).
__global__ void batch_classify_kernel(const BatchOrderArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int total = a.cell_begin[a.nmech];
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < total; i += warps) {
    int m = 0;
    while (m + 1 < a.nmech && i >= a.cell_begin[m + 1]) ++m;
    const double *Ac = a.A[m] + (size_t)(i - a.cell_begin[m]) * a.nnz[m];
    unsigned worst = 0;
    for (int r = lane; r < a.n[m]; r += 32) {
      const unsigned hi = diag_departure_hi(__ldg(Ac + __ldg(a.diag[m] + r)));
      worst = hi > worst ? hi : worst;
    }
    worst = __reduce_max_sync(kFull, worst);
    if (lane == 0) {
      const int k = difficulty_class(worst);
      a.cls[i] = (unsigned char)k;
      atomicAdd(a.counts + m * 2 * kClasses + k, 1);
    }
  }
}

__global__ void batch_scatter_kernel(const BatchOrderArgs a) {
  __shared__ int start[kMaxMech][kClasses];
  for (int m = threadIdx.x >> 5; m < a.nmech; m += blockDim.x >> 5) {
    const int l = threadIdx.x & 31;
    const int *cnt = a.counts + m * 2 * kClasses;
    const int x = cnt[2 * l], y = cnt[2 * l + 1];
    int s = x + y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, s, o);
      if (l >= o) s += t;
    }
    start[m][2 * l] = s - x - y;
    start[m][2 * l + 1] = s - y;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.cell_begin[a.nmech]) {
    int m = 0;
    while (m + 1 < a.nmech && i >= a.cell_begin[m + 1]) ++m;
    const int k = a.cls[i];
    const int pos = start[m][k] + atomicAdd(a.counts + m * 2 * kClasses + kClasses + k, 1);
    a.order[a.cell_begin[m] + pos] = i - a.cell_begin[m];
  }
}

}  // namespace

const void *batch_classify_kernel_fn() { return (const void *)batch_classify_kernel; }
const void *batch_scatter_kernel_fn() { return (const void *)batch_scatter_kernel; }

size_t difficulty_scratch_bytes(int cells) {
  // class bytes (rounded to 16), the order, the class totals and cursors
  return (((size_t)cells + 15) & ~(size_t)15) + (size_t)cells * sizeof(int) +
         2 * kClasses * sizeof(int);
}

cudaError_t launch_difficulty_order(const double *A, int cells, int n, int nnz,
                                    const int *diag, void *scratch, int **order,
                                    cudaStream_t st) {
  unsigned char *cls = (unsigned char *)scratch;
  int *ord = (int *)(cls + (((size_t)cells + 15) & ~(size_t)15));
  int *counts = ord + cells;
  *order = ord;
  if (cells <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * kClasses * sizeof(int), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (cells * 32 + 255) / 256;
  if (blocks > sms * 8) blocks = sms * 8;
  classify_kernel<<<blocks, 256, 0, st>>>(A, cells, n, nnz, diag, cls, counts);
  scatter_kernel<<<(cells + 255) / 256, 256, 0, st>>>(cls, cells, counts, ord);
  return cudaGetLastError();
}

}  // namespace camp
