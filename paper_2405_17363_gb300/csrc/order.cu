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

}  // namespace

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
