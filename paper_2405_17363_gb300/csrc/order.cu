// Difficulty ordering of the cells for the warp-packed solve.  The cells that
// share a warp run in lockstep until the last one converges, so pairing cells
// of similar iteration counts wastes fewer lanes, and solving the hardest
// first shortens the tail.  The estimate is the largest Jacobi-scaled
// off-diagonal row sum, max_i sum_{j != i} |A_ij| / |A_ii|, formed in FP32
// (the FP64 pipe is left to the solve); cells are then bucketed on log2 of it
// by one thread block (order inside a bucket is arbitrary: a cell's result
// does not depend on where it is solved).
#include "warp_common.cuh"

namespace camp {

namespace {

constexpr int kBuckets = 1024;

__global__ void difficulty_kernel(const double *__restrict__ A, int cells, int n,
                                  int nnz, const int *__restrict__ rp,
                                  const int *__restrict__ diag,
                                  float *__restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < cells; c += warps) {
    const double *Ac = A + (size_t)c * nnz;
    float worst = 0.0f;
    for (int i = lane; i < n; i += 32) {
      const int d = __ldg(diag + i);
      float off = 0.0f;
      for (int k = __ldg(rp + i); k < __ldg(rp + i + 1); ++k)
        if (k != d) off += fabsf(d2f_rn(__ldg(Ac + k)));
      const float dd = fabsf(d2f_rn(__ldg(Ac + d)));
      const float ratio = dd > 0.0f ? off / dd : 3.0e38f;
      worst = fmaxf(worst, ratio);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(kFull, worst, o));
    if (lane == 0) keys[c] = worst;
  }
}

__device__ __forceinline__ int bucket_of(float key) {
  // decreasing difficulty: larger keys get smaller bucket indices
  const float l = key > 0.0f ? __log2f(key) : -1000.0f;
  int b = (int)floorf(l * 32.0f) + 800;
  b = b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
  return kBuckets - 1 - b;
}

__global__ void __launch_bounds__(kBuckets) order_kernel(const float *__restrict__ keys,
                                                         int cells, int *__restrict__ order) {
  __shared__ int hist[kBuckets];
  __shared__ int scan[kBuckets];
  const int t = threadIdx.x;
  hist[t] = 0;
  __syncthreads();
  for (int c = t; c < cells; c += blockDim.x) atomicAdd(&hist[bucket_of(keys[c])], 1);
  __syncthreads();
  // exclusive scan (Hillis-Steele on the inclusive sums, then shift)
  scan[t] = hist[t];
  __syncthreads();
  for (int off = 1; off < kBuckets; off <<= 1) {
    const int v = t >= off ? scan[t - off] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  hist[t] = scan[t] - hist[t];   // start of bucket t
  __syncthreads();
  for (int c = t; c < cells; c += blockDim.x) {
    const int p = atomicAdd(&hist[bucket_of(keys[c])], 1);
    order[p] = c;
  }
}

}  // namespace

cudaError_t launch_difficulty_order(const double *A, int cells, int n, int nnz,
                                    const int *row_ptr, const int *diag,
                                    float *keys, int *order, cudaStream_t st) {
  if (cells <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int warps_needed = cells;
  int blocks = (warps_needed * 32 + 255) / 256;
  if (blocks > sms * 8) blocks = sms * 8;
  difficulty_kernel<<<blocks, 256, 0, st>>>(A, cells, n, nnz, row_ptr, diag, keys);
  order_kernel<<<1, kBuckets, 0, st>>>(keys, cells, order);
  return cudaGetLastError();
}

}  // namespace camp
