// Block-cells(k) kernel: the paper's arrangement (Sec. 3.2, Table GPU1 and
// Table GPU): cpb cells per thread block, one thread per species row, the
// rows of cell j on threads [j*n, j*n + n); cpb = 1 is Block-cells(1).  The
// whole solve of every cell runs in one launch with per-cell convergence on
// the device (Sec. 3.1).  Unlike the paper's Block-cells(N), the cells of a
// block keep separate scalars and convergence tests, so each cell's result
// does not depend on how the cells are packed.
//
// Reductions: every thread writes its terms to shared memory, one warp per
// cell sums them (warp shuffles instead of the paper's power-of-two Harris
// tree, Table GPU2), and every thread reads its cell's total; two barriers per
// reduction round.
//
// Also here: the pattern-gradient kernel gA[k] = -lambda[row k] x[col k].
#include "camp_internal.h"

namespace camp {

namespace {

constexpr unsigned kFullB = 0xffffffffu;

__device__ __forceinline__ bool fin_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return ((u >> 52) & 0x7ffull) != 0x7ffull;
}
__device__ __forceinline__ bool tiny_bits(double v) {
  const unsigned long long u =
      (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return u < 0x01a56e1fc2f8f359ull;  // 1e-300
}
__device__ __forceinline__ bool le_nn(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}

// Per-cell sums of NV values: v holds this thread's terms on entry and the
// totals of its cell on return (threads outside any cell get zeros).
template <int NV>
__device__ __forceinline__ void cell_sum(double (&v)[NV], double *prod,
                                         double *tot, int n, int cpb, int j,
                                         bool in_block) {
  const int t = threadIdx.x, bd = blockDim.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) prod[q * bd + t] = in_block ? v[q] : 0.0;
  __syncthreads();
  const int w = t >> 5, lane = t & 31, nw = bd >> 5;
  for (int jj = w; jj < cpb; jj += nw) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double acc = 0.0;
      for (int ii = lane; ii < n; ii += 32) acc += prod[q * bd + jj * n + ii];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        acc += __shfl_xor_sync(kFullB, acc, off);
      if (lane == 0) tot[q * cpb + jj] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = in_block ? tot[q * cpb + j] : 0.0;
}

// Coupled mode (the paper's Block-cells(N) semantics, Sec. 3.2): one total
// over every row of the block's present cells, i.e. the cells of a block form
// one block-diagonal system with shared scalars and one convergence test.
// Warp shuffles, one partial per warp in shared memory, warp 0 sums them.
template <int NV>
__device__ __forceinline__ void block_total(double (&v)[NV], double *prod,
                                            double *tot, bool contrib) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double acc = contrib ? v[q] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFullB, acc, off);
    if (lane == 0) prod[q * 32 + w] = acc;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double acc = lane < nw ? prod[q * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFullB, acc, off);
      if (lane == 0) tot[q] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = tot[q];
}

}  // namespace

__global__ void __launch_bounds__(1024) block_bicgstab_kernel(const BlockArgs a) {
  extern __shared__ __align__(16) double bsm[];
  const int n = a.n, nnz = a.nnz, cpb = a.cpb;
  const int t = threadIdx.x, bd = blockDim.x;
  const int c0 = blockIdx.x * cpb;
  const int here = min(cpb, a.cells - c0);
  const int j = t / n, i = t - j * n;
  const bool in_block = j < cpb;
  const bool has = j < here;  // this thread's row belongs to a real cell
  const int c = c0 + j;

  double *As = bsm;                         // [cpb x nnz]
  double *gs = As + (size_t)cpb * nnz;      // [cpb x n]
  double *o1 = gs + (size_t)cpb * n;        // [cpb x n]
  double *o2 = o1 + (size_t)cpb * n;        // [cpb x n]
  double *prod = o2 + (size_t)cpb * n;      // [3 x bd]
  double *tot = prod + 3 * (size_t)bd;      // [3 x cpb]

  // stage the block's cells (consecutive in memory)
  if (a.a_perm) {
    for (int k = t; k < here * nnz; k += bd) {
      const int jj = k / nnz, kk = k - jj * nnz;
      As[k] = __ldg(a.A + (size_t)(c0 + jj) * nnz + __ldg(a.a_perm + kk));
    }
  } else {
    const double *Ab = a.A + (size_t)c0 * nnz;
    for (int k = t; k < here * nnz; k += bd) As[k] = __ldg(Ab + k);
  }
  __syncthreads();

  const double *Ac = As + (size_t)j * nnz;
  int rlo = 0, rhi = 0;
  if (in_block) {
    rlo = __ldg(a.row_ptr + i);
    rhi = __ldg(a.row_ptr + i + 1);
  }
  double *g = gs + (size_t)j * n, *v1 = o1 + (size_t)j * n, *v2 = o2 + (size_t)j * n;

  const double bi = has ? __ldg(a.b + (size_t)c * n + i) : 0.0;
  double dinv = 0.0;
  if (has) {
    const double d = Ac[__ldg(a.diag + i)];
    dinv = (d != 0.0) ? 1.0 / d : 1.0;
  }
  double xv = (has && a.x0_given) ? a.x[(size_t)c * n + i] : 0.0;
  double r = bi, rh = 0.0, p = 0.0, s = 0.0;

  auto spmv = [&](const double *src, double *dst) {
    if (in_block) {
      double acc = 0.0;
      for (int k = rlo; k < rhi; ++k) acc = fma(Ac[k], src[__ldg(a.col_idx + k)], acc);
      dst[i] = acc;
    }
  };

  double bbv[1] = {bi * bi};
  if (a.coupled) block_total<1>(bbv, prod, tot, has);
      else cell_sum<1>(bbv, prod, tot, n, cpb, j, in_block);
  const double bb = bbv[0];
  const double bnorm = sqrt(bb);
  const double thr = (a.tol * bnorm) * (a.tol * bnorm);
  int st = -1, it = 0, nbreak = 0;
  double resid = 0.0;
  bool done = !has;
  if (has) {
    if (!fin_bits(bb)) {
      st = CAMP_CELL_NONFINITE;
      resid = __longlong_as_double(0x7ff8000000000000ll);
      done = true;
    } else if (bb == 0.0) {
      st = CAMP_CELL_CONVERGED;
      done = true;
      xv = 0.0;
    }
  }
  if (a.x0_given) {
    if (in_block) g[i] = xv;
    __syncthreads();
    spmv(g, v1);
    __syncthreads();
    if (in_block) r -= v1[i];
  }

  bool restart = !done, first = true, fin = false, active = false, broke = false,
       nonfin = false;
  double rho = 1.0, rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (;;) {
    {
      double rr[1] = {r * r};
      if (a.coupled) block_total<1>(rr, prod, tot, has);
      else cell_sum<1>(rr, prod, tot, n, cpb, j, in_block);
      if (restart) {
        rh = r;
        p = 0.0;
        rho = rr[0];
        rho_prev = alpha = omega = 1.0;
        broke = nonfin = false;
        fin = true;
        // a restart follows a failed true-residual test: always iterate
        active = first ? !le_nn(rr[0], thr) : true;
        restart = false;
        first = false;
      }
    }
    while (__syncthreads_or(active)) {
      if (active) {
        if (it >= a.maxit) {
          active = false;
        } else if (!fin_bits(rho)) {
          nonfin = true;
          active = false;
        } else if (tiny_bits(rho)) {
          broke = true;
          active = false;
        }
      }
      const double beta = (rho / rho_prev) * (alpha / omega);
      if (active) p = fma(beta, p, r);
      const double ph = dinv * p;
      if (in_block) g[i] = ph;
      __syncthreads();
      spmv(g, v1);
      __syncthreads();
      if (active) ++it;
      const double v = in_block ? v1[i] : 0.0;
      double sg[1] = {rh * v};
      if (a.coupled) block_total<1>(sg, prod, tot, has);
      else cell_sum<1>(sg, prod, tot, n, cpb, j, in_block);
      if (active) {
        if (!fin_bits(sg[0])) {
          nonfin = true;
          active = false;
        } else if (tiny_bits(sg[0])) {
          broke = true;
          active = false;
        }
      }
      const double al = rho / sg[0];
      if (active) {
        alpha = al;
        xv = fma(al, ph, xv);
        s = fma(-al, v, r);
      }
      const double sh = dinv * s;
      if (in_block) g[i] = sh;
      __syncthreads();
      spmv(g, v2);
      __syncthreads();
      const double tv = in_block ? v2[i] : 0.0;
      double q3[3] = {s * s, tv * s, tv * tv};
      if (a.coupled) block_total<3>(q3, prod, tot, has);
      else cell_sum<3>(q3, prod, tot, n, cpb, j, in_block);
      bool full = false;
      if (active) {
        if (le_nn(q3[0], thr)) {
          active = false;
        } else if (!fin_bits(q3[1]) || !fin_bits(q3[2])) {
          nonfin = true;
          active = false;
        } else if (q3[2] == 0.0) {
          broke = true;
          active = false;
        } else {
          full = true;
        }
      }
      const double om = q3[1] / q3[2];
      if (full) {
        omega = om;
        xv = fma(om, sh, xv);
        r = fma(-om, tv, s);
        p = fma(-om, v, p);
      }
      double q2[2] = {rh * r, r * r};
      if (a.coupled) block_total<2>(q2, prod, tot, has);
      else cell_sum<2>(q2, prod, tot, n, cpb, j, in_block);
      if (full) {
        nbreak = 0;
        if (le_nn(q2[1], thr)) {
          active = false;
        } else if (om == 0.0) {
          broke = true;
          active = false;
        } else {
          rho_prev = rho;
          rho = q2[0];
        }
      }
    }
    // true residual
    if (in_block) g[i] = xv;
    __syncthreads();
    spmv(g, v1);
    __syncthreads();
    const double rt = bi - (in_block ? v1[i] : 0.0);
    double rt2[1] = {rt * rt};
    if (a.coupled) block_total<1>(rt2, prod, tot, has);
      else cell_sum<1>(rt2, prod, tot, n, cpb, j, in_block);
    if (fin) {
      fin = false;
      resid = sqrt(rt2[0]) / bnorm;
      if (nonfin || !fin_bits(resid)) {
        st = CAMP_CELL_NONFINITE;
      } else if (resid <= a.tol) {
        st = CAMP_CELL_CONVERGED;
      } else if (it >= a.maxit) {
        st = CAMP_CELL_MAXIT;
      } else if (broke && ++nbreak >= 2) {
        st = CAMP_CELL_BREAKDOWN;
      } else {
        r = rt;
        restart = true;
      }
    }
    if (!__syncthreads_or(restart)) break;
  }
  if (has) {
    a.x[(size_t)c * n + i] = xv;
    if (i == 0) {
      a.iters[c] = it;
      a.resid[c] = resid;
      if (a.status) a.status[c] = st;
    }
  }
}

cudaError_t block_set_smem(size_t smem) {
  (void)smem;
  return ensure_max_smem((const void *)block_bicgstab_kernel);
}

cudaError_t launch_block(const BlockArgs &a, int threads, size_t smem,
                         cudaStream_t st) {
  cudaError_t e = block_set_smem(smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.cells + a.cpb - 1) / a.cpb;
  block_bicgstab_kernel<<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// gA[c, k] = -lambda[c, row k] * x[c, col k]; one thread per entry, grid-stride.
__global__ void grad_A_kernel(const GradArgs a) {
  const size_t total = (size_t)a.cells * a.nnz;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const size_t c = q / a.nnz;
    const int k = (int)(q - c * a.nnz);
    const double lam = __ldg(a.lambda + c * a.n + __ldg(a.row_of + k));
    const double xv = __ldg(a.x + c * a.n + __ldg(a.col_idx + k));
    a.gA[q] = -lam * xv;
  }
}

cudaError_t launch_grad(const GradArgs &a, cudaStream_t st) {
  const size_t total = (size_t)a.cells * a.nnz;
  if (total == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t blocks = (total + 255) / 256;
  const size_t cap = (size_t)sms * 8;
  if (blocks > cap) blocks = cap;
  grad_A_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace camp
