// Self-test entry point: runs the warp kernels' numerical building blocks
// (reciprocals, FP64<->FP32 conversions on the integer pipe, segment sums) on
// caller data so tests can compare them with exact host references.
#include "warp_common.cuh"

namespace camp {
namespace {

__global__ void selftest_kernel(int op, int n, const double *in, double *out, int lanes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < n;
  const double v = ok ? in[i] : 0.0;
  double r = 0.0;
  if (op == 0) r = recip64(v);
  else if (op == 1) r = recip64s(v);
  else if (op == 2) r = f2d_exact(d2f_rn(v));
  else if (op == 3) r = seg_sum_exact(v, lanes);     // whole warp takes part
  else if (op == 4) {
    double a[1] = {v};
    seg_sum<1>(a, lanes);
    r = a[0];
  } else if (op == 5) {  // the whole warp takes part
    switch (lanes) {
      case 1: r = seg_sum_exact_redux<32>(v); break;
      case 2: r = seg_sum_exact_redux<16>(v); break;
      case 4: r = seg_sum_exact_redux<8>(v); break;
      case 8: r = seg_sum_exact_redux<4>(v); break;
      case 16: r = seg_sum_exact_redux<2>(v); break;
      default: r = seg_sum_exact_redux<1>(v); break;
    }
  }
  if (ok) out[i] = r;
}

// FP64 issue-rate probe: four independent dependent-FMA chains per thread,
// steps * 4 DFMAs in all; the caller times the launch.
__global__ void dfma_rate_kernel(int n, const double *in, double *out, int steps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = in[i], b = a + 1.0, c = a + 2.0, d = a + 3.0;
  const double m = 0.999999999, q = 1e-9;
  for (int s = 0; s < steps; ++s) {
    a = fma(a, m, q);
    b = fma(b, m, q);
    c = fma(c, m, q);
    d = fma(d, m, q);
  }
  out[i] = a + b + c + d;
}

}  // namespace
}  // namespace camp

extern "C" camp_status camp_selftest(int op, int n, const double *in, double *out,
                                     int lanes, void *stream) {
  if (op < 0 || op > 6 || n < 0 || !in || !out) return CAMP_EINVAL;
  if (op == 6) {
    if (lanes < 1 || lanes > (1 << 20)) return CAMP_EINVAL;
    if (n == 0) return CAMP_OK;
    camp::dfma_rate_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, in, out, lanes);
    return cudaGetLastError() == cudaSuccess ? CAMP_OK : CAMP_ECUDA;
  }
  if (op >= 3 && (lanes < 1 || lanes > 32 || (lanes & (lanes - 1)) || n % 32)) return CAMP_EINVAL;
  if (n == 0) return CAMP_OK;
  camp::selftest_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(op, n, in, out, lanes);
  return cudaGetLastError() == cudaSuccess ? CAMP_OK : CAMP_ECUDA;
}
