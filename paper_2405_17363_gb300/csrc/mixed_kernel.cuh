// FP32-inner / FP64-outer iterative refinement, warp-packed layout (see
// warp_kernel.cuh for the lane/segment arrangement).  Per cell and sweep: the
// FP64 true residual r = b - A x and its norm decide convergence; otherwise an
// FP32 right-Jacobi BiCGSTAB solves A32 d = r / ||r|| to a relative inner
// tolerance (or an inner iteration cap) and x += ||r|| d in FP64.  The FP64
// pipe only sees the residual products, norms and updates; the inner
// iterations run on the FP32 pipe.
//
// Shared memory per cell: A in FP32 [segA] and, when a.a64_smem is set, in
// FP64 [segA] (otherwise the FP64 residual product reads A through L1 from
// the cell's row in global memory, which the staging has just brought into
// L2: it runs two or three times per cell, against tens of FP32 products, and
// the smaller footprint lets more warps run), the FP64 product input/output
// vectors [segV each] and three FP32 vectors [segV each].
#pragma once
#include "warp_common.cuh"

namespace camp {

template <int E, int LC>
__device__ __forceinline__ void mixed_body(const MixedArgs &a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SchedWord *sch_s = reinterpret_cast<SchedWord *>(smem_raw);
  const int nsch = a.L * a.Lc;
  for (int i = threadIdx.x; i < nsch; i += blockDim.x) sch_s[i] = a.sched[i];

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int Lc = LC ? LC : a.Lc;  // lanes per cell (compile-time when LC > 0)
  const int seg = LC ? lane / LC : lane >> a.log2Lc;
  const int sl = lane & (Lc - 1);
  const int n = a.n, nnz = a.nnz;
  // bytes per cell: (12 or 4) segA + 16 segV + 12 segV (FP64 A when staged,
  // FP32 A, 2 FP64 + 3 FP32 vectors)
  const size_t cellBytes = (size_t)(a.a64_smem ? 12 : 4) * a.segA + (size_t)28 * a.segV;
  unsigned char *wb = smem_raw + sched_smem_bytes(nsch) +
                      ((size_t)warp * a.k + seg) * cellBytes;
  double *As = reinterpret_cast<double *>(wb);
  double *g64 = As + (a.a64_smem ? a.segA : 0);
  double *o64 = g64 + a.segV;
  float *As32 = reinterpret_cast<float *>(o64 + a.segV);
  float *g32 = As32 + a.segA;
  float *o1 = g32 + a.segV;
  float *o2 = o1 + a.segV;
  // in-launch difficulty ordering first: it borrows the start of the warp
  // regions (and ends with a block barrier)
  if (a.ord_ws)
    order_prologue<false>(a, reinterpret_cast<int *>(smem_raw + sched_smem_bytes(nsch)));
  for (int i = sl; i < a.segV; i += Lc) {
    g64[i] = 0.0; o64[i] = 0.0; g32[i] = 0.0f; o1[i] = 0.0f; o2[i] = 0.0f;
  }
  __syncthreads();
  const SchedWord *sch = sch_s + sl;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  constexpr int K = LC ? 32 / LC : 0;  // cells per warp (0: a.k)

  auto refine_group = [&](int g) {
    const int pos = g * (K ? K : a.k) + seg;
    const bool has = pos < a.cells;
    // the order may have been written earlier in this launch (cell + 1 from
    // the in-launch ordering): read it through L2, clamped in range
    const int c = (has && a.order)
                      ? (int)min((unsigned)(__ldcg(a.order + pos) - (a.ord_ws ? 1 : 0)),
                                 (unsigned)a.cells - 1u)
                      : pos;
    const double *Ac = a.A + (size_t)(has ? c : 0) * nnz;
    if (a.a64_smem) {  // stage A in slot order, FP64 and its FP32 rounding
      stage_scatter(Ac, a.dst, nnz, sl, Lc, has, [&](int t, double v) {
        As[t] = v;
        As32[t] = d2f_rn(v);
      });
      zero_padding(As, a.padfrom, a.L, Lc, sl);
    } else {  // the FP32 rounding only
      stage_scatter(Ac, a.dst, nnz, sl, Lc, has, [&](int t, double v) { As32[t] = d2f_rn(v); });
    }
    zero_padding(As32, a.padfrom, a.L, Lc, sl);
    __syncwarp();
    double xv[E];
    float dinv[E];
    double bb;
    {
      double acc[1] = {0.0};
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        const bool v = has && i < n;
        const double bi = v ? __ldg(a.b + (size_t)c * n + i) : 0.0;
        const float d = v ? As32[__ldg(a.dslot + i)] : 0.0f;
        dinv[e] = v ? (d != 0.0f ? 1.0f / d : 1.0f) : 0.0f;
        xv[e] = 0.0;
        acc[0] = fma(bi, bi, acc[0]);
      }
      bb = seg_sum_x<LC>(acc[0], Lc);
    }
    const double thr = (a.tol * a.tol) * bb;  // (tol ||b||)^2
    int st = -1, sweeps = 0, inner = 0;
    double resid = 0.0;
    bool done = !has;
    if (has && !is_finite_bits(bb)) {
      st = CAMP_CELL_NONFINITE;
      resid = __longlong_as_double(0x7ff8000000000000ll);
      done = true;
    } else if (has && is_zero_bits(bb)) {
      st = CAMP_CELL_CONVERGED;
      done = true;
    }
    for (int pass = 0;; ++pass) {
      // ---- FP64 true residual r = b - A x (x = 0 on the first pass)
      double r[E];
      if (pass > 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) g64[sl + e * Lc] = xv[e];
        __syncwarp();
        if (a.a64_smem) seg_spmv(sch, a.L, Lc, As + sl, g64, o64);
        else seg_spmv_gather(sch, a.src + sl, a.L, Lc, Ac, g64, o64);
        __syncwarp();
      }
      double rr[1] = {0.0};
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        const double bi = (has && i < n) ? __ldg(a.b + (size_t)c * n + i) : 0.0;
        r[e] = pass > 0 ? bi - o64[i] : bi;
        rr[0] = fma(r[e], r[e], rr[0]);
      }
      rr[0] = seg_sum_x<LC>(rr[0], Lc);
      if (!done) {
        // ||r|| <= tol ||b|| on the bit patterns; the relative residual itself
        // (a square root and a division) is formed once, at the end
        if (!is_finite_bits(rr[0])) {
          st = CAMP_CELL_NONFINITE;
          done = true;
        } else if (le_nonneg(rr[0], thr)) {
          st = CAMP_CELL_CONVERGED;
          done = true;
        } else if (sweeps >= a.max_sweeps) {
          st = CAMP_CELL_MAXIT;
          done = true;
        }
        if (done) resid = sqrt(rr[0] * recip64(bb));
      }
      if (!__any_sync(kFull, !done)) break;
      // ---- FP32 inner solve of A d = r / ||r||.  The scale only sets the
      // size of the FP32 right-hand side, so it is formed in FP32 (FP64 when
      // ||r||^2 is outside the FP32 range).
      float rn32, rinv32;
      bool wide = false;
      {
        const int ex = (int)(((unsigned long long)__double_as_longlong(rr[0]) >> 52) & 0x7ffull) - 1023;
        wide = ex < -120 || ex > 120;
        const float rr32 = d2f_rn(rr[0]);
        rinv32 = rsqrtf(rr32);
        rn32 = rr32 * rinv32;
      }
      const double rn64 = wide ? sqrt(rr[0]) : 0.0;
      const double sc64 = wide ? 1.0 / rn64 : 0.0;
      float rf[E], rh[E], p[E], s[E], d[E];
      float cc[1] = {0.0f};
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const float ce = done ? 0.0f : (wide ? d2f_rn(r[e] * sc64) : d2f_rn(r[e]) * rinv32);
        rf[e] = ce;
        rh[e] = ce;
        p[e] = 0.0f;
        s[e] = 0.0f;
        d[e] = 0.0f;
        cc[0] = fmaf(ce, ce, cc[0]);
      }
      seg_sumf<1>(cc, Lc);
      const float thr = a.tol_in * a.tol_in * cc[0];
      float rho = cc[0], rho_prev = 1.0f, alpha = 1.0f, omega = 1.0f;
      bool act = !done && cc[0] > 0.0f && isfinite(cc[0]);
      int it = 0;
      while (__any_sync(kFull, act)) {
        if (act) {
          if (it >= a.maxit_in || !isfinite(rho) || fabsf(rho) < 1e-37f) act = false;
        }
        const float beta = (rho / rho_prev) * (alpha / omega);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (act) p[e] = fmaf(beta, p[e], rf[e]);
          g32[sl + e * Lc] = dinv[e] * p[e];
        }
        __syncwarp();
        seg_spmvf(sch, a.L, Lc, As32 + sl, g32, o1);
        __syncwarp();
        if (act) ++it;
        float sg[1] = {0.0f};
#pragma unroll
        for (int e = 0; e < E; ++e) sg[0] = fmaf(rh[e], o1[sl + e * Lc], sg[0]);
        seg_sumf<1>(sg, Lc);
        if (act && (!isfinite(sg[0]) || fabsf(sg[0]) < 1e-37f)) act = false;
        const float al = rho / sg[0];
        if (act) alpha = al;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = sl + e * Lc;
          if (act) {
            d[e] = fmaf(al, g32[i], d[e]);
            s[e] = fmaf(-al, o1[i], rf[e]);
          }
          g32[i] = dinv[e] * s[e];
        }
        __syncwarp();
        seg_spmvf(sch, a.L, Lc, As32 + sl, g32, o2);
        __syncwarp();
        float q3[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const float t = o2[sl + e * Lc];
          q3[0] = fmaf(s[e], s[e], q3[0]);
          q3[1] = fmaf(t, s[e], q3[1]);
          q3[2] = fmaf(t, t, q3[2]);
        }
        seg_sumf<3>(q3, Lc);
        bool full = false;
        if (act) {
          if (q3[0] <= thr || !isfinite(q3[1]) || !isfinite(q3[2]) || q3[2] == 0.0f)
            act = false;
          else
            full = true;
        }
        const float om = q3[1] / q3[2];
        if (full) omega = om;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = sl + e * Lc;
          if (full) {
            d[e] = fmaf(om, g32[i], d[e]);
            rf[e] = fmaf(-om, o2[i], s[e]);
            p[e] = fmaf(-om, o1[i], p[e]);
          }
        }
        float q2[2] = {0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < E; ++e) {
          q2[0] = fmaf(rh[e], rf[e], q2[0]);
          q2[1] = fmaf(rf[e], rf[e], q2[1]);
        }
        seg_sumf<2>(q2, Lc);
        if (full) {
          if (q2[1] <= thr || om == 0.0f) {
            act = false;
          } else {
            rho_prev = rho;
            rho = q2[0];
          }
        }
      }
      if (!done) {
        inner += it;
        ++sweeps;
#pragma unroll
        for (int e = 0; e < E; ++e)
          xv[e] += wide ? rn64 * f2d_exact(d[e]) : f2d_exact(rn32 * d[e]);
      }
    }
    if (has) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        if (i < n) a.x[(size_t)c * n + i] = xv[e];
      }
      if (sl == 0) {
        a.iters[c] = inner;
        if (a.sweeps) a.sweeps[c] = sweeps;
        a.resid[c] = resid;
        if (a.status) a.status[c] = st;
      }
    }
    __syncwarp();
  };

  if (!a.queue) {
    for (int g = blockIdx.x * (blockDim.x >> 5) + warp; g < a.ngroups; g += warps_total)
      refine_group(g);
    return;
  }
  // dynamic assignment (an ordered launch first gives every warp one group
  // of a stratified wave)
  bool first = true;
  unsigned g = 0;
  while (take_group(a, warp, lane, first, g)) {
    const bool mine = await_order_entries(a, g, K ? K : a.k, lane);
    refine_group((int)g);
    if (mine) a.ord_out[g * (K ? K : a.k) + lane] = 0;
  }
  finish_queue(a, true, warps_total, lane);
}

template <int E>
__global__ void __launch_bounds__(256, 2) mixed_refine_kernel(const MixedArgs a) {
  // the automatic choice (at most 3 rows per lane on 8, 16 or 32 lanes) runs
  // code with the lane count fixed at compile time
  if constexpr (E >= 2 && E <= 3) {
    if (a.Lc == 32) return mixed_body<E, 32>(a);
    if (a.Lc == 16) return mixed_body<E, 16>(a);
    if (a.Lc == 8) return mixed_body<E, 8>(a);
  }
  mixed_body<E, 0>(a);
}

}  // namespace camp
