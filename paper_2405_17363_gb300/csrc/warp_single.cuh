// One cell on all 32 lanes of a warp, bit for bit as its pair solve at 16
// lanes per cell (solve_group<E16, kSrcStaged, 16>): the end of a large
// batch and small batches, where a warp runs nearly alone and its latency,
// not the FP64 units' throughput, decides the launch's length.
//
// The 16-lane layout gives lane v (v = 0..15) the vector rows v + 16e,
// e = 0..E16-1, and the SpMV rows of its schedule column.  Here lane v keeps
// rows e = 0..E0-1 and lane v + 16 takes rows e = E0..E16-1 (E0 = ceil(E16 /
// 2)); the SpMV runs on the split schedule, which gives each of lanes v and
// v + 16 whole rows of 16-lane lane v with their slots in the same order.
// Every quantity is then computed by the same operations in the same order:
//   - element-wise updates act on the same rows with the same scalars;
//   - each row's product is the same chain of multiply-adds;
//   - a dot product's per-lane partial is the chain over e = 0..E16-1: lane v
//     runs e < E0, hands its partial to lane v + 16 (one shuffle), which runs
//     the rest, and the exact cross-lane sum sees the same 16 partials (the
//     other lanes add zero, which changes neither the exponent maximum nor
//     the integer sum);
//   - the scalars and tests follow from those values as in solve_group.
// The iteration, its guards and its readings are those of solve_group.
#pragma once
#include "warp_common.cuh"

namespace camp {

// Lane v's partial of a chained dot product handed to lane v + 16, which
// continues it; lanes v then hold zero.  acc: this lane's value after the
// first stage (the upper lanes' is ignored).
__device__ __forceinline__ double split_handoff(double acc, int h, int v) {
  const double in = __shfl_sync(kFull, acc, v);
  return h ? in : acc;
}

template <int E16>
__device__ __forceinline__ void solve_single(const WarpArgs &a, int pos, double *wbase) {
  constexpr int E0 = (E16 + 1) / 2;     // rows of the lower lanes (registers per lane)
  const int lane = threadIdx.x & 31;
  const int h = lane >> 4, v = lane & 15;
  const int EJ = h ? E16 - E0 : E0;     // this lane's rows
  const int n = a.n, nnz = a.nnz;
  const double tol = a.tol;
  // region: the split slots, then g, o1, o2 (rows 0 .. 16 E16 - 1)
  const int segA2 = (a.L2 * 32 + 1) & ~1;
  const int segV2 = ((16 * E16 + 1) + 1) & ~1;
  double *Abase = wbase;
  double *gs = Abase + segA2;
  double *o1 = gs + segV2;
  double *o2 = o1 + segV2;
  const bool has = pos < a.cells;
  const int c = (has && a.order)
                    ? (int)min((unsigned)(__ldcg(a.order + pos) - (a.ord_ws ? 1 : 0)),
                               (unsigned)a.cells - 1u)
                    : pos;
  const double *Ac = a.A + (size_t)(has ? c : 0) * nnz;
  const SchedWord *sch = a.sched2 + lane;
  const double *Asl = Abase + lane;
  // row of register slot j (the upper lanes' spare slot, when E16 is odd,
  // maps to row v: it is never read or written, and no address it could
  // form leaves the region)
  auto row = [&](int j) { return v + 16 * (h ? (j < E16 - E0 ? E0 + j : 0) : j); };
  auto spmv = [&](double *out) { seg_spmv(sch, a.L2, 32, Asl, gs, out); };
  // the chained dot products: stage one on the lower lanes, the hand-off,
  // stage two on the upper lanes, then the exact sum over the warp
#define CHAIN(acc, X, Y)                                             \
  do {                                                               \
    _Pragma("unroll") for (int j = 0; j < E0; ++j)                   \
      if (h == 0) acc = fma(X, Y, acc);                              \
    acc = split_handoff(acc, h, v);                                  \
    _Pragma("unroll") for (int j = 0; j < E0; ++j)                   \
      if (h == 1 && j < EJ) acc = fma(X, Y, acc);                    \
    acc = h ? acc : 0.0;                                             \
  } while (0)

  double xv[E0], rhs[E0], dvs[E0];
  int st = -1, it = 0;
  double resid = 0.0;
  const bool live = has;

  // ---- stage the cell's matrix values in split-slot order
  stage_scatter(Ac, a.dst2, nnz, lane, 32, live, [&](int t, double x) { Abase[t] = x; });
  zero_padding(Abase, a.padfrom2, a.L2, 32, lane);
  // pad rows of the product vectors are never written by the SpMV
  for (int i = n + lane; i < 16 * E16; i += 32) {
    o1[i] = 0.0;
    o2[i] = 0.0;
  }
  __syncwarp();

  double r[E0], p[E0], s[E0];
  double bb;
  {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < E0; ++j) {
      const int i = row(j);
      const bool ok = live && j < EJ && i < n;
      const double bi = ok ? __ldg(a.b + (size_t)c * n + i) : 0.0;
      const double d = ok ? Abase[__ldg(a.dslot2 + i)] : 0.0;
      dvs[j] = ok ? (!is_zero_bits(d) ? recip64(d) : 1.0) : 0.0;
      xv[j] = (ok && a.x0_given) ? a.x[(size_t)c * n + i] : 0.0;
      r[j] = bi;
      p[j] = 0.0;
      s[j] = 0.0;
      rhs[j] = 0.0;
    }
    CHAIN(acc, r[j], r[j]);
    bb = seg_sum_exact_redux<1>(acc);
  }
  const double thr = (tol * tol) * bb;  // (tol ||b||)^2
  int nbreak = 0;
  bool done = !live;
  if (live) {
    if (!is_finite_bits(bb)) {
      st = CAMP_CELL_NONFINITE;
      resid = __longlong_as_double(0x7ff8000000000000ll);
      done = true;
    } else if (is_zero_bits(bb)) {
      st = CAMP_CELL_CONVERGED;
      done = true;
#pragma unroll
      for (int j = 0; j < E0; ++j) xv[j] = 0.0;
    }
  }
  if (a.x0_given) {  // r = b - A x0
#pragma unroll
    for (int j = 0; j < E0; ++j)
      if (j < EJ) gs[row(j)] = xv[j];
    __syncwarp();
    spmv(o1);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E0; ++j)
      if (j < EJ) r[j] -= o1[row(j)];
  }

  bool restart = !done, first = true;
  bool pass0 = true;  // the solve's first (re)start
  bool fin = false, active = false, broke = false, nonfin = false;
  double rho = 1.0, rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (;;) {
    {  // (re)start from the current residual r
      double acc = 0.0;
      if (pass0 && !a.x0_given) {
        acc = bb;  // r = b: the same chain and exact sum as ||b||^2
      } else {
        CHAIN(acc, r[j], r[j]);
        acc = seg_sum_exact_redux<1>(acc);
      }
      pass0 = false;
      if (restart) {
#pragma unroll
        for (int j = 0; j < E0; ++j) {
          rhs[j] = r[j];
          p[j] = 0.0;
        }
        rho = acc;
        rho_prev = alpha = omega = 1.0;
        broke = nonfin = false;
        fin = true;
        active = first ? !le_nonneg(acc, thr) : true;
        restart = false;
        first = false;
      }
    }
    while (__any_sync(kFull, active)) {
      if (active) {
        if (it >= a.maxit) {
          active = false;
        } else if (!is_finite_bits(rho)) {
          nonfin = true;
          active = false;
        } else if (abs_tiny(rho)) {
          broke = true;
          active = false;
        }
      }
      // p = r + beta (p - omega v); the bracket is kept in p
      const double beta = (rho * alpha) * recip64s(rho_prev * omega);
#pragma unroll
      for (int j = 0; j < E0; ++j) {
        if (active) p[j] = fma(beta, p[j], r[j]);
        if (j < EJ) gs[row(j)] = dvs[j] * p[j];
      }
      __syncwarp();
      spmv(o1);  // v = A p^
      __syncwarp();
      if (active) ++it;
      double sg = 0.0;
      CHAIN(sg, rhs[j], o1[row(j)]);
      sg = seg_sum_exact_redux<1>(sg);
      if (active) {
        if (!is_finite_bits(sg)) {
          nonfin = true;
          active = false;
        } else if (abs_tiny(sg)) {
          broke = true;
          active = false;
        }
      }
      const double al = rho * recip64s(sg);
      if (active) alpha = al;
#pragma unroll
      for (int j = 0; j < E0; ++j) {
        if (j < EJ) {
          const int i = row(j);
          if (active) {
            xv[j] = fma(al, gs[i], xv[j]);
            s[j] = fma(-al, o1[i], r[j]);
          }
          gs[i] = dvs[j] * s[j];
        }
      }
      __syncwarp();
      spmv(o2);  // t = A s^
      __syncwarp();
      double q0 = 0.0, q1 = 0.0, q2 = 0.0;
      {
        double t[E0];
#pragma unroll
        for (int j = 0; j < E0; ++j) t[j] = j < EJ ? o2[row(j)] : 0.0;
#pragma unroll
        for (int j = 0; j < E0; ++j)
          if (h == 0) {
            q0 = fma(s[j], s[j], q0);
            q1 = fma(t[j], s[j], q1);
            q2 = fma(t[j], t[j], q2);
          }
        q0 = split_handoff(q0, h, v);
        q1 = split_handoff(q1, h, v);
        q2 = split_handoff(q2, h, v);
#pragma unroll
        for (int j = 0; j < E0; ++j)
          if (h == 1 && j < EJ) {
            q0 = fma(s[j], s[j], q0);
            q1 = fma(t[j], s[j], q1);
            q2 = fma(t[j], t[j], q2);
          }
        q0 = h ? q0 : 0.0;
        q1 = h ? q1 : 0.0;
        q2 = h ? q2 : 0.0;
      }
      q0 = seg_sum_exact_redux<1>(q0);
      q1 = seg_sum_exact_redux<1>(q1);
      q2 = seg_sum_exact_redux<1>(q2);
      bool full = false;
      if (active) {
        if (le_nonneg(q0, thr)) {
          active = false;  // converged on the half step (x live alpha p^)
        } else if (!is_finite_bits(q1) || !is_finite_bits(q2)) {
          nonfin = true;
          active = false;
        } else if (is_zero_bits(q2)) {
          broke = true;  // keep the half step, restart
          active = false;
        } else {
          full = true;
        }
      }
      const double om = q1 * recip64s(q2);
      if (full) omega = om;
#pragma unroll
      for (int j = 0; j < E0; ++j) {
        if (full && j < EJ) {
          const int i = row(j);
          xv[j] = fma(om, gs[i], xv[j]);
          r[j] = fma(-om, o2[i], s[j]);
          p[j] = fma(-om, o1[i], p[j]);
        }
      }
      double hr = 0.0, rr = 0.0;
#pragma unroll
      for (int j = 0; j < E0; ++j)
        if (h == 0) {
          hr = fma(rhs[j], r[j], hr);
          rr = fma(r[j], r[j], rr);
        }
      hr = split_handoff(hr, h, v);
      rr = split_handoff(rr, h, v);
#pragma unroll
      for (int j = 0; j < E0; ++j)
        if (h == 1 && j < EJ) {
          hr = fma(rhs[j], r[j], hr);
          rr = fma(r[j], r[j], rr);
        }
      hr = h ? hr : 0.0;
      rr = h ? rr : 0.0;
      hr = seg_sum_exact_redux<1>(hr);
      rr = seg_sum_exact_redux<1>(rr);
      if (full) {
        nbreak = 0;
        if (le_nonneg(rr, thr)) {
          active = false;
        } else if (is_zero_bits(om)) {
          broke = true;
          active = false;
        } else {
          rho_prev = rho;
          rho = hr;
        }
      }
    }
    // ---- true residual
#pragma unroll
    for (int j = 0; j < E0; ++j)
      if (j < EJ) gs[row(j)] = xv[j];
    __syncwarp();
    spmv(o1);
    __syncwarp();
    double rt2 = 0.0;
#pragma unroll
    for (int j = 0; j < E0; ++j) {
      const int i = row(j);
      const double bi = (live && j < EJ && i < n) ? __ldg(a.b + (size_t)c * n + i) : 0.0;
      s[j] = j < EJ ? bi - o1[i] : 0.0;  // s holds the true residual here
    }
    CHAIN(rt2, s[j], s[j]);
    rt2 = seg_sum_exact_redux<1>(rt2);
    if (fin) {
      fin = false;
      resid = sqrt(rt2 * recip64(bb));
      if (nonfin || !is_finite_bits(resid)) {
        st = CAMP_CELL_NONFINITE;
      } else if (resid <= tol) {
        st = CAMP_CELL_CONVERGED;
      } else if (it >= a.maxit) {
        st = CAMP_CELL_MAXIT;
      } else if (broke && ++nbreak >= 2) {
        st = CAMP_CELL_BREAKDOWN;
      } else {
#pragma unroll
        for (int j = 0; j < E0; ++j) r[j] = s[j];
        restart = true;
      }
    }
    if (!__any_sync(kFull, restart)) break;
  }
  // ---- write the cell's results
  if (has) {
#pragma unroll
    for (int j = 0; j < E0; ++j) {
      const int i = row(j);
      if (j < EJ && i < n) a.x[(size_t)c * n + i] = xv[j];
    }
    if (lane == 0) {
      a.iters[c] = it;
      a.resid[c] = resid;
      if (a.status) a.status[c] = st;
    }
  }
  __syncwarp();
#undef CHAIN
}

}  // namespace camp
