// Warp-packed batched Jacobi-BiCGSTAB kernel.
//
// One warp solves k = 32/Lc cells at a time; each cell ("segment") owns Lc
// consecutive lanes, and lane sl of a segment owns rows i = sl + e*Lc,
// e = 0..E-1 (rows >= n are zero padding).  A cell's whole solve stays inside
// its segment, so cells never communicate (Block-cells, Sec. 3.1), and the
// convergence test runs on the device (Sec. 3.1, Fig. UMLMultiBlock).  The
// per-cell scalars (rho, alpha, omega, ...) are replicated in the segment's
// lanes; every FP64 instruction is issued once for all k cells of the warp.
//
// Shared memory per cell: its matrix values A_s [segA] (unless read through
// L1 from global memory), the gathered vector g_s and the products o1_s = A p^
// and o2_s = A s^ [segV each]; the shadow residual and the Jacobi reciprocals
// are lane-local and stay in registers up to kRegVecMaxE rows per lane (two
// more shared vectors beyond).
// The plain launch also keeps the SpMV schedule in shared memory; the
// persistent launch (several mechanisms) reads each mechanism's schedule
// through L1.
//
// The iteration is right-preconditioned BiCGSTAB with M = diag(A); see the
// header of the oracle for the readings of the paper (relative 2-norm test on
// s and r, true-residual check with residual replacement, breakdown and
// non-finite rules, iteration count = products v = A p^).
#pragma once
#include <type_traits>
#include "warp_common.cuh"
#include "warp_single.cuh"

namespace camp {

#ifndef CAMP_EXACT_SUMS
#define CAMP_EXACT_SUMS 1  // segment sums on the integer pipe (0: FP64 shuffle tree)
#endif

template <int LC>
__device__ __forceinline__ double ssum1(double v, int Lc) {
  if (CAMP_EXACT_SUMS) return seg_sum_x<LC>(v, Lc);
  double a[1] = {v};
  seg_sum<1>(a, Lc);
  return a[0];
}
template <int LC>
__device__ __forceinline__ void ssum2(double &a, double &b, int Lc) {
  if (CAMP_EXACT_SUMS) {
    a = seg_sum_x<LC>(a, Lc);
    b = seg_sum_x<LC>(b, Lc);
  } else {
    seg_sum2(a, b, Lc);
  }
}
template <int LC>
__device__ __forceinline__ void ssum3(double &a, double &b, double &c, int Lc) {
  if (CAMP_EXACT_SUMS) {
    a = seg_sum_x<LC>(a, Lc);
    b = seg_sum_x<LC>(b, Lc);
    c = seg_sum_x<LC>(c, Lc);
  } else {
    seg_sum3(a, b, c, Lc);
  }
}

#ifndef CAMP_WARP_MINB
#define CAMP_WARP_MINB 2  // with 256 threads per CTA at most: <= 128 registers
#endif

// Where a group's matrix values come from (template parameter SRC of
// solve_group): staged from A into shared memory in slot order, read from A
// through L1 by the SpMV, or assembled in shared memory from the cell's
// concentrations (A = I - gamma J).
constexpr int kSrcStaged = 0, kSrcGlobal = 1, kSrcAssembled = 2, kSrcNewton = 3;

// A lane's rows e = 0..E-1 of a per-cell vector: in registers, or in the
// cell's shared-memory vector (element sl + e*Lc).
template <int E, bool REG>
struct LaneRows;
template <int E>
struct LaneRows<E, true> {
  double v[E];
  __device__ __forceinline__ double &operator[](int e) { return v[e]; }
};
template <int E>
struct LaneRows<E, false> {
  double *p;
  int Lc;
  __device__ __forceinline__ void bind(double *q, int lc) { p = q; Lc = lc; }
  __device__ __forceinline__ double &operator[](int e) { return p[e * Lc]; }
};

// Newton corrector of the implicit step G(y) = y - gamma f(y) - a = 0 for
// the segment's cell (a: history term in b; y: initial guess in x, replaced
// by the solution): each iteration evaluates the mass-action rates f(y),
// sets the right-hand side -G(y), assembles A = I - gamma J(y) and solves
// A d = -G(y) through stage_and_solve, then y += d; converged when
// ||d|| <= newton_tol ||y||.  Status 0 converged, 1 iterations exhausted,
// 2 linear solve failed, 3 non-finite; iters = BiCGSTAB iterations summed.
// The iterate lives in the caller's x (it holds the guess on entry and the
// solution on return): read at the start of an iteration and written back
// after the update, so no register holds it across the linear solve.
template <int E, class Solve>
__device__ __forceinline__ void newton_loop(const WarpArgs &a, bool has, bool &live, int c,
                                            int sl, int Lc, int n, double *o1, double *o2,
                                            double *nrh, double (&xv)[E], int &st, int &it,
                                            double &resid, Solve &stage_and_solve) {
  double *yc = a.x + (size_t)c * n;  // the iterate (c is in range whenever has)
  const double gam = has ? __ldg(a.gamma + c) : 0.0;
  const double nt2 = a.newton_tol * a.newton_tol;
  const bool any = a.max_newton > 0;
  int nst = has ? (any ? -1 : 1) : 0, nit = 0, lin = 0;
  double upd = 0.0, lres = 0.0;
  bool act = has && any;
  while (__any_sync(kFull, act)) {
    // the iterate to the concentration buffer, f(y) accumulated in o1 (each
    // lane adds the terms of its own rows)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      o2[i] = (has && i < n) ? yc[i] : 0.0;
      o1[i] = 0.0;
    }
    __syncwarp();
    const double *rv = a.rval + sl;
    const int *rm = a.rmeta + sl;
    for (int q = 0; q < a.rcount; ++q) {
      const int meta = __ldg(rm + q * Lc);
      const int ya = (meta & 0x7ff) - 1, yb = ((meta >> 11) & 0x7ff) - 1;
      const int row = sl + ((meta >> 22) & 0xff) * Lc;
      double term = __ldg(rv + q * Lc) * (ya >= 0 ? o2[ya] : 1.0);
      if (yb >= 0) term *= o2[yb];
      o1[row] += term;
    }
    // right-hand side -G(y) = a - (y - gamma f(y))
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      const double ai = (act && i < n) ? __ldg(a.b + (size_t)c * n + i) : 0.0;
      nrh[i] = ai - fma(-gam, o1[i], o2[i]);
    }
    __syncwarp();
    live = act;
    stage_and_solve();
    const bool ok = act && st == CAMP_CELL_CONVERGED;
    double d2 = 0.0, y2 = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      double ye = (has && i < n) ? yc[i] : 0.0;
      if (ok) {
        ye += xv[e];
        if (i < n) yc[i] = ye;
      }
      d2 = fma(xv[e], xv[e], d2);
      y2 = fma(ye, ye, y2);
    }
    d2 = seg_sum_exact(d2, Lc);
    y2 = seg_sum_exact(y2, Lc);
    if (act) {
      ++nit;
      lin += it;
      lres = resid;
      if (!ok) {
        nst = (st == CAMP_CELL_NONFINITE) ? 3 : 2;
        act = false;
      } else if (!is_finite_bits(d2) || !is_finite_bits(y2)) {
        nst = 3;
        act = false;
      } else {
        // ||d|| <= tol ||y|| (||d|| <= tol when y = 0) on the squares
        const bool y0 = is_zero_bits(y2);
        upd = y0 ? sqrt(d2) : sqrt(d2 * recip64(y2));
        if (le_nonneg(d2, y0 ? nt2 : nt2 * y2)) {
          nst = 0;
          act = false;
        } else if (nit >= a.max_newton) {
          nst = 1;
          act = false;
        }
      }
    }
  }
  if (has && sl == 0) {
    a.newton_iters[c] = nit;
    a.iters[c] = lin;
    a.upd[c] = upd;
    a.resid[c] = lres;
    if (a.status) a.status[c] = nst;
  }
  __syncwarp();
}

// Solve the k = 32/Lc cells of group g (cells g*k .. g*k+k-1) of one
// mechanism with this warp.  wbase: the warp's shared-memory region; sch: this
// lane's column of the SpMV schedule (shared or global memory).
template <int E, int SRC, int LC = 0>
__device__ __forceinline__ void solve_group(const WarpArgs &a, int g,
                                            double *wbase,
                                            const SchedWord *sch) {
  const int lane = threadIdx.x & 31;
  const int Lc = LC ? LC : a.Lc;   // lanes per cell (compile-time when LC > 0)
  const int seg = LC ? lane / LC : lane >> a.log2Lc;
  const int sl = lane & (Lc - 1);
  const int n = a.n, nnz = a.nnz;
  const double tol = a.tol;
  double *Abase = wbase + (size_t)seg * a.segStride;
  double *gs = Abase + a.segA;   // gathered vector (p^, s^ or x)
  double *o1 = gs + a.segV;      // v = A p^
  double *o2 = o1 + a.segV;      // t = A s^
  constexpr bool kVR = E <= kRegVecMaxE;
  LaneRows<E, kVR> rhs, dvs;     // shadow residual r^, Jacobi reciprocals
  if constexpr (!kVR) {
    rhs.bind(o2 + a.segV + sl, Lc);
    dvs.bind(o2 + 2 * a.segV + sl, Lc);
  }
  double *nrh = o2 + (kVR ? 1 : 3) * a.segV;  // Newton right-hand side
  const int pos = g * (LC ? 32 / LC : a.k) + seg;
  const bool has = pos < a.cells;
  // The order may have been written earlier in this launch: read it through
  // L2.  The in-launch ordering stores cell + 1 (0: not yet written).
  // Clamped, so that even an order left incomplete indexes in bounds.
  const int c = (has && a.order)
                    ? (int)min((unsigned)(__ldcg(a.order + pos) - (a.ord_ws ? 1 : 0)),
                               (unsigned)a.cells - 1u)
                    : pos;
#define SPMV(out)                                                    \
  do {                                                               \
    if (ASMEM) seg_spmv(sch, a.L, Lc, Asl, gs, out);                 \
    else seg_spmv_gather(sch, srcl, a.L, Lc, Ac, gs, out);           \
  } while (0)
  const double *Ac = a.A + (size_t)(has ? c : 0) * nnz;
  const int *srcl = a.src + sl;
  const int LL = a.L * Lc;
  constexpr bool ASMEM = SRC != kSrcGlobal;
  const double *Asl = Abase + sl;  // this lane's slots (stride Lc)
  double xv[E];
  int st = -1, it = 0;
  double resid = 0.0;
  bool live = has;  // the cell takes part in the next solve
  // Stage (or assemble) the cell's matrix and run BiCGSTAB on it: x in xv,
  // status, iterations and true relative residual in st, it, resid.  The
  // right-hand side comes from b, or from nrh in the Newton launch; a segment
  // whose cell is not live only follows the warp's shuffles.
  auto stage_and_solve = [&]() {
  st = -1;
  it = 0;
  resid = 0.0;
  // ---- stage the cell's matrix values in slot order (Sec. 3.1: one cell,
  // one team); the transposed view's permutation is folded into src
  if (SRC == kSrcAssembled || SRC == kSrcNewton) {
    // J accumulates in place in the lane's own slots, then A = I - gamma J
    for (int t = sl; t < LL; t += Lc) Abase[t] = 0.0;
    // the cell's concentrations go to the (not yet used) t-product buffer
    // (the Newton launch has put the current iterate there)
    if (SRC == kSrcAssembled && live)
      for (int i = sl; i < n; i += Lc) o2[i] = __ldg(a.conc + (size_t)c * n + i);
    __syncwarp();
    const double gam = live ? __ldg(a.gamma + c) : 0.0;
    const double *tv = a.tval + sl;
    const int *tm = a.tmeta + sl;
    for (int p = 0; p < a.tcount; ++p) {
      const int meta = __ldg(tm + p * Lc);
      const int sp = (meta & 0x7ff) - 1;
      double *dst = Abase + ((meta >> 11) & 0x7ff) * Lc + sl;
      *dst = fma(__ldg(tv + p * Lc), sp >= 0 ? o2[sp] : 1.0, *dst);
    }
    for (int t = sl; t < LL; t += Lc) {
      const SchedWord w = sch[t - sl];  // this lane's word for slot t
      const bool dg = __ldg(a.src + t) >= 0 && (w & 0x7ffu) == ((w >> 11) & 0x7ffu);
      Abase[t] = fma(-gam, Abase[t], dg ? 1.0 : 0.0);
    }
  } else if (ASMEM) {
    // coalesced read of the cell's A row, scattered into slot order; each lane
    // zeroes its own padding slots (never a scatter target)
    stage_scatter(Ac, a.dst, nnz, sl, Lc, live, [&](int t, double v) { Abase[t] = v; });
    zero_padding(Abase, a.padfrom, a.L, Lc, sl);
  }
  // pad rows of the product vectors are never written by the SpMV
  for (int i = n + sl; i < E * Lc; i += Lc) {
    o1[i] = 0.0;
    o2[i] = 0.0;
  }
  __syncwarp();

  double r[E], p[E], s[E];
  double bb;
  {
    double acc[1] = {0.0};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      const bool v = live && i < n;
      const double bi = v ? (SRC == kSrcNewton ? nrh[i] : __ldg(a.b + (size_t)c * n + i)) : 0.0;
      const double d = v ? (ASMEM ? Abase[__ldg(a.dslot + i)]
                               : __ldg(Ac + __ldg(a.src + __ldg(a.dslot + i)))) : 0.0;
      dvs[e] = v ? (!is_zero_bits(d) ? recip64(d) : 1.0) : 0.0;
      xv[e] = (v && a.x0_given) ? a.x[(size_t)c * n + i] : 0.0;
      r[e] = bi;
      p[e] = 0.0;
      s[e] = 0.0;
      acc[0] = fma(bi, bi, acc[0]);
    }
    bb = ssum1<LC>(acc[0], Lc);
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
      for (int e = 0; e < E; ++e) xv[e] = 0.0;
    }
  }
  if (a.x0_given) {  // r = b - A x0
#pragma unroll
    for (int e = 0; e < E; ++e) gs[sl + e * Lc] = xv[e];
    __syncwarp();
    SPMV(o1);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) r[e] -= o1[sl + e * Lc];
  }

  bool restart = !done, first = true;
  bool pass0 = true;  // the solve's first (re)start, the same for every segment
  bool fin = false, active = false, broke = false, nonfin = false;
  double rho = 1.0, rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (;;) {
    {  // (re)start from the current residual r
      double acc[1] = {0.0};
      if (pass0 && !a.x0_given) {
        acc[0] = bb;  // r = b: the same chain and exact sum as ||b||^2
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) acc[0] = fma(r[e], r[e], acc[0]);
        acc[0] = ssum1<LC>(acc[0], Lc);
      }
      pass0 = false;
      if (restart) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          rhs[e] = r[e];
          p[e] = 0.0;
        }
        rho = acc[0];
        rho_prev = alpha = omega = 1.0;
        broke = nonfin = false;
        fin = true;
        // a restart follows a failed true-residual test: always iterate
        active = first ? !le_nonneg(acc[0], thr) : true;
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
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        if (active) p[e] = fma(beta, p[e], r[e]);
        gs[i] = dvs[e] * p[e];
      }
      __syncwarp();
      SPMV(o1);  // v = A p^
      __syncwarp();
      if (active) ++it;
      double sg[1] = {0.0};
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        sg[0] = fma(rhs[e], o1[i], sg[0]);
      }
      sg[0] = ssum1<LC>(sg[0], Lc);
      if (active) {
        if (!is_finite_bits(sg[0])) {
          nonfin = true;
          active = false;
        } else if (abs_tiny(sg[0])) {
          broke = true;
          active = false;
        }
      }
      const double al = rho * recip64s(sg[0]);
      if (active) alpha = al;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        if (active) {
          xv[e] = fma(al, gs[i], xv[e]);
          s[e] = fma(-al, o1[i], r[e]);
        }
        gs[i] = dvs[e] * s[e];
      }
      __syncwarp();
      SPMV(o2);  // t = A s^
      __syncwarp();
      double q0 = 0.0, q1 = 0.0, q2 = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const double t = o2[sl + e * Lc];
        q0 = fma(s[e], s[e], q0);
        q1 = fma(t, s[e], q1);
        q2 = fma(t, t, q2);
      }
      ssum3<LC>(q0, q1, q2, Lc);
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
      for (int e = 0; e < E; ++e) {
        const int i = sl + e * Lc;
        if (full) {
          xv[e] = fma(om, gs[i], xv[e]);
          r[e] = fma(-om, o2[i], s[e]);
          p[e] = fma(-om, o1[i], p[e]);
        }
      }
      double hr = 0.0, rr = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        hr = fma(rhs[e], r[e], hr);
        rr = fma(r[e], r[e], rr);
      }
      ssum2<LC>(hr, rr, Lc);
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
    // ---- true residual of the segments that stopped iterating
#pragma unroll
    for (int e = 0; e < E; ++e) gs[sl + e * Lc] = xv[e];
    __syncwarp();
    SPMV(o1);
    __syncwarp();
    double rt2[1] = {0.0};
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      const double bi = (live && i < n) ? (SRC == kSrcNewton ? nrh[i] : __ldg(a.b + (size_t)c * n + i)) : 0.0;
      s[e] = bi - o1[i];  // s holds the true residual here
      rt2[0] = fma(s[e], s[e], rt2[0]);
    }
    rt2[0] = ssum1<LC>(rt2[0], Lc);
    if (fin) {
      fin = false;
      resid = sqrt(rt2[0] * recip64(bb));
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
        for (int e = 0; e < E; ++e) r[e] = s[e];
        restart = true;
      }
    }
    if (!__any_sync(kFull, restart)) break;
  }
  };  // stage_and_solve

  if (SRC == kSrcNewton) {
    newton_loop<E>(a, has, live, c, sl, Lc, n, o1, o2, nrh, xv, st, it, resid,
                   stage_and_solve);
    return;
  }
  stage_and_solve();
  // ---- write the cell's results
  if (has) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = sl + e * Lc;
      if (i < n) a.x[(size_t)c * n + i] = xv[e];
    }
    if (sl == 0) {
      a.iters[c] = it;
      a.resid[c] = resid;
      if (a.status) a.status[c] = st;
    }
  }
  __syncwarp();
#undef SPMV
}

// Plain launch: one mechanism, the SpMV schedule in shared memory, groups of
// k cells taken by warps from the dynamic queue (or a grid-stride loop).
template <int E, int SRC>
__device__ __forceinline__ void plain_launch_body(const WarpArgs &a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SchedWord *sch_s = reinterpret_cast<SchedWord *>(smem_raw);
  const int nsch = a.L * a.Lc;
  for (int i = threadIdx.x; i < nsch; i += blockDim.x) sch_s[i] = a.sched[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  double *wbase = reinterpret_cast<double *>(smem_raw + sched_smem_bytes(nsch)) +
                  (size_t)warp * a.k * a.segStride;
  const SchedWord *sch = sch_s + (lane & (a.Lc - 1));
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  if (a.ord_ws)
    order_prologue<SRC != kSrcStaged>(a, reinterpret_cast<int *>(smem_raw + sched_smem_bytes(nsch)));
  auto run = [&](auto lc) {
    constexpr int LC = decltype(lc)::value;
    if (!a.queue) {
      for (int g = blockIdx.x * (blockDim.x >> 5) + warp; g < a.ngroups; g += warps_total)
        solve_group<E, SRC, LC>(a, g, wbase, sch);
      return;
    }
    // dynamic assignment: warps take the next group until none is left (an
    // ordered launch first gives every warp one group of a stratified wave).
    // The steps of take_group / await_order_entries, written out: built from
    // those helpers this kernel ran its first-wave groups far slower (272
    // against 212 us at 80 species x 10,000 cells).
    const bool strat = a.order && a.ord_stride == 0 && a.ord_wave > 0;
    bool first = strat;
    for (;;) {
      unsigned g = 0;
      if (first) {
        first = false;
        const unsigned B = gridDim.x, b = blockIdx.x, w = (unsigned)warp;
        g = w * B + ((w & 1u) ? B - 1u - b : b);
      } else {
        if (lane == 0) g = atomicAdd(a.queue, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (strat) g += (unsigned)a.ord_wave;
        if (g >= (unsigned)a.ngroups) break;
        if (a.order && a.ord_stride && g < (unsigned)a.ord_wave)
          g = (unsigned)((unsigned long long)g * (unsigned)a.ord_stride % (unsigned)a.ord_wave);
      }
      if constexpr (SRC == kSrcStaged && LC == 16 && E <= kRegVecMaxE) {
        if (a.sched2 && (int)g >= a.single_from) {
          // a single-cell ticket: one cell on all 32 lanes (warp_single.cuh)
          const int ps = 2 * a.single_from + ((int)g - a.single_from);
          const bool one = a.ord_ws && lane == 0 && ps < a.cells;
          if (one) wait_order_entry(a.order + ps, a.ord_ws + kOrdFlag, a.ord_err, a.ord_wait);
          __syncwarp();
          solve_single<E>(a, ps, wbase);
          if (one) a.ord_out[ps] = 0;
          continue;
        }
      }
      // in-launch ordering: wait for this group's order entries, solve,
      // then clear them
      const int p = (int)g * (LC ? 32 / LC : a.k) + lane;
      const bool mine = a.ord_ws && lane < (LC ? 32 / LC : a.k) && p < a.cells;
      if (mine) wait_order_entry(a.order + p, a.ord_ws + kOrdFlag, a.ord_err, a.ord_wait);
      __syncwarp();
      solve_group<E, SRC, LC>(a, (int)g, wbase, sch);
      if (mine) a.ord_out[p] = 0;
    }
  };
  // The arrangements the automatic choice makes for 21..160 rows (3 to 5 rows
  // per lane on 8, 16 or 32 lanes) run code with Lc fixed at compile time:
  // constant strides fold into the shared-memory addressing.
  if constexpr (E >= 3 && E <= kRegVecMaxE) {
    if (a.Lc == 16) run(std::integral_constant<int, 16>());
    else if (a.Lc == 32) run(std::integral_constant<int, 32>());
    else if (a.Lc == 8) run(std::integral_constant<int, 8>());
    else run(std::integral_constant<int, 0>());
  } else {
    run(std::integral_constant<int, 0>());
  }
  if (!a.queue) return;
  // the last warp resets the queue and the ordering workspace (and, after a
  // time-out of the ordering, marks the launch's cells invalid)
  finish_queue(a, true, warps_total, lane);
}

template <int E>
__global__ void __launch_bounds__(256, CAMP_WARP_MINB)
    warp_bicgstab_kernel(const WarpArgs a) {
  plain_launch_body<E, kSrcStaged>(a);
}

// Device Newton corrector of the implicit step around the assembly + solve.
template <int E>
__global__ void __launch_bounds__(256, CAMP_WARP_MINB)
    newton_bicgstab_kernel(const WarpArgs a) {
  plain_launch_body<E, kSrcNewton>(a);
}

// Fused Jacobian assembly and solve (A = I - gamma J(conc) built per cell).
template <int E>
__global__ void __launch_bounds__(256, CAMP_WARP_MINB)
    assemble_bicgstab_kernel(const WarpArgs a) {
  plain_launch_body<E, kSrcAssembled>(a);
}

// Persistent launch over several mechanisms (uneven batching): every warp
// takes the next work item (one group of one mechanism) from a device queue
// head until the queue is empty.  Items are ordered mechanism by mechanism,
// largest cells first, so the long items start early and the short ones fill
// the tail.  The only wait is the atomic increment: no spin, no barrier.
template <int E, bool ASMEM>
__global__ void __launch_bounds__(256, CAMP_WARP_MINB)
    batch_bicgstab_kernel(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  double *wbase = reinterpret_cast<double *>(smem_raw) + (size_t)warp * b.warp_doubles;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(b.counter, 1u);
    item = __shfl_sync(kFull, item, 0);
    if (item >= (unsigned)b.total_items) break;
    int m = 0;
    while (m + 1 < b.nmech && item >= (unsigned)b.item_begin[m + 1]) ++m;
    const WarpArgs &a = b.m[m];
    const SchedWord *sch = a.sched + (lane & (a.Lc - 1));
    solve_group<E, ASMEM ? kSrcStaged : kSrcGlobal>(a, (int)item - b.item_begin[m], wbase, sch);
  }
}

}  // namespace camp
