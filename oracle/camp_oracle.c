/*
 * CPU oracle for the batched Jacobi-preconditioned BiCGSTAB solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (the paper, Sec. 2.2 and Sec. 3.1): every grid cell c holds
 * an independent sparse linear system A_c x_c = b_c (the Newton system of the
 * BDF step of the chemistry ODE); all cells share one CSR sparsity pattern and
 * each cell is solved on its own (Block-cells: one cell, one solve, no coupling
 * between cells).  The paper names the iterative solver "Biconjugate Gradient
 * (BCG)" (Sec. 3.1) built from SpMV, dot products, vector updates and
 * reductions, with a per-cell convergence test and the iteration count of the
 * slowest cell as the reported figure (Sec. 3.2).  It prints no algorithm text,
 * so the iteration is the stabilised variant BiCGSTAB (van der Vorst, SIAM J.
 * Sci. Stat. Comput. 13, 1992) preconditioned on the right with the Jacobi
 * matrix M = diag(A) (the paper runs without a preconditioner and names one as
 * future work, Sec. 5.2).  Plain FP64, natural row order, one cell at a time,
 * nine work vectors per cell (the paper's "nine auxiliary arrays", Sec. 5.1).
 *
 * Readings where the paper is silent (all stated in the design notes):
 *  - tol is relative: ||b - A x||_2 <= tol ||b||_2.  It is tested on the
 *    recursive residual after the half step (s) and after the full step (r);
 *    on exit the true residual is recomputed and, if it fails while iterations
 *    remain, the iteration restarts from r = b - A x, r^ = r (residual
 *    replacement).  resid_out is always the true relative residual.
 *  - iteration count = number of v = A p^ products; restarts keep counting;
 *    the final true-residual product is not counted.
 *  - breakdown: |rho| < 1e-300, |r^.v| < 1e-300, t.t == 0 or omega == 0 causes
 *    a restart; a second breakdown with no completed iteration in between ends
 *    the cell with status BREAKDOWN.
 *  - a non-finite scalar ends the cell with status NONFINITE.
 *  - x0 = 0 unless an initial guess is supplied; b == 0 gives x = 0, 0 iters.
 *  - Jacobi guard: a zero diagonal entry uses 1 in place of 1/A_ii.
 *
 * Mixed precision (workload with FP32 inner solves): iterative refinement.
 * Outer sweeps in FP64: r = b - A x; stop when ||r|| <= tol ||b||; otherwise
 * solve A d = r/||r|| in FP32 with the same BiCGSTAB (FP32 A, FP32 Jacobi) to
 * an inner relative tolerance or an inner iteration cap, then x += ||r|| d in
 * FP64.
 *
 * Adjoint: lambda = A^{-T} w by the same BiCGSTAB on the transposed pattern
 * (built here, independently of the library), dL/db = lambda and
 * dL/dA_k = -lambda[row k] * x[col k] on the pattern.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CONVERGED 0
#define ORC_MAXIT 1
#define ORC_BREAKDOWN 2
#define ORC_NONFINITE 3

#define ORC_TINY 1e-300

/* y = A x for one cell (CSR, natural row order). */
static void spmv(int n, const int *rp, const int *ci, const double *a,
                 const double *x, double *y) {
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc += a[k] * x[ci[k]];
    y[i] = acc;
  }
}

static double dot(int n, const double *u, const double *w) {
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += u[i] * w[i];
  return acc;
}

/*
 * One cell.  x holds the initial guess on entry when x0_given != 0; x is the
 * solution on return.  Returns the status code.  restarts_out (or NULL)
 * receives the number of restarts from r = b - A x (residual replacement
 * after a failed true-residual test, or after a breakdown).
 */
int orc_bicgstab_cell_r(int n, const int *rp, const int *ci, const double *a,
                        const double *b, double tol, int maxit, int x0_given,
                        double *x, int *iters_out, double *resid_out,
                        int *restarts_out) {
  /* the nine work arrays */
  double *work = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  double *r = work, *rh = r + n, *p = rh + n, *v = p + n, *s = v + n,
         *t = s + n, *ph = t + n, *sh = ph + n, *dinv = sh + n;
  int status = ORC_MAXIT, iters = 0, restarts = 0;
  double resid = 0.0;

  /* Jacobi preconditioner M = diag(A), applied on the right */
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d = a[k];
    dinv[i] = (d != 0.0) ? 1.0 / d : 1.0;
  }
  if (!x0_given)
    for (int i = 0; i < n; ++i) x[i] = 0.0;

  const double bnorm = sqrt(dot(n, b, b));
  if (!isfinite(bnorm)) {
    status = ORC_NONFINITE;
    resid = NAN;
    goto done;
  }
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    status = ORC_CONVERGED;
    resid = 0.0;
    goto done;
  }

  /* r = b - A x */
  spmv(n, rp, ci, a, x, t);
  for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];

  int nbreak = 0; /* breakdowns since the last completed iteration */
  for (;;) {
    /* (re)start from the current residual r */
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    for (int i = 0; i < n; ++i) {
      rh[i] = r[i];
      p[i] = 0.0;
      v[i] = 0.0;
    }
    int conv = (sqrt(dot(n, r, r)) / bnorm <= tol);
    int broke = 0, nonfin = 0;
    while (!conv && iters < maxit) {
      const double rho = dot(n, rh, r);
      if (!isfinite(rho)) { nonfin = 1; break; }
      if (fabs(rho) < ORC_TINY) { broke = 1; break; }
      const double beta = (rho / rho_prev) * (alpha / omega);
      for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      for (int i = 0; i < n; ++i) ph[i] = dinv[i] * p[i];
      spmv(n, rp, ci, a, ph, v);
      ++iters;
      const double sigma = dot(n, rh, v);
      if (!isfinite(sigma)) { nonfin = 1; break; }
      if (fabs(sigma) < ORC_TINY) { broke = 1; break; }
      alpha = rho / sigma;
      for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      if (sqrt(dot(n, s, s)) / bnorm <= tol) {
        for (int i = 0; i < n; ++i) x[i] += alpha * ph[i];
        conv = 1;
        break;
      }
      for (int i = 0; i < n; ++i) sh[i] = dinv[i] * s[i];
      spmv(n, rp, ci, a, sh, t);
      const double tt = dot(n, t, t);
      const double ts = dot(n, t, s);
      if (!isfinite(tt) || !isfinite(ts)) { nonfin = 1; break; }
      if (tt == 0.0) {
        /* keep the valid half step, then restart */
        for (int i = 0; i < n; ++i) x[i] += alpha * ph[i];
        broke = 1;
        break;
      }
      omega = ts / tt;
      for (int i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
      for (int i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
      nbreak = 0;
      if (sqrt(dot(n, r, r)) / bnorm <= tol) { conv = 1; break; }
      if (omega == 0.0) { broke = 1; break; }
      rho_prev = rho;
    }
    /* true residual */
    spmv(n, rp, ci, a, x, t);
    for (int i = 0; i < n; ++i) t[i] = b[i] - t[i];
    resid = sqrt(dot(n, t, t)) / bnorm;
    if (nonfin || !isfinite(resid)) { status = ORC_NONFINITE; break; }
    if (resid <= tol) { status = ORC_CONVERGED; break; }
    if (iters >= maxit) { status = ORC_MAXIT; break; }
    if (broke && ++nbreak >= 2) { status = ORC_BREAKDOWN; break; }
    (void)conv;
    for (int i = 0; i < n; ++i) r[i] = t[i]; /* residual replacement */
    ++restarts;
  }
done:
  *iters_out = iters;
  *resid_out = resid;
  if (restarts_out) *restarts_out = restarts;
  free(work);
  return status;
}

int orc_bicgstab_cell(int n, const int *rp, const int *ci, const double *a,
                      const double *b, double tol, int maxit, int x0_given,
                      double *x, int *iters_out, double *resid_out) {
  return orc_bicgstab_cell_r(n, rp, ci, a, b, tol, maxit, x0_given, x, iters_out,
                             resid_out, NULL);
}

/* ---- FP32 inner solve for the mixed-precision refinement ---------------- */

static void spmv_f(int n, const int *rp, const int *ci, const float *a,
                   const float *x, float *y) {
  for (int i = 0; i < n; ++i) {
    float acc = 0.0f;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc += a[k] * x[ci[k]];
    y[i] = acc;
  }
}

static float dot_f(int n, const float *u, const float *w) {
  float acc = 0.0f;
  for (int i = 0; i < n; ++i) acc += u[i] * w[i];
  return acc;
}

/* FP32 right-Jacobi BiCGSTAB on A d = c with x0 = 0, stopping on the recursive
 * residual only (the FP64 outer sweep checks the true residual).  Returns the
 * number of iterations. */
static int inner_f32(int n, const int *rp, const int *ci, const float *a,
                     const float *dinv, const float *c, float tol_in,
                     int maxit_in, float *d, float *work) {
  float *r = work, *rh = r + n, *p = rh + n, *v = p + n, *s = v + n,
        *t = s + n, *ph = t + n, *sh = ph + n;
  for (int i = 0; i < n; ++i) {
    d[i] = 0.0f;
    r[i] = c[i];
    rh[i] = c[i];
    p[i] = 0.0f;
    v[i] = 0.0f;
  }
  const float cnorm = sqrtf(dot_f(n, c, c));
  if (!(cnorm > 0.0f) || !isfinite(cnorm)) return 0;
  float rho_prev = 1.0f, alpha = 1.0f, omega = 1.0f;
  int it = 0;
  while (it < maxit_in) {
    const float rho = dot_f(n, rh, r);
    if (!isfinite(rho) || fabsf(rho) < 1e-37f) break;
    const float beta = (rho / rho_prev) * (alpha / omega);
    for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    for (int i = 0; i < n; ++i) ph[i] = dinv[i] * p[i];
    spmv_f(n, rp, ci, a, ph, v);
    ++it;
    const float sigma = dot_f(n, rh, v);
    if (!isfinite(sigma) || fabsf(sigma) < 1e-37f) break;
    alpha = rho / sigma;
    for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    if (sqrtf(dot_f(n, s, s)) / cnorm <= tol_in) {
      for (int i = 0; i < n; ++i) d[i] += alpha * ph[i];
      break;
    }
    for (int i = 0; i < n; ++i) sh[i] = dinv[i] * s[i];
    spmv_f(n, rp, ci, a, sh, t);
    const float tt = dot_f(n, t, t);
    const float ts = dot_f(n, t, s);
    if (!isfinite(tt) || !isfinite(ts) || tt == 0.0f) {
      for (int i = 0; i < n; ++i) d[i] += alpha * ph[i];
      break;
    }
    omega = ts / tt;
    for (int i = 0; i < n; ++i) d[i] += alpha * ph[i] + omega * sh[i];
    for (int i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
    if (sqrtf(dot_f(n, r, r)) / cnorm <= tol_in) break;
    if (omega == 0.0f) break;
    rho_prev = rho;
  }
  return it;
}

/*
 * Mixed-precision refinement for one cell.  iters_out = total inner FP32
 * iterations, sweeps_out = outer FP64 sweeps that ran an inner solve.
 */
int orc_mixed_cell(int n, const int *rp, const int *ci, const double *a,
                   const double *b, double tol, int max_sweeps, double tol_in,
                   int maxit_in, double *x, int *iters_out, int *sweeps_out,
                   double *resid_out) {
  int nnz = rp[n];
  float *af = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  float *fw = (float *)malloc(sizeof(float) * 11 * (size_t)(n > 0 ? n : 1));
  double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  float *dinv = fw + 8 * n, *c = dinv + n, *d = c + n;
  int status = ORC_MAXIT, iters = 0, sweeps = 0;
  double resid = 0.0;
  for (int k = 0; k < nnz; ++k) af[k] = (float)a[k];
  for (int i = 0; i < n; ++i) {
    float dg = 0.0f;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) dg = af[k];
    dinv[i] = (dg != 0.0f) ? 1.0f / dg : 1.0f;
    x[i] = 0.0;
  }
  const double bnorm = sqrt(dot(n, b, b));
  if (!isfinite(bnorm)) { status = ORC_NONFINITE; resid = NAN; goto done; }
  if (bnorm == 0.0) { status = ORC_CONVERGED; goto done; }
  for (;;) {
    spmv(n, rp, ci, a, x, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    const double rn = sqrt(dot(n, r, r));
    resid = rn / bnorm;
    if (!isfinite(resid)) { status = ORC_NONFINITE; break; }
    if (resid <= tol) { status = ORC_CONVERGED; break; }
    if (sweeps >= max_sweeps) { status = ORC_MAXIT; break; }
    for (int i = 0; i < n; ++i) c[i] = (float)(r[i] / rn);
    iters += inner_f32(n, rp, ci, af, dinv, c, (float)tol_in, maxit_in, d, fw);
    ++sweeps;
    for (int i = 0; i < n; ++i) x[i] += rn * (double)d[i];
  }
done:
  *iters_out = iters;
  *sweeps_out = sweeps;
  *resid_out = resid;
  free(af);
  free(fw);
  free(r);
  return status;
}

/* ---- adjoint ----------------------------------------------------------- */

/* Transposed CSR of the pattern: rpt[n+1], cit[nnz] and src[nnz] with
 * AT_vals[k] = A_vals[src[k]].  Counting sort over columns. */
void orc_transpose_pattern(int n, const int *rp, const int *ci, int *rpt,
                           int *cit, int *src) {
  int nnz = rp[n];
  for (int j = 0; j <= n; ++j) rpt[j] = 0;
  for (int k = 0; k < nnz; ++k) rpt[ci[k] + 1]++;
  for (int j = 0; j < n; ++j) rpt[j + 1] += rpt[j];
  int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) fill[j] = rpt[j];
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      int q = fill[ci[k]]++;
      cit[q] = i;
      src[q] = k;
    }
  free(fill);
}

/* gA[k] = -lambda[row k] * x[col k] for one cell */
void orc_grad_A_cell(int n, const int *rp, const int *ci, const double *lambda,
                     const double *x, double *gA) {
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) gA[k] = -lambda[i] * x[ci[k]];
}

/* ---- batches over cells, threaded ------------------------------------- */

typedef struct {
  int kind; /* 0 = FP64 solve, 1 = mixed */
  int cells, n, nnz;
  const int *rp, *ci;
  const double *a, *b;
  double tol, tol_in;
  int maxit, maxit_in, max_sweeps, x0_given;
  double *x, *resid;
  int *iters, *status, *sweeps, *restarts;
  int next; /* shared cell counter */
} batch_t;

static void *batch_worker(void *arg) {
  batch_t *B = (batch_t *)arg;
  for (;;) {
    int c = __atomic_fetch_add(&B->next, 1, __ATOMIC_RELAXED);
    if (c >= B->cells) break;
    const double *a = B->a + (size_t)c * B->nnz;
    const double *b = B->b + (size_t)c * B->n;
    double *x = B->x + (size_t)c * B->n;
    if (B->kind == 0) {
      B->status[c] = orc_bicgstab_cell_r(B->n, B->rp, B->ci, a, b, B->tol,
                                         B->maxit, B->x0_given, x, &B->iters[c],
                                         &B->resid[c],
                                         B->restarts ? &B->restarts[c] : NULL);
    } else {
      int sw = 0;
      B->status[c] = orc_mixed_cell(B->n, B->rp, B->ci, a, b, B->tol,
                                    B->max_sweeps, B->tol_in, B->maxit_in, x,
                                    &B->iters[c], &sw, &B->resid[c]);
      if (B->sweeps) B->sweeps[c] = sw;
    }
  }
  return NULL;
}

static int run_batch(batch_t *B, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  B->next = 0;
  if (nthreads == 1) {
    batch_worker(B);
    return 0;
  }
  pthread_t th[512];
  int started = 0;
  for (int i = 0; i < nthreads; ++i) {
    if (pthread_create(&th[i], NULL, batch_worker, B) != 0) break;
    ++started;
  }
  if (started == 0) batch_worker(B);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  return started;
}

/* All cells of a batch: a [cells x nnz], b/x [cells x n]; cells are claimed
 * from a shared counter by nthreads threads.  restarts [cells] (or NULL)
 * receives each cell's restart count.  Returns the threads used. */
int orc_bicgstab_batch(int cells, int n, int nnz, const int *rp, const int *ci,
                       const double *a, const double *b, double tol, int maxit,
                       int x0_given, double *x, int *iters, double *resid,
                       int *status, int *restarts, int nthreads) {
  batch_t B;
  memset(&B, 0, sizeof B);
  B.kind = 0; B.cells = cells; B.n = n; B.nnz = nnz; B.rp = rp; B.ci = ci;
  B.a = a; B.b = b; B.tol = tol; B.maxit = maxit; B.x0_given = x0_given;
  B.x = x; B.iters = iters; B.resid = resid; B.status = status;
  B.restarts = restarts;
  int used = run_batch(&B, nthreads);
  return used > 0 ? used : 1;
}

int orc_mixed_batch(int cells, int n, int nnz, const int *rp, const int *ci,
                    const double *a, const double *b, double tol,
                    int max_sweeps, double tol_in, int maxit_in, double *x,
                    int *iters, int *sweeps, double *resid, int *status,
                    int nthreads) {
  batch_t B;
  memset(&B, 0, sizeof B);
  B.kind = 1; B.cells = cells; B.n = n; B.nnz = nnz; B.rp = rp; B.ci = ci;
  B.a = a; B.b = b; B.tol = tol; B.max_sweeps = max_sweeps; B.tol_in = tol_in;
  B.maxit_in = maxit_in; B.x = x; B.iters = iters; B.sweeps = sweeps;
  B.resid = resid; B.status = status;
  int used = run_batch(&B, nthreads);
  return used > 0 ? used : 1;
}

/* ---- mass-action Jacobian assembly (the step before the solve) --------- */

/* Position of (row i, column j) in the CSR pattern, or -1. */
static int csr_pos(const int *rp, const int *ci, int i, int j) {
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    if (ci[k] == j) return k;
  return -1;
}

/*
 * A = I - gamma J(conc) for one cell on the CSR pattern, J the mass-action
 * Jacobian of R reactions: reaction r consumes ra[r] (and rb[r] when
 * rb[r] >= 0) and produces pr[r] at rate k[r] y_a (first order) or
 * k[r] y_a y_b (second order), so dy_i/dt sums -rate over consumed and +rate
 * over produced species (the paper's f_i = sum_j (dy_i/dt)_j, Sec. 2.2) and J
 * is its derivative in y.  J is accumulated in reaction order, each term a
 * separately rounded product and sum.  Returns 0, or -1 if a Jacobian entry
 * falls outside the pattern.
 */
int orc_assemble_cell(int n, const int *rp, const int *ci, int R,
                      const int *ra, const int *rb, const int *pr,
                      const double *k, const double *conc, double gamma,
                      double *A) {
  int nnz = rp[n];
  for (int q = 0; q < nnz; ++q) A[q] = 0.0; /* J accumulates here first */
  for (int r = 0; r < R; ++r) {
    const int a = ra[r], b = rb[r], c = pr[r];
    if (b < 0) {
      /* rate = k y_a: d/dy_a of -rate (row a) and +rate (row c) */
      int p1 = csr_pos(rp, ci, a, a), p2 = csr_pos(rp, ci, c, a);
      if (p1 < 0 || p2 < 0) return -1;
      A[p1] = A[p1] - k[r];
      A[p2] = A[p2] + k[r];
    } else {
      /* rate = k y_a y_b: d/dy_a = k y_b, d/dy_b = k y_a; rows a, b lose, c gains */
      const double da = k[r] * conc[b], db = k[r] * conc[a];
      int paa = csr_pos(rp, ci, a, a), pab = csr_pos(rp, ci, a, b);
      int pba = csr_pos(rp, ci, b, a), pbb = csr_pos(rp, ci, b, b);
      int pca = csr_pos(rp, ci, c, a), pcb = csr_pos(rp, ci, c, b);
      if (paa < 0 || pab < 0 || pba < 0 || pbb < 0 || pca < 0 || pcb < 0) return -1;
      A[paa] = A[paa] - da;
      A[pab] = A[pab] - db;
      A[pba] = A[pba] - da;
      A[pbb] = A[pbb] - db;
      A[pca] = A[pca] + da;
      A[pcb] = A[pcb] + db;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int q = rp[i]; q < rp[i + 1]; ++q)
      A[q] = ((ci[q] == i) ? 1.0 : 0.0) - gamma * A[q];
  return 0;
}

/* ---- Newton corrector of the implicit step around the solve ------------ */

/* f_i(y) = dy_i/dt: every reaction r has rate k[r] y_a (first order) or
 * k[r] y_a y_b (second order); it is subtracted from its reactants' rows and
 * added to its product's row (Sec. 2.2: f_i sums the reactions' terms). */
void orc_rates_cell(int n, int R, const int *ra, const int *rb, const int *pr,
                    const double *k, const double *y, double *f) {
  for (int i = 0; i < n; ++i) f[i] = 0.0;
  for (int r = 0; r < R; ++r) {
    const int a = ra[r], b = rb[r], c = pr[r];
    const double rate = (b < 0) ? k[r] * y[a] : k[r] * y[a] * y[b];
    f[a] = f[a] - rate;
    if (b >= 0) f[b] = f[b] - rate;
    f[c] = f[c] + rate;
  }
}

/*
 * The nonlinear system of one implicit (BDF) step, G(y) = y - gamma f(y) - a
 * = 0 (a: the step's history term, e.g. y^n for backward Euler), by Newton's
 * method from the initial guess in y: each iteration assembles the Newton
 * matrix A = I - gamma J(y), solves A d = -G(y) with the BiCGSTAB above
 * (lin_tol, lin_maxit) and sets y += d; converged when ||d||_2 <= newton_tol
 * ||y||_2.  The paper's CVODE/BDF step needs exactly these linear systems
 * (Sec. 2.2); the solver loop around them is its future work (Sec. 6).
 * Returns 0 converged, 1 iterations exhausted, 2 linear solve failed,
 * 3 non-finite.  newton_iters = iterations run, lin_iters = BiCGSTAB
 * iterations summed, upd = final ||d|| / ||y||.
 */
int orc_newton_cell(int n, const int *rp, const int *ci, int R, const int *ra,
                    const int *rb, const int *pr, const double *k,
                    const double *a_hist, double gamma, double *y,
                    double newton_tol, int max_newton, double lin_tol,
                    int lin_maxit, int *newton_iters, int *lin_iters,
                    double *upd) {
  const int nnz = rp[n];
  double *A = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double *w = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double *f = w, *rhs = w + n, *d = w + 2 * n;
  int status = 1, it = 0, lin = 0;
  double u = 0.0;
  for (it = 0; it < max_newton;) {
    orc_rates_cell(n, R, ra, rb, pr, k, y, f);
    for (int i = 0; i < n; ++i) rhs[i] = -(y[i] - gamma * f[i] - a_hist[i]);
    if (orc_assemble_cell(n, rp, ci, R, ra, rb, pr, k, y, gamma, A) != 0) { status = 2; break; }
    int li = 0;
    double res = 0.0;
    const int ls = orc_bicgstab_cell(n, rp, ci, A, rhs, lin_tol, lin_maxit, 0, d, &li, &res);
    lin += li;
    ++it;
    if (ls != ORC_CONVERGED) { status = (ls == ORC_NONFINITE) ? 3 : 2; break; }
    for (int i = 0; i < n; ++i) y[i] += d[i];
    const double dn = sqrt(dot(n, d, d)), yn = sqrt(dot(n, y, y));
    u = (yn > 0.0) ? dn / yn : dn;
    if (!isfinite(u)) { status = 3; break; }
    if (u <= newton_tol) { status = 0; break; }
  }
  *newton_iters = it;
  *lin_iters = lin;
  *upd = u;
  free(A);
  free(w);
  return status;
}
