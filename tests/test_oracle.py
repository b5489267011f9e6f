"""Pins of the CPU oracle against facts fixed by mathematics, not by the
oracle itself: dense direct solves (LAPACK through numpy), closed forms
(diagonal systems, b = 0, A = I), exact-termination properties of Krylov
methods, constructed solutions, the residual invariant, SciPy's BiCGSTAB, and
finite differences for the adjoint."""
import numpy as np
import pytest

import oracle
import synth


def dense_of(rp, ci, vals, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = vals[rp[i]:rp[i + 1]]
    return A


def csr_of(A, keep=None):
    n = A.shape[0]
    mask = (A != 0) if keep is None else keep
    mask = mask | np.eye(n, dtype=bool)
    rp = [0]
    ci = []
    vals = []
    for i in range(n):
        cols = np.nonzero(mask[i])[0]
        ci += list(cols)
        vals += list(A[i, cols])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(vals)


def random_system(n, density, seed, dominance=1.5):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(M, 0.0)
    d = np.abs(M).sum(axis=1) * dominance + rng.uniform(0.5, 2.0, n)
    M[np.arange(n), np.arange(n)] = d * rng.choice([-1.0, 1.0], n)
    return M


def true_resid(A, x, b):
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_dense_lu_small(n, seed):
    A = random_system(n, 0.5, 100 * n + seed)
    rp, ci, vals = csr_of(A)
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n)
    out = oracle.solve(rp, ci, vals[None], b[None], tol=1e-12, maxit=200)
    x_lu = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A, 1)
    assert out["status"][0] == oracle.CONVERGED
    err = np.linalg.norm(out["x"][0] - x_lu) / np.linalg.norm(x_lu)
    assert err <= max(1e-9, 2 * kappa * 1e-12)
    assert out["resid"][0] <= 1e-12


def test_matches_dense_lu_workload0_shape():
    cbs, tol, maxit = synth.workload(0, cells=8)
    cb = cbs[0]
    m = cb.mech
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit)
    for c in range(8):
        A = m.dense(cb.A_vals[c])
        x_lu = np.linalg.solve(A, cb.b[c])
        err = np.linalg.norm(out["x"][c] - x_lu) / np.linalg.norm(x_lu)
        kappa = np.linalg.cond(A, 1)
        assert err <= max(1e-9, 2 * kappa * tol), (c, err, kappa)


def test_diagonal_system_is_one_half_step():
    """A diagonal: right-Jacobi makes A M^-1 = I, so v = r, alpha = 1, s = 0 and
    the solve ends on the half step of iteration 1 with x = b / diag."""
    n = 17
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 4.0, n) * rng.choice([-1, 1], n)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    b = rng.standard_normal((3, n))
    vals = np.tile(d, (3, 1))
    out = oracle.solve(rp, ci, vals, b, tol=1e-10, maxit=50)
    assert np.all(out["iters"] == 1)
    assert np.all(out["status"] == oracle.CONVERGED)
    np.testing.assert_allclose(out["x"], b / d, rtol=4e-16, atol=0)


def test_identity_and_zero_rhs():
    n = 9
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    b = np.vstack([np.linspace(-1, 1, n), np.zeros(n)])
    out = oracle.solve(rp, ci, np.ones((2, n)), b, tol=1e-10, maxit=5)
    assert out["iters"][0] == 1 and out["status"][0] == oracle.CONVERGED
    np.testing.assert_array_equal(out["x"][0], b[0])
    assert out["iters"][1] == 0 and out["status"][1] == oracle.CONVERGED
    assert out["resid"][1] == 0.0
    np.testing.assert_array_equal(out["x"][1], np.zeros(n))


@pytest.mark.parametrize("seed", range(5))
def test_two_step_termination_with_jacobi(seed):
    """A = (I + u v^T) D with u, v of disjoint support: diag(A) = D, so the
    right-Jacobi operator is I + u v^T whose minimal polynomial is (z-1)^2;
    BiCG, hence BiCGSTAB, terminates within 2 iterations.  Without the
    preconditioner (or with a wrong beta/omega) it would not."""
    n = 24
    rng = np.random.default_rng(seed)
    u = np.zeros(n)
    v = np.zeros(n)
    u[: n // 2] = rng.standard_normal(n // 2)
    v[n // 2:] = rng.standard_normal(n - n // 2)
    D = np.diag(rng.uniform(0.2, 5.0, n))
    A = (np.eye(n) + np.outer(u, v)) @ D
    rp, ci, vals = csr_of(A)
    b = rng.standard_normal(n)
    out = oracle.solve(rp, ci, vals[None], b[None], tol=1e-10, maxit=50)
    assert out["status"][0] == oracle.CONVERGED
    assert out["iters"][0] <= 2
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"][0] - x) / np.linalg.norm(x) < 1e-9


@pytest.mark.parametrize("n", [2, 3, 4])
def test_terminates_within_n_iterations(n):
    """In exact arithmetic BiCGSTAB (no breakdown) ends within n iterations."""
    for seed in range(6):
        A = random_system(n, 1.0, 7 * n + seed, dominance=1.2)
        rp, ci, vals = csr_of(A)
        b = np.random.default_rng(seed).standard_normal(n)
        out = oracle.solve(rp, ci, vals[None], b[None], tol=1e-11, maxit=50)
        assert out["status"][0] == oracle.CONVERGED
        assert out["iters"][0] <= n


def test_constructed_solution_and_residual_invariant():
    cbs, tol, maxit = synth.workload(1, cells=64)
    cb = cbs[0]
    m = cb.mech
    rng = np.random.default_rng(9)
    xs = rng.standard_normal((64, m.n))
    b = np.stack([m.dense(cb.A_vals[c]) @ xs[c] for c in range(64)])
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, b, tol, maxit)
    for c in range(64):
        A = m.dense(cb.A_vals[c])
        r = true_resid(A, out["x"][c], b[c])
        assert out["status"][c] == oracle.CONVERGED
        assert r <= tol
        # both residuals carry rounding of order eps * (|A||x| + |b|)
        slack = 64 * np.finfo(float).eps * np.linalg.norm(
            np.abs(A) @ np.abs(out["x"][c]) + np.abs(b[c])) / np.linalg.norm(b[c])
        assert abs(out["resid"][c] - r) <= slack
        kappa = np.linalg.cond(A, 1)
        err = np.linalg.norm(out["x"][c] - xs[c]) / np.linalg.norm(xs[c])
        assert err <= kappa * tol, (c, err, kappa)


def test_scipy_bicgstab_agrees():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    cbs, tol, maxit = synth.workload(2, cells=6)
    for cb in cbs:
        m = cb.mech
        out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit)
        for c in range(cb.cells):
            A = scipy_sparse.csr_matrix((cb.A_vals[c], m.col_idx, m.row_ptr),
                                        shape=(m.n, m.n))
            Minv = scipy_sparse.diags(1.0 / A.diagonal())
            xs, info = spla.bicgstab(A, cb.b[c], rtol=1e-13, atol=0.0, M=Minv,
                                     maxiter=1000)
            assert info == 0
            kappa = np.linalg.cond(A.toarray(), 1)
            err = np.linalg.norm(out["x"][c] - xs) / np.linalg.norm(xs)
            assert err <= max(1e-9, 2 * kappa * tol)


def test_nonfinite_inputs():
    cbs, tol, maxit = synth.workload(0, cells=3)
    cb = cbs[0]
    m = cb.mech
    A = cb.A_vals.copy()
    b = cb.b.copy()
    b[0, 3] = np.nan
    A[1, 5] = np.inf
    out = oracle.solve(m.row_ptr, m.col_idx, A, b, tol, maxit)
    assert out["status"][0] == oracle.NONFINITE
    assert out["status"][1] == oracle.NONFINITE
    assert out["status"][2] == oracle.CONVERGED


def test_singular_zero_row_terminates():
    cbs, tol, maxit = synth.workload(0, cells=1)
    cb = cbs[0]
    m = cb.mech
    A = cb.A_vals.copy()
    A[0, m.row_ptr[4]:m.row_ptr[5]] = 0.0   # row 4 all zero (diag too)
    out = oracle.solve(m.row_ptr, m.col_idx, A, cb.b, tol, 40)
    assert out["status"][0] in (oracle.MAXIT, oracle.BREAKDOWN)
    assert out["iters"][0] <= 40
    assert out["resid"][0] > tol


def test_skew_system_breaks_down_twice():
    """A = [[0, 1], [-1, 0]]: zero diagonal (Jacobi guard uses 1) and
    r^T A r = 0 for every r, so sigma = r^.v = 0 on the first iteration of every
    restart; the second breakdown ends the cell after 2 iterations."""
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    vals = np.array([[0.0, 1.0, -1.0, 0.0]])
    out = oracle.solve(rp, ci, vals, np.array([[1.0, 2.0]]), tol=1e-10, maxit=50)
    assert out["status"][0] == oracle.BREAKDOWN
    assert out["iters"][0] == 2


def test_maxit_and_identical_cells():
    cbs, tol, maxit = synth.workload(0, cells=2)
    cb = cbs[0]
    m = cb.mech
    A = np.repeat(cb.A_vals[:1], 4, axis=0)
    b = np.repeat(cb.b[:1], 4, axis=0)
    out = oracle.solve(m.row_ptr, m.col_idx, A, b, tol, maxit, threads=4)
    assert np.all(out["iters"] == out["iters"][0])
    for c in range(1, 4):
        np.testing.assert_array_equal(out["x"][c], out["x"][0])
    one = oracle.solve(m.row_ptr, m.col_idx, A[:1], b[:1], tol, 1)
    assert one["status"][0] == oracle.MAXIT and one["iters"][0] == 1


def test_initial_guess():
    cbs, tol, maxit = synth.workload(0, cells=2)
    cb = cbs[0]
    m = cb.mech
    x_lu = np.stack([np.linalg.solve(m.dense(cb.A_vals[c]), cb.b[c]) for c in range(2)])
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, x0=x_lu)
    assert np.all(out["iters"] == 0) and np.all(out["status"] == oracle.CONVERGED)
    x0 = x_lu + 1e-3
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, x0=x0)
    assert np.all(out["status"] == oracle.CONVERGED)
    assert np.all(out["iters"] >= 1)


def test_transpose_pattern_rebuilds_dense_transpose():
    cbs, _, _ = synth.workload(1, cells=2)
    cb = cbs[0]
    m = cb.mech
    rpt, cit, src = oracle.transpose_pattern(m.row_ptr, m.col_idx)
    assert sorted(src) == list(range(m.nnz))
    for c in range(2):
        AT = dense_of(rpt, cit, cb.A_vals[c][src], m.n)
        np.testing.assert_array_equal(AT, m.dense(cb.A_vals[c]).T)


def test_adjoint_against_dense_and_finite_differences():
    """L = w . x, x = A^{-1} b: dL/db = A^{-T} w, dL/dA_ij = -lambda_i x_j.
    Checked against dense LAPACK solves and central differences of L computed
    with dense solves (forward error far below the difference step)."""
    cbs, tol, maxit = synth.workload(3, cells=4)
    cb = cbs[0]
    m = cb.mech
    rng = np.random.default_rng(3000)
    w = rng.standard_normal((4, m.n))
    fwd = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, 1e-14, maxit)
    adj = oracle.adjoint(m.row_ptr, m.col_idx, cb.A_vals, fwd["x"], w, tol=1e-14, maxit=maxit)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    for c in range(4):
        A = m.dense(cb.A_vals[c])
        lam = np.linalg.solve(A.T, w[c])
        x = np.linalg.solve(A, cb.b[c])
        np.testing.assert_allclose(adj["lam"][c], lam, rtol=1e-9, atol=1e-12 * np.abs(lam).max())
        gA = -lam[rows] * x[m.col_idx]
        np.testing.assert_allclose(adj["gA"][c], gA, rtol=1e-8, atol=1e-11 * np.abs(gA).max())
        # central differences on a few entries and b components
        for k in rng.choice(m.nnz, 6, replace=False):
            a = cb.A_vals[c, k]
            h = 1e-6 * max(1.0, abs(a))
            Ap = A.copy(); Ap[rows[k], m.col_idx[k]] += h
            Am = A.copy(); Am[rows[k], m.col_idx[k]] -= h
            fd = (w[c] @ np.linalg.solve(Ap, cb.b[c]) - w[c] @ np.linalg.solve(Am, cb.b[c])) / (2 * h)
            assert abs(fd - adj["gA"][c, k]) <= 1e-6 * max(1.0, abs(fd))
        for i in rng.choice(m.n, 4, replace=False):
            bp = cb.b[c].copy(); bp[i] += 1e-6
            bm = cb.b[c].copy(); bm[i] -= 1e-6
            fd = (w[c] @ np.linalg.solve(A, bp) - w[c] @ np.linalg.solve(A, bm)) / 2e-6
            assert abs(fd - adj["gb"][c, i]) <= 1e-6 * max(1.0, abs(fd))


def test_mixed_precision_refinement():
    """FP32 inner solves cannot reach 1e-10 alone (FP32 unit round-off 6e-8);
    the FP64 refinement must, in a few sweeps, and agree with a dense solve."""
    cbs, tol, _ = synth.workload(4, cells=16)
    cb = cbs[0]
    m = cb.mech
    out = oracle.solve_mixed(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol)
    assert np.all(out["status"] == oracle.CONVERGED)
    assert np.all(out["resid"] <= tol)
    assert np.all(out["sweeps"] >= 2) and np.all(out["sweeps"] <= 6)
    for c in range(16):
        A = m.dense(cb.A_vals[c])
        x = np.linalg.solve(A, cb.b[c])
        kappa = np.linalg.cond(A, 1)
        err = np.linalg.norm(out["x"][c] - x) / np.linalg.norm(x)
        assert err <= max(1e-9, 2 * kappa * tol)
        assert true_resid(A, out["x"][c], cb.b[c]) <= tol


def test_threads_do_not_change_results():
    cbs, tol, maxit = synth.workload(1, cells=200)
    cb = cbs[0]
    m = cb.mech
    a = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=1)
    b = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["iters"], b["iters"])


def _scipy_count(A, b, tol, maxit, x0=None):
    """SciPy's BiCGSTAB (right preconditioning with M^-1 = diag(A)^-1, stop on
    ||s|| or ||r|| against rtol*||b||): the textbook iteration in a library.
    Returns (iterations, x, info); iterations = products v = A p^ (half-step
    exits count as one), derived from the number of matrix-vector calls."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    scipy_sparse = pytest.importorskip("scipy.sparse")
    n = A.shape[0]
    calls = [0]

    def mv(v):
        calls[0] += 1
        return A @ v

    op = spla.LinearOperator((n, n), matvec=mv, dtype=float)
    Minv = scipy_sparse.diags(1.0 / A.diagonal())
    x, info = spla.bicgstab(op, b, x0=x0, rtol=tol, atol=0.0, M=Minv, maxiter=maxit)
    init = 1 if x0 is not None else 0   # SciPy forms b - A x0 when x0 is given
    return (calls[0] - init + 1) // 2, x, info


@pytest.mark.parametrize("wid", [1, 2])
def test_iteration_counts_equal_scipy(wid):
    """Same algorithm, same stopping rule: the per-cell iteration counts agree
    exactly (a wrong alpha, beta, omega, preconditioner or test changes them)."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    cbs, tol, maxit = synth.workload(wid, cells=40)
    for cb in cbs:
        m = cb.mech
        out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit)
        for c in range(cb.cells):
            A = scipy_sparse.csr_matrix((cb.A_vals[c], m.col_idx, m.row_ptr),
                                        shape=(m.n, m.n))
            it, xs, info = _scipy_count(A, cb.b[c], tol, maxit)
            assert info == 0
            assert out["iters"][c] == it, (c, out["iters"][c], it)
            np.testing.assert_allclose(out["x"][c], xs, rtol=1e-9,
                                       atol=1e-9 * np.abs(xs).max())


def test_residual_replacement_matches_scipy_restart():
    """When the recursive residual meets tol but the true one does not, the
    oracle restarts from r = b - A x, r^ = r: exactly a second SciPy call with
    x0 = x.  Only cells whose decisions are clear of rounding are compared."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    tol = 1e-15
    cbs, _, maxit = synth.workload(2, cells=200)
    checked = 0
    for cb in cbs:
        m = cb.mech
        out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit)
        for c in range(cb.cells):
            A = scipy_sparse.csr_matrix((cb.A_vals[c], m.col_idx, m.row_ptr),
                                        shape=(m.n, m.n))
            b = cb.b[c]
            it1, x1, info1 = _scipy_count(A, b, tol, maxit)
            r1 = np.linalg.norm(b - A @ x1) / np.linalg.norm(b)
            if info1 != 0 or r1 <= 1.02 * tol:
                continue
            it2, x2, info2 = _scipy_count(A, b, tol, maxit - it1, x0=x1)
            r2 = np.linalg.norm(b - A @ x2) / np.linalg.norm(b)
            if info2 != 0 or r2 >= 0.5 * tol:
                continue
            checked += 1
            assert out["status"][c] == oracle.CONVERGED
            assert out["iters"][c] == it1 + it2, (c, out["iters"][c], it1, it2)
            assert out["restarts"][c] == 1
    assert checked >= 1


def test_initial_guess_iteration_counts_equal_scipy():
    """With x0 given, r0 = b - A x0 and the shadow vector r^ = r0 (SciPy does
    the same): counts and solutions agree."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    cbs, tol, maxit = synth.workload(1, cells=30)
    cb = cbs[0]
    m = cb.mech
    x0 = np.random.default_rng(5).standard_normal((30, m.n))
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, x0=x0)
    for c in range(30):
        A = scipy_sparse.csr_matrix((cb.A_vals[c], m.col_idx, m.row_ptr), shape=(m.n, m.n))
        it, xs, info = _scipy_count(A, cb.b[c], tol, maxit, x0=x0[c].copy())
        assert info == 0
        assert out["iters"][c] == it, (c, out["iters"][c], it)
        np.testing.assert_allclose(out["x"][c], xs, rtol=1e-9, atol=1e-9 * np.abs(xs).max())


def test_assembly_matches_independent_numpy_jacobian():
    """The oracle's C mass-action assembly against the generator's NumPy one
    (itself pinned by Euler's identity and finite differences of the rates):
    two codings of the same Jacobian agree to rounding."""
    for wid in (0, 1, 4):
        cbs, _, _ = synth.workload(wid, cells=12)
        cb = cbs[0]
        m = cb.mech
        A = oracle.assemble(m.row_ptr, m.col_idx, m.reactants[:, 0], m.reactants[:, 1],
                            m.products, m.k, cb.conc, cb.gamma)
        scale = np.abs(cb.A_vals).max(axis=1, keepdims=True)
        assert np.all(np.abs(A - cb.A_vals) <= 1e-15 * scale)


def test_assembly_rejects_entries_outside_the_pattern():
    m = synth.make_mechanism(8, 6, 3)
    # drop one off-diagonal coupling from the pattern
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    k = int(np.nonzero(rows != m.col_idx)[0][0])
    keep = np.ones(m.nnz, bool)
    keep[k] = False
    ci = m.col_idx[keep]
    rp = np.r_[0, np.cumsum(np.bincount(rows[keep], minlength=m.n))].astype(np.int32)
    with pytest.raises(ValueError):
        oracle.assemble(rp, ci, m.reactants[:, 0], m.reactants[:, 1], m.products, m.k,
                        np.ones((1, m.n)), [0.1])


def test_rates_match_independent_numpy_rates():
    cbs, _, _ = synth.workload(1, cells=5)
    cb = cbs[0]
    m = cb.mech
    F = oracle.rates(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k, cb.conc)
    np.testing.assert_allclose(F, m.rates(cb.conc), rtol=1e-13, atol=1e-30)


def test_newton_linear_mechanism_is_one_step():
    """First-order reactions only: f is linear, G(y) = (I - gamma J) y - a, so
    Newton lands on the dense solution in one step and confirms it with a
    negligible second update."""
    m = synth.make_mechanism(12, 16, 3)
    keep = m.reactants[:, 1] < 0
    ra, rb, pr, k = m.reactants[keep, 0], m.reactants[keep, 1], m.products[keep], m.k[keep]
    rng = np.random.default_rng(0)
    a = rng.uniform(0.1, 1.0, (4, m.n))
    gam = np.array([1e-3, 1e-2, 0.1, 1.0])
    out = oracle.newton(m.row_ptr, m.col_idx, ra, rb, pr, k, a, gam, a.copy(),
                        newton_tol=1e-9, lin_tol=1e-13)
    assert np.all(out["status"] == 0) and np.all(out["newton_iters"] == 2)
    for c in range(4):
        J = np.zeros((m.n, m.n))
        for r in range(len(k)):
            J[ra[r], ra[r]] -= k[r]
            J[pr[r], ra[r]] += k[r]
        y = np.linalg.solve(np.eye(m.n) - gam[c] * J, a[c])
        np.testing.assert_allclose(out["y"][c], y, rtol=1e-11)


def test_newton_root_satisfies_the_step_equation():
    """The full (second-order) mechanism: the converged y makes the implicit
    step's residual y - gamma f(y) - a vanish, with f evaluated by the
    generator's independent rate code, and agrees with SciPy's root finder."""
    optimize = pytest.importorskip("scipy.optimize")
    cbs, _, _ = synth.workload(1, cells=6)
    cb = cbs[0]
    m = cb.mech
    a = cb.conc
    out = oracle.newton(m.row_ptr, m.col_idx, m.reactants[:, 0], m.reactants[:, 1],
                        m.products, m.k, a, cb.gamma, a.copy(), newton_tol=1e-12)
    assert np.all(out["status"] == 0)
    for c in range(6):
        y = out["y"][c]
        G = y - cb.gamma[c] * m.rates(y) - a[c]
        assert np.linalg.norm(G) <= 1e-10 * np.linalg.norm(a[c])
        sol = optimize.root(lambda z: z - cb.gamma[c] * m.rates(z) - a[c], a[c], tol=1e-15)
        np.testing.assert_allclose(y, sol.x, rtol=1e-8, atol=1e-12 * np.abs(a[c]).max())


def test_restart_count_is_zero_without_replacement():
    """Cells that converge on their first run (true residual within tol at
    the first exit) report no restart; SciPy needs one call for them."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    cbs, tol, maxit = synth.workload(1, cells=40)
    cb = cbs[0]
    m = cb.mech
    out = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit)
    for c in range(cb.cells):
        A = scipy_sparse.csr_matrix((cb.A_vals[c], m.col_idx, m.row_ptr), shape=(m.n, m.n))
        it1, x1, info1 = _scipy_count(A, cb.b[c], tol, maxit)
        r1 = np.linalg.norm(cb.b[c] - A @ x1) / np.linalg.norm(cb.b[c])
        if info1 == 0 and r1 <= 0.5 * tol:
            assert out["restarts"][c] == 0


def test_hard_regime_is_sensitive_to_rounding():
    """The reading behind the hard-regime parity bar: on stiff, strongly
    coupled systems (the hard workload) the oracle itself, given right-hand
    sides one rounding away, takes iteration counts more than two apart on
    many cells while every converged solution stays within the 1e-8 bar; on
    the benchmark's systems the counts do not move."""
    from tests import parity
    cbs, tol, maxit = synth.workload(5, cells=2000)
    cb = cbs[0]
    m = cb.mech
    o = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    p = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, parity.perturbed_rhs(cb.b, 1), tol,
                     maxit, threads=8)
    assert o["iters"].mean() >= 30 and o["iters"].max() >= 150
    sp = parity.spread(o, p)
    assert sp["frac_iters_off"] >= 0.05 and sp["max_iters_off"] >= 20
    assert np.all(o["status"] == 0) and np.all(p["status"] == 0)
    assert parity.rel_err(p["x"], o["x"]).max() <= parity.REL_TOL
    cbs, tol, maxit = synth.workload(1, cells=2000)
    cb = cbs[0]
    m = cb.mech
    o = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    p = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, parity.perturbed_rhs(cb.b, 1), tol,
                     maxit, threads=8)
    assert parity.spread(o, p)["max_iters_off"] <= 1


def test_sensitive_bar_accepts_rounding_and_rejects_planted_mistakes():
    """compare_sensitive accepts the oracle on a third one-rounding change of
    b (a correct implementation with different rounding) and rejects: counts
    raised by three, a right-hand side off by 1e-6 (x misses the 1e-8 bar),
    the oracle run to a looser tolerance (converged residuals above tol), and
    an implementation that gives up early (a lower iteration cap)."""
    from tests import parity
    cbs, tol, maxit = synth.workload(5, cells=2000)
    cb = cbs[0]
    m = cb.mech

    def run(b, t=tol):
        return oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, b, t, maxit, threads=8)

    o = run(cb.b)
    pert = [run(parity.perturbed_rhs(cb.b, s)) for s in (1, 2)]
    ok = run(parity.perturbed_rhs(cb.b, 3))
    parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit, ok, o, pert, "third perturbation")
    shifted = dict(ok, iters=np.minimum(ok["iters"] + 3, maxit))
    with pytest.raises(AssertionError):
        parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit,
                                 oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, 60,
                                              threads=8), o, pert, "early cap")
    with pytest.raises(AssertionError):
        parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit, shifted, o, pert, "shift")
    with pytest.raises(AssertionError):
        parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit, run(cb.b * (1 + 1e-6)), o,
                                 pert, "wrong b")
    with pytest.raises(AssertionError):
        parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit, run(cb.b, 1e-6), o, pert,
                                 "loose tol")
