"""Adjoint through the transposed solve: the autograd Function's gradients
against the oracle adjoint, dense LAPACK gradients and central differences;
the host-memory entry point against the device one."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_autograd_gradients(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(3, cells=64)
    cb = cbs[0]
    m = cb.mech
    w = np.random.default_rng(3000).standard_normal((64, m.n))
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=cuda).requires_grad_(True)
    b = torch.as_tensor(cb.b, device=cuda).requires_grad_(True)
    x, it, res, st = camp.solve(A, b, s, 1e-13, maxit)
    L = (x * torch.as_tensor(w, device=cuda)).sum()
    L.backward()
    gA = A.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()
    fwd = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, 1e-13, maxit)
    adj = oracle.adjoint(m.row_ptr, m.col_idx, cb.A_vals, fwd["x"], w, tol=1e-13, maxit=maxit)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    for c in range(64):
        Ad = m.dense(cb.A_vals[c])
        lam = np.linalg.solve(Ad.T, w[c])
        xd = np.linalg.solve(Ad, cb.b[c])
        kappa = np.linalg.cond(Ad, 1)
        bar = max(1e-8, 4 * kappa * 1e-13)
        assert np.linalg.norm(gb[c] - lam) <= bar * np.linalg.norm(lam)
        assert np.linalg.norm(gb[c] - adj["gb"][c]) <= bar * np.linalg.norm(lam)
        g_ref = -lam[rows] * xd[m.col_idx]
        assert np.linalg.norm(gA[c] - g_ref) <= bar * np.linalg.norm(g_ref)
        assert np.linalg.norm(gA[c] - adj["gA"][c]) <= bar * np.linalg.norm(g_ref)
    # central differences of L on 16 sampled cells (dense forward solves)
    rng = np.random.default_rng(7)
    for c in rng.choice(64, 16, replace=False):
        Ad = m.dense(cb.A_vals[c])
        for k in rng.choice(m.nnz, 3, replace=False):
            a = cb.A_vals[c, k]
            h = 1e-6 * max(1.0, abs(a))
            Ap = Ad.copy(); Ap[rows[k], m.col_idx[k]] += h
            Am = Ad.copy(); Am[rows[k], m.col_idx[k]] -= h
            fd = (w[c] @ np.linalg.solve(Ap, cb.b[c]) - w[c] @ np.linalg.solve(Am, cb.b[c])) / (2 * h)
            assert abs(fd - gA[c, k]) <= 1e-6 * max(1.0, abs(fd))
    s.close()


def test_grad_kernel_exact(cuda):
    """gA[k] = -lambda[row k] x[col k] is a single product: bitwise equal to NumPy."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, _, _ = synth.workload(1, cells=333)
    m = cbs[0].mech
    rng = np.random.default_rng(1)
    lam = rng.standard_normal((333, m.n))
    x = rng.standard_normal((333, m.n))
    s = camp.Solver(m.row_ptr, m.col_idx)
    gA = s.grad_A(torch.as_tensor(lam, device=cuda), torch.as_tensor(x, device=cuda)).cpu().numpy()
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    np.testing.assert_array_equal(gA, -lam[:, rows] * x[:, m.col_idx])
    s.close()


@pytest.mark.parametrize("cells,pinned_out", [(5000, True), (10000, True), (700, True),
                                              (5000, False)])
def test_solve_host_equals_device(cuda, cells, pinned_out):
    """The host-memory entry point (chunked copies, outputs written in place
    when the host arrays are device-addressable, staged and copied back
    otherwise) gives the device solve's bits."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1, cells=cells)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    xd, itd, rd, sd = s.solve(torch.as_tensor(cb.A_vals, device=cuda),
                              torch.as_tensor(cb.b, device=cuda), tol, maxit)
    torch.cuda.synchronize()
    C = cb.cells
    hA = torch.as_tensor(cb.A_vals).pin_memory()
    hb = torch.as_tensor(cb.b).pin_memory()
    pin = (lambda t: t.pin_memory()) if pinned_out else (lambda t: t)
    hx = pin(torch.full((C, m.n), np.nan, dtype=torch.float64))
    hit = pin(torch.full((C,), -7, dtype=torch.int32))
    hr = pin(torch.full((C,), np.nan, dtype=torch.float64))
    hs = pin(torch.full((C,), -7, dtype=torch.int32))
    camp.camp_solver_solve_host(s.h, C, hA, hb, hx, tol, maxit, hit, hr, hs)
    np.testing.assert_array_equal(hx.numpy(), xd.cpu().numpy())
    np.testing.assert_array_equal(hit.numpy(), itd.cpu().numpy())
    np.testing.assert_array_equal(hr.numpy(), rd.cpu().numpy())
    np.testing.assert_array_equal(hs.numpy(), sd.cpu().numpy())
    s.close()


def test_adjoint_full_size_all_cells(cuda):
    """Adjoint workload at full size (80 species, 10000 cells, tol 1e-10): the
    gradients of L = sum_c w_c . x_c from the autograd Function, every cell
    against the oracle's adjoint (x, lambda = dL/db and dL/dA_vals each within
    the 1e-8 bar, no cell needing a conditioning fallback), and 16 sampled
    cells against dense LAPACK gradients and central differences (step 1e-6,
    dense forward solves)."""
    import os
    import torch
    from paper_2405_17363_gb300 import camp
    from tests import parity
    cbs, tol, maxit = synth.workload(3)
    cb = cbs[0]
    m = cb.mech
    w = np.random.default_rng(3000).standard_normal((cb.cells, m.n))
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=cuda).requires_grad_(True)
    b = torch.as_tensor(cb.b, device=cuda).requires_grad_(True)
    x, it, res, st = camp.solve(A, b, s, tol, maxit)
    (x * torch.as_tensor(w, device=cuda)).sum().backward()
    assert int((st == 0).sum()) == cb.cells
    X = x.detach().cpu().numpy()
    gA = A.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()
    threads = os.cpu_count() or 8
    fwd = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=threads)
    adj = oracle.adjoint(m.row_ptr, m.col_idx, cb.A_vals, fwd["x"], w, tol=tol, maxit=maxit,
                         threads=threads)
    assert np.all(adj["status"] == 0)
    e_x = parity.rel_err(X, fwd["x"])
    e_l = parity.rel_err(gb, adj["gb"])
    e_g = parity.rel_err(gA, adj["gA"])
    assert e_x.max() <= parity.REL_TOL, e_x.max()
    assert e_l.max() <= parity.REL_TOL, e_l.max()
    # gA = -lambda[row] x[col] on the pattern: ||d gA|| <= ||d lambda|| ||x_gpu||
    # + ||lambda|| ||d x||, so relative to ||gA|| the error is bounded by the
    # two relative errors times q = ||lambda|| ||x|| / ||gA||
    q = (np.linalg.norm(adj["gb"], axis=1) * np.linalg.norm(fwd["x"], axis=1)
         / np.linalg.norm(adj["gA"], axis=1))
    bound = (e_l * (1 + e_x) + e_x) * q * (1 + 1e-6) + 1e-14
    assert np.all(e_g <= bound), np.max(e_g / bound)
    print(f"adjoint 80 sp x 10000 cells: max error x {e_x.max():.2e}, lambda {e_l.max():.2e}, "
          f"gA {e_g.max():.2e}")
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    rng = np.random.default_rng(16)
    for c in rng.choice(cb.cells, 16, replace=False):
        Ad = m.dense(cb.A_vals[c])
        lam = np.linalg.solve(Ad.T, w[c])
        xd = np.linalg.solve(Ad, cb.b[c])
        kappa = np.linalg.cond(Ad, 1)
        bar = max(1e-8, 4 * kappa * tol)
        assert np.linalg.norm(gb[c] - lam) <= bar * np.linalg.norm(lam)
        g_ref = -lam[rows] * xd[m.col_idx]
        assert np.linalg.norm(gA[c] - g_ref) <= bar * np.linalg.norm(g_ref)
        for k in rng.choice(m.nnz, 3, replace=False):
            h = 1e-6 * max(1.0, abs(cb.A_vals[c, k]))
            Ap = Ad.copy(); Ap[rows[k], m.col_idx[k]] += h
            Am = Ad.copy(); Am[rows[k], m.col_idx[k]] -= h
            fd = (w[c] @ np.linalg.solve(Ap, cb.b[c]) - w[c] @ np.linalg.solve(Am, cb.b[c])) / (2 * h)
            assert abs(fd - gA[c, k]) <= 1e-6 * max(1.0, abs(fd))
    s.close()
