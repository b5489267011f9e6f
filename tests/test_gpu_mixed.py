"""FP32-inner / FP64-outer refinement on the GPU against the oracle: the
refined solution must meet the FP64 bar against the FP64 oracle, statuses must
match the refinement oracle and outer sweep counts agree within one."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wid,cells", [(4, 300), (1, 515), (0, 64)])
def test_mixed_matches_fp64_oracle(cuda, wid, cells):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(wid, cells=cells)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    x, it, sw, res, st = s.solve_mixed(A, b, tol)
    torch.cuda.synchronize()
    gpu = dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
               status=st.cpu().numpy())
    sweeps = sw.cpu().numpy()
    mix = oracle.solve_mixed(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, threads=8)
    f64 = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    assert np.array_equal(gpu["status"], mix["status"])
    assert np.all(np.abs(sweeps - mix["sweeps"]) <= 1)
    assert np.all(gpu["status"] == 0)
    r = parity.true_resid(m, cb.A_vals, gpu["x"], cb.b)
    assert np.all(r <= tol * 1.0001)
    # the error against the FP64 oracle, per cell, with the parity bar
    gpu_cmp = dict(gpu, iters=f64["iters"])   # inner FP32 counts are not FP64 counts
    parity.compare(m, cb.A_vals, cb.b, tol, gpu_cmp, f64, f"mixed wid{wid}")
    err = np.linalg.norm(gpu["x"] - f64["x"], axis=1) / np.linalg.norm(f64["x"], axis=1)
    print(f"mixed wid{wid}: error vs FP64 oracle max {err.max():.2e} p99 "
          f"{np.percentile(err, 99):.2e}; sweeps mean {sweeps.mean():.2f}")
    s.close()


def test_mixed_full_size_all_cells(cuda):
    """Mixed-precision workload at full size (150 species, 100000 cells): every
    cell's FP64 true residual on the host, every cell against the FP64 oracle
    (the 1e-8 bar) and against the refinement oracle (sweeps within one)."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(4)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    x, it, sw, res, st = s.solve_mixed(A, b, tol)
    torch.cuda.synchronize()
    X = x.cpu().numpy()
    status = st.cpu().numpy()
    sweeps = sw.cpu().numpy()
    assert np.all(status == 0)
    for lo in range(0, cb.cells, 20000):
        hi = lo + 20000
        r = parity.true_resid(m, cb.A_vals[lo:hi], X[lo:hi], cb.b[lo:hi])
        assert np.all(r <= tol * 1.0001)
    threads = os.cpu_count() or 8
    f64 = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=threads)
    mix = oracle.solve_mixed(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, threads=threads)
    assert np.array_equal(status, mix["status"])
    assert np.all(np.abs(sweeps - mix["sweeps"]) <= 1)
    gpu = dict(x=X, iters=f64["iters"], resid=res.cpu().numpy(), status=status)
    parity.compare(m, cb.A_vals, cb.b, tol, gpu, f64, "mixed full")
    err = parity.rel_err(X, f64["x"])
    print(f"mixed 150 sp x 100000 cells: error vs FP64 oracle max {err.max():.2e} "
          f"p99 {np.percentile(err, 99):.2e}")
    s.close()


@pytest.mark.parametrize("wid,cells", [(1, 10000), (0, 300), (4, 3001)])
def test_mixed_ordering_gives_identical_results(cuda, wid, cells):
    """The refinement kernel under the three orderings (index order, ordered
    inside the cooperative launch, separate ordering pass) and the explicit
    16-lanes-per-cell arrangement (2 cells per warp): bitwise identical
    outputs, since a cell's refinement does not depend on where it runs."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(wid, cells=cells)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    for lanes in (0, 16):
        if lanes:
            s.set_arrangement(camp.CAMP_ARR_WARP, lanes, 1, 0)
        s.set_ordering(0)
        ref = [t.clone() for t in s.solve_mixed(A, b, tol)]
        out = [torch.empty_like(t) for t in ref]
        for mode in (1, 2, 1, 1):
            s.set_ordering(mode)
            for t in out:  # a cell the launch skipped keeps the poison
                t.fill_(float("nan") if t.is_floating_point() else -7)
            got = s.solve_mixed(A, b, tol, out=out)
            torch.cuda.synchronize()
            for r, g in zip(ref, got):
                assert torch.equal(r, g), (lanes, mode)
    s.close()
