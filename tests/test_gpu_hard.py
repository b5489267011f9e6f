"""Parity in the hard regime: stiff, strongly coupled systems (rate constants
up to 1e4, gamma up to 10, concentrations up to 1) on which Jacobi-BiCGSTAB
needs tens to hundreds of iterations per cell, at the full 10,000-cell size, in
the benchmark's launch configuration (automatic arrangement, in-launch
ordering), every cell against the oracle.

On these systems the iteration in finite precision depends on rounding: the
oracle itself, given right-hand sides one rounding away, takes iteration counts
more than two apart on about a fifth of the cells and changes the status of
cells near the iteration cap.  The bar (``parity.compare_sensitive``) is then:
every converged cell meets the 1e-8 bar against the oracle, every status is
consistent with the cell's own true residual and count, and the CUDA path's
spread from the oracle stays within twice the oracle's own spread (where it
converges cells the oracle does not, each is checked against a dense solve).  Three
cases: convergence at 1e-10 (mean iterations above 30), the iteration cap
reached by most cells (maxit 30), and tol 1e-15, where the recursive residual
meets the tolerance before the true one does and the residual-replacement
restart runs on thousands of cells.  A well-conditioned workload at tol 1e-15
(the benchmark's cells) keeps the strict per-cell bar, restarts included."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def camp(cuda):
    from paper_2405_17363_gb300 import camp as c
    return c


@pytest.fixture(scope="module")
def hard():
    cbs, tol, maxit = synth.workload(5)
    return cbs[0]


def _gpu(camp, m, A, b, tol, maxit, dev):
    import torch
    s = camp.Solver(m.row_ptr, m.col_idx)
    cells = b.shape[0]
    out = (torch.full((cells, m.n), float("nan"), dtype=torch.float64, device=dev),
           torch.full((cells,), -7, dtype=torch.int32, device=dev),
           torch.full((cells,), float("nan"), dtype=torch.float64, device=dev),
           torch.full((cells,), -7, dtype=torch.int32, device=dev))
    x, it, res, st = s.solve(torch.as_tensor(A, device=dev), torch.as_tensor(b, device=dev),
                             tol, maxit, out=out)
    torch.cuda.synchronize()
    s.close()
    return dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
                status=st.cpu().numpy())


def _oracles(m, A, b, tol, maxit):
    orc = oracle.solve(m.row_ptr, m.col_idx, A, b, tol, maxit, threads=THREADS)
    pert = [oracle.solve(m.row_ptr, m.col_idx, A, parity.perturbed_rhs(b, seed), tol, maxit,
                         threads=THREADS) for seed in (1, 2)]
    return orc, pert


@pytest.mark.parametrize("tol,maxit", [(1e-10, 500), (1e-10, 30), (1e-15, 500)])
def test_hard_regime_all_cells(camp, cuda, hard, tol, maxit):
    cb = hard
    m = cb.mech
    gpu = _gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda)
    orc, pert = _oracles(m, cb.A_vals, cb.b, tol, maxit)
    # every cell's true residual recomputed on the host matches the kernel's,
    # up to the rounding of the two residual computations
    r = parity.true_resid(m, cb.A_vals, gpu["x"], cb.b)
    fl = parity.resid_rounding(m, cb.A_vals, gpu["x"], cb.b)
    bad = np.nonzero(~(np.abs(gpu["resid"] - r) <= 1e-3 * r + fl))[0]
    assert bad.size == 0, (bad[:5], gpu["resid"][bad[:5]], r[bad[:5]], fl[bad[:5]])
    res = parity.compare_sensitive(m, cb.A_vals, cb.b, tol, maxit, gpu, orc, pert,
                                   f"hard tol {tol} maxit {maxit}")
    it_o = orc["iters"]
    if maxit == 500 and tol == 1e-10:
        # the regime this test exists for: long iterations, every cell converged
        assert it_o.mean() >= 30 and it_o.max() >= 200
        assert np.all(orc["status"] == 0) and np.all(gpu["status"] == 0)
        assert gpu["iters"].max() >= 200
    if maxit == 30:
        # most cells exhaust the cap, the rest converge before it
        assert (orc["status"] == 1).sum() >= 5000 and (gpu["status"] == 1).sum() >= 5000
        assert (gpu["status"] == 0).sum() >= 1000
    if tol == 1e-15:
        # residual replacement on thousands of cells; some still converge
        assert (orc["restarts"] > 0).sum() >= 1000
        assert (gpu["status"] == 0).sum() >= 1000 and (gpu["status"] == 1).sum() >= 1000
    print(f"hard tol {tol} maxit {maxit}: oracle mean iters {it_o.mean():.2f} max "
          f"{it_o.max()}, gpu mean {gpu['iters'].mean():.2f} max {gpu['iters'].max()}; "
          f"statuses gpu {np.bincount(gpu['status'], minlength=4).tolist()} oracle "
          f"{np.bincount(orc['status'], minlength=4).tolist()}; {res}")


def test_residual_replacement_well_conditioned_strict(camp, cuda):
    """The benchmark's 10,000 cells at tol 1e-15: the oracle restarts some
    cells from the true residual after the recursive one met the tolerance;
    on these systems the iteration is not sensitive to rounding, so every
    cell, the restarted ones included, meets the strict bar (status, +-2
    iterations, 1e-8)."""
    cbs, _, maxit = synth.workload(1)
    cb = cbs[0]
    m = cb.mech
    tol = 1e-15
    gpu = _gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda)
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=THREADS)
    restarted = np.nonzero(orc["restarts"] > 0)[0]
    assert restarted.size >= 10
    parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, "tol 1e-15")
    assert np.all(gpu["status"][restarted] == 0)
