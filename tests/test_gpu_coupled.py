"""Coupled Block-cells(k) (the paper's Block-cells(N) semantics: the cells of
a block share scalars and one convergence test) against the oracle solving
each block as one block-diagonal system, and the paper's trade-off: sharing
costs iterations on varied cells, none on identical cells."""
import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu


def _run(camp, m, A, b, tol, maxit, cpb, dev, coupled=True):
    import torch
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_arrangement(camp.CAMP_ARR_BLOCK_COUPLED if coupled else camp.CAMP_ARR_BLOCK, 0, cpb, 0)
    x, it, res, st = s.solve(torch.as_tensor(A, device=dev), torch.as_tensor(b, device=dev), tol, maxit)
    torch.cuda.synchronize()
    out = dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
               status=st.cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("cpb", [2, 3, 12])
def test_coupled_matches_block_diagonal_oracle(cuda, cpb):
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1, cells=12 * 9 + 5)   # ragged last block
    cb = cbs[0]
    m = cb.mech
    gpu = _run(camp, m, cb.A_vals, cb.b, tol, maxit, cpb, cuda)
    for c0 in range(0, cb.cells, cpb):
        k = min(cpb, cb.cells - c0)
        rp, ci, vals, rhs = parity.block_diagonal(m, cb.A_vals, cb.b, c0, k)
        orc = oracle.solve(rp, ci, vals, rhs, tol, maxit)
        blk = slice(c0, c0 + k)
        assert np.all(gpu["status"][blk] == orc["status"][0])
        assert np.all(gpu["iters"][blk] == gpu["iters"][c0])
        assert abs(int(gpu["iters"][c0]) - int(orc["iters"][0])) <= parity.ITER_SLACK
        xg = gpu["x"][blk].reshape(-1)
        xo = orc["x"][0]
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
        if err > parity.REL_TOL:
            mech_blk = synth.Mechanism(n=k * m.n, R=0, reactants=None, products=None, k=None,
                                       row_ptr=rp, col_idx=ci)
            Ad = mech_blk.dense(vals[0])
            xt = np.linalg.solve(Ad, rhs[0])
            assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 2 * np.linalg.cond(Ad, 1) * tol
        assert gpu["resid"][c0] <= tol


def test_coupling_costs_iterations_only_on_varied_cells(cuda):
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1, cells=1200)
    cb = cbs[0]
    m = cb.mech
    per_cell = _run(camp, m, cb.A_vals, cb.b, tol, maxit, 1, cuda, coupled=False)
    mean_it = {}
    for cpb in (1, 2, 3, 12):
        mean_it[cpb] = float(_run(camp, m, cb.A_vals, cb.b, tol, maxit, cpb, cuda)["iters"].mean())
    # "realistic" (varied) cells: the block system needs more iterations as it grows
    assert mean_it[1] == pytest.approx(per_cell["iters"].mean())
    assert mean_it[12] > mean_it[3] > mean_it[1]
    print("mean iterations by cells per block (coupled):", mean_it)
    # "ideal" cells (all identical): sharing the scalars changes nothing
    A = np.repeat(cb.A_vals[:1], 240, axis=0)
    b = np.repeat(cb.b[:1], 240, axis=0)
    one = _run(camp, m, A[:1], b[:1], tol, maxit, 1, cuda)
    for cpb in (2, 3, 12):
        g = _run(camp, m, A, b, tol, maxit, cpb, cuda)
        assert np.all(np.abs(g["iters"] - one["iters"][0]) <= 1)


@pytest.mark.parametrize("cpb", [2, 3, 12])
def test_coupled_hard_regime_against_block_diagonal_oracle(cuda, cpb):
    """Coupled Block-cells(k) on the hard cells (600 of them, blocks of k):
    every block against the oracle on its block-diagonal system, with the
    rounding-sensitive bar (the blocks' systems iterate tens to hundreds of
    times, where rounding moves counts); all cells of a block report the
    block's count, residual and status."""
    import os
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(5)
    cb = cbs[0]
    m = cb.mech
    C = 600
    A, b = cb.A_vals[:C], cb.b[:C]
    gpu = _run(camp, m, A, b, tol, maxit, cpb, cuda)
    nb = C // cpb
    for key in ("iters", "resid", "status"):
        per = gpu[key].reshape(nb, cpb)
        assert np.all(per == per[:, :1]), key
    rp, ci, _, _ = parity.block_diagonal(m, A, b, 0, cpb)
    mblk = synth.Mechanism(n=cpb * m.n, R=0, reactants=None, products=None, k=None,
                           row_ptr=rp, col_idx=ci)
    Ab = np.ascontiguousarray(A.reshape(nb, cpb * m.nnz))
    bb = np.ascontiguousarray(b.reshape(nb, cpb * m.n))
    gblk = dict(x=gpu["x"].reshape(nb, cpb * m.n), iters=gpu["iters"][::cpb],
                resid=gpu["resid"][::cpb], status=gpu["status"][::cpb])
    threads = os.cpu_count() or 8
    orc = oracle.solve(rp, ci, Ab, bb, tol, maxit, threads=threads)
    pert = [oracle.solve(rp, ci, Ab, parity.perturbed_rhs(bb, seed), tol, maxit, threads=threads)
            for seed in (1, 2)]
    assert orc["iters"].mean() >= 30
    res = parity.compare_sensitive(mblk, Ab, bb, tol, maxit, gblk, orc, pert,
                                   f"coupled hard k={cpb}")
    print(f"coupled hard k={cpb}: oracle mean iters {orc['iters'].mean():.1f}, gpu "
          f"{gblk['iters'].mean():.1f}; {res['gpu']} vs oracle {res['oracle_perturbed']}")
