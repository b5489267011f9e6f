"""Single-cell tickets of the plain 16-lane launch (warp_single.cuh): a cell
solved alone on all 32 lanes must give bit for bit what its pair solve gives
(same operations in the same order: the split schedule keeps every row's
chain, the dot products hand their partials across the two half-warps), for
any number of single tickets, under every ordering, on ragged and tiny
batches, the hard cells, a given initial guess, the transposed solve and the
edge cases (b = 0, non-finite b, a zero row)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ALL = 1 << 30  # more single tickets than any batch has pairs: every cell alone


def _solve(camp, s, A, b, tol, maxit, tail, ordering, **kw):
    import torch
    s.set_single_tail(tail)
    s.set_ordering(ordering)
    cells = b.shape[0]
    out = (torch.full((cells, b.shape[1]), float("nan"), dtype=torch.float64, device=b.device),
           torch.full((cells,), -7, dtype=torch.int32, device=b.device),
           torch.full((cells,), float("nan"), dtype=torch.float64, device=b.device),
           torch.full((cells,), -7, dtype=torch.int32, device=b.device))
    got = s.solve(A, b, tol, maxit, out=out, **kw)
    torch.cuda.synchronize()
    return [t.clone() for t in got]


def _assert_same(ref, got, label):
    import torch
    names = ("x", "iters", "resid", "status")
    for nm, r, g in zip(names, ref, got):
        if nm in ("x", "resid"):
            same = torch.equal(r.view(torch.int64), g.view(torch.int64))  # NaN bits too
        else:
            same = torch.equal(r, g)
        assert same, f"{label}: {nm} differs"


@pytest.mark.parametrize("wid,cells", [(1, 10000), (1, 4001), (1, 777), (1, 3), (1, 2), (1, 1),
                                       (5, 10000), (2, 3000)])
def test_single_tickets_are_bitwise_the_pair_solve(cuda, wid, cells):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(wid, cells=cells)
    cb = cbs[1] if wid == 2 else cbs[0]   # workload 2: its 80-species mechanism
    m = cb.mech
    assert 32 < m.n <= 80  # 16 lanes per cell, at most 5 rows per lane
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    ref = _solve(camp, s, A, b, tol, maxit, 0, 0)
    for tail in (1, 137, 1000, ALL, -1):
        for ordering in (0, 1):
            got = _solve(camp, s, A, b, tol, maxit, tail, ordering)
            _assert_same(ref, got, f"wid {wid} cells {cells} tail {tail} ordering {ordering}")
    s.close()


def test_single_tickets_hard_guess_and_transpose(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(5, cells=3001)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    x0 = torch.as_tensor(np.random.default_rng(4).standard_normal(cb.b.shape), device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    for kw in ({"x0": x0}, {"transpose": True}, {"x0": x0, "transpose": True}):
        ref = _solve(camp, s, A, b, tol, maxit, 0, 0, **kw)
        for tail in (500, ALL):
            got = _solve(camp, s, A, b, tol, maxit, tail, 1, **kw)
            _assert_same(ref, got, f"hard {sorted(kw)} tail {tail}")
    # the iteration cap and tol 1e-15 (residual-replacement restarts)
    for t, mi in ((1e-10, 30), (1e-15, 500)):
        ref = _solve(camp, s, A, b, t, mi, 0, 0)
        got = _solve(camp, s, A, b, t, mi, ALL, 0)
        _assert_same(ref, got, f"hard tol {t} maxit {mi}")
    s.close()


def test_single_tickets_edge_cases(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1, cells=9)
    cb = cbs[0]
    m = cb.mech
    Ah = cb.A_vals.copy()
    bh = cb.b.copy()
    bh[1] = 0.0                                  # b = 0
    bh[2, 4] = np.nan                            # non-finite
    Ah[3, m.row_ptr[5]:m.row_ptr[6]] = 0.0       # a zero row (zero diagonal)
    Ah[4] = Ah[5]                                # identical cells
    bh[4] = bh[5]
    A = torch.as_tensor(Ah, device=cuda)
    b = torch.as_tensor(bh, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    ref = _solve(camp, s, A, b, tol, 30, 0, 0)
    got = _solve(camp, s, A, b, tol, 30, ALL, 0)
    _assert_same(ref, got, "edge cases")
    assert int(got[3][2]) == camp.CAMP_CELL_NONFINITE and int(got[1][1]) == 0
    s.close()


@pytest.mark.parametrize("n,R", [(12, 20), (24, 48), (40, 90), (56, 130), (80, 200)])
def test_single_tickets_every_rows_per_lane(cuda, n, R):
    """At 16 lanes per cell with 1 to 5 rows per lane (the split gives the
    upper lanes 0, 1, 1, 2 and 2 rows; odd counts leave them a spare slot):
    single tickets bit for bit the pair solve, on 1,001 cells."""
    import torch
    from paper_2405_17363_gb300 import camp
    m = synth.make_mechanism(n, R, 500 + n)
    cb = synth.make_cells(m, 1001, 600 + n, gamma=(1e-4, 1e-1))
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_arrangement(camp.CAMP_ARR_WARP, 16, 1, 0)
    ref = _solve(camp, s, A, b, 1e-10, 500, 0, 0)
    for tail in (77, ALL):
        for ordering in (0, 1):
            got = _solve(camp, s, A, b, 1e-10, 500, tail, ordering)
            _assert_same(ref, got, f"n {n} tail {tail} ordering {ordering}")
    assert int((ref[3] == 0).sum()) == 1001
    s.close()
