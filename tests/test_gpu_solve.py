"""Parity of the CUDA batched solve with the oracle (element by element on the
same seeded inputs), for every arrangement, the workloads' shapes and the edge
cases.  Every call goes through the C ABI (ctypes binding)."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu

KEYS = ("x", "iters", "resid", "status")
THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def camp(cuda):
    from paper_2405_17363_gb300 import camp as c
    return c


def to_dev(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def run_gpu(camp, mech, A_vals, b, tol, maxit, dev, arrangement=None, x0=None,
            transpose=False):
    import torch
    s = camp.Solver(mech.row_ptr, mech.col_idx)
    if arrangement is not None:
        s.set_arrangement(*arrangement)
    cells = b.shape[0]
    # outputs poisoned (NaN, -7): a cell the launch skipped cannot pass
    poison = (torch.full((cells, mech.n), float("nan"), dtype=torch.float64, device=dev),
              torch.full((cells,), -7, dtype=torch.int32, device=dev),
              torch.full((cells,), float("nan"), dtype=torch.float64, device=dev),
              torch.full((cells,), -7, dtype=torch.int32, device=dev))
    x, it, res, st = s.solve(to_dev(A_vals, dev), to_dev(b, dev), tol, maxit,
                             x0=None if x0 is None else to_dev(x0, dev),
                             transpose=transpose, out=poison)
    torch.cuda.synchronize()
    out = dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
               status=st.cpu().numpy())
    s.close()
    return out


def arrangements(n):
    out = [("auto", None)]
    for lc in (1, 2, 4, 8, 16, 32):
        if (n + lc - 1) // lc <= 16:
            out.append((f"warp{lc}", (1, lc, 0, 0)))
    for cpb in (1, 2, 3):
        if cpb * n <= 1024:
            out.append((f"block{cpb}", (2, 0, cpb, 0)))
    nmax = 1024 // n
    if nmax > 3:
        out.append((f"blockN{nmax}", (2, 0, nmax, 0)))
    return out


@pytest.mark.parametrize("wid,cells", [(0, 64), (1, 515), (4, 131)])
def test_parity_all_arrangements(camp, cuda, wid, cells):
    cbs, tol, maxit = synth.workload(wid, cells=cells)
    cb = cbs[0]
    m = cb.mech
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    for name, arr in arrangements(m.n):
        gpu = run_gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda, arr)
        parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, f"wid{wid}/{name}")


def test_parity_uneven_mechanisms(camp, cuda):
    cbs, tol, maxit = synth.workload(2, cells=300)
    for cb in cbs:
        m = cb.mech
        orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
        gpu = run_gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda)
        parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, f"n{m.n}")


def test_full_size_all_cells(camp, cuda):
    """The benchmark's workload at full size (80 species, 10000 cells) in the
    launch configuration the benchmark times: every cell's residual checked on
    the host and every cell against the oracle, with no cell needing the
    conditioning fallback."""
    cbs, tol, maxit = synth.workload(1)
    cb = cbs[0]
    m = cb.mech
    gpu = run_gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda)
    assert np.all(gpu["status"] == 0)
    r = parity.true_resid(m, cb.A_vals, gpu["x"], cb.b)
    assert np.all(r <= tol * 1.0001)
    np.testing.assert_allclose(gpu["resid"], r, rtol=1e-3, atol=1e-15)
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=THREADS)
    assert parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, "full") == 0


def test_edge_cases(camp, cuda):
    import torch
    cbs, tol, maxit = synth.workload(0, cells=9)
    cb = cbs[0]
    m = cb.mech
    A = cb.A_vals.copy()
    b = cb.b.copy()
    b[1] = 0.0                               # b = 0 -> x = 0, 0 iterations
    b[2, 4] = np.nan                         # non-finite
    A[3, m.row_ptr[5]:m.row_ptr[6]] = 0.0    # singular: zero row
    A[4] = A[5]; b[4] = b[5]                 # identical cells
    for name, arr in arrangements(m.n):
        orc = oracle.solve(m.row_ptr, m.col_idx, A, b, tol, 30)
        gpu = run_gpu(camp, m, A, b, tol, 30, cuda, arr)
        assert np.array_equal(gpu["status"], orc["status"]), name
        assert gpu["iters"][1] == 0 and np.all(gpu["x"][1] == 0) and gpu["resid"][1] == 0
        assert gpu["status"][2] == 3
        assert gpu["status"][3] in (1, 2)
        np.testing.assert_array_equal(gpu["x"][4], gpu["x"][5])
        assert gpu["iters"][4] == gpu["iters"][5]
        keep = [0, 5, 6, 7, 8]
        parity.compare(m, A[keep], b[keep], tol, {k: gpu[k][keep] for k in KEYS},
                       {k: orc[k][keep] for k in KEYS}, name)
    # a single cell, and zero cells (nothing enqueued)
    gpu = run_gpu(camp, m, A[:1], b[:1], tol, maxit, cuda)
    orc = oracle.solve(m.row_ptr, m.col_idx, A[:1], b[:1], tol, maxit)
    parity.compare(m, A[:1], b[:1], tol, gpu, orc, "one cell")
    s = camp.Solver(m.row_ptr, m.col_idx)
    e = torch.empty(0, dtype=torch.float64, device=cuda)
    ei = torch.empty(0, dtype=torch.int32, device=cuda)
    camp.camp_solver_solve(s.h, 0, e, e, e, tol, maxit, ei, e)
    with pytest.raises(camp.CampError) as ex:
        camp.camp_solver_solve(s.h, 1, to_dev(A[:1], cuda), to_dev(b[:1], cuda),
                               torch.empty((1, m.n), dtype=torch.float64, device=cuda),
                               0.0, maxit, torch.empty(1, dtype=torch.int32, device=cuda),
                               torch.empty(1, dtype=torch.float64, device=cuda))
    assert ex.value.code == camp.CAMP_EINVAL
    s.close()


def test_diagonal_and_tiny_patterns(camp, cuda):
    rng = np.random.default_rng(4)
    for n in (1, 2, 31, 32, 33, 64):
        rp = np.arange(n + 1, dtype=np.int32)
        ci = np.arange(n, dtype=np.int32)
        mech = synth.Mechanism(n=n, R=0, reactants=None, products=None, k=None,
                               row_ptr=rp, col_idx=ci)
        d = rng.uniform(0.5, 3.0, (37, n))
        b = rng.standard_normal((37, n))
        for name, arr in arrangements(n):
            gpu = run_gpu(camp, mech, d, b, 1e-10, 20, cuda, arr)
            assert np.all(gpu["iters"] == 1), (n, name)
            # x = alpha * b / d with alpha = 1 up to the iteration scalars'
            # one-step Newton reciprocal (relative error about 2^-44)
            np.testing.assert_allclose(gpu["x"], b / d, rtol=2.0 ** -43, atol=0)


def test_skew_breakdown(camp, cuda):
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    mech = synth.Mechanism(n=2, R=0, reactants=None, products=None, k=None,
                           row_ptr=rp, col_idx=ci)
    A = np.array([[0.0, 1.0, -1.0, 0.0]] * 5)
    b = np.array([[1.0, 2.0]] * 5)
    for name, arr in arrangements(2):
        gpu = run_gpu(camp, mech, A, b, 1e-10, 50, cuda, arr)
        assert np.all(gpu["status"] == 2) and np.all(gpu["iters"] == 2), name


def test_initial_guess_and_transpose(camp, cuda):
    cbs, tol, maxit = synth.workload(1, cells=100)
    cb = cbs[0]
    m = cb.mech
    x0 = np.random.default_rng(5).standard_normal((100, m.n))
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, x0=x0)
    for name, arr in arrangements(m.n)[:4] + [arrangements(m.n)[-1]]:
        gpu = run_gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda, arr, x0=x0)
        parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, f"x0/{name}")
    rpt, cit, src = oracle.transpose_pattern(m.row_ptr, m.col_idx)
    AT = cb.A_vals[:, src]
    orcT = oracle.solve(rpt, cit, AT, cb.b, tol, maxit)
    mT = synth.Mechanism(n=m.n, R=0, reactants=None, products=None, k=None,
                         row_ptr=rpt, col_idx=cit)
    for name, arr in arrangements(m.n)[:4] + [arrangements(m.n)[-1]]:
        gpu = run_gpu(camp, m, cb.A_vals, cb.b, tol, maxit, cuda, arr, transpose=True)
        parity.compare(mT, AT, cb.b, tol, gpu, orcT, f"T/{name}")


def _poison(out):
    """Fill output buffers with values no solve writes (NaN, -7), so that a
    cell a launch skipped cannot pass for a solved one."""
    for t in out:
        t.fill_(float("nan") if t.is_floating_point() else -7)


@pytest.mark.parametrize("wid", [1, 4])
def test_difficulty_ordering_gives_identical_results(camp, cuda, wid):
    """Handing cells to warps hardest first changes which cells share a warp,
    never a cell's result: bitwise identical outputs, transposed solves too,
    for both the in-launch ordering (1) and the separate pass (2).  The batch
    sizes change from call to call (ragged, tiny, larger than one ordering
    piece per CTA), so a workspace or order entry left over from the previous
    launch would misplace cells."""
    import torch
    cbs, tol, maxit = synth.workload(wid, cells=2001)
    cb = cbs[0]
    m = cb.mech
    A0 = torch.as_tensor(cb.A_vals, device=cuda)
    b0 = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    for cells in (2001, 2, 1500, 33, 2001, 2001 * 90):
        reps = (cells + 2000) // 2001
        A = A0.repeat(reps, 1)[:cells].contiguous()
        b = b0.repeat(reps, 1)[:cells].contiguous()
        for transpose in (False, True):
            s.set_ordering(0)
            ref = [t.clone() for t in s.solve(A, b, tol, maxit, transpose=transpose)]
            out = [torch.empty_like(t) for t in ref]
            for mode in (1, 2, 1):
                s.set_ordering(mode)
                _poison(out)  # a cell the launch skipped keeps the poison
                got = s.solve(A, b, tol, maxit, transpose=transpose, out=out)
                torch.cuda.synchronize()
                for r, g in zip(ref, got):
                    assert torch.equal(r, g), (cells, transpose, mode)
    s.close()


def test_ordering_sample_and_recalibration(camp, cuda):
    """The in-launch ordering reads the whole diagonal on its first ordered
    solve, then only the rows where the estimate peaked, and the whole
    diagonal again every 64 ordered solves: through 140 solves (two
    recalibrations) every result stays bitwise that of index order.  A
    mechanism with no more rows than the sample always reads them all."""
    import torch
    cbs, tol, maxit = synth.workload(1, cells=3001)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    ref = [t.clone() for t in s.solve(A, b, tol, maxit)]
    out = [torch.empty_like(t) for t in ref]
    s.set_ordering(1)
    for rep in range(140):
        _poison(out)
        got = s.solve(A, b, tol, maxit, transpose=False, out=out)
        for r, g in zip(ref, got):
            assert torch.equal(r, g), rep
    s.close()
    mech = synth.make_mechanism(6, 12, 5)
    small = synth.make_cells(mech, 777, 6, gamma=(1e-4, 1e-1))
    A = torch.as_tensor(small.A_vals, device=cuda)
    b = torch.as_tensor(small.b, device=cuda)
    s = camp.Solver(mech.row_ptr, mech.col_idx)
    ref = [t.clone() for t in s.solve(A, b, tol, maxit)]
    out = [torch.empty_like(t) for t in ref]
    s.set_ordering(1)
    for rep in range(3):
        _poison(out)
        got = s.solve(A, b, tol, maxit, out=out)
        for r, g in zip(ref, got):
            assert torch.equal(r, g), rep
    s.close()


def test_ordered_solve_in_cuda_graph(camp, cuda):
    """The ordered (cooperative) solve captured in a CUDA graph: replays give
    bitwise the eager index-order results, also after the inputs change in
    place (the order entries are cleared by every replay)."""
    import torch
    cbs, tol, maxit = synth.workload(1, cells=4000)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_ordering(0)
    ref = [t.clone() for t in s.solve(A, b, tol, maxit)]
    ref2 = [t.clone() for t in s.solve(A.flip(0).contiguous(), b.flip(0).contiguous(), tol, maxit)]
    s.set_ordering(1)
    out = [torch.empty_like(t) for t in ref]
    for _ in range(3):  # allocate the ordering state and pick the sampled rows
        s.solve(A, b, tol, maxit, out=out)
        torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            s.solve(A, b, tol, maxit, out=out)
    torch.cuda.current_stream().wait_stream(stream)
    for rep in range(3):
        for t in out:
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            assert torch.equal(r, o), rep
    A.copy_(A.flip(0).clone())
    b.copy_(b.flip(0).clone())
    g.replay()
    torch.cuda.synchronize()
    for r, o in zip(ref2, out):
        assert torch.equal(r, o)
    s.close()


@pytest.mark.parametrize("n,R", [(400, 1000), (700, 1600)])
def test_large_mechanisms(camp, cuda, n, R):
    """Mechanisms far beyond the benchmark's: 400 species (automatic choice:
    32 lanes, 13 rows per lane) and 700 species (beyond 16 rows per lane: the
    automatic choice falls back to one thread per row), against the oracle."""
    mech = synth.make_mechanism(n, R, 77 + n)
    cb = synth.make_cells(mech, 24, 78 + n, gamma=(1e-4, 1e-1))
    tol, maxit = 1e-10, 500
    orc = oracle.solve(mech.row_ptr, mech.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    gpu = run_gpu(camp, mech, cb.A_vals, cb.b, tol, maxit, cuda)
    parity.compare(mech, cb.A_vals, cb.b, tol, gpu, orc, f"n={n}")


def test_large_batch_all_cells(camp, cuda):
    """480,000 cells of 80 species in one launch (A alone is 2.2 GB, so byte
    offsets pass 2^31): every cell converges and matches the oracle."""
    import torch
    cbs, tol, maxit = synth.workload(1, cells=480000)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    x, it, res, st = s.solve(to_dev(cb.A_vals, cuda), to_dev(cb.b, cuda), tol, maxit)
    torch.cuda.synchronize()
    gpu = dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
               status=st.cpu().numpy())
    s.close()
    assert np.all(gpu["status"] == 0) and np.all(gpu["resid"] <= tol)
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=THREADS)
    parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, "480k")
