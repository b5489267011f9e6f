"""camp_solve_noalloc, the entry point for callers that cannot allocate device
memory (a host model that hands out all device memory from its own pool, or a
time loop that must not call cudaMalloc once it runs): called through the C
ABI on consecutive calls that re-stage its static scratch with different
patterns, every cell must match the oracle (the same per-cell bar as every
parity test) and be bitwise equal to the handle-based camp_solver_solve_ex in
index order (both run the same kernel).  While its stream captures a CUDA
graph it must refuse to run.  Collected last so that a failure here leaves
every other test already run; it also passes alone in a fresh process, where
its first call performs the per-device set-up."""
import ctypes

import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu

KEYS = ("x", "iters", "resid", "status")


def _noalloc(lib, mech, A, b, tol, maxit, torch, dev, out=None, stream=None):
    f = lib.camp_solve_noalloc
    f.restype = ctypes.c_int
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f.argtypes = [I, I, P, P, I, P, P, P, D, I, P, P, P, P]
    cells = b.shape[0]
    if out is None:
        out = (torch.full((cells, mech.n), float("nan"), dtype=torch.float64, device=dev),
               torch.full((cells,), -7, dtype=torch.int32, device=dev),
               torch.full((cells,), -1.0, dtype=torch.float64, device=dev),
               torch.full((cells,), -7, dtype=torch.int32, device=dev))
    x, it, res, st = out
    rp = np.ascontiguousarray(mech.row_ptr, np.int32)
    ci = np.ascontiguousarray(mech.col_idx, np.int32)
    s = stream if stream is not None else torch.cuda.current_stream()
    code = f(mech.n, mech.nnz, rp.ctypes.data, ci.ctypes.data, cells, A.data_ptr(),
             b.data_ptr(), x.data_ptr(), tol, maxit, it.data_ptr(), res.data_ptr(),
             st.data_ptr(), s.cuda_stream)
    return code, (x, it, res, st)


def _np(t):
    return dict(zip(KEYS, (v.cpu().numpy() for v in t)))


def test_noalloc_matches_oracle_and_handle_on_consecutive_calls(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    lib = camp._lib
    # two calls in a row with different patterns (the second re-stages the
    # static scratch), then the first pattern again
    for wid, cells in ((1, 3001), (0, 64), (1, 517)):
        cbs, tol, maxit = synth.workload(wid, cells=cells)
        cb = cbs[0]
        m = cb.mech
        A = torch.as_tensor(cb.A_vals, device=cuda)
        b = torch.as_tensor(cb.b, device=cuda)
        code, out = _noalloc(lib, m, A, b, tol, maxit, torch, cuda)
        assert code == camp.CAMP_OK, camp.camp_last_error()
        s = camp.Solver(m.row_ptr, m.col_idx)
        s.set_ordering(0)  # index order, as the allocation-free launch
        ref = s.solve(A, b, tol, maxit)
        torch.cuda.synchronize()
        got = _np(out)
        orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit,
                           threads=os.cpu_count() or 8)
        parity.compare(m, cb.A_vals, cb.b, tol, got, orc, f"noalloc wid{wid}")
        for g, r in zip(out, ref):
            assert torch.equal(g, r), f"noalloc wid{wid}: not bitwise the handle's result"
        s.close()


def test_noalloc_refuses_to_run_while_capturing(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    lib = camp._lib
    cbs, tol, maxit = synth.workload(0, cells=8)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        code, out = _noalloc(lib, m, A, b, tol, maxit, torch, cuda, stream=stream)
        assert code == camp.CAMP_OK, camp.camp_last_error()
    torch.cuda.synchronize()
    want = [t.clone() for t in out]
    marker = torch.zeros(1, device=cuda)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        code, _ = _noalloc(lib, m, A, b, tol, maxit, torch, cuda, out=out, stream=stream)
        marker.add_(1.0)  # the graph holds this op only
    assert code == camp.CAMP_EUNSUPPORTED
    assert "capturing" in camp.camp_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert marker.item() == 1.0
    for t, w in zip(out, want):
        assert torch.equal(t, w)


def test_noalloc_rejects_a_pattern_larger_than_its_scratch(cuda):
    from paper_2405_17363_gb300 import camp
    lib = camp._lib
    n, per_row = 512, 80          # 40960 entries: the schedule alone exceeds 256 KiB
    rng = np.random.default_rng(0)
    rows = []
    for i in range(n):
        cols = set(rng.choice(n, per_row - 1, replace=False).tolist()) | {i}
        while len(cols) < per_row:
            cols.add(int(rng.integers(n)))
        rows.append(sorted(cols))
    rp = np.r_[0, np.cumsum([len(r) for r in rows])].astype(np.int32)
    ci = np.concatenate(rows).astype(np.int32)
    mech = synth.Mechanism(n=n, R=0, reactants=None, products=None, k=None,
                           row_ptr=rp, col_idx=ci)
    import torch
    A = torch.zeros((1, len(ci)), dtype=torch.float64, device=cuda)
    b = torch.zeros((1, n), dtype=torch.float64, device=cuda)
    code, _ = _noalloc(lib, mech, A, b, 1e-10, 10, torch, cuda)
    assert code == camp.CAMP_EUNSUPPORTED
    assert "static scratch" in camp.camp_last_error()


def test_noalloc_hard_regime_bitwise_handle(cuda):
    """The hard cells (tens to hundreds of iterations per cell, residual
    replacement on some): the allocation-free call gives bitwise the handle's
    index-order results, whose parity with the oracle the hard-regime tests
    check."""
    import torch
    from paper_2405_17363_gb300 import camp
    lib = camp._lib
    cbs, tol, maxit = synth.workload(5)
    cb = cbs[0]
    m = cb.mech
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    code, out = _noalloc(lib, m, A, b, tol, maxit, torch, cuda)
    assert code == camp.CAMP_OK, camp.camp_last_error()
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_ordering(0)
    ref = s.solve(A, b, tol, maxit)
    torch.cuda.synchronize()
    assert float(ref[1].double().mean().item()) >= 30
    for g, r in zip(out, ref):
        assert torch.equal(g, r)
    s.close()
