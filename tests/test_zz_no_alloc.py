"""camp_solve_noalloc, the entry point for callers that cannot allocate device
memory (a host model that hands out all device memory from its own pool, or a
time loop that must not call cudaMalloc once it runs): called through the C
ABI, its results must equal those of the handle-based camp_solver_solve_ex on
the same inputs, on consecutive calls that re-stage its static scratch with
different patterns.  Collected last so that a failure here leaves every other
test already run; it also passes alone in a fresh process, where its first
call performs the per-device set-up."""
import ctypes

import numpy as np
import pytest

import synth
from tests import parity

pytestmark = pytest.mark.gpu

KEYS = ("x", "iters", "resid", "status")


def _noalloc(lib, mech, A, b, tol, maxit, torch, dev):
    f = lib.camp_solve_noalloc
    f.restype = ctypes.c_int
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f.argtypes = [I, I, P, P, I, P, P, P, D, I, P, P, P, P]
    cells = b.shape[0]
    x = torch.full((cells, mech.n), float("nan"), dtype=torch.float64, device=dev)
    it = torch.full((cells,), -7, dtype=torch.int32, device=dev)
    res = torch.full((cells,), -1.0, dtype=torch.float64, device=dev)
    st = torch.full((cells,), -7, dtype=torch.int32, device=dev)
    rp = np.ascontiguousarray(mech.row_ptr, np.int32)
    ci = np.ascontiguousarray(mech.col_idx, np.int32)
    code = f(mech.n, mech.nnz, rp.ctypes.data, ci.ctypes.data, cells, A.data_ptr(),
             b.data_ptr(), x.data_ptr(), tol, maxit, it.data_ptr(), res.data_ptr(),
             st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return code, (x, it, res, st)


def _np(t):
    return dict(zip(KEYS, (v.cpu().numpy() for v in t)))


def test_noalloc_matches_handle_on_consecutive_calls(cuda):
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
        ref = s.solve(A, b, tol, maxit)
        torch.cuda.synchronize()
        got, want = _np(out), _np(ref)
        # same per-cell bar as every parity test (relative 1e-8, iterations +-2)
        parity.compare(m, cb.A_vals, cb.b, tol, got, want, f"noalloc wid{wid}")
        assert np.array_equal(got["status"], want["status"])
        s.close()


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
