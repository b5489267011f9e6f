"""FP32-inner / FP64-outer refinement on the GPU against the oracle: the
refined solution must meet the FP64 bar against the FP64 oracle, statuses must
match the refinement oracle and outer sweep counts agree within one."""
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
