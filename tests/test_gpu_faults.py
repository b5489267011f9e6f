"""The rare paths of an ordered solve, driven on the GPU through the test hooks
(include/camp_testing.h) without faulting or hanging it:

- the in-launch ordering's bounded waits running out (a limit of a few clock
  cycles, so every wait ends at once): the same call reports it (every cell
  CAMP_CELL_INVALID with a NaN residual; camp_solver_get_fault without
  synchronising), and the next call, also when enqueued right behind it,
  gives bitwise the index-order results;
- a refused cooperative launch: the solve falls back to the separate ordering
  pass and gives bitwise the index-order results, which match the oracle.

Both for the plain FP64 solve and for the FP32-inner refinement with two cells
per warp (the arrangement in which that kernel orders)."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu

WAIT_CYCLES = 16  # far below any real wait: every wait of the launch runs out


@pytest.fixture(scope="module")
def setup(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1)
    cb = cbs[0]
    A = torch.as_tensor(cb.A_vals, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    return camp, cb, tol, maxit, A, b


def _poison(out):
    for t in out:
        t.fill_(float("nan") if t.is_floating_point() else -7)


def _solver(camp, m, mixed):
    s = camp.Solver(m.row_ptr, m.col_idx)
    if mixed:
        s.set_arrangement(camp.CAMP_ARR_WARP, 16, 1, 0)  # two cells per warp: ordered
    return s


def _solve(s, A, b, tol, maxit, mixed, out=None):
    if mixed:
        return s.solve_mixed(A, b, tol, out=out)
    return s.solve(A, b, tol, maxit, out=out)


def _status_resid(got, mixed):
    # solve: (x, iters, resid, status); solve_mixed: (x, iters, sweeps, resid, status)
    return (got[4], got[3]) if mixed else (got[3], got[2])


@pytest.mark.parametrize("mixed", [False, True])
def test_ordering_timeout_is_reported_on_the_call(setup, mixed):
    import torch
    camp, cb, tol, maxit, A, b = setup
    s = _solver(camp, cb.mech, mixed)
    s.set_ordering(0)
    ref = [t.clone() for t in _solve(s, A, b, tol, maxit, mixed)]
    out = [torch.empty_like(t) for t in ref]
    s.set_ordering(1)
    _solve(s, A, b, tol, maxit, mixed, out=out)  # a normal ordered solve first
    torch.cuda.synchronize()
    assert not s.get_fault()
    for rep in range(2):
        s.set_test_hooks(ordering_wait_cycles=WAIT_CYCLES)
        _poison(out)
        got = _solve(s, A, b, tol, maxit, mixed, out=out)
        torch.cuda.synchronize()
        assert s.get_fault(), rep
        assert not s.get_fault()  # the query clears the report
        st, res = _status_resid(got, mixed)
        assert torch.all(st == camp.CAMP_CELL_INVALID), rep
        assert torch.all(torch.isnan(res)), rep
        # back to the default limit: the next solve is clean and exact
        s.set_test_hooks(0)
        _poison(out)
        got = _solve(s, A, b, tol, maxit, mixed, out=out)
        torch.cuda.synchronize()
        assert not s.get_fault()
        for r, g in zip(ref, got):
            assert torch.equal(r, g), rep
    # a timed-out launch and a normal one enqueued back to back, no host sync
    out2 = [torch.empty_like(t) for t in ref]
    _poison(out)
    _poison(out2)
    s.set_test_hooks(ordering_wait_cycles=WAIT_CYCLES)
    bad = _solve(s, A, b, tol, maxit, mixed, out=out)
    s.set_test_hooks(0)
    good = _solve(s, A, b, tol, maxit, mixed, out=out2)
    torch.cuda.synchronize()
    assert s.get_fault()
    assert torch.all(_status_resid(bad, mixed)[0] == camp.CAMP_CELL_INVALID)
    for r, g in zip(ref, good):
        assert torch.equal(r, g)
    s.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_refused_cooperative_launch_falls_back(setup, mixed):
    import torch
    camp, cb, tol, maxit, A, b = setup
    m = cb.mech
    s = _solver(camp, m, mixed)
    s.set_ordering(0)
    ref = [t.clone() for t in _solve(s, A, b, tol, maxit, mixed)]
    out = [torch.empty_like(t) for t in ref]
    s.set_ordering(1)
    s.set_test_hooks(refuse_cooperative=True)
    for rep in range(3):
        _poison(out)
        got = _solve(s, A, b, tol, maxit, mixed, out=out)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            assert torch.equal(r, g), rep
    assert not s.get_fault()
    s.close()
    if mixed:
        return
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit,
                       threads=os.cpu_count() or 8)
    gpu = dict(x=out[0].cpu().numpy(), iters=out[1].cpu().numpy(),
               resid=out[2].cpu().numpy(), status=out[3].cpu().numpy())
    parity.compare(m, cb.A_vals, cb.b, tol, gpu, orc, "refused cooperative launch")


def test_test_hooks_reject_bad_arguments(setup):
    camp, cb, tol, maxit, A, b = setup
    s = camp.Solver(cb.mech.row_ptr, cb.mech.col_idx)
    with pytest.raises(camp.CampError) as ex:
        s.set_test_hooks(ordering_wait_cycles=-1)
    assert ex.value.code == camp.CAMP_EINVAL
    s.close()
    assert np.all(np.isfinite(cb.b))
