"""Fused Jacobian assembly and solve against the oracle's plain-C mass-action
assembly followed by the oracle solve, per cell."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu


def _case(cuda, wid, cells):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(wid, cells=cells)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k)
    conc = torch.as_tensor(cb.conc, device=cuda)
    gam = torch.as_tensor(cb.gamma, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    x, it, res, st = s.assemble_solve(conc, gam, b, tol, maxit)
    torch.cuda.synchronize()
    gpu = dict(x=x.cpu().numpy(), iters=it.cpu().numpy(), resid=res.cpu().numpy(),
               status=st.cpu().numpy())
    return camp, s, cb, m, tol, maxit, gpu


@pytest.mark.parametrize("wid,cells", [(0, 64), (1, 301), (4, 127)])
def test_assemble_solve_matches_oracle(cuda, wid, cells):
    camp, s, cb, m, tol, maxit, gpu = _case(cuda, wid, cells)
    A = oracle.assemble(m.row_ptr, m.col_idx, m.reactants[:, 0], m.reactants[:, 1],
                        m.products, m.k, cb.conc, cb.gamma)
    orc = oracle.solve(m.row_ptr, m.col_idx, A, cb.b, tol, maxit, threads=8)
    parity.compare(m, A, cb.b, tol, gpu, orc, f"assemble wid{wid}")
    # the residual of the returned x against the oracle-assembled matrices
    r = parity.true_resid(m, A, gpu["x"], cb.b)
    assert np.all(r[gpu["status"] == 0] <= tol * 1.0001)
    s.close()


def test_assemble_solve_full_size_all_cells(cuda):
    """80 species x 10000 cells assembled in the kernel: every cell against the
    oracle's assembly followed by the oracle's solve."""
    camp, s, cb, m, tol, maxit, gpu = _case(cuda, 1, None)
    assert np.all(gpu["status"] == 0)
    A = oracle.assemble(m.row_ptr, m.col_idx, m.reactants[:, 0], m.reactants[:, 1],
                        m.products, m.k, cb.conc, cb.gamma)
    orc = oracle.solve(m.row_ptr, m.col_idx, A, cb.b, tol, maxit, threads=os.cpu_count() or 8)
    parity.compare(m, A, cb.b, tol, gpu, orc, "assemble full")
    s.close()


def test_mechanism_outside_pattern_is_rejected(cuda):
    from paper_2405_17363_gb300 import camp
    m = synth.make_mechanism(8, 6, 3)
    n = m.n
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)   # diagonal pattern only
    s = camp.Solver(rp, ci)
    with pytest.raises(camp.CampError) as ex:
        s.set_mechanism(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k)
    assert ex.value.code == camp.CAMP_EPATTERN
    s.close()


def test_assemble_ordering_is_bitwise_neutral(cuda):
    """The fused launch orders its cells hardest first by gamma inside the
    launch (orderings 1 and 2): bitwise the index-order results, with batch
    sizes that change from call to call; a refused cooperative launch runs in
    index order; a wait that runs out marks the call's cells invalid and the
    next call is exact again."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(1, cells=4001)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k)
    conc = torch.as_tensor(cb.conc, device=cuda)
    gam = torch.as_tensor(cb.gamma, device=cuda)
    b = torch.as_tensor(cb.b, device=cuda)
    for cells in (4001, 2, 777, 4001):
        args = (conc[:cells].contiguous(), gam[:cells].contiguous(), b[:cells].contiguous(), tol,
                maxit)
        s.set_ordering(0)
        ref = [t.clone() for t in s.assemble_solve(*args)]
        out = [torch.empty_like(t) for t in ref]
        for mode, hooks in ((1, {}), (2, {}), (1, {"refuse_cooperative": True})):
            s.set_ordering(mode)
            s.set_test_hooks(**hooks)
            for t in out:
                t.fill_(float("nan") if t.is_floating_point() else -7)
            got = s.assemble_solve(*args, out=out)
            torch.cuda.synchronize()
            for r, g in zip(ref, got):
                assert torch.equal(r, g), (cells, mode, hooks)
            s.set_test_hooks()
    s.set_ordering(1)
    s.set_test_hooks(ordering_wait_cycles=16)
    got = s.assemble_solve(conc, gam, b, tol, maxit)
    torch.cuda.synchronize()
    assert s.get_fault() and torch.all(got[3] == camp.CAMP_CELL_INVALID)
    s.set_test_hooks()
    got = s.assemble_solve(conc, gam, b, tol, maxit)
    s.set_ordering(0)
    ref = s.assemble_solve(conc, gam, b, tol, maxit)
    torch.cuda.synchronize()
    for r, g in zip(ref, got):
        assert torch.equal(r, g)
    s.close()
