"""Device Newton corrector of the implicit step against the oracle's Newton
loop (rates, assembly and BiCGSTAB in plain C), per cell.

Bar: statuses equal; Newton iterations within +-1 (the stopping test compares
||d|| with tol ||y||, and the two sides round ||d|| differently); summed
BiCGSTAB iterations within +-2 per Newton iteration; the converged y within
1e-8 relative of the oracle's, and the step residual y - gamma f(y) - a,
with f from the generator's own rate code, small against ||a||."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NEWTON_TOL = 1e-10
REL_TOL = 1e-8


def _run(cuda, m, ra, rb, pr, k, a, gamma, y0, **kw):
    import torch
    from paper_2405_17363_gb300 import camp
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(ra, rb, pr, k)
    out = s.newton_solve(torch.as_tensor(a, device=cuda), torch.as_tensor(gamma, device=cuda),
                         torch.as_tensor(y0, device=cuda), **kw)
    torch.cuda.synchronize()
    s.close()
    return {key: v.cpu().numpy() for key, v in out.items()}


def _oracle(m, ra, rb, pr, k, a, gamma, y0, **kw):
    return oracle.newton(m.row_ptr, m.col_idx, ra, rb, pr, k, a, gamma, y0.copy(), **kw)


def _compare(gpu, orc, label):
    st_g, st_o = gpu["status"], orc["status"]
    assert np.array_equal(st_g, st_o), f"{label}: status differs at {np.nonzero(st_g != st_o)[0][:10]}"
    dn = np.abs(gpu["newton_iters"].astype(int) - orc["newton_iters"].astype(int))
    assert dn.max(initial=0) <= 1, f"{label}: Newton iterations differ by {dn.max()}"
    same = dn == 0
    dl = np.abs(gpu["lin_iters"].astype(int) - orc["lin_iters"].astype(int))
    assert np.all(dl[same] <= 2 * orc["newton_iters"][same]), f"{label}: BiCGSTAB iterations"
    ok = st_o == 0
    nrm = np.linalg.norm(orc["y"], axis=1)
    err = np.linalg.norm(gpu["y"] - orc["y"], axis=1) / np.where(nrm > 0, nrm, 1.0)
    assert np.all(err[ok] <= REL_TOL), f"{label}: max y error {err[ok].max()}"
    assert np.all(gpu["upd"][ok] <= NEWTON_TOL)


def _mech_args(m):
    return m.reactants[:, 0], m.reactants[:, 1], m.products, m.k


@pytest.mark.parametrize("wid,cells", [(0, 64), (1, 301), (4, 37)])
def test_newton_matches_oracle(cuda, wid, cells):
    cbs, _, _ = synth.workload(wid, cells=cells)
    cb = cbs[0]
    m = cb.mech
    a = cb.conc
    rng = np.random.default_rng(100 + wid)
    y0 = a * rng.uniform(0.9, 1.1, a.shape)       # a perturbed predictor
    args = _mech_args(m)
    gpu = _run(cuda, m, *args, a, cb.gamma, y0, newton_tol=NEWTON_TOL)
    orc = _oracle(m, *args, a, cb.gamma, y0, newton_tol=NEWTON_TOL)
    _compare(gpu, orc, f"newton wid{wid}")
    assert np.all(gpu["status"] == 0)
    for c in range(cells):
        y = gpu["y"][c]
        G = y - cb.gamma[c] * m.rates(y) - a[c]
        assert np.linalg.norm(G) <= 1e-8 * np.linalg.norm(a[c]), f"cell {c}"


def test_newton_full_size_all_cells(cuda):
    """80 species x 10000 cells in one launch; every cell re-run by the
    oracle's Newton loop."""
    cbs, _, _ = synth.workload(1)
    cb = cbs[0]
    m = cb.mech
    args = _mech_args(m)
    gpu = _run(cuda, m, *args, cb.conc, cb.gamma, cb.conc, newton_tol=NEWTON_TOL)
    assert np.all(gpu["status"] == 0)
    orc = _oracle(m, *args, cb.conc, cb.gamma, cb.conc, newton_tol=NEWTON_TOL)
    _compare(gpu, orc, "newton full")


def test_newton_linear_mechanism_is_one_step(cuda):
    """First-order reactions only: one Newton step reaches the dense solution
    of (I - gamma J) y = a, the second confirms it."""
    m = synth.make_mechanism(12, 16, 3)
    keep = m.reactants[:, 1] < 0
    ra, rb, pr, k = m.reactants[keep, 0], m.reactants[keep, 1], m.products[keep], m.k[keep]
    rng = np.random.default_rng(0)
    a = rng.uniform(0.1, 1.0, (4, m.n))
    gam = np.array([1e-3, 1e-2, 0.1, 1.0])
    gpu = _run(cuda, m, ra, rb, pr, k, a, gam, a.copy(), newton_tol=1e-9, lin_tol=1e-13)
    assert np.all(gpu["status"] == 0) and np.all(gpu["newton_iters"] == 2)
    for c in range(4):
        J = np.zeros((m.n, m.n))
        for r in range(len(k)):
            J[ra[r], ra[r]] -= k[r]
            J[pr[r], ra[r]] += k[r]
        np.testing.assert_allclose(gpu["y"][c], np.linalg.solve(np.eye(m.n) - gam[c] * J, a[c]),
                                   rtol=1e-11)


def test_newton_edge_cases(cuda):
    """Per cell: zero state (f(0) = 0, converged at once), a non-finite
    history term (status 3), and in separate calls max_newton = 0 (status 1,
    y untouched) and a one-iteration linear cap (status 2, y untouched)."""
    cbs, _, _ = synth.workload(0, cells=6)
    cb = cbs[0]
    m = cb.mech
    args = _mech_args(m)
    a = cb.conc.copy()
    y0 = a.copy()
    a[1] = 0.0
    y0[1] = 0.0
    a[3, 5] = np.nan
    gpu = _run(cuda, m, *args, a, cb.gamma, y0, newton_tol=NEWTON_TOL)
    orc = _oracle(m, *args, a, cb.gamma, y0, newton_tol=NEWTON_TOL)
    assert list(gpu["status"]) == list(orc["status"]) == [0, 0, 0, 3, 0, 0]
    assert gpu["newton_iters"][1] == 1 and np.all(gpu["y"][1] == 0.0)
    _compare(gpu, orc, "edge")

    gpu = _run(cuda, m, *args, cb.conc, cb.gamma, cb.conc, max_newton=0)
    assert np.all(gpu["status"] == 1) and np.all(gpu["newton_iters"] == 0)
    assert np.array_equal(gpu["y"], cb.conc)

    y0 = cb.conc * 1.05
    gpu = _run(cuda, m, *args, cb.conc, cb.gamma, y0, lin_maxit=1)
    orc = _oracle(m, *args, cb.conc, cb.gamma, y0, lin_maxit=1)
    assert np.all(gpu["status"] == 2) and np.array_equal(gpu["status"], orc["status"])
    assert np.array_equal(gpu["y"], y0) and np.all(gpu["newton_iters"] == 1)


def test_newton_argument_errors(cuda):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, _, _ = synth.workload(0, cells=4)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(*_mech_args(m))
    a = torch.as_tensor(cb.conc, device=cuda)
    g = torch.as_tensor(cb.gamma, device=cuda)
    for kw in (dict(newton_tol=0.0), dict(lin_tol=float("nan")), dict(max_newton=-1),
               dict(lin_maxit=0)):
        with pytest.raises(camp.CampError) as ex:
            s.newton_solve(a, g, a, **kw)
        assert ex.value.code == camp.CAMP_EINVAL
    s.close()


def test_newton_ordering_is_bitwise_neutral(cuda):
    """The Newton launch orders its cells hardest first by gamma inside the
    launch: bitwise the index-order results (orderings 1 and 2, and a refused
    cooperative launch, which runs in index order)."""
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, _, _ = synth.workload(1, cells=3001)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(*_mech_args(m))
    a = torch.as_tensor(cb.conc, device=cuda)
    g = torch.as_tensor(cb.gamma, device=cuda)

    def run():
        out = s.newton_solve(a, g, a.clone(), newton_tol=NEWTON_TOL)
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in out.items()}
    s.set_ordering(0)
    ref = run()
    for mode, hooks in ((1, {}), (2, {}), (1, {"refuse_cooperative": True})):
        s.set_ordering(mode)
        s.set_test_hooks(**hooks)
        got = run()
        for k in ref:
            assert torch.equal(ref[k], got[k]), (k, mode, hooks)
        s.set_test_hooks()
    s.close()
