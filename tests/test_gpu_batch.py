"""Persistent multi-mechanism launch (uneven batching under a CUDA graph):
every mechanism's cells against the oracle, bitwise agreement with the plain
per-mechanism launch, graph replay with new pointers, and every launch
configuration the tuner can pick."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

pytestmark = pytest.mark.gpu


def _setup(cuda, cells):
    import torch
    from paper_2405_17363_gb300 import camp
    cbs, tol, maxit = synth.workload(2, cells=cells)
    solvers = [camp.Solver(cb.mech.row_ptr, cb.mech.col_idx) for cb in cbs]
    A = [torch.as_tensor(cb.A_vals, device=cuda) for cb in cbs]
    b = [torch.as_tensor(cb.b, device=cuda) for cb in cbs]
    return camp, cbs, tol, maxit, solvers, A, b


def _np(o):
    return dict(x=o[0].cpu().numpy(), iters=o[1].cpu().numpy(), resid=o[2].cpu().numpy(),
                status=o[3].cpu().numpy())


@pytest.mark.parametrize("cfg", [(0, 0, 1), (5, 4, 1), (6, 2, 1), (8, 8, 1), (5, 4, 0), (3, 4, 0)])
def test_batch_matches_oracle(cuda, cfg):
    import torch
    camp, cbs, tol, maxit, solvers, A, b = _setup(cuda, 97)
    if cfg[0] == 3:
        # 150 species need E >= 5 with 32 lanes: E=3 must be refused
        batch = camp.Batch(solvers)
        batch.set_config(*cfg)
        with pytest.raises(camp.CampError):
            batch.solve(A, b, tol, maxit)
        batch.close()
        return
    batch = camp.Batch(solvers)
    batch.set_config(*cfg)
    out = batch.solve(A, b, tol, maxit)
    torch.cuda.synchronize()
    for cb, o in zip(cbs, out):
        m = cb.mech
        orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
        parity.compare(m, cb.A_vals, cb.b, tol, _np(o), orc, f"batch {cfg} n{m.n}")
    batch.close()


def test_batch_equals_plain_and_replays(cuda):
    import torch
    camp, cbs, tol, maxit, solvers, A, b = _setup(cuda, 301)
    batch = camp.Batch(solvers)
    out1 = batch.solve(A, b, tol, maxit)
    # replay the captured graph with new output buffers and permuted inputs
    A2 = [a.flip(0).contiguous() for a in A]
    b2 = [v.flip(0).contiguous() for v in b]
    out2 = batch.solve(A2, b2, tol, maxit)
    torch.cuda.synchronize()
    for sv, a, v, o1, o2 in zip(solvers, A, b, out1, out2):
        x, it, res, st = sv.solve(a, v, tol, maxit)
        torch.cuda.synchronize()
        assert torch.equal(x, o1[0]) and torch.equal(it, o1[1]) and torch.equal(st, o1[3])
        assert torch.equal(o2[0], o1[0].flip(0)) and torch.equal(o2[1], o1[1].flip(0))
    # uneven counts, one mechanism empty
    out3 = batch.solve([A[0], A[1][:0], A[2][:7]], [b[0], b[1][:0], b[2][:7]], tol, maxit)
    torch.cuda.synchronize()
    assert torch.equal(out3[0][0], out1[0][0])
    assert torch.equal(out3[2][0], out1[2][0][:7])
    batch.close()


def test_batch_full_size_all_cells(cuda):
    """The uneven workload at full size (20000 + 5000 + 500 cells, gamma up to
    1, so iteration counts diverge): every cell converges, its residual is
    checked on the host and it matches the oracle."""
    import torch
    camp, cbs, tol, maxit, solvers, A, b = _setup(cuda, None)
    batch = camp.Batch(solvers)
    out = batch.solve(A, b, tol, maxit)
    torch.cuda.synchronize()
    for cb, o in zip(cbs, out):
        m = cb.mech
        g = _np(o)
        assert np.all(g["status"] == 0)
        r = parity.true_resid(m, cb.A_vals, g["x"], cb.b)
        assert np.all(r <= tol * 1.0001)
        orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit,
                           threads=os.cpu_count() or 8)
        parity.compare(m, cb.A_vals, cb.b, tol, g, orc, f"batch full n{m.n}")
    batch.close()


def test_batch_ordering_is_bitwise_neutral(cuda):
    """Hardest-first ordering of each mechanism's cells (the default) changes
    which cells share a warp, never a cell's result: bitwise the index-order
    outputs, at full size, for every launch configuration kind, across graph
    replays with new pointers and with cell counts that change (the ordering
    scratch grows and the graph is rebuilt)."""
    import torch
    camp, cbs, tol, maxit, solvers, A, b = _setup(cuda, None)
    batch = camp.Batch(solvers)
    for cfg in ((0, 0, 1), (5, 8, 0)):
        batch.set_config(*cfg)
        batch.set_ordering(0)
        ref = [[t.clone() for t in o] for o in batch.solve(A, b, tol, maxit)]
        batch.set_ordering(1)
        for rep in range(2):
            out = batch.solve(A, b, tol, maxit)
            torch.cuda.synchronize()
            for r, o in zip(ref, out):
                for x, y in zip(r, o):
                    assert torch.equal(x, y), (cfg, rep)
        # fewer cells, then more than ever before
        part = [a[: a.shape[0] // 3] for a in A], [v[: v.shape[0] // 3] for v in b]
        out = batch.solve(part[0], part[1], tol, maxit)
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            for x, y in zip(r, o):
                assert torch.equal(x[: y.shape[0]], y), cfg
        big = [torch.cat([a, a]) for a in A], [torch.cat([v, v]) for v in b]
        out = batch.solve(big[0], big[1], tol, maxit)
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            for x, y in zip(r, o):
                assert torch.equal(torch.cat([x, x]), y), cfg
    with pytest.raises(camp.CampError):
        batch.set_ordering(2)
    batch.close()


def test_tuner_picks_a_valid_config(cuda, tmp_path, monkeypatch):
    import torch
    from paper_2405_17363_gb300 import tune
    monkeypatch.setenv("CAMP_TUNE_CACHE", str(tmp_path / "tune.json"))
    camp, cbs, tol, maxit, solvers, A, b = _setup(cuda, 400)
    cb = cbs[1]
    s = solvers[1]
    res = tune.tune_solver(s, cb.mech.row_ptr, cb.mech.col_idx, A[1], b[1], tol, maxit, reps=3)
    assert res["table"] and res["ms"] == min(t for _, t in res["table"])
    again = tune.tune_solver(s, cb.mech.row_ptr, cb.mech.col_idx, A[1], b[1], tol, maxit)
    assert again["cached"] and again["best"] == res["best"]
    x, it, r, st = s.solve(A[1], b[1], tol, maxit)
    orc = oracle.solve(cb.mech.row_ptr, cb.mech.col_idx, cb.A_vals, cb.b, tol, maxit, threads=8)
    parity.compare(cb.mech, cb.A_vals, cb.b, tol, _np((x, it, r, st)), orc, "tuned")
    batch = camp.Batch(solvers)
    bres = tune.tune_batch(batch, A, b, tol, maxit, reps=2)
    assert len(bres["table"]) >= 6
    out = batch.solve(A, b, tol, maxit)
    torch.cuda.synchronize()
    for cb2, o in zip(cbs, out):
        m = cb2.mech
        orc = oracle.solve(m.row_ptr, m.col_idx, cb2.A_vals, cb2.b, tol, maxit, threads=8)
        parity.compare(m, cb2.A_vals, cb2.b, tol, _np(o), orc, f"tuned batch n{m.n}")
    batch.close()
