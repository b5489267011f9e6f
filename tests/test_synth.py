"""Pins for the synthetic workload generator (input side, shared by both
paths): mass-action Jacobian checked against rates it does not use, pattern
invariants, determinism."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("n,R,seed", [(30, 60, 1000), (80, 200, 1001), (6, 4, 7)])
def test_pattern_invariants(n, R, seed):
    m = synth.make_mechanism(n, R, seed)
    rp, ci = m.row_ptr, m.col_idx
    assert rp[0] == 0 and rp[-1] == len(ci)
    for i in range(n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0), "columns sorted, no duplicates"
        assert i in row, "diagonal present"
    # union of couplings: every (row, col) a reaction touches is present
    dense = np.zeros((n, n), bool)
    for i in range(n):
        dense[i, ci[rp[i]:rp[i + 1]]] = True
    for r in range(R):
        a, b = m.reactants[r]
        c = m.products[r]
        if b < 0:
            assert dense[a, a] and dense[c, a]
            assert a != c
        else:
            assert len({a, b, c}) == 3
            for (i, j) in [(a, a), (a, b), (b, a), (b, b), (c, a), (c, b)]:
                assert dense[i, j]


def test_jacobian_matches_euler_identity_and_fd():
    """Mass action: unimolecular rates are degree-1 and bimolecular degree-2
    homogeneous in y, so J(y) y = f_uni(y) + 2 f_bi(y) (Euler); and J is the
    derivative of the independently coded rates f (central differences)."""
    m = synth.make_mechanism(12, 20, 5)
    rng = np.random.default_rng(0)
    y = rng.uniform(0.1, 1.0, m.n)
    J = m.dense(m.jacobian_values(y[None])[0])
    f_uni = np.zeros(m.n)
    f_bi = np.zeros(m.n)
    for r in range(m.R):
        a, b = m.reactants[r]
        c = m.products[r]
        if b < 0:
            w = m.k[r] * y[a]
            f_uni[a] -= w
            f_uni[c] += w
        else:
            w = m.k[r] * y[a] * y[b]
            f_bi[a] -= w
            f_bi[b] -= w
            f_bi[c] += w
    np.testing.assert_allclose(J @ y, f_uni + 2 * f_bi, rtol=1e-12, atol=1e-12 * np.abs(J).max())
    h = 1e-6
    for j in range(m.n):
        e = np.zeros(m.n)
        e[j] = h
        fd = (m.rates(y + e) - m.rates(y - e)) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-8 * max(1, np.abs(J).max()))


def test_unimolecular_columns_conserve_mass():
    """With only A -> B reactions every column of J sums to zero, so every
    column of A = I - gamma J sums to one."""
    m = synth.make_mechanism(10, 16, 3)
    m.R = 8   # keep only the unimolecular half
    keep = m.contrib_rxn < 8
    m.contrib_pos, m.contrib_rxn = m.contrib_pos[keep], m.contrib_rxn[keep]
    m.contrib_spec, m.contrib_sign = m.contrib_spec[keep], m.contrib_sign[keep]
    cb = synth.make_cells(m, 4, 11, gamma=(1e-3, 1.0))
    for c in range(4):
        A = m.dense(cb.A_vals[c])
        np.testing.assert_allclose(A.sum(axis=0), np.ones(m.n), rtol=0, atol=1e-12)


def test_determinism_and_shapes():
    a, tol, maxit = synth.workload(1, cells=16)
    b, _, _ = synth.workload(1, cells=16)
    assert tol == 1e-10 and maxit == 500
    np.testing.assert_array_equal(a[0].A_vals, b[0].A_vals)
    np.testing.assert_array_equal(a[0].b, b[0].b)
    cb = a[0]
    assert cb.A_vals.shape == (16, cb.mech.nnz) and cb.b.shape == (16, 80)
    assert cb.A_vals.flags["C_CONTIGUOUS"]
    g = cb.gamma
    assert np.all((g >= 1e-4) & (g <= 1e-1))
    assert np.all((cb.conc >= 1e-12) & (cb.conc <= 1e-3))
    # A_ii = 1 + gamma * (loss rates) >= 1
    assert np.all(cb.A_vals[:, cb.mech.diag_pos()] >= 1.0)
