"""Comparison of the CUDA path with the oracle, per cell.

Bar (floating point, FP64): relative error ||x_gpu - x_orc|| / ||x_orc|| <= 1e-8
per cell and iteration counts within +-2.  Two solutions that each meet the
relative residual tol may differ by up to about 2 kappa(A) tol, so a cell that
misses the 1e-8 bar while both true residuals meet tol is re-checked against a
dense LAPACK solve: its error must stay within 2 kappa_1(A) tol.  Such cells are
counted; a caller states how many it accepts (none by default), so a kernel that
drifts into the fallback fails instead of passing silently.  Status codes must
agree exactly; cells the oracle reports NONFINITE are compared on status only.

Hard (ill-conditioned, many-iteration) systems need a second form of the bar:
there the iteration of BiCGSTAB in finite precision is sensitive to rounding,
so two correct FP64 implementations that sum in different orders take
different iteration counts on some cells, and a cell near the iteration cap may
end converged in one and exhausted in the other.  ``compare_sensitive`` measures
that sensitivity with the oracle itself (the oracle on right-hand sides changed
by one unit in the last place) and holds the CUDA path to the same spread.
"""
import numpy as np

REL_TOL = 1e-8
ITER_SLACK = 2


def rel_err(x_g, x_o):
    """||x_g - x_o|| / ||x_o|| per cell (the norm of x_o, or 1 where x_o = 0)."""
    nrm = np.linalg.norm(x_o, axis=1)
    return np.linalg.norm(x_g - x_o, axis=1) / np.where(nrm > 0, nrm, 1.0)


def _lu_fallback(mech, A_vals, b, x_g, c, tol, label, err):
    """The conditioning fallback for cell c: error against a dense LU solve
    within 2 kappa_1(A) (tol + n u), u = 2^-53 (n u: the LU solve's own
    rounding, which matters only at tolerances near FP64 precision)."""
    A = mech.dense(A_vals[c])
    xt = np.linalg.solve(A, b[c])
    kappa = np.linalg.cond(A, 1)
    e_g = np.linalg.norm(x_g[c] - xt) / np.linalg.norm(xt)
    bound = 2 * kappa * (tol + mech.n * 2.0 ** -53)
    assert e_g <= bound, f"{label}: cell {c} err {err}, vs LU {e_g}, kappa {kappa}"


def compare(mech, A_vals, b, tol, gpu, orc, label="", max_fallback=0):
    """gpu/orc: dicts of numpy arrays x, iters, resid, status.  Asserts the
    bar on every cell and that at most max_fallback cells needed the
    conditioning fallback; returns that number."""
    x_g, x_o = gpu["x"], orc["x"]
    st_g, st_o = gpu["status"], orc["status"]
    assert np.array_equal(st_g, st_o), f"{label}: status differs at cells {np.nonzero(st_g != st_o)[0][:10]}"
    fin = st_o != 3
    d_it = np.abs(gpu["iters"].astype(np.int64) - orc["iters"].astype(np.int64))
    bad = np.nonzero(fin & (d_it > ITER_SLACK))[0]
    assert bad.size == 0, \
        f"{label}: cell {bad[0]} iters gpu {gpu['iters'][bad[0]]} oracle {orc['iters'][bad[0]]}"
    conv = st_o == 0
    bad = np.nonzero(conv & ~(gpu["resid"] <= tol))[0]
    assert bad.size == 0, f"{label}: cell {bad[0]} resid {gpu['resid'][bad[0]]}"
    err = rel_err(x_g, x_o)
    over = np.nonzero(fin & ~(err <= REL_TOL))[0]
    for c in over:
        assert st_o[c] == 0, f"{label}: cell {c} err {err[c]} (status {st_o[c]})"
        _lu_fallback(mech, A_vals, b, x_g, c, tol, label, err[c])
    assert over.size <= max_fallback, \
        f"{label}: {over.size} cells needed the conditioning fallback (accepted {max_fallback})"
    return int(over.size)


def perturbed_rhs(b, seed):
    """b with every entry moved by one unit in the last place, up or down at
    random (seeded): a change of the size of one rounding."""
    sgn = np.random.default_rng(seed).choice([-1.0, 1.0], size=b.shape)
    return np.where(sgn > 0, np.nextafter(b, np.inf), np.nextafter(b, -np.inf))


def spread(ref, other):
    """How far two solves of the same cells are apart: the share of cells
    whose iteration counts differ by more than ITER_SLACK, the largest
    difference, the cells the reference converged and the other did not
    (flips_lost) and the reverse (flips_won), and the other's mean iteration
    count minus the reference's (shift)."""
    d = np.abs(ref["iters"].astype(np.int64) - other["iters"].astype(np.int64))
    c_r, c_o = ref["status"] == 0, other["status"] == 0
    return {"frac_iters_off": float(np.mean(d > ITER_SLACK)), "max_iters_off": int(d.max()),
            "flips_lost": int(np.sum(c_r & ~c_o)), "flips_won": int(np.sum(~c_r & c_o)),
            "shift": float(other["iters"].mean()) - float(ref["iters"].mean())}


def compare_sensitive(mech, A_vals, b, tol, maxit, gpu, orc, orc_perturbed, label="",
                      max_fallback=0):
    """Parity on systems whose iteration is sensitive to rounding.

    orc: the oracle on (A_vals, b); orc_perturbed: the oracle on inputs one
    rounding away (``perturbed_rhs``: the right-hand sides, and an initial
    guess where one is given, since r0 = b - A x0 then rounds at the scale of
    A x0), a list of at least one.

    Per cell, every cell: a converged status means a true residual <= tol, a
    MAXIT status means maxit iterations and a residual above tol; where both
    the CUDA path and the oracle converged, x meets the 1e-8 bar (or the
    conditioning fallback, at most max_fallback cells); a cell that only the
    CUDA path converged must be within 2 kappa_1(A) tol of a dense LU solve.

    Over the batch, against the largest spread a one-rounding change of b
    gives the oracle itself (times two, plus a small absolute margin): the
    share of cells more than ITER_SLACK iterations off; the cells the oracle
    converged and the CUDA path did not; and the rise of the mean iteration
    count.  The other direction is not bounded: near the limit of FP64
    accuracy (tol 1e-15) an implementation whose dot products are more
    accurate than the oracle's plain sums reaches a lower true residual, so it
    converges more cells in fewer iterations, and every such cell is checked
    on its own above.  Returns the spreads and the fallback count."""
    st_g, st_o = gpu["status"], orc["status"]
    it_g = gpu["iters"].astype(np.int64)
    assert np.all((st_g >= 0) & (st_g <= 3)), f"{label}: invalid status"
    conv_g = st_g == 0
    bad = np.nonzero(conv_g & ~(gpu["resid"] <= tol))[0]
    assert bad.size == 0, f"{label}: converged cell {bad[0]} resid {gpu['resid'][bad[0]]}"
    mx = st_g == 1
    bad = np.nonzero(mx & ((it_g != maxit) | ~(gpu["resid"] > tol)))[0]
    assert bad.size == 0, \
        f"{label}: MAXIT cell {bad[0]} iters {it_g[bad[0]]} resid {gpu['resid'][bad[0]]}"
    assert np.all(it_g <= maxit) and np.all(it_g >= 0), f"{label}: iteration count out of range"
    both = conv_g & (st_o == 0)
    err = rel_err(gpu["x"], orc["x"])
    over = np.nonzero(both & ~(err <= REL_TOL))[0]
    for c in over:
        _lu_fallback(mech, A_vals, b, gpu["x"], c, tol, label, err[c])
    assert over.size <= max_fallback, \
        f"{label}: {over.size} cells needed the conditioning fallback (accepted {max_fallback})"
    won = np.nonzero(conv_g & (st_o != 0))[0]
    for c in won:
        _lu_fallback(mech, A_vals, b, gpu["x"], c, tol, label, err[c])
    g = spread(orc, gpu)
    ps = [spread(orc, p) for p in orc_perturbed]
    p = {k: max(abs(s[k]) for s in ps) for k in g}
    flips_p = max(max(s["flips_lost"], s["flips_won"]) for s in ps)
    cells = len(st_o)
    assert g["frac_iters_off"] <= 2 * p["frac_iters_off"] + 0.005, (label, g, p)
    assert g["flips_lost"] <= 2 * flips_p + max(2, cells // 2000), (label, g, p)
    assert g["shift"] <= 2 * p["shift"] + 0.002 * float(orc["iters"].mean()) + 0.01, (label, g, p)
    return {"gpu": g, "oracle_perturbed": p, "fallback": int(over.size),
            "won_checked_by_lu": int(won.size),
            "max_err_converged": float(err[both].max()) if both.any() else 0.0}


def true_resid(mech, A_vals, x, b):
    """||b - A x|| / ||b|| per cell, recomputed on the host in NumPy."""
    rows = np.repeat(np.arange(mech.n), np.diff(mech.row_ptr))
    Ax = np.zeros_like(b)
    prod = A_vals * x[:, mech.col_idx]
    np.add.at(Ax, (slice(None), rows), prod)
    return np.linalg.norm(b - Ax, axis=1) / np.linalg.norm(b, axis=1)


def resid_rounding(mech, A_vals, x, b):
    """Per cell, a bound on how far two computations of ||b - A x|| / ||b||
    may differ through rounding alone: each computed entry of b - A x is off
    by at most (m + 1) u (|b| + |A| |x|) (m entries in the longest row,
    u = 2^-53), so two of them differ by at most twice that."""
    rows = np.repeat(np.arange(mech.n), np.diff(mech.row_ptr))
    m = int(np.diff(mech.row_ptr).max())
    ax = np.zeros_like(b)
    np.add.at(ax, (slice(None), rows), np.abs(A_vals) * np.abs(x[:, mech.col_idx]))
    bound = 2 * (m + 1) * 2.0 ** -53 * np.linalg.norm(np.abs(b) + ax, axis=1)
    return bound / np.linalg.norm(b, axis=1)


def block_diagonal(mech, A_vals, b, c0, k):
    """The cells c0 .. c0+k-1 as one block-diagonal system (the coupled
    Block-cells(k) reading): CSR (row_ptr, col_idx), values [1, k*nnz] and
    right-hand side [1, k*n]."""
    n, nnz = mech.n, mech.nnz
    rp = np.concatenate([[0]] + [mech.row_ptr[1:] + j * nnz for j in range(k)]).astype(np.int32)
    ci = np.concatenate([mech.col_idx + j * n for j in range(k)]).astype(np.int32)
    vals = np.ascontiguousarray(A_vals[c0:c0 + k].reshape(1, k * nnz))
    rhs = np.ascontiguousarray(b[c0:c0 + k].reshape(1, k * n))
    return rp, ci, vals, rhs
