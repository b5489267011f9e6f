"""Synthetic stiff-chemistry linear systems shaped like the paper's workload.

The paper (Sec. 2.2) solves, at every BDF/Newton step of a stiff chemistry ODE
``y' = f(t, y)`` with ``f_i = sum_j (dy_i/dt)_j`` over reactions j, one sparse
linear system per grid cell; all cells share one sparsity pattern (Sec. 3.1: the
cells are gathered into one data structure of identical arrays, Sec. 5.1).  The
chemical mechanism itself (CB05 + isoprene SOA, Sec. 4.2) is not available, so
this module draws synthetic mechanisms:

* ``R`` reactions, the first ``R//2`` unimolecular ``A -> B`` and the rest
  bimolecular ``A + B -> C``; the species of one reaction are distinct and drawn
  uniformly (without replacement) from ``n`` species;
* rate constants ``k_r`` log-uniform in [1e-6, 1e2], one per reaction, shared by
  all cells;
* per-cell concentrations log-uniform in [1e-12, 1e-3];
* the mass-action Jacobian ``J = df/dy``; for ``A -> B`` (rate ``k y_A``):
  ``J[A,A] -= k, J[B,A] += k``; for ``A + B -> C`` (rate ``k y_A y_B``):
  ``J[A,A] -= k y_B, J[A,B] -= k y_A, J[B,A] -= k y_B, J[B,B] -= k y_A,
  J[C,A] += k y_B, J[C,B] += k y_A``;
* the Newton matrix ``A = I - gamma J`` with a per-cell ``gamma``;
* the CSR pattern is the union of all couplings plus the full diagonal, columns
  sorted; a structural position stays even where its value cancels;
* ``b ~ N(0, 1)`` per cell.

Every draw comes from ``numpy.random.default_rng`` (PCG64) with a fixed seed, in
the order documented in ``make_mechanism`` and ``make_cells``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Mechanism", "CellBatch", "make_mechanism", "make_cells", "workload",
           "WORKLOADS"]


@dataclass
class Mechanism:
    n: int                      # species (rows of A)
    R: int                      # reactions
    reactants: np.ndarray       # int32 [R, 2]; second column -1 for unimolecular
    products: np.ndarray        # int32 [R]
    k: np.ndarray               # float64 [R] rate constants
    row_ptr: np.ndarray         # int32 [n+1]
    col_idx: np.ndarray         # int32 [nnz], sorted within each row
    # contributions: J_vals[:, pos] += sign * k[r] * (conc[:, spec] if spec >= 0 else 1)
    contrib_pos: np.ndarray = field(repr=False, default=None)
    contrib_rxn: np.ndarray = field(repr=False, default=None)
    contrib_spec: np.ndarray = field(repr=False, default=None)
    contrib_sign: np.ndarray = field(repr=False, default=None)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def diag_pos(self) -> np.ndarray:
        """CSR position of each diagonal entry."""
        out = np.empty(self.n, dtype=np.int64)
        for i in range(self.n):
            lo, hi = self.row_ptr[i], self.row_ptr[i + 1]
            out[i] = lo + int(np.searchsorted(self.col_idx[lo:hi], i))
        return out

    def rates(self, conc: np.ndarray) -> np.ndarray:
        """f(y) = dy/dt for concentrations ``conc`` [..., n] (mass action)."""
        conc = np.asarray(conc, dtype=np.float64)
        f = np.zeros_like(conc)
        for r in range(self.R):
            a, b2 = self.reactants[r]
            c = self.products[r]
            w = self.k[r] * conc[..., a] * (conc[..., b2] if b2 >= 0 else 1.0)
            f[..., a] -= w
            if b2 >= 0:
                f[..., b2] -= w
            f[..., c] += w
        return f

    def jacobian_values(self, conc: np.ndarray) -> np.ndarray:
        """Values of J = df/dy on the CSR pattern, shape [cells, nnz]."""
        conc = np.atleast_2d(np.asarray(conc, dtype=np.float64))
        cells = conc.shape[0]
        J = np.zeros((cells, self.nnz), dtype=np.float64)
        ones = np.ones(cells)
        for pos, r, s, sg in zip(self.contrib_pos, self.contrib_rxn,
                                 self.contrib_spec, self.contrib_sign):
            col = conc[:, s] if s >= 0 else ones
            J[:, pos] += sg * self.k[r] * col
        return J

    def dense(self, vals: np.ndarray) -> np.ndarray:
        """Scatter one cell's pattern values [nnz] into a dense n x n array."""
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            lo, hi = self.row_ptr[i], self.row_ptr[i + 1]
            A[i, self.col_idx[lo:hi]] = vals[lo:hi]
        return A


def make_mechanism(n: int, R: int, seed: int,
                   log10_k: tuple[float, float] = (-6.0, 2.0)) -> Mechanism:
    """Draw a mechanism.  Draw order: for r = 0..R-1 the species of reaction r
    (``rng.choice(n, 2 or 3, replace=False)``: reactant(s) first, product last),
    then all ``R`` log10 rate constants ``rng.uniform(*log10_k, R)`` (by
    default rate constants in [1e-6, 1e2])."""
    if n < 3:
        raise ValueError("a bimolecular A+B->C reaction needs n >= 3 species")
    rng = np.random.default_rng(seed)
    n_uni = R // 2
    reactants = np.full((R, 2), -1, dtype=np.int32)
    products = np.empty(R, dtype=np.int32)
    for r in range(R):
        if r < n_uni:
            a, b = rng.choice(n, 2, replace=False)
            reactants[r, 0] = a
            products[r] = b
        else:
            a, b, c = rng.choice(n, 3, replace=False)
            reactants[r] = (a, b)
            products[r] = c
    k = 10.0 ** rng.uniform(log10_k[0], log10_k[1], R)

    # (row, col, reaction, species multiplying k or -1, sign)
    contrib = []
    for r in range(R):
        a, b = int(reactants[r, 0]), int(reactants[r, 1])
        c = int(products[r])
        if b < 0:
            contrib += [(a, a, r, -1, -1.0), (c, a, r, -1, +1.0)]
        else:
            contrib += [(a, a, r, b, -1.0), (a, b, r, a, -1.0),
                        (b, a, r, b, -1.0), (b, b, r, a, -1.0),
                        (c, a, r, b, +1.0), (c, b, r, a, +1.0)]
    rows_cols = {(i, i) for i in range(n)} | {(t[0], t[1]) for t in contrib}
    per_row = [[] for _ in range(n)]
    for i, j in rows_cols:
        per_row[i].append(j)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for i in range(n):
        cs = sorted(per_row[i])
        cols += cs
        row_ptr[i + 1] = row_ptr[i] + len(cs)
    col_idx = np.asarray(cols, dtype=np.int32)
    pos_of = {}
    for i in range(n):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            pos_of[(i, int(col_idx[p]))] = p
    mech = Mechanism(n=n, R=R, reactants=reactants, products=products, k=k,
                     row_ptr=row_ptr, col_idx=col_idx)
    mech.contrib_pos = np.array([pos_of[(t[0], t[1])] for t in contrib], dtype=np.int64)
    mech.contrib_rxn = np.array([t[2] for t in contrib], dtype=np.int64)
    mech.contrib_spec = np.array([t[3] for t in contrib], dtype=np.int64)
    mech.contrib_sign = np.array([t[4] for t in contrib], dtype=np.float64)
    return mech


@dataclass
class CellBatch:
    mech: Mechanism
    conc: np.ndarray     # [C, n]
    gamma: np.ndarray    # [C]
    A_vals: np.ndarray   # [C, nnz]  A = I - gamma J, pattern order, C-contiguous
    b: np.ndarray        # [C, n]

    @property
    def cells(self) -> int:
        return int(self.b.shape[0])


def make_cells(mech: Mechanism, cells: int, seed: int,
               gamma: float | tuple[float, float] = 1e-2,
               conc_range: tuple[float, float] = (1e-12, 1e-3)) -> CellBatch:
    """Draw ``cells`` systems on ``mech``.  Draw order: concentrations
    ``rng.uniform(log10 lo, log10 hi, (cells, n))``; then gamma
    (``rng.uniform(log10 lo, log10 hi, cells)`` when a range is given, no draw
    when it is fixed); then ``b = rng.standard_normal((cells, n))``."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log10(conc_range[0]), np.log10(conc_range[1])
    conc = 10.0 ** rng.uniform(lo, hi, (cells, mech.n))
    if isinstance(gamma, tuple):
        g = 10.0 ** rng.uniform(np.log10(gamma[0]), np.log10(gamma[1]), cells)
    else:
        g = np.full(cells, float(gamma))
    b = rng.standard_normal((cells, mech.n))
    J = mech.jacobian_values(conc)
    A = -g[:, None] * J
    A[:, mech.diag_pos()] += 1.0
    return CellBatch(mech=mech, conc=conc, gamma=g, A_vals=np.ascontiguousarray(A),
                     b=np.ascontiguousarray(b))


# Workloads: (name, [(n, R, cells, gamma[, options])], tol, maxit).  Mechanism
# seed 1000+id (+10 per extra mechanism), cell seed 2000+id (+10 per extra
# mechanism).  Options: "log10_k" (rate-constant exponent range, default
# (-6, 2)) and "conc" (concentration range, default (1e-12, 1e-3)).
WORKLOADS = {
    0: ("30 species / 60 reactions, 64 cells, gamma 1e-2",
        [(30, 60, 64, 1e-2)], 1e-10, 200),
    1: ("80 species / 200 reactions, 10000 cells, gamma logU[1e-4,1e-1]",
        [(80, 200, 10000, (1e-4, 1e-1))], 1e-10, 500),
    2: ("uneven: 40/90 x 20000 + 80/200 x 5000 + 150/400 x 500, gamma logU[1e-4,1]",
        [(40, 90, 20000, (1e-4, 1.0)), (80, 200, 5000, (1e-4, 1.0)),
         (150, 400, 500, (1e-4, 1.0))], 1e-10, 500),
    3: ("adjoint: 80 species / 200 reactions, 10000 cells, gamma logU[1e-4,1e-1]",
        [(80, 200, 10000, (1e-4, 1e-1))], 1e-10, 500),
    4: ("mixed precision: 150 species / 400 reactions, 100000 cells, gamma logU[1e-4,1e-1]",
        [(150, 400, 100000, (1e-4, 1e-1))], 1e-10, 500),
    # Hard regime (parity only): stiffer and more strongly coupled systems
    # (rate constants up to 1e4, gamma up to 10, concentrations up to 1), so
    # that Jacobi-BiCGSTAB needs tens to hundreds of iterations per cell.
    5: ("hard: 80 species / 200 reactions, 10000 cells, k logU[1e-4,1e4], "
        "gamma logU[1e-2,10], conc logU[1e-3,1]",
        [(80, 200, 10000, (1e-2, 10.0), {"log10_k": (-4.0, 4.0), "conc": (1e-3, 1.0)})],
        1e-10, 500),
}


def workload(wid: int, cells: int | None = None):
    """Build the mechanisms and cell batches of workload ``wid``.  ``cells``
    overrides the cell count of every mechanism (for small parity cases).
    Returns (list[CellBatch], tol, maxit)."""
    _, mechs, tol, maxit = WORKLOADS[wid]
    out = []
    for j, spec in enumerate(mechs):
        n, R, C, g = spec[:4]
        opt = spec[4] if len(spec) > 4 else {}
        mech = make_mechanism(n, R, 1000 + wid + 10 * j,
                              log10_k=opt.get("log10_k", (-6.0, 2.0)))
        out.append(make_cells(mech, C if cells is None else cells,
                              2000 + wid + 10 * j, gamma=g,
                              conc_range=opt.get("conc", (1e-12, 1e-3))))
    return out, tol, maxit
