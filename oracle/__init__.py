"""CPU oracle for the batched Jacobi-preconditioned BiCGSTAB solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check and
by the benchmark's CPU-baseline / reference leg.  The library's product path never
imports it, and it imports nothing from the library.

The arithmetic lives in plain C (``camp_oracle.c``, FP64, natural row order, one
cell at a time, threads over cells); this module compiles it with gcc on first
use and marshals NumPy arrays to it.  See ``camp_oracle.c`` for the algorithm and
the readings of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "camp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED, MAXIT, BREAKDOWN, NONFINITE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_bicgstab_cell.restype = I
            lib.orc_bicgstab_cell.argtypes = [I, P, P, P, P, D, I, I, P, P, P]
            lib.orc_bicgstab_batch.restype = I
            lib.orc_bicgstab_batch.argtypes = [I, I, I, P, P, P, P, D, I, I, P, P,
                                               P, P, P, I]
            lib.orc_mixed_batch.restype = I
            lib.orc_mixed_batch.argtypes = [I, I, I, P, P, P, P, D, I, D, I, P, P,
                                            P, P, P, I]
            lib.orc_transpose_pattern.restype = None
            lib.orc_transpose_pattern.argtypes = [I, P, P, P, P, P]
            lib.orc_assemble_cell.restype = I
            lib.orc_assemble_cell.argtypes = [I, P, P, I, P, P, P, P, P, D, P]
            lib.orc_rates_cell.restype = None
            lib.orc_rates_cell.argtypes = [I, I, P, P, P, P, P, P]
            lib.orc_newton_cell.restype = I
            lib.orc_newton_cell.argtypes = [I, P, P, I, P, P, P, P, P, D, P, D, I, D, I, P, P, P]
            lib.orc_grad_A_cell.restype = None
            lib.orc_grad_A_cell.argtypes = [I, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def solve(row_ptr, col_idx, A_vals, b, tol=1e-10, maxit=500, x0=None,
          threads=1):
    """Solve every cell.  A_vals [cells, nnz], b [cells, n] (FP64).

    Returns dict(x, iters, resid, status, restarts, threads); restarts counts
    each cell's restarts from r = b - A x (residual replacement or breakdown)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    A, B = _f64(np.atleast_2d(A_vals)), _f64(np.atleast_2d(b))
    cells, n = B.shape
    nnz = int(rp[-1])
    assert A.shape == (cells, nnz) and rp.shape == (n + 1,)
    x = np.zeros((cells, n)) if x0 is None else _f64(np.array(x0, dtype=np.float64,
                                                                copy=True).reshape(cells, n))
    iters = np.zeros(cells, dtype=np.int32)
    resid = np.zeros(cells)
    status = np.zeros(cells, dtype=np.int32)
    restarts = np.zeros(cells, dtype=np.int32)
    used = lib.orc_bicgstab_batch(cells, n, nnz, _p(rp), _p(ci), _p(A), _p(B),
                                  float(tol), int(maxit), int(x0 is not None),
                                  _p(x), _p(iters), _p(resid), _p(status),
                                  _p(restarts), int(threads))
    return dict(x=x, iters=iters, resid=resid, status=status, restarts=restarts,
                threads=used)


def solve_mixed(row_ptr, col_idx, A_vals, b, tol=1e-10, max_sweeps=20,
                tol_in=1e-5, maxit_in=50, threads=1):
    """FP32-inner / FP64-outer iterative refinement for every cell.

    Returns dict(x, iters (inner FP32 total), sweeps, resid, status, threads)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    A, B = _f64(np.atleast_2d(A_vals)), _f64(np.atleast_2d(b))
    cells, n = B.shape
    nnz = int(rp[-1])
    x = np.zeros((cells, n))
    iters = np.zeros(cells, dtype=np.int32)
    sweeps = np.zeros(cells, dtype=np.int32)
    resid = np.zeros(cells)
    status = np.zeros(cells, dtype=np.int32)
    used = lib.orc_mixed_batch(cells, n, nnz, _p(rp), _p(ci), _p(A), _p(B),
                               float(tol), int(max_sweeps), float(tol_in),
                               int(maxit_in), _p(x), _p(iters), _p(sweeps),
                               _p(resid), _p(status), int(threads))
    return dict(x=x, iters=iters, sweeps=sweeps, resid=resid, status=status,
                threads=used)


def transpose_pattern(row_ptr, col_idx):
    """Transposed CSR (rpt, cit) and the source map src: AT_vals = A_vals[..., src]."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    rpt = np.zeros(n + 1, dtype=np.int32)
    cit = np.zeros(nnz, dtype=np.int32)
    src = np.zeros(nnz, dtype=np.int32)
    lib.orc_transpose_pattern(n, _p(rp), _p(ci), _p(rpt), _p(cit), _p(src))
    return rpt, cit, src


def assemble(row_ptr, col_idx, reactant_a, reactant_b, product, k, conc, gamma):
    """A_vals [cells, nnz] = I - gamma_c J(conc_c) on the pattern (mass action;
    reactant_b = -1 marks a first-order reaction)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    ra, rb, pr = _i32(reactant_a), _i32(reactant_b), _i32(product)
    kk = _f64(k)
    C = _f64(np.atleast_2d(conc))
    g = _f64(np.atleast_1d(gamma))
    cells, n = C.shape
    nnz = int(rp[-1])
    A = np.zeros((cells, nnz))
    for c in range(cells):
        code = lib.orc_assemble_cell(n, _p(rp), _p(ci), int(ra.shape[0]), _p(ra), _p(rb),
                                     _p(pr), _p(kk), _p(np.ascontiguousarray(C[c])),
                                     float(g[c]), _p(A[c]))
        if code != 0:
            raise ValueError("a Jacobian entry lies outside the pattern")
    return A


def rates(reactant_a, reactant_b, product, k, y):
    """f(y) [cells, n] of the mass-action mechanism."""
    lib = _load()
    ra, rb, pr = _i32(reactant_a), _i32(reactant_b), _i32(product)
    kk = _f64(k)
    Y = _f64(np.atleast_2d(y))
    F = np.zeros_like(Y)
    for c in range(Y.shape[0]):
        lib.orc_rates_cell(Y.shape[1], int(ra.shape[0]), _p(ra), _p(rb), _p(pr), _p(kk),
                           _p(np.ascontiguousarray(Y[c])), _p(F[c]))
    return F


def newton(row_ptr, col_idx, reactant_a, reactant_b, product, k, a_hist, gamma, y0,
           newton_tol=1e-10, max_newton=20, lin_tol=1e-10, lin_maxit=500):
    """Newton corrector of G(y) = y - gamma f(y) - a = 0 per cell (see
    camp_oracle.c).  Returns dict(y, newton_iters, lin_iters, upd, status)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    ra, rb, pr = _i32(reactant_a), _i32(reactant_b), _i32(product)
    kk = _f64(k)
    Ah = _f64(np.atleast_2d(a_hist))
    g = _f64(np.atleast_1d(gamma))
    Y = np.array(np.atleast_2d(y0), dtype=np.float64, copy=True)
    cells = Y.shape[0]
    out = dict(y=Y, newton_iters=np.zeros(cells, np.int32), lin_iters=np.zeros(cells, np.int32),
               upd=np.zeros(cells), status=np.zeros(cells, np.int32))
    ni, li, up = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    for c in range(cells):
        yc = np.ascontiguousarray(Y[c])
        st = lib.orc_newton_cell(Y.shape[1], _p(rp), _p(ci), int(ra.shape[0]), _p(ra), _p(rb),
                                 _p(pr), _p(kk), _p(np.ascontiguousarray(Ah[c])), float(g[c]),
                                 _p(yc), float(newton_tol), int(max_newton), float(lin_tol),
                                 int(lin_maxit), ctypes.byref(ni), ctypes.byref(li),
                                 ctypes.byref(up))
        Y[c] = yc
        out["newton_iters"][c] = ni.value
        out["lin_iters"][c] = li.value
        out["upd"][c] = up.value
        out["status"][c] = st
    return out


def adjoint(row_ptr, col_idx, A_vals, x, w, tol=1e-10, maxit=500, threads=1):
    """Adjoint of L = sum_c w_c . x_c through x_c = A_c^{-1} b_c.

    lambda_c = A_c^{-T} w_c (BiCGSTAB on the transposed pattern);
    dL/db = lambda; dL/dA_vals[c, k] = -lambda_c[row k] * x_c[col k].
    Returns dict(lam, gA, gb, iters, resid, status)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    A = _f64(np.atleast_2d(A_vals))
    X, W = _f64(np.atleast_2d(x)), _f64(np.atleast_2d(w))
    cells, n = W.shape
    rpt, cit, src = transpose_pattern(rp, ci)
    AT = np.ascontiguousarray(A[:, src])
    out = solve(rpt, cit, AT, W, tol=tol, maxit=maxit, threads=threads)
    lam = out["x"]
    gA = np.zeros_like(A)
    for c in range(cells):
        lib.orc_grad_A_cell(n, _p(rp), _p(ci), _p(np.ascontiguousarray(lam[c])),
                            _p(np.ascontiguousarray(X[c])), _p(gA[c]))
    return dict(lam=lam, gA=gA, gb=lam.copy(), iters=out["iters"],
                resid=out["resid"], status=out["status"])
