"""Thin Python binding of the C ABI in ``include/camp_solver.h``.

Argument marshalling only: every step of a solve runs in ``libcampsolve.so``.
Device arrays are torch CUDA tensors (contiguous, float64 / int32); the calls
are enqueued on torch's current CUDA stream.  The library must have been built
(``python -m paper_2405_17363_gb300.build`` or ``__graft_entry__.build()``);
importing this module without it raises ``ImportError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("CAMP_LIBRARY") or os.path.join(_HERE, "_lib", "libcampsolve.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcampsolve.so is not built ({LIB_PATH}); run "
                      "`python -m paper_2405_17363_gb300.build`")

_lib = ctypes.CDLL(LIB_PATH)

CAMP_OK, CAMP_EINVAL, CAMP_ECUDA, CAMP_ENOMEM, CAMP_EPATTERN, CAMP_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5
CAMP_CELL_CONVERGED, CAMP_CELL_MAXIT, CAMP_CELL_BREAKDOWN, CAMP_CELL_NONFINITE = \
    0, 1, 2, 3
CAMP_CELL_INVALID = 4
CAMP_TRANSPOSE, CAMP_X0_GIVEN = 1, 2
CAMP_ARR_AUTO, CAMP_ARR_WARP, CAMP_ARR_BLOCK, CAMP_ARR_BLOCK_COUPLED = 0, 1, 2, 3

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def _sig(name, args, res=_I):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_create = _sig("camp_solver_create", [ctypes.POINTER(_P), _I, _I, _P, _P])
_destroy = _sig("camp_solver_destroy", [_P])
_set_stream = _sig("camp_solver_set_stream", [_P, _P])
_set_arr = _sig("camp_solver_set_arrangement", [_P, _I, _I, _I, _I])
_set_ordering = _sig("camp_solver_set_ordering", [_P, _I])
_get_fault = _sig("camp_solver_get_fault", [_P, ctypes.POINTER(_I)])
_set_test_hooks = _sig("camp_solver_set_test_hooks", [_P, ctypes.c_longlong, _I])
_set_single_tail = _sig("camp_solver_set_single_tail", [_P, _I])
_solve = _sig("camp_solver_solve", [_P, _I, _P, _P, _P, _D, _I, _P, _P])
_solve_ex = _sig("camp_solver_solve_ex", [_P, _I, _P, _P, _P, _D, _I, _P, _P, _P, _I])
_grad_A = _sig("camp_solver_grad_A", [_P, _I, _P, _P, _P])
_solve_host = _sig("camp_solver_solve_host", [_P, _I, _P, _P, _P, _D, _I, _P, _P, _P])
_solve_mixed = _sig("camp_solver_solve_mixed",
                    [_P, _I, _P, _P, _P, _D, _I, _D, _I, _P, _P, _P, _P])
_set_mech = _sig("camp_solver_set_mechanism", [_P, _I, _P, _P, _P, _P])
_assemble_solve = _sig("camp_solver_assemble_solve", [_P, _I, _P, _P, _P, _P, _D, _I, _P, _P, _P])
_newton_solve = _sig("camp_solver_newton_solve",
                     [_P, _I, _P, _P, _P, _D, _I, _D, _I, _P, _P, _P, _P, _P])
_batch_create = _sig("camp_batch_create", [ctypes.POINTER(_P), _I, _P])
_batch_destroy = _sig("camp_batch_destroy", [_P])
_batch_set_stream = _sig("camp_batch_set_stream", [_P, _P])
_batch_set_config = _sig("camp_batch_set_config", [_P, _I, _I, _I])
_batch_set_ordering = _sig("camp_batch_set_ordering", [_P, _I])
_batch_solve = _sig("camp_batch_solve", [_P, _P, _P, _P, _P, _D, _I, _P, _P, _P])
_last_error = _sig("camp_last_error", [], ctypes.c_char_p)
_version = _sig("camp_version", [], ctypes.c_char_p)


class CampError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")


def _check(code: int, where: str):
    if code != CAMP_OK:
        raise CampError(code, where)


def camp_last_error() -> str:
    return _last_error().decode(errors="replace")


def camp_version() -> str:
    return _version().decode()


def _host_i32(a):
    import numpy as np
    arr = np.ascontiguousarray(a, dtype=np.int32)
    return arr, arr.ctypes.data_as(_P)


def _dptr(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _hptr(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CPU tensor")
    return t.data_ptr()


# ---- C-ABI names ---------------------------------------------------------

def camp_solver_create(row_ptr, col_idx) -> int:
    """Create a solver for the shared CSR pattern (host int arrays); returns
    the opaque handle."""
    rp, prp = _host_i32(row_ptr)
    ci, pci = _host_i32(col_idx)
    h = _P()
    _check(_create(ctypes.byref(h), int(rp.shape[0] - 1), int(ci.shape[0]), prp, pci),
           "camp_solver_create")
    return h.value


def camp_solver_destroy(h: int):
    _check(_destroy(h), "camp_solver_destroy")


def camp_solver_set_stream(h: int, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_set_stream(h, s.cuda_stream if hasattr(s, "cuda_stream") else s),
           "camp_solver_set_stream")


def camp_solver_set_arrangement(h: int, arrangement: int, lanes_per_cell: int = 0,
                                cells_per_block: int = 1, warps_per_block: int = 0):
    _check(_set_arr(h, arrangement, lanes_per_cell, cells_per_block, warps_per_block),
           "camp_solver_set_arrangement")


def camp_solver_set_ordering(h: int, ordering: int):
    _check(_set_ordering(h, int(ordering)), "camp_solver_set_ordering")


def camp_solver_get_fault(h: int) -> bool:
    """Whether an in-launch ordering wait of this handle ran out since the
    last query (no synchronisation; see include/camp_solver.h)."""
    v = _I(0)
    _check(_get_fault(h, ctypes.byref(v)), "camp_solver_get_fault")
    return bool(v.value)


def camp_solver_set_single_tail(h: int, pairs: int) -> None:
    """Single-cell tickets of the plain 16-lane launch (include/camp_testing.h):
    pairs < 0 automatic, 0 none, k > 0 the last k pairs as single cells."""
    _check(_set_single_tail(h, int(pairs)), "camp_solver_set_single_tail")


def camp_solver_set_test_hooks(h: int, ordering_wait_cycles: int = 0,
                               refuse_cooperative: bool = False):
    """Test hooks (include/camp_testing.h): the ordering's wait limit in SM
    cycles (0: default) and a switch that treats cooperative launches as
    refused."""
    _check(_set_test_hooks(h, int(ordering_wait_cycles), int(bool(refuse_cooperative))),
           "camp_solver_set_test_hooks")


def camp_solver_solve(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out):
    camp_solver_set_stream(h)
    _check(_solve(h, int(cells), _dptr(A_vals, torch.float64, "A_vals"),
                  _dptr(b, torch.float64, "b"), _dptr(x, torch.float64, "x"),
                  float(tol), int(maxit), _dptr(iters_out, torch.int32, "iters_out"),
                  _dptr(resid_out, torch.float64, "resid_out")), "camp_solver_solve")


def camp_solver_solve_ex(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out,
                         status_out=None, flags=0):
    camp_solver_set_stream(h)
    _check(_solve_ex(h, int(cells), _dptr(A_vals, torch.float64, "A_vals"),
                     _dptr(b, torch.float64, "b"), _dptr(x, torch.float64, "x"),
                     float(tol), int(maxit),
                     _dptr(iters_out, torch.int32, "iters_out"),
                     _dptr(resid_out, torch.float64, "resid_out"),
                     _dptr(status_out, torch.int32, "status_out"), int(flags)),
           "camp_solver_solve_ex")


def camp_solver_grad_A(h, cells, lam, x, gA):
    camp_solver_set_stream(h)
    _check(_grad_A(h, int(cells), _dptr(lam, torch.float64, "lambda"),
                   _dptr(x, torch.float64, "x"), _dptr(gA, torch.float64, "gA")),
           "camp_solver_grad_A")


def camp_solver_solve_host(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out,
                           status_out=None):
    camp_solver_set_stream(h)
    _check(_solve_host(h, int(cells), _hptr(A_vals, torch.float64, "A_vals"),
                       _hptr(b, torch.float64, "b"), _hptr(x, torch.float64, "x"),
                       float(tol), int(maxit), _hptr(iters_out, torch.int32, "iters_out"),
                       _hptr(resid_out, torch.float64, "resid_out"),
                       _hptr(status_out, torch.int32, "status_out")),
           "camp_solver_solve_host")


def camp_solver_solve_mixed(h, cells, A_vals, b, x, tol, max_sweeps, tol_inner,
                            maxit_inner, iters_out, sweeps_out, resid_out,
                            status_out=None):
    camp_solver_set_stream(h)
    _check(_solve_mixed(h, int(cells), _dptr(A_vals, torch.float64, "A_vals"),
                        _dptr(b, torch.float64, "b"), _dptr(x, torch.float64, "x"),
                        float(tol), int(max_sweeps), float(tol_inner), int(maxit_inner),
                        _dptr(iters_out, torch.int32, "iters_out"),
                        _dptr(sweeps_out, torch.int32, "sweeps_out"),
                        _dptr(resid_out, torch.float64, "resid_out"),
                        _dptr(status_out, torch.int32, "status_out")),
           "camp_solver_solve_mixed")


def camp_solver_set_mechanism(h, reactant_a, reactant_b, product, rate_k):
    """Attach a mass-action mechanism (host arrays [R]; reactant_b = -1 for
    first-order reactions) for camp_solver_assemble_solve."""
    import numpy as np
    ra, pra = _host_i32(reactant_a)
    rb, prb = _host_i32(reactant_b)
    pr, ppr = _host_i32(product)
    k = np.ascontiguousarray(rate_k, dtype=np.float64)
    _check(_set_mech(h, int(ra.shape[0]), pra, prb, ppr, k.ctypes.data_as(_P)),
           "camp_solver_set_mechanism")


def camp_solver_assemble_solve(h, cells, conc, gamma, b, x, tol, maxit, iters_out,
                               resid_out, status_out=None):
    camp_solver_set_stream(h)
    _check(_assemble_solve(h, int(cells), _dptr(conc, torch.float64, "conc"),
                           _dptr(gamma, torch.float64, "gamma"), _dptr(b, torch.float64, "b"),
                           _dptr(x, torch.float64, "x"), float(tol), int(maxit),
                           _dptr(iters_out, torch.int32, "iters_out"),
                           _dptr(resid_out, torch.float64, "resid_out"),
                           _dptr(status_out, torch.int32, "status_out")),
           "camp_solver_assemble_solve")


def camp_solver_newton_solve(h, cells, a_hist, gamma, y, newton_tol, max_newton, lin_tol,
                             lin_maxit, newton_iters_out, lin_iters_out, upd_out, resid_out,
                             status_out=None):
    camp_solver_set_stream(h)
    _check(_newton_solve(h, int(cells), _dptr(a_hist, torch.float64, "a_hist"),
                         _dptr(gamma, torch.float64, "gamma"), _dptr(y, torch.float64, "y"),
                         float(newton_tol), int(max_newton), float(lin_tol), int(lin_maxit),
                         _dptr(newton_iters_out, torch.int32, "newton_iters_out"),
                         _dptr(lin_iters_out, torch.int32, "lin_iters_out"),
                         _dptr(upd_out, torch.float64, "upd_out"),
                         _dptr(resid_out, torch.float64, "resid_out"),
                         _dptr(status_out, torch.int32, "status_out")),
           "camp_solver_newton_solve")


def camp_batch_create(solver_handles) -> int:
    arr = (_P * len(solver_handles))(*solver_handles)
    h = _P()
    _check(_batch_create(ctypes.byref(h), len(solver_handles), arr), "camp_batch_create")
    return h.value


def camp_batch_destroy(h: int):
    _check(_batch_destroy(h), "camp_batch_destroy")


def camp_batch_set_config(h: int, rows_per_lane=0, warps_per_block=0, stage_A_in_smem=1):
    _check(_batch_set_config(h, rows_per_lane, warps_per_block, stage_A_in_smem),
           "camp_batch_set_config")


def camp_batch_set_ordering(h: int, ordering: int):
    _check(_batch_set_ordering(h, int(ordering)), "camp_batch_set_ordering")


def camp_batch_solve(h, cells, A_vals, b, x, tol, maxit, iters_out, resid_out,
                     status_out=None):
    """cells: list of ints; the other arguments are lists of CUDA tensors
    (one per mechanism)."""
    nm = len(cells)
    s = torch.cuda.current_stream()
    _check(_batch_set_stream(h, s.cuda_stream), "camp_batch_set_stream")

    def arr(ts, dtype, name):
        return (_P * nm)(*[_dptr(t, dtype, name) if t is not None else None for t in ts])

    c_cells = (_I * nm)(*[int(c) for c in cells])
    st = arr(status_out, torch.int32, "status_out") if status_out is not None else None
    _check(_batch_solve(h, c_cells, arr(A_vals, torch.float64, "A_vals"),
                        arr(b, torch.float64, "b"), arr(x, torch.float64, "x"),
                        float(tol), int(maxit), arr(iters_out, torch.int32, "iters_out"),
                        arr(resid_out, torch.float64, "resid_out"), st),
           "camp_batch_solve")


# ---- convenience wrapper ------------------------------------------------

class Solver:
    """One shared sparsity pattern; solves batches of cells on the GPU."""

    def __init__(self, row_ptr, col_idx):
        self.h = camp_solver_create(row_ptr, col_idx)
        self.n = int(len(row_ptr) - 1)
        self.nnz = int(len(col_idx))

    def close(self):
        if getattr(self, "h", None):
            camp_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_arrangement(self, arrangement, lanes_per_cell=0, cells_per_block=1,
                        warps_per_block=0):
        camp_solver_set_arrangement(self.h, arrangement, lanes_per_cell,
                                    cells_per_block, warps_per_block)

    def set_ordering(self, ordering: int):
        camp_solver_set_ordering(self.h, ordering)

    def get_fault(self) -> bool:
        return camp_solver_get_fault(self.h)

    def set_test_hooks(self, ordering_wait_cycles: int = 0, refuse_cooperative: bool = False):
        camp_solver_set_test_hooks(self.h, ordering_wait_cycles, refuse_cooperative)

    def set_single_tail(self, pairs: int):
        camp_solver_set_single_tail(self.h, pairs)

    def solve(self, A_vals, b, tol=1e-10, maxit=500, x0=None, transpose=False,
              out=None):
        """Returns (x, iters, resid, status) as CUDA tensors."""
        cells = b.shape[0]
        dev = b.device
        if out is None:
            x = torch.empty((cells, self.n), dtype=torch.float64, device=dev)
            iters = torch.empty(cells, dtype=torch.int32, device=dev)
            resid = torch.empty(cells, dtype=torch.float64, device=dev)
            status = torch.empty(cells, dtype=torch.int32, device=dev)
        else:
            x, iters, resid, status = out
        flags = CAMP_TRANSPOSE if transpose else 0
        if x0 is not None:
            x.copy_(x0)
            flags |= CAMP_X0_GIVEN
        camp_solver_solve_ex(self.h, cells, A_vals, b, x, tol, maxit, iters, resid,
                             status, flags)
        return x, iters, resid, status

    def set_mechanism(self, reactant_a, reactant_b, product, rate_k):
        camp_solver_set_mechanism(self.h, reactant_a, reactant_b, product, rate_k)

    def assemble_solve(self, conc, gamma, b, tol=1e-10, maxit=500, out=None):
        """Solve (I - gamma_c J(conc_c)) x_c = b_c with the matrices built in the
        kernel; returns (x, iters, resid, status)."""
        cells = b.shape[0]
        dev = b.device
        if out is None:
            out = (torch.empty((cells, self.n), dtype=torch.float64, device=dev),
                   torch.empty(cells, dtype=torch.int32, device=dev),
                   torch.empty(cells, dtype=torch.float64, device=dev),
                   torch.empty(cells, dtype=torch.int32, device=dev))
        camp_solver_assemble_solve(self.h, cells, conc, gamma, b, out[0], tol, maxit,
                                   out[1], out[2], out[3])
        return out

    def newton_solve(self, a_hist, gamma, y0, newton_tol=1e-10, max_newton=20, lin_tol=1e-10,
                     lin_maxit=500):
        """Newton corrector of y - gamma_c f(y) - a_c = 0 per cell from y0 (one
        launch); returns dict(y, newton_iters, lin_iters, upd, resid, status)."""
        cells = a_hist.shape[0]
        dev = a_hist.device
        y = y0.clone()
        out = dict(y=y,
                   newton_iters=torch.empty(cells, dtype=torch.int32, device=dev),
                   lin_iters=torch.empty(cells, dtype=torch.int32, device=dev),
                   upd=torch.empty(cells, dtype=torch.float64, device=dev),
                   resid=torch.empty(cells, dtype=torch.float64, device=dev),
                   status=torch.empty(cells, dtype=torch.int32, device=dev))
        camp_solver_newton_solve(self.h, cells, a_hist, gamma, y, newton_tol, max_newton,
                                 lin_tol, lin_maxit, out["newton_iters"], out["lin_iters"],
                                 out["upd"], out["resid"], out["status"])
        return out

    def grad_A(self, lam, x, out=None):
        gA = out if out is not None else torch.empty(
            (lam.shape[0], self.nnz), dtype=torch.float64, device=lam.device)
        camp_solver_grad_A(self.h, lam.shape[0], lam, x, gA)
        return gA

    def solve_mixed(self, A_vals, b, tol=1e-10, max_sweeps=20, tol_inner=1e-5,
                    maxit_inner=50, out=None):
        """Returns (x, iters, sweeps, resid, status) as CUDA tensors (into
        `out` when given)."""
        cells = b.shape[0]
        dev = b.device
        if out is None:
            x = torch.empty((cells, self.n), dtype=torch.float64, device=dev)
            iters = torch.empty(cells, dtype=torch.int32, device=dev)
            sweeps = torch.empty(cells, dtype=torch.int32, device=dev)
            resid = torch.empty(cells, dtype=torch.float64, device=dev)
            status = torch.empty(cells, dtype=torch.int32, device=dev)
        else:
            x, iters, sweeps, resid, status = out
        camp_solver_solve_mixed(self.h, cells, A_vals, b, x, tol, max_sweeps, tol_inner,
                                maxit_inner, iters, sweeps, resid, status)
        return x, iters, sweeps, resid, status


class Batch:
    """Several mechanisms solved by one persistent launch (uneven batching)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.h = camp_batch_create([sv.h for sv in self.solvers])

    def close(self):
        if getattr(self, "h", None):
            camp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, rows_per_lane=0, warps_per_block=0, stage_A_in_smem=1):
        camp_batch_set_config(self.h, rows_per_lane, warps_per_block, stage_A_in_smem)

    def set_ordering(self, ordering: int):
        """1 (default): each mechanism's cells hardest first; 0: index order."""
        camp_batch_set_ordering(self.h, ordering)

    def solve(self, A_list, b_list, tol=1e-10, maxit=500, out=None):
        """Returns a list of (x, iters, resid, status), one per mechanism."""
        if out is None:
            out = []
            for sv, b in zip(self.solvers, b_list):
                c = b.shape[0]
                out.append((torch.empty((c, sv.n), dtype=torch.float64, device=b.device),
                            torch.empty(c, dtype=torch.int32, device=b.device),
                            torch.empty(c, dtype=torch.float64, device=b.device),
                            torch.empty(c, dtype=torch.int32, device=b.device)))
        camp_batch_solve(self.h, [b.shape[0] for b in b_list], A_list, b_list,
                         [o[0] for o in out], tol, maxit, [o[1] for o in out],
                         [o[2] for o in out], [o[3] for o in out])
        return out


class CampSolve(torch.autograd.Function):
    """x = A^{-1} b per cell, differentiable in A_vals (pattern entries) and b.

    Backward: lambda = A^{-T} dL/dx by the same kernel on the transposed
    pattern, dL/db = lambda, dL/dA_vals[k] = -lambda[row k] x[col k]."""

    @staticmethod
    def forward(ctx, A_vals, b, solver: Solver, tol: float, maxit: int):
        x, iters, resid, status = solver.solve(A_vals, b, tol, maxit)
        ctx.solver, ctx.tol, ctx.maxit = solver, tol, maxit
        ctx.save_for_backward(A_vals, x)
        ctx.mark_non_differentiable(iters, resid, status)
        return x, iters, resid, status

    @staticmethod
    def backward(ctx, gx, _gi, _gr, _gs):
        A_vals, x = ctx.saved_tensors
        s = ctx.solver
        lam, _, _, _ = s.solve(A_vals, gx.contiguous(), ctx.tol, ctx.maxit,
                               transpose=True)
        gA = s.grad_A(lam, x) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gA, gb, None, None, None


def solve(A_vals, b, solver: Solver, tol=1e-10, maxit=500):
    """Differentiable batched solve; returns (x, iters, resid, status)."""
    return CampSolve.apply(A_vals, b, solver, tol, maxit)
