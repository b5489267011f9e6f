"""Autotuner for the launch arrangement (the paper's kernel-configuration
study, Sec. 3.2 and Sec. 5.2, made automatic).

For one pattern and batch size it times every admissible arrangement -- cells
per warp (lanes per cell) and warps per block of the warp-packed kernel, cells
per block of the Block-cells(k) kernel; for the persistent batch, rows per
lane, warps per block and shared-memory staging of A -- with CUDA events on
the current stream (L2 flushed before each timed solve), keeps the fastest and
sets it on the handle.  Results are cached per (pattern, GPU, batch size, mode)
in a JSON file (``CAMP_TUNE_CACHE``, default ``~/.cache/campsolve/tune.json``).

The paper picks its configuration by profiling device bandwidth; here the
solve is bound by the FP64 pipe, not by HBM, so the measured solve time is the
criterion.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import camp

_FLUSH = {}


def _flush(dev):
    buf = _FLUSH.get(dev)
    if buf is None:
        buf = _FLUSH[dev] = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    buf.zero_()


def time_call(fn, dev, reps=7, warmup=2):
    """Median CUDA-event time (ms) of fn() with L2 flushed before each call."""
    for _ in range(warmup):
        _flush(dev)
        fn()
    times = []
    for _ in range(reps):
        _flush(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def _cache_path():
    return os.environ.get("CAMP_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "campsolve", "tune.json")


def _load_cache():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(cache):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def pattern_key(row_ptr, col_idx, cells, mode, dev):
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(row_ptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(col_idx, np.int32).tobytes())
    bucket = int(np.ceil(np.log2(max(cells, 1))))
    return f"{h.hexdigest()[:16]}:{torch.cuda.get_device_name(dev)}:c2^{bucket}:{mode}"


def solver_candidates(n):
    out = []
    for lc in (1, 2, 4, 8, 16, 32):
        e = (n + lc - 1) // lc
        if e <= 12:
            for wpb in (2, 4, 8):
                out.append(("warp", lc, wpb))
    for cpb in (1, 2, 3):
        if cpb * n <= 1024:
            out.append(("block", cpb, 0))
    return out


def _apply(solver, cand):
    kind, a, b = cand
    if kind == "warp":
        solver.set_arrangement(camp.CAMP_ARR_WARP, a, 0, b)
    elif kind == "block":
        solver.set_arrangement(camp.CAMP_ARR_BLOCK, 0, a, 0)
    else:
        solver.set_arrangement(camp.CAMP_ARR_AUTO)


def tune_solver(solver, row_ptr, col_idx, A_vals, b, tol=1e-10, maxit=500,
                mode="fp64", use_cache=True, reps=7):
    """Pick and set the fastest arrangement for this pattern and batch.
    mode: "fp64" (camp_solver_solve) or "mixed" (FP32-inner refinement; the
    Block-cells kernel has no mixed form, so only warp arrangements are
    tried).  Returns dict(best=(kind, a, b), ms=..., table=[...])."""
    dev = b.device
    cells = b.shape[0]
    key = pattern_key(row_ptr, col_idx, cells, mode, dev)
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        best = tuple(cache[key]["best"])
        _apply(solver, best)
        return dict(cache[key], cached=True)
    out = solver.solve(A_vals, b, tol, maxit) if mode == "fp64" else None
    table = []
    for cand in solver_candidates(solver.n):
        if mode == "mixed" and cand[0] != "warp":
            continue
        try:
            _apply(solver, cand)
            if mode == "fp64":
                ms = time_call(lambda: solver.solve(A_vals, b, tol, maxit, out=out), dev, reps)
            else:
                ms = time_call(lambda: solver.solve_mixed(A_vals, b, tol), dev, reps)
        except camp.CampError:
            continue
        table.append((cand, ms))
    table.sort(key=lambda t: t[1])
    best, ms = table[0]
    _apply(solver, best)
    res = {"best": list(best), "ms": ms, "table": [[list(c), t] for c, t in table]}
    if use_cache:
        cache[key] = res
        _store_cache(cache)
    return dict(res, cached=False)


def tune_batch(batch, A_list, b_list, tol=1e-10, maxit=500, reps=5):
    """Pick and set the fastest (rows per lane, warps per block, A staging)
    for a persistent multi-mechanism batch.  Returns dict(best, ms, table)."""
    dev = b_list[0].device
    max_n = max(s.n for s in batch.solvers)
    out = batch.solve(A_list, b_list, tol, maxit)
    table = []
    for E in (3, 4, 5, 6, 8):
        if (max_n + 31) // 32 > E:
            continue
        for wpb in (2, 4, 8):
            for stage in (1, 0):
                cand = (E, wpb, stage)
                try:
                    batch.set_config(*cand)
                    ms = time_call(lambda: batch.solve(A_list, b_list, tol, maxit, out=out),
                                   dev, reps)
                except camp.CampError:
                    continue
                table.append((cand, ms))
    table.sort(key=lambda t: t[1])
    best, ms = table[0]
    batch.set_config(*best)
    return {"best": list(best), "ms": ms, "table": [[list(c), t] for c, t in table]}
