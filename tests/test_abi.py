"""The C-ABI library builds, loads and exports every function that
include/*.h declares; host-side argument and pattern checks run without a GPU
(they return before any CUDA call)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_17363_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(camp_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("camp_solver_create", "camp_solver_destroy", "camp_solver_solve",
                     "camp_solver_solve_ex", "camp_solver_grad_A", "camp_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _create(lib, n, rp, ci):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    lib.camp_solver_create.restype = ctypes.c_int
    lib.camp_solver_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    code = lib.camp_solver_create(ctypes.byref(h), n, len(ci), rp.ctypes.data, ci.ctypes.data)
    return code, h


def _msg(lib):
    lib.camp_last_error.restype = ctypes.c_char_p
    return lib.camp_last_error().decode()


def test_pattern_validation_without_gpu(lib):
    EINVAL, EPATTERN = -1, -4
    # unsorted columns
    code, h = _create(lib, 2, [0, 2, 4], [1, 0, 0, 1])
    assert code == EPATTERN and "increasing" in _msg(lib) and not h.value
    # missing diagonal
    code, _ = _create(lib, 2, [0, 1, 2], [1, 0])
    assert code == EPATTERN and "diagonal" in _msg(lib)
    # column out of range
    code, _ = _create(lib, 2, [0, 2, 3], [0, 2, 1])
    assert code == EPATTERN
    # row_ptr inconsistent with nnz
    code, _ = _create(lib, 2, [0, 1, 3], [0, 1])
    assert code in (EPATTERN, EINVAL)
    # sizes
    code, _ = _create(lib, 0, [0], [])
    assert code == EINVAL
    # null pointers
    lib.camp_solver_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.camp_solver_create(ctypes.byref(h), 2, 2, None, None) == EINVAL


def test_null_handle_calls_are_rejected(lib):
    EINVAL = -1
    f = lib.camp_solver_solve
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    assert f(None, 4, None, None, None, 1e-10, 10, None, None) == EINVAL
    lib.camp_solver_set_stream.restype = ctypes.c_int
    lib.camp_solver_set_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.camp_solver_set_stream(None, None) == EINVAL
    lib.camp_solver_destroy.restype = ctypes.c_int
    lib.camp_solver_destroy.argtypes = [ctypes.c_void_p]
    assert lib.camp_solver_destroy(None) == 0
    lib.camp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.camp_version()


@pytest.mark.parametrize("wid", [0, 1, 4])
def test_spmv_schedule_replays_the_product(lib, wid):
    """Replaying the exported SpMV schedule on the host reproduces y = A x for
    every lanes-per-cell choice: every entry used exactly once, each row stored
    exactly once, after all of its entries."""
    import synth
    cbs, _, _ = synth.workload(wid, cells=1)
    m = cbs[0].mech
    vals = cbs[0].A_vals[0]
    x = np.random.default_rng(0).standard_normal(m.n)
    y_ref = m.dense(vals) @ x
    f = lib.camp_schedule_build
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    rp = np.ascontiguousarray(m.row_ptr, np.int32)
    ci = np.ascontiguousarray(m.col_idx, np.int32)
    for lc in (1, 2, 4, 8, 16, 32):
        L = ctypes.c_int()
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, None, 0, ctypes.byref(L)) == 0
        words = np.zeros(2 * L.value * lc, np.uint32)
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, words.ctypes.data,
                 L.value * lc, ctypes.byref(L)) == 0
        w = words.reshape(L.value, lc, 2)
        y = np.full(m.n, np.nan)
        used = np.zeros(m.nnz, int)
        for lane in range(lc):
            acc = 0.0
            for j in range(L.value):
                src, w1 = int(w[j, lane, 0]), int(w[j, lane, 1])
                col = w1 & 0x7FF
                if src != 0xFFFFFFFF:
                    acc += vals[src] * x[col]
                    used[src] += 1
                    assert col == m.col_idx[src]
                if w1 >> 31:
                    row = (w1 >> 11) & 0x7FF
                    assert np.isnan(y[row])
                    y[row] = acc
                    acc = 0.0
                    # the row ends after every one of its entries
                    assert np.all(used[m.row_ptr[row]:m.row_ptr[row + 1]] == 1)
        assert np.all(used == 1)
        np.testing.assert_allclose(y, y_ref, rtol=1e-13, atol=1e-13 * np.abs(y_ref).max())
        # balance: no lane exceeds the mean by more than the longest row
        lens = np.diff(m.row_ptr)
        assert L.value <= int(np.ceil(m.nnz / lc)) + lens.max()


def test_row_ptr_rising_past_nnz_is_rejected_before_reading_columns(lib):
    """A row_ptr that rises above nnz in the middle and comes back to nnz at
    the end is rejected on that row, before any column index beyond nnz is
    read: by camp_solver_create, camp_schedule_build and camp_solve_noalloc
    (with zero cells its checks run without a GPU)."""
    EPATTERN = -4
    n, nnz = 3, 3
    rp = np.array([0, 3, 3, 3], np.int32)
    rp_bad = np.array([0, 1, 60, 3], np.int32)   # rises to 60 > nnz, not monotone
    rp_bad2 = np.array([0, 2, 50, 50], np.int32)  # monotone, past nnz, ends != nnz
    ci = np.array([0, 1, 2], np.int32)
    for r in (rp_bad, rp_bad2):
        code, h = _create(lib, n, r, ci)
        assert code == EPATTERN and not h.value
    # rows past nnz in the middle, back to nnz at the end
    rp_mid = np.array([0, 1, 2, 3], np.int32)
    rp_mid_bad = np.array([0, 40, 40, 3], np.int32)
    code, _ = _create(lib, n, rp_mid_bad, ci)
    assert code == EPATTERN and ("exceeds" in _msg(lib) or "decreases" in _msg(lib))
    f = lib.camp_schedule_build
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L = ctypes.c_int()
    assert f(n, nnz, rp_mid_bad.ctypes.data, ci.ctypes.data, 1, None, 0, ctypes.byref(L)) == EPATTERN
    g = lib.camp_solve_noalloc
    g.restype = ctypes.c_int
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    g.argtypes = [I, I, P, P, I, P, P, P, D, I, P, P, P, P]
    assert g(n, nnz, rp_mid_bad.ctypes.data, ci.ctypes.data, 0, None, None, None, 1e-10, 10,
             None, None, None, None) == EPATTERN
    assert "exceeds" in _msg(lib)
    # the valid diagonal pattern passes every check (no cells: no GPU work)
    assert g(n, nnz, rp_mid.ctypes.data, ci.ctypes.data, 0, None, None, None, 1e-10, 10,
             None, None, None, None) == 0
    del rp


def test_testing_hooks_validate_without_gpu(lib):
    EINVAL = -1
    f = lib.camp_solver_set_test_hooks
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]
    assert f(None, 0, 0) == EINVAL
    q = lib.camp_solver_get_fault
    q.restype = ctypes.c_int
    q.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert q(None, None) == EINVAL


@pytest.mark.parametrize("wid", [0, 1, 2, 4, 5])
def test_spmv_schedule_spreads_gathers_over_banks(lib, wid):
    """The schedule orders each row's entries so that the lanes reading the
    gathered vector in one slot hit distinct shared-memory bank pairs: a
    model of the 8-byte accesses (16 lanes per 128-byte wavefront; the cells
    of a half-warp Lc doubles apart modulo 16) gives at most 1.3 wavefronts
    per half-warp on average at the automatic lanes per cell up to 16 lanes,
    1.6 at 32 lanes (1 is conflict-free; bin-packed rows in CSR order gave
    1.7 to 3.8)."""
    import synth
    cbs, _, _ = synth.workload(wid, cells=1)
    f = lib.camp_schedule_build
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    for cb in cbs:
        m = cb.mech
        lc = 1
        while (m.n + lc - 1) // lc > 5:
            lc *= 2
        rp = np.ascontiguousarray(m.row_ptr, np.int32)
        ci = np.ascontiguousarray(m.col_idx, np.int32)
        L = ctypes.c_int()
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, None, 0, ctypes.byref(L)) == 0
        words = np.zeros(2 * L.value * lc, np.uint32)
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, words.ctypes.data,
                 L.value * lc, ctypes.byref(L)) == 0
        col = (words.reshape(L.value, lc, 2)[:, :, 1] & 0x7FF).astype(int)
        soff = lc % 16
        total = 0
        for j in range(L.value):
            for h0 in (0, 16):
                per_bank = {}
                for lane in range(h0, h0 + 16):
                    s, q = divmod(lane, lc)
                    per_bank.setdefault((s * soff + col[j, q]) % 16, set()).add((s, col[j, q]))
                total += max(len(v) for v in per_bank.values())
        mean = total / (2 * L.value)
        assert mean <= (1.3 if lc <= 16 else 1.6), (m.n, lc, mean)


def test_committed_traffic_figure_matches_the_library_revision(lib):
    """bench.py reports the headline kernel's DRAM traffic from the committed
    ncu summary only when it was captured on this library revision: the
    summary must name the revision the library reports."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    lib.camp_version.restype = ctypes.c_char_p
    version = lib.camp_version().decode()
    traffic = bench.measured_traffic(version)
    assert traffic is not None and 40e6 < traffic < 80e6, (version, traffic)
    assert bench.measured_traffic("campsolve 0.0 (none)") is None


def test_schedule_build_rejects_columns_out_of_range(lib):
    """camp_schedule_build checks every column index against [0, n) before
    the schedule builder uses it (a negative or too large column would index
    its residue tables out of range)."""
    EPATTERN = -4
    f = lib.camp_schedule_build
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    rp = np.array([0, 2, 4, 5], np.int32)
    L = ctypes.c_int()
    for bad in (-1, 3, 4000):
        ci = np.array([0, bad, 0, 1, 2], np.int32)
        assert f(3, 5, rp.ctypes.data, ci.ctypes.data, 1, None, 0, ctypes.byref(L)) == EPATTERN
        assert "out of range" in _msg(lib)
    ci = np.array([0, 2, 0, 1, 2], np.int32)
    assert f(3, 5, rp.ctypes.data, ci.ctypes.data, 1, None, 0, ctypes.byref(L)) == 0


def _rows_of_schedule(w, L, lanes):
    """Per row, the sequence of entries its sum multiplies, in slot order."""
    rows = {}
    for lane in range(lanes):
        cur = []
        for j in range(L):
            src, w1 = int(w[j, lane, 0]), int(w[j, lane, 1])
            if src == 0xFFFFFFFF:
                assert not w1 >> 31
                continue
            cur.append(src)
            if w1 >> 31:
                row = (w1 >> 11) & 0x7FF
                assert row not in rows
                rows[row] = cur
                cur = []
        assert not cur, "entries after a lane's last row end"
    return rows


@pytest.mark.parametrize("wid", [0, 1, 2, 5])
def test_split_schedule_keeps_every_row_chain(lib, wid):
    """The split schedule behind single-cell tickets (one cell on 32 lanes)
    gives every row exactly the entries, in exactly the order, of the 16-lane
    schedule (so each row's sum is the same chain of multiply-adds), lane
    v + 16 takes only rows of 16-lane lane v, and the split halves the slots
    per lane to within the longest row."""
    import synth
    cbs, _, _ = synth.workload(wid, cells=1)
    for cb in cbs:
        m = cb.mech
        if (m.n + 15) // 16 > 5:
            continue
        L16, w16 = _schedule(lib, "camp_schedule_build", m, 16)
        f = lib.camp_schedule_build_split
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        rp = np.ascontiguousarray(m.row_ptr, np.int32)
        ci = np.ascontiguousarray(m.col_idx, np.int32)
        L = ctypes.c_int()
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, None, 0, ctypes.byref(L)) == 0
        words = np.zeros(2 * L.value * 32, np.uint32)
        assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, words.ctypes.data, L.value * 32,
                 ctypes.byref(L)) == 0
        w2 = words.reshape(L.value, 32, 2)
        r16 = _rows_of_schedule(w16, L16, 16)
        r2 = _rows_of_schedule(w2, L.value, 32)
        assert r16 == r2
        assert set(r16) == set(range(m.n))
        # lane v + 16 holds rows of 16-lane lane v
        lane16 = {}
        for lane in range(16):
            for j in range(L16):
                if w16[j, lane, 0] != 0xFFFFFFFF:
                    lane16[(int(w16[j, lane, 1]) >> 11) & 0x7FF] = lane
        for lane in range(32):
            for j in range(L.value):
                if w2[j, lane, 0] != 0xFFFFFFFF:
                    assert lane16[(int(w2[j, lane, 1]) >> 11) & 0x7FF] == lane % 16
        longest = int(np.diff(m.row_ptr).max())
        assert L.value <= (L16 + 1) // 2 + longest, (L.value, L16, longest)


def _schedule(lib, fn, m, lc):
    f = getattr(lib, fn)
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    rp = np.ascontiguousarray(m.row_ptr, np.int32)
    ci = np.ascontiguousarray(m.col_idx, np.int32)
    L = ctypes.c_int()
    assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, None, 0, ctypes.byref(L)) == 0
    words = np.zeros(2 * max(1, L.value * lc), np.uint32)
    assert f(m.n, m.nnz, rp.ctypes.data, ci.ctypes.data, lc, words.ctypes.data,
             L.value * lc, ctypes.byref(L)) == 0
    return L.value, words[:2 * L.value * lc].reshape(L.value, lc, 2)


def test_single_tail_and_split_export_validate_without_gpu(lib):
    """camp_solver_set_single_tail rejects a null handle; the split-schedule
    export rejects patterns its 16-lane layout cannot take (more than 5 rows
    per lane: EUNSUPPORTED) and bad patterns (EPATTERN), before any work."""
    EINVAL, EPATTERN, EUNSUPPORTED = -1, -4, -5
    f = lib.camp_solver_set_single_tail
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert f(None, 3) == EINVAL
    g = lib.camp_schedule_build_split
    g.restype = ctypes.c_int
    g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L = ctypes.c_int()
    n = 81  # 6 rows per lane at 16 lanes
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    assert g(n, n, rp.ctypes.data, ci.ctypes.data, None, 0, ctypes.byref(L)) == EUNSUPPORTED
    n = 40
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    ci[7] = 8  # row 7 without its diagonal entry
    assert g(n, n, rp.ctypes.data, ci.ctypes.data, None, 0, ctypes.byref(L)) == EPATTERN
    ci[7] = 7
    assert g(n, n, rp.ctypes.data, ci.ctypes.data, None, 0, ctypes.byref(L)) == 0
    assert L.value >= 1


def test_split_schedule_with_many_rows_on_one_lane(lib):
    """A pattern whose 16-lane schedule puts more than 32 rows on one lane
    (15 long rows fill 15 lanes, 65 diagonal-only rows go to the 16th): the
    split (greedy past 16 rows per lane) still keeps every row's chain."""
    import synth
    n = 80
    rows = [sorted(set(range(0, 60)) | {i}) for i in range(15)] + [[i] for i in range(15, n)]
    rp = np.r_[0, np.cumsum([len(r) for r in rows])].astype(np.int32)
    ci = np.concatenate([np.array(r, np.int32) for r in rows])
    m = synth.Mechanism(n=n, R=0, reactants=None, products=None, k=None, row_ptr=rp, col_idx=ci)
    L16, w16 = _schedule(lib, "camp_schedule_build", m, 16)
    lanes_rows = [sum(1 for j in range(L16) if w16[j, q, 0] != 0xFFFFFFFF and w16[j, q, 1] >> 31)
                  for q in range(16)]
    assert max(lanes_rows) > 32
    f = lib.camp_schedule_build_split
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L = ctypes.c_int()
    assert f(n, m.nnz, rp.ctypes.data, ci.ctypes.data, None, 0, ctypes.byref(L)) == 0
    words = np.zeros(2 * L.value * 32, np.uint32)
    assert f(n, m.nnz, rp.ctypes.data, ci.ctypes.data, words.ctypes.data, L.value * 32,
             ctypes.byref(L)) == 0
    w2 = words.reshape(L.value, 32, 2)
    assert _rows_of_schedule(w16, L16, 16) == _rows_of_schedule(w2, L.value, 32)
    assert L.value <= L16
