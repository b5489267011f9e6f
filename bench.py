#!/usr/bin/env python
"""Benchmark: batched Jacobi-BiCGSTAB solve of the per-cell chemistry systems.

Workload: 80 species / 200 reactions synthetic mechanism (stand-in for the
paper's intermediate-complexity mechanism, Sec. 4.2), 10,000 cells, FP64,
relative residual 1e-10, maxit 500.  One step = one batched solve of all cells
(one kernel launch).  Prints one JSON line (see the keys below).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch under torchrun: every rank solves its own batch (weak
scaling, no collective on the data path); the time is the max over ranks.
--impl reference times the CPU oracle (plain C, FP64) on this host's cores on
the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "solved cell-systems/s (80 species, 10k cells, 1e-10) and % of HBM roofline"
UNIT = "cell-systems/s"
WORKLOAD_ID = 1
DEFAULT_ORDERING = 1  # the library default of camp_solver_set_ordering
HBM_PEAK_FALLBACK = 6800.0
# FP64 pipe: 2 DFMA per clock per SM (4 flops) x 152 SMs x 2.07 GHz max clock
FP64_PEAK_GFLOPS = 4 * 152 * 2.07
# The committed ncu summary of the headline kernel states its DRAM bytes
# (read + write) per launch and the library revision they were taken on.
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "warp_bicgstab_80sp_10k.md")


def measured_traffic(version):
    """DRAM bytes per launch of the headline kernel from the committed ncu
    summary (dram__bytes_read.sum + dram__bytes_write.sum of one capture), or
    None if the summary was taken on another library revision."""
    import re
    try:
        with open(TRAFFIC_PROFILE) as f:
            for line in f:
                m = re.match(r"traffic_bytes_per_launch: (\d+) \(library `(.+)`\)", line.strip())
                if m and m.group(2) == version:
                    return float(m.group(1))
    except OSError:
        pass
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def algorithmic(mech, cells, iters):
    """Algorithmic FP64 flops and HBM bytes of one batched solve.
    Per iteration: two SpMVs (2 nnz flops each) and 26 n flops of vector work
    (p update 4n, two Jacobi scalings 2n, six dot products 12n, s 2n, x 4n, r 2n);
    per cell: the final true residual (2 nnz + 3 n) and ||b|| (2 n) and the
    Jacobi reciprocals (n).  Bytes: A_vals, b read once, x written once, iters
    and resid written once per cell, plus the shared pattern once."""
    n, nnz = mech.n, mech.nnz
    flops = float(np.sum(iters, dtype=np.float64)) * (4 * nnz + 26 * n) + cells * (2 * nnz + 6 * n)
    bytes_ = cells * (8 * nnz + 16 * n + 12) + 4 * (n + 1 + nnz)
    return flops, bytes_


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower().startswith("active"):
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(mech, A, b, tol, maxit, min_seconds=10.0, single_seconds=3.0):
    import oracle
    threads = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    used = threads
    while True:
        out = oracle.solve(mech.row_ptr, mech.col_idx, A, b, tol, maxit, threads=threads)
        used = out["threads"]
        done += A.shape[0]
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    # one core, on leading slices of the same cells
    one, t1, chunk = 0, time.perf_counter(), min(A.shape[0], 1000)
    while True:
        oracle.solve(mech.row_ptr, mech.col_idx, A[:chunk], b[:chunk], tol, maxit, threads=1)
        one += chunk
        el1 = time.perf_counter() - t1
        if el1 >= single_seconds:
            break
    return {"value": done / el, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"the full {A.shape[0]}-cell workload solved {done // A.shape[0]}x "
                      f"({el:.1f} s, {used} threads, plain C FP64)",
            "value_1core": one / el1,
            "sample_1core": f"the first {chunk} cells solved {one // chunk}x ({el1:.1f} s, 1 thread)"}


def run_reference(args, rank, world):
    cbs, tol, maxit = synth.workload(WORKLOAD_ID)
    cb = cbs[0]
    m = cb.mech
    if rank != 0:
        return
    import oracle
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit, threads=threads)
    t0 = time.perf_counter()
    used = threads
    for _ in range(args.steps):
        used = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit,
                            threads=threads)["threads"]
    el = time.perf_counter() - t0
    value = cb.cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": synth.WORKLOADS[WORKLOAD_ID][0], "cells": cb.cells,
                       "n": m.n, "nnz": m.nnz, "tol": tol, "maxit": maxit},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(used),
                             "kind": "oracle",
                             "sample": f"the full {cb.cells}-cell workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over all ranks (the job's time is its slowest
    rank's); identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, cells: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every rank solves its own `cells` per step."""
    return world * cells * steps / (total_ms * 1e-3)


def set_arrangement(camp, solver, spec):
    parts = spec.split(":")
    if parts[0] == "auto":
        return "auto"
    if parts[0] == "warp":
        lc = int(parts[1])
        wpb = int(parts[2]) if len(parts) > 2 else 0
        solver.set_arrangement(camp.CAMP_ARR_WARP, lc, 0, wpb)
        return f"warp-packed, {lc} lanes per cell, {32 // lc} cells per warp"
    if parts[0] == "block":
        cpb = int(parts[1])
        solver.set_arrangement(camp.CAMP_ARR_BLOCK, 0, cpb, 0)
        return f"Block-cells({cpb}): one thread per row"
    raise SystemExit(f"bad --arrangement {spec}")


def time_steps(fn, flush, stream, steps, warmup):
    """CUDA-event time of each step on the launching stream; the L2 flush
    between steps is outside the events.  Returns the per-step times (ms)."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        fn()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def time_e2e(camp, solver, cb, C, tol, maxit, steps, world, dev):
    """Same metric end to end through the public host-memory entry point:
    every step copies A_vals and b from pinned host memory and copies x,
    iters, resid and status back."""
    import torch
    import torch.distributed as dist
    m = cb.mech
    hA = torch.as_tensor(cb.A_vals).pin_memory()
    hb = torch.as_tensor(cb.b).pin_memory()
    hx = torch.empty((C, m.n), dtype=torch.float64).pin_memory()
    hit = torch.empty(C, dtype=torch.int32).pin_memory()
    hres = torch.empty(C, dtype=torch.float64).pin_memory()
    hst = torch.empty(C, dtype=torch.int32).pin_memory()
    for _ in range(3):
        camp.camp_solver_solve_host(solver.h, C, hA, hb, hx, tol, maxit, hit, hres, hst)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        camp.camp_solver_solve_host(solver.h, C, hA, hb, hx, tol, maxit, hit, hres, hst)
    el = max_over_ranks(time.perf_counter() - t0, dev)
    return {"value": world * C * steps / el, "unit": UNIT,
            "h2d_bytes_per_step": C * (m.nnz + m.n) * 8,
            "d2h_bytes_per_step": C * (m.n * 8 + 4 + 8 + 4)}


def difficulty_order(mech, A):
    """Host model of the library's cell ordering: the difficulty class of a
    cell (half octaves of max_i |A_ii - 1|, from the high word of its bit
    pattern; class 0 hardest) and the cells sorted hardest class first (index
    order inside a class; the kernels' order inside a class is arbitrary)."""
    d = np.abs(A[:, mech.diag_pos()] - 1.0).max(axis=1)
    hi = (np.ascontiguousarray(d).view(np.uint64) >> np.uint64(32)).astype(np.int64)
    top = ((1023 + 3) << 1) | 1
    cls = np.clip(top - (hi >> 19), 0, 63)
    return np.argsort(cls, kind="stable")


def time_uneven(camp, dev, flush, stream, steps=50, tune=True):
    """The uneven-batching workload (40/90 x 20000 + 80/200 x 5000 + 150/400 x
    500 cells, gamma up to 1): the persistent launch under a CUDA graph with
    the launch configuration picked by the autotuner (tune.tune_batch, timed
    here with each mechanism's cells ordered hardest first), the same in index
    order, and three plain FP64 launches back to back, all to the 1e-10 true
    residual.  Lockstep waste per mechanism (lane-iterations spent waiting for
    the slowest cell of a warp, over useful ones) for index order and for the
    host model of the hardest-first order."""
    import torch
    from paper_2405_17363_gb300 import tune as tuner
    cbs, tol, maxit = synth.workload(2)
    solvers = [camp.Solver(cb.mech.row_ptr, cb.mech.col_idx) for cb in cbs]
    A = [torch.as_tensor(cb.A_vals, device=dev) for cb in cbs]
    b = [torch.as_tensor(cb.b, device=dev) for cb in cbs]
    batch = camp.Batch(solvers)
    tuned = tuner.tune_batch(batch, A, b, tol, maxit, reps=3) if tune else None
    out = batch.solve(A, b, tol, maxit)
    t_batch = time_steps(lambda: batch.solve(A, b, tol, maxit, out=out), flush, stream, steps, 3)
    batch.set_ordering(0)
    t_index = time_steps(lambda: batch.solve(A, b, tol, maxit, out=out), flush, stream, steps, 3)
    batch.set_ordering(1)
    outs = [sv.solve(a, v, tol, maxit) for sv, a, v in zip(solvers, A, b)]

    def plain():
        for sv, a, v, o in zip(solvers, A, b, outs):
            sv.solve(a, v, tol, maxit, out=o)
    t_plain = time_steps(plain, flush, stream, steps, 3)
    cells = sum(cb.cells for cb in cbs)
    mb, mi, mp = (sum(t) / steps for t in (t_batch, t_index, t_plain))
    conv = sum(int((o[3] == 0).sum().item()) for o in out)
    its = [o[1].cpu().numpy() for o in out]
    iters = np.concatenate(its)
    waste = {"index": [], "hardest_first": []}
    for cb, it in zip(cbs, its):
        k = 32 // sv_lanes(cb.mech.n)
        waste["index"].append(lockstep_waste(it, k))
        waste["hardest_first"].append(lockstep_waste(it[difficulty_order(cb.mech, cb.A_vals)], k))
    batch.close()
    for sv in solvers:
        sv.close()
    res = {"workload": synth.WORKLOADS[2][0], "cells": cells,
           "persistent_graph": {"ms_per_step": mb, "value": cells / (mb * 1e-3), "unit": UNIT,
                                "ordering": "hardest first per mechanism"},
           "persistent_graph_index_order": {"ms_per_step": mi, "value": cells / (mi * 1e-3),
                                            "unit": UNIT},
           "three_plain_launches": {"ms_per_step": mp, "value": cells / (mp * 1e-3), "unit": UNIT},
           "lockstep_waste_by_mechanism": waste, "mechanisms_species": [cb.mech.n for cb in cbs],
           "converged": conv, "iters_mean": float(iters.mean()), "iters_max": int(iters.max())}
    if tuned is not None:
        res["tuned_config"] = {"rows_per_lane": tuned["best"][0],
                               "warps_per_block": tuned["best"][1],
                               "stage_A_in_smem": tuned["best"][2],
                               "configs_timed": len(tuned["table"])}
    return res


def variability(camp, dev, flush, stream, steps):
    """'Realistic' cells (per-cell concentrations and gamma, as generated)
    against 'ideal' cells (every cell a copy of the first one), as in the
    paper's two initial-condition set-ups (Sec. 4.2): the spread of iteration
    counts, the lockstep waste it causes in the warp-packed solve (index order
    and the host model of hardest first) and the throughput of the plain
    launches (one per mechanism, the library's default in-launch ordering) and
    of the persistent launch (its default hardest-first ordering)."""
    import torch
    rows = []
    for wid in (WORKLOAD_ID, 2):
        cbs, tol, maxit = synth.workload(wid)
        for setup in ("realistic", "ideal"):
            solvers, As, bs, hostA, cells = [], [], [], [], 0
            for cb in cbs:
                A, b = cb.A_vals, cb.b
                if setup == "ideal":
                    A = np.repeat(A[:1], cb.cells, axis=0)
                    b = np.repeat(b[:1], cb.cells, axis=0)
                hostA.append(A)
                solvers.append(camp.Solver(cb.mech.row_ptr, cb.mech.col_idx))
                As.append(torch.as_tensor(np.ascontiguousarray(A), device=dev))
                bs.append(torch.as_tensor(np.ascontiguousarray(b), device=dev))
                cells += cb.cells
            outs = [sv.solve(a, v, tol, maxit) for sv, a, v in zip(solvers, As, bs)]

            def plain():
                for sv, a, v, o in zip(solvers, As, bs, outs):
                    sv.solve(a, v, tol, maxit, out=o)
            tp = sum(time_steps(plain, flush, stream, steps, 3)) / steps
            batch = camp.Batch(solvers)
            bo = batch.solve(As, bs, tol, maxit)
            tb = sum(time_steps(lambda: batch.solve(As, bs, tol, maxit, out=bo), flush, stream,
                                steps, 3)) / steps
            its = [o[1].cpu().numpy() for o in outs]
            it = np.concatenate(its)
            w_idx, w_ord = [], []
            for cb, A, i1 in zip(cbs, hostA, its):
                k = 32 // sv_lanes(cb.mech.n)
                w_idx.append(lockstep_waste(i1, k))
                w_ord.append(lockstep_waste(i1[difficulty_order(cb.mech, A)], k))
            rows.append({"workload": synth.WORKLOADS[wid][0], "setup": setup, "cells": cells,
                         "iters_mean": float(it.mean()), "iters_std": float(it.std()),
                         "iters_p99": float(np.percentile(it, 99)), "iters_max": int(it.max()),
                         "lockstep_waste_index_order": w_idx,
                         "lockstep_waste_hardest_first": w_ord,
                         "plain_ms": tp, "plain_value": cells / (tp * 1e-3),
                         "persistent_ms": tb, "persistent_value": cells / (tb * 1e-3)})
            batch.close()
            for sv in solvers:
                sv.close()
    return rows


def time_cfg4(camp, dev, flush, stream, steps=10, threads=None):
    """The mixed-precision workload at full size (150 species / 400 reactions,
    100,000 cells, gamma logU[1e-4,1e-1]): the FP32-inner refinement against
    the plain FP64 solve, both to the 1e-10 true residual, in cells/s; and the
    per-cell relative error ||x - x_oracle|| / ||x_oracle|| of both against
    the FP64 oracle over all cells (max and p99; the oracle runs outside the
    timed regions)."""
    import torch
    import oracle
    cbs, tol, maxit = synth.workload(4)
    cb = cbs[0]
    m = cb.mech
    C = cb.cells
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=dev)
    b = torch.as_tensor(cb.b, device=dev)
    f64 = s.solve(A, b, tol, maxit)
    t64 = sum(time_steps(lambda: s.solve(A, b, tol, maxit, out=f64), flush, stream, steps, 3)) / steps
    mix = s.solve_mixed(A, b, tol)
    t32 = sum(time_steps(lambda: s.solve_mixed(A, b, tol, out=mix), flush, stream, steps, 3)) / steps
    torch.cuda.synchronize()
    x64 = f64[0].cpu().numpy()
    x32 = mix[0].cpu().numpy()
    orc = oracle.solve(m.row_ptr, m.col_idx, cb.A_vals, cb.b, tol, maxit,
                       threads=threads or os.cpu_count() or 1)
    nrm = np.linalg.norm(orc["x"], axis=1)
    e32 = np.linalg.norm(x32 - orc["x"], axis=1) / nrm
    e64 = np.linalg.norm(x64 - orc["x"], axis=1) / nrm
    res = {"workload": synth.WORKLOADS[4][0], "cells": C, "n": m.n, "nnz": m.nnz, "tol": tol,
           "fp32_inner": {"ms_per_step": t32, "value": C / (t32 * 1e-3), "unit": UNIT,
                          "converged": int((mix[4] == 0).sum().item()),
                          "sweeps_mean": float(mix[2].double().mean().item()),
                          "inner_iters_mean": float(mix[1].double().mean().item()),
                          "rel_err_vs_fp64_oracle_max": float(e32.max()),
                          "rel_err_vs_fp64_oracle_p99": float(np.percentile(e32, 99))},
           "fp64": {"ms_per_step": t64, "value": C / (t64 * 1e-3), "unit": UNIT,
                    "converged": int((f64[3] == 0).sum().item()),
                    "iters_mean": float(f64[1].double().mean().item()),
                    "rel_err_vs_fp64_oracle_max": float(e64.max()),
                    "rel_err_vs_fp64_oracle_p99": float(np.percentile(e64, 99))},
           "speedup_fp32_inner_vs_fp64": t64 / t32,
           "l2": "inputs (1.0 GB) larger than L2, flushed between timed steps"}
    s.close()
    return res


def time_small_batches(camp, cb, tol, maxit, flush, stream, dev, steps=200, sizes=(64, 608)):
    """Small batches of the headline cells (by default 64 and 608 cells, where
    one pair per warp would keep at most a quarter of the GPU's warps busy):
    the library's automatic launch, which solves each cell alone on a warp
    (single-cell tickets, bit for bit the pair solve), against the same
    launch with pairs only.  Median microseconds per solve, L2 flushed."""
    import torch
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    out = {}
    for C in sizes:
        A = torch.as_tensor(cb.A_vals[:C], device=dev)
        b = torch.as_tensor(cb.b[:C], device=dev)
        row = {"cells": C}
        for name, tail in (("automatic_us", -1), ("pairs_only_us", 0)):
            s.set_single_tail(tail)
            res = s.solve(A, b, tol, maxit)
            t = time_steps(lambda: s.solve(A, b, tol, maxit, out=res), flush, stream, steps, 5)
            row[name] = float(np.median(t)) * 1000.0
        s.set_single_tail(-1)
        out[str(C)] = row
    s.close()
    return out


def time_adjoint(camp, dev, flush, stream, steps=50):
    """The adjoint workload (80 species / 200 reactions, 10,000 cells): one
    forward solve and the backward of L = sum_c w_c . x_c as the library's
    autograd Function runs it (the transposed solve A^T lambda = w and
    dL/dA_vals = -lambda[row] x[col]), through the C ABI, L2 flushed before
    each step; cells/s of forward + backward and the backward's share."""
    import torch
    cbs, tol, maxit = synth.workload(3)
    cb = cbs[0]
    m = cb.mech
    C = cb.cells
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=dev)
    b = torch.as_tensor(cb.b, device=dev)
    w = torch.as_tensor(np.random.default_rng(3000).standard_normal((C, m.n)), device=dev)
    x = torch.empty_like(b)
    lam = torch.empty_like(b)
    gA = torch.empty_like(A)
    it = [torch.empty(C, dtype=torch.int32, device=dev) for _ in range(2)]
    res = [torch.empty(C, dtype=torch.float64, device=dev) for _ in range(2)]
    st = [torch.empty(C, dtype=torch.int32, device=dev) for _ in range(2)]

    def fwd():
        camp.camp_solver_solve_ex(s.h, C, A, b, x, tol, maxit, it[0], res[0], st[0], 0)

    def bwd():
        camp.camp_solver_solve_ex(s.h, C, A, w, lam, tol, maxit, it[1], res[1], st[1],
                                  camp.CAMP_TRANSPOSE)
        camp.camp_solver_grad_A(s.h, C, lam, x, gA)

    def both():
        fwd()
        bwd()
    tt = sum(time_steps(both, flush, stream, steps, 3)) / steps
    tb = sum(time_steps(bwd, flush, stream, steps, 3)) / steps
    out = {"workload": synth.WORKLOADS[3][0], "cells": C,
           "value": C / (tt * 1e-3), "unit": "cells/s (forward + backward)", "ms_per_step": tt,
           "backward_ms": tb, "backward_share": tb / tt,
           "converged_forward": int((st[0] == 0).sum().item()),
           "converged_transposed": int((st[1] == 0).sum().item()),
           "iters_mean_forward": float(it[0].double().mean().item()),
           "iters_mean_transposed": float(it[1].double().mean().item())}
    s.close()
    return out


def fp64_rate(camp, dev):
    """Measured FP64 FMA rate of this GPU (GFLOP/s, 2 flops per FMA): the
    library's probe of independent dependent-FMA chains, 64 warps per SM on
    every SM, timed with CUDA events (median of 5)."""
    import ctypes
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n, steps = sms * 2048, 4096
    x = torch.rand(n, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    f = camp._lib.camp_selftest
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    s = torch.cuda.current_stream(dev)
    ts = []
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        assert f(6, n, x.data_ptr(), y.data_ptr(), steps, s.cuda_stream) == 0
        e1.record(s)
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    ms = sorted(ts[1:])[2]
    return 2.0 * 4 * n * steps / (ms * 1e-3) / 1e9


def time_fused(camp, cb, tol, maxit, flush, stream, dev, steps=200, ordering=None):
    """The same cells solved with the matrices assembled in the kernel from
    the concentrations (A = I - gamma J) instead of read from HBM."""
    import torch
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k)
    if ordering is not None:
        s.set_ordering(ordering)
    conc = torch.as_tensor(cb.conc, device=dev)
    gam = torch.as_tensor(cb.gamma, device=dev)
    b = torch.as_tensor(cb.b, device=dev)
    out = s.assemble_solve(conc, gam, b, tol, maxit)
    t = time_steps(lambda: s.assemble_solve(conc, gam, b, tol, maxit, out=out), flush, stream,
                   steps, 5)
    ms = sum(t) / steps
    conv = int((out[3] == 0).sum().item())
    s.close()
    return {"value": cb.cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "what": "matrices assembled in shared memory from concentrations and gamma",
            "hbm_bytes_per_cell": 8 * m.n + 8 + 16 * m.n + 12, "converged": conv}


def time_newton(camp, cb, flush, stream, dev, steps=50, newton_tol=1e-10, lin_tol=1e-10,
                lin_maxit=500, ordering=None):
    """The device Newton corrector of the implicit step on the same cells:
    history term a = the cells' concentrations, initial guess y = a; every
    step copies the guess in and runs all Newton iterations of all cells in
    one launch.  The unit is Newton solves (cells) per second."""
    import torch
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    s.set_mechanism(m.reactants[:, 0], m.reactants[:, 1], m.products, m.k)
    if ordering is not None:
        s.set_ordering(ordering)
    a = torch.as_tensor(cb.conc, device=dev)
    gam = torch.as_tensor(cb.gamma, device=dev)
    out = s.newton_solve(a, gam, a, newton_tol, 20, lin_tol, lin_maxit)
    y = out["y"]

    def step():
        y.copy_(a)
        camp.camp_solver_newton_solve(s.h, cb.cells, a, gam, y, newton_tol, 20, lin_tol,
                                      lin_maxit, out["newton_iters"], out["lin_iters"],
                                      out["upd"], out["resid"], out["status"])
    t = time_steps(step, flush, stream, steps, 5)
    ms = sum(t) / steps
    ni = out["newton_iters"].double()
    res = {"value": cb.cells / (ms * 1e-3), "unit": "cell Newton solves/s", "ms_per_step": ms,
           "what": "Newton corrector of y - gamma f(y) - a = 0 per cell on the device "
                   "(rates, assembly, BiCGSTAB per iteration), newton_tol 1e-10",
           "newton_iters_mean": float(ni.mean().item()),
           "newton_iters_max": int(ni.max().item()),
           "lin_iters_per_newton": float((out["lin_iters"].double() / ni.clamp(min=1))
                                         .mean().item()),
           "converged": int((out["status"] == 0).sum().item())}
    s.close()
    return res


def run_step_case(args):
    """--case fused / --case newton: the in-kernel assembly + solve, or the
    device Newton corrector, alone on the 80-species cells (for profiling)."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    cbs, tol, maxit = synth.workload(WORKLOAD_ID)
    st = torch.cuda.current_stream()
    if args.case == "fused":
        res = time_fused(camp, cbs[0], tol, maxit, flush, st, dev, steps=args.steps,
                         ordering=args.ordering)
    else:
        res = time_newton(camp, cbs[0], flush, st, dev, steps=args.steps,
                          ordering=args.ordering)
    ordering = args.ordering if args.ordering is not None else DEFAULT_ORDERING
    print(json.dumps({"case": args.case, "ordering": ordering, **res}), flush=True)


def run_side_case(args):
    """--case cfg4 / --case adjoint: the 150-species mixed-precision block or
    the adjoint block alone (for profiling)."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    if args.case == "cfg4":
        res = time_cfg4(camp, dev, flush, st, steps=args.steps)
    else:
        res = time_adjoint(camp, dev, flush, st, steps=args.steps)
    print(json.dumps({"case": args.case, **res}), flush=True)


def run_small_case(args):
    """--case small: the small-batch block alone (automatic launch against
    pairs only) at the sizes --cells lists, e.g. for profiling a lone warp."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    cbs, tol, maxit = synth.workload(WORKLOAD_ID)
    sizes = tuple(int(c) for c in args.cells.split(","))
    if not sizes or min(sizes) < 1 or max(sizes) > cbs[0].cells:
        raise SystemExit(f"--cells must list sizes in [1, {cbs[0].cells}]")
    res = time_small_batches(camp, cbs[0], tol, maxit, flush, torch.cuda.current_stream(), dev,
                             steps=args.steps, sizes=sizes)
    print(json.dumps({"case": "small", "workload": synth.WORKLOADS[WORKLOAD_ID][0],
                      "unit": "us per solve", "sizes": res}), flush=True)


def run_uneven_case(args):
    """--case uneven: the persistent batch alone, timed as the step."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    res = time_uneven(camp, dev, flush, torch.cuda.current_stream(), steps=args.steps,
                      tune=not args.no_tune)
    print(json.dumps({"case": "uneven", **res}), flush=True)


def lockstep_waste(iters, k):
    """Lane-iterations idle because the k cells sharing a warp run until the
    slowest converges, as a fraction of the useful ones (consecutive cells of
    the given order share a warp)."""
    it = np.asarray(iters, dtype=np.float64)
    pad = (-len(it)) % k
    grp = np.concatenate([it, np.zeros(pad)]).reshape(-1, k)
    return float((grp.max(axis=1, keepdims=True) - grp).sum() / max(it.sum(), 1.0))


def run_variability_case(args):
    """--case variability: the realistic vs ideal rows alone."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    rows = variability(camp, dev, flush, torch.cuda.current_stream(), args.steps)
    print(json.dumps({"case": "variability", "unit": UNIT, "rows": rows}), flush=True)


def sv_lanes(n):
    """Lanes per cell of the automatic warp arrangement (at most five rows per lane)."""
    lc = 1
    while (n + lc - 1) // lc > 5 and lc < 32:
        lc *= 2
    return lc


def run_arrangements_case(args):
    """--case arrangements: the paper's kernel-configuration study (Sec. 3.2,
    Sec. 5.2) on the headline workload: every arrangement's solve time and
    iterations, per-cell scalars and coupled (shared-scalar) Block-cells(k)."""
    import torch
    from paper_2405_17363_gb300 import camp
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    cbs, tol, maxit = synth.workload(WORKLOAD_ID)
    cb = cbs[0]
    m = cb.mech
    s = camp.Solver(m.row_ptr, m.col_idx)
    A = torch.as_tensor(cb.A_vals, device=dev)
    b = torch.as_tensor(cb.b, device=dev)
    nmax = 1024 // m.n
    arrs = [("warp-packed auto", (camp.CAMP_ARR_AUTO, 0, 1, 0)),
            ("warp per cell (32 lanes)", (camp.CAMP_ARR_WARP, 32, 0, 0))]
    for cpb in (1, 2, 3, nmax):
        arrs.append((f"Block-cells({cpb}) per-cell scalars", (camp.CAMP_ARR_BLOCK, 0, cpb, 0)))
    for cpb in (2, 3, nmax):
        arrs.append((f"Block-cells({cpb}) coupled", (camp.CAMP_ARR_BLOCK_COUPLED, 0, cpb, 0)))
    rows = []
    for name, arr in arrs:
        s.set_arrangement(*arr)
        out = s.solve(A, b, tol, maxit)
        ms = sum(time_steps(lambda: s.solve(A, b, tol, maxit, out=out), flush, stream,
                            args.steps, 3)) / args.steps
        it = out[1].cpu().numpy()
        rows.append({"arrangement": name, "ms": ms, "value": cb.cells / (ms * 1e-3),
                     "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                     "converged": int((out[3] == 0).sum().item())})
    s.close()
    print(json.dumps({"case": "arrangements", "workload": synth.WORKLOADS[WORKLOAD_ID][0],
                      "unit": UNIT, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--arrangement", default="auto",
                    help="auto | warp:<lanes per cell>[:<warps per block>] | block:<cells per block>")
    ap.add_argument("--mode", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: plain FP64 solve (the headline); mixed: FP32-inner refinement")
    ap.add_argument("--case", default="headline",
                    choices=["headline", "uneven", "arrangements", "variability", "fused",
                             "newton", "cfg4", "adjoint", "small"],
                    help="headline: the 80-species 10k-cell FP64 solve; uneven: time the "
                         "persistent multi-mechanism batch as the step; fused / newton: the "
                         "in-kernel assembly or the device Newton corrector alone (for "
                         "profiling); small: small batches (--cells) automatic against pairs "
                         "only")
    ap.add_argument("--cells", default="64,608",
                    help="--case small: comma-separated batch sizes of headline cells")
    ap.add_argument("--ordering", type=int, default=None, choices=[0, 1, 2],
                    help="cell ordering: 0 index order, 1 hardest first ordered inside the "
                         "solve launch, 2 hardest first by a separate pass (default: the "
                         "library's)")
    ap.add_argument("--no-tune", action="store_true",
                    help="--case uneven: keep the batch's automatic launch configuration "
                         "(no autotuning launches, e.g. for profiling)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the device solve only (no e2e, CPU baseline or mixed side run)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.case == "uneven":
        return run_uneven_case(args)
    if args.case == "arrangements":
        return run_arrangements_case(args)
    if args.case == "variability":
        return run_variability_case(args)
    if args.case in ("fused", "newton"):
        return run_step_case(args)
    if args.case in ("cfg4", "adjoint"):
        return run_side_case(args)
    if args.case == "small":
        return run_small_case(args)

    import torch
    import torch.distributed as dist
    from paper_2405_17363_gb300 import camp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    cbs, tol, maxit = synth.workload(WORKLOAD_ID)
    cb = cbs[0]
    m = cb.mech
    C = cb.cells
    solver = camp.Solver(m.row_ptr, m.col_idx)
    arr_desc = set_arrangement(camp, solver, args.arrangement)
    if args.ordering is not None:
        solver.set_ordering(args.ordering)
    ordering = args.ordering if args.ordering is not None else DEFAULT_ORDERING
    A = torch.as_tensor(cb.A_vals, device=dev)
    b = torch.as_tensor(cb.b, device=dev)
    x = torch.empty((C, m.n), dtype=torch.float64, device=dev)
    it = torch.empty(C, dtype=torch.int32, device=dev)
    res = torch.empty(C, dtype=torch.float64, device=dev)
    st = torch.empty(C, dtype=torch.int32, device=dev)
    sweeps = torch.empty(C, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def solve_fp64():
        camp.camp_solver_solve_ex(solver.h, C, A, b, x, tol, maxit, it, res, st, 0)

    def solve_mixed():
        camp.camp_solver_solve_mixed(solver.h, C, A, b, x, tol, 20, 1e-5, 50, it, sweeps,
                                     res, st)

    step = solve_fp64 if args.mode == "fp64" else solve_mixed
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = time_steps(step, flush, stream, args.steps, args.warmup)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dev)
    iters = it.cpu().numpy()
    status = st.cpu().numpy()
    sw = sweeps.cpu().numpy()
    value = weak_value(world, C, args.steps, total_ms)
    ms_step = total_ms / args.steps
    kernel_s = ms_step * 1e-3
    hbm_peak, hbm_src = peaks()
    flops, nbytes = algorithmic(m, C, iters)

    mixed_side = None
    e2e = None
    uneven = var_rows = cfg4 = adjoint = small = None
    fused = None
    newton = None
    fp64_measured = None
    if not args.skip_extras:
        if args.mode == "fp64":
            mt = time_steps(solve_mixed, flush, stream, 200, 5)
            mms = sum(mt) / len(mt)
            mixed_side = {
                "value": world * C / (mms * 1e-3), "unit": UNIT, "ms_per_step": mms,
                "what": "FP32-inner BiCGSTAB with FP64 residual and refinement sweeps "
                        "to the same 1e-10 true residual",
                "sweeps_mean": float(sweeps.float().mean().item()),
                "inner_iters_mean": float(it.float().mean().item()),
                "converged": int((st == 0).sum().item()),
                "speedup_vs_fp64": ms_step / mms}
        e2e = time_e2e(camp, solver, cb, C, tol, maxit, args.e2e_steps, world, dev)
        fp64_measured = fp64_rate(camp, dev)
        fused = time_fused(camp, cb, tol, maxit, flush, stream, dev)
        newton = time_newton(camp, cb, flush, stream, dev)
        if rank == 0:
            uneven = time_uneven(camp, dev, flush, stream)
            var_rows = variability(camp, dev, flush, stream, 20)
            cfg4 = time_cfg4(camp, dev, flush, stream)
            adjoint = time_adjoint(camp, dev, flush, stream)
            small = time_small_batches(camp, cb, tol, maxit, flush, stream, dev)

    if rank == 0:
        cpu = cpu_baseline(m, cb.A_vals, cb.b, tol, maxit, args.cpu_seconds) \
            if world == 1 and not args.skip_extras else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": synth.WORKLOADS[WORKLOAD_ID][0], "cells": C,
                       "n": m.n, "nnz": m.nnz, "tol": tol, "maxit": maxit,
                       "mode": args.mode, "arrangement": arr_desc,
                       "ordering": ["index", "hardest first, in the solve launch",
                                    "hardest first, separate pass"][ordering],
                       "l2": "flushed between timed steps (512 MB write)",
                       "iters_max": int(iters.max()), "iters_mean": float(iters.mean()),
                       "converged": int((status == 0).sum())},
            "roofline": {"bound": "alu", "achieved": flops / kernel_s / 1e9,
                         "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": flops / kernel_s / 1e9 / FP64_PEAK_GFLOPS,
                         "traffic": measured_traffic(camp.camp_version())
                         if args.arrangement == "auto" and args.mode == "fp64" else None,
                         "peak_source": "FP64 pipe 4 flop/clk/SM x 152 SMs x 2.07 GHz"},
            "hbm_roofline": {"bound": "hbm", "achieved": nbytes / kernel_s / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": nbytes / kernel_s / 1e9 / hbm_peak,
                             "peak_source": hbm_src},
            "e2e": e2e,
            # the classify and scatter pass adds two launches per solve
            "gpu_launches": args.steps * (3 if ordering == 2 and args.mode == "fp64" else 1),
            "clocks": clk,
        }
        if args.mode == "mixed":
            line["config"]["sweeps_mean"] = float(sw.mean())
            line["roofline"] = None
        if fp64_measured is not None and line["roofline"] is not None:
            # the same achieved rate against the FMA rate measured on this GPU
            line["roofline"]["peak_measured"] = fp64_measured
            line["roofline"]["frac_of_measured"] = line["roofline"]["achieved"] / fp64_measured
        if mixed_side is not None:
            line["mixed_fp32_inner"] = mixed_side
        if uneven is not None:
            line["uneven_batch"] = uneven
        if var_rows is not None:
            line["variability"] = var_rows
        if cfg4 is not None:
            line["mixed_cfg4"] = cfg4
        if adjoint is not None:
            line["adjoint"] = adjoint
        if small is not None:
            line["small_batches"] = small
        if fused is not None:
            line["fused_assembly"] = fused
        if newton is not None:
            line["newton_step"] = newton
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    solver.close()


if __name__ == "__main__":
    main()
