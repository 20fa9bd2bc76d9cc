#!/usr/bin/env python3
"""Benchmark of the multi-RHS pressure-Poisson hot path on one GB300 (or N replicas).

One step = one GSpMV sweep Y = A X over m in {1, 2, 4, 8, 16, 32} (FP64, Section 2.3) on the
variable-coefficient channel operator 256 x 128 x 128 (n = 4,194,304, nnz = 29,294,592), with
all inputs resident in HBM. `value` is the sweep's algorithmic HBM throughput:
    bytes(m) = 4(n+1) + 12 nnz + 16 m n      (matrix once, X in once, Y out once)
summed over the sweep, divided by the device time (CUDA events, max over ranks). Every launch
moves >= 435 MB, more than the 129 MB L2, so no flush is needed between launches.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on the host instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSpMV HBM GB/s vs m; multi-RHS Poisson solves/s at rel.res 1e-8; p99 latency"
WORKLOAD = "channel256x128x128"
M_SWEEP = (1, 2, 4, 8, 16, 32)
FALLBACK_HBM_GBS = 6800.0
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "gspmv_tile_m32_channel.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1711_10622_gb300", "csrc", f) for f in ("rowprod.cuh", "gspmv.cu")]


def alg_bytes(n: int, nnz: int, m: int, sv: int = 8, sx: int = 8) -> int:
    """Matrix once (row_ptr, col_idx, val), X read once, Y written once."""
    return 4 * (n + 1) + (4 + sv) * nnz + 2 * sx * m * n


def paper_traffic(n: int, nnz: int, m: int) -> float:
    """Sigma_m of Section 2.3 (X re-read for every nonzero)."""
    return 4.0 * n * (2 * m + 1) + 12.0 * nnz + 8.0 * m * nnz


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    try:
        text = open(PROFILE_SUMMARY).read()
        h = hashlib.sha256()
        for p in KERNEL_SOURCES:
            h.update(open(p, "rb").read())
        src_hash = h.hexdigest()
    except OSError:
        return None
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not h or not t or h.group(1) != src_hash:
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    QUERY = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL,
                text=True,
            )
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


def replica_throughput(dist, seconds: float, units_per_step: float, steps: int, device="cuda"):
    """Whole-job throughput of N independent replicas: every rank processed units_per_step * steps
    in its own `seconds`; the job took the slowest rank's time. Returns (max seconds, total units
    per second). dist = torch.distributed (initialised) or None for one process."""
    world = 1
    if dist is not None:
        import torch

        world = dist.get_world_size()
        t = torch.tensor([seconds], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return seconds, world * units_per_step * steps / seconds


def host_info():
    """Core count and CPU model of this host (recorded beside every CPU number)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": os.uname().machine}


def cpu_baseline_sweep(op, seconds_cap: float = 30.0, reps: int = 10):
    """The oracle (C, FP64) on the host, as it stands: (i) the serial build on one core, column by
    column, one full m-sweep on the full channel operator (capped at `seconds_cap`); (ii) the OpenMP
    build of the same source on all host cores, column by column and with the columns of a row
    together (the loop order of Fig. GSpMV): 2 untimed sweeps, then the median of `reps` timed sweeps
    (the row-wise one; the column-wise one, ~0.5 s a sweep, is capped at `seconds_cap` of timed
    sweeps); (iii) the oracle's per-column BiCGStab on the plain-method workload (32^3, m = 4, tol
    1e-8), serial and all cores. `value` is the faster all-core product (GB/s of algorithmic bytes)."""
    import gen
    import oracle

    n, nnz = op.n, op.nnz
    Xs = {m: gen.rhs_normal(n, m, 20000 + m) for m in M_SWEEP}

    def sweep(fn, cap=None):
        total_bytes, total_t, done = 0, 0.0, []
        for m in M_SWEEP:
            t0 = time.perf_counter()
            fn(Xs[m])
            total_t += time.perf_counter() - t0
            total_bytes += alg_bytes(n, nnz, m)
            done.append(m)
            if cap is not None and total_t > cap:
                break
        return total_bytes / total_t / 1e9, done, total_t

    serial_gbs, serial_done, _ = sweep(lambda X: oracle.gspmv(op, X), seconds_cap)
    out = {
        "value": serial_gbs,
        "unit": "GB/s",
        "cores": 1,
        "kind": "oracle",
        "sample": f"one FP64 GSpMV per m in {serial_done} on the full {WORKLOAD} operator (serial C oracle, column by column)",
        "serial": {"gbs": serial_gbs, "cores": 1, "widths": serial_done},
        "host": host_info(),
    }
    def median_sweeps(fn, cap=None):
        for _ in range(2):
            sweep(fn)
        runs, spent = [], 0.0
        while len(runs) < reps and (cap is None or spent < cap or len(runs) < 1):
            gbs, _, t = sweep(fn)
            runs.append(gbs)
            spent += t
        return statistics.median(runs), len(runs)

    if oracle.lib_omp() is not None:
        threads = oracle.threads(parallel=True)
        col_gbs, col_n = median_sweeps(lambda X: oracle.gspmv(op, X, parallel=True), seconds_cap)
        row_gbs, row_n = median_sweeps(lambda X: oracle.gspmv_rowwise(op, X, parallel=True))
        out.update(
            {
                "value": max(col_gbs, row_gbs),
                "cores": threads,
                "sample": f"one FP64 GSpMV per m in {list(M_SWEEP)} on the full {WORKLOAD} operator per sweep, OpenMP build "
                f"of the oracle on {threads} threads, median of {row_n} sweeps after 2 untimed ones (rows split; columns of a "
                f"row together = {row_gbs:.2f} GB/s, column by column = {col_gbs:.2f} GB/s, median of {col_n}); the serial "
                f"build on 1 core, one sweep: {serial_gbs:.2f} GB/s",
                "all_cores": {"threads": threads, "rowwise_gbs": row_gbs, "columnwise_gbs": col_gbs,
                              "rowwise_sweeps": row_n, "columnwise_sweeps": col_n},
            }
        )
    # oracle block solves: RHS-solves/s of the per-column BiCGStab on the plain-method workload
    w = gen.WORKLOADS["dirichlet32_m4"]
    dop = w["op"]()
    B = w["rhs"](dop.n, 4)
    solves = {}
    for par in (False, True):
        if par and oracle.lib_omp() is None:
            continue
        t0 = time.perf_counter()
        _, it, _, st = oracle.solve_block(dop, B, w["tol"], parallel=par)
        dt = time.perf_counter() - t0
        solves["all_cores" if par else "serial"] = {"rhs_solves_per_s": 4 / dt, "seconds": dt, "threads": oracle.threads(par),
                                                    "iters": it.tolist(), "converged": int((st == 0).sum())}
    out["solves_dirichlet32_m4"] = solves
    return out


def oracle_references(level: str = "default") -> dict:
    """FP64 oracle solutions that the bench's GPU results are compared with (run in a spawned process
    on the host cores while the GPU sections run). Each entry: the oracle's X for the columns listed,
    solved to a tolerance tighter than the GPU's (so its own error does not mask the GPU's):
      dirichlet32_m4         all 4 columns, unpreconditioned, tol 1e-12
      cubes192x128x96_m8     all 8 columns, oracle AMG preconditioner, tol 1e-11
      batch                  64^3 all 4 columns; 128^3 and 96x160x96 column 0 (AMG, tol 1e-12);
                             256x192x192 column 0 only with level 'full' (minutes on the host)
      serving                the sampled requests (see serving_samples), AMG, tol 1e-12
    """
    import numpy as np

    import gen
    import oracle

    out, t_all = {}, time.perf_counter()
    par = oracle.lib_omp() is not None
    w = gen.WORKLOADS["dirichlet32_m4"]
    op = w["op"]()
    t0 = time.perf_counter()
    X, it, rr, st = oracle.solve_block(op, w["rhs"](op.n, 4), 1e-12, parallel=par)
    out["dirichlet32_m4"] = {"X": X, "cols": [0, 1, 2, 3], "tol": 1e-12, "precond": "none", "status": st.tolist(),
                             "seconds": time.perf_counter() - t0}
    w = gen.WORKLOADS["cubes192x128x96_m8"]
    op = w["op"]()
    t0 = time.perf_counter()
    H = oracle.AMG(op)
    X, it, rr, st = oracle.solve_block(op, w["rhs"](op.n, 8), 1e-11, precond="amg", amg=H, parallel=par)
    H.close()
    out["cubes192x128x96_m8"] = {"X": X, "cols": list(range(8)), "tol": 1e-11, "precond": "amg", "status": st.tolist(),
                                 "seconds": time.perf_counter() - t0}
    batch = {}
    for i, (dims, m) in enumerate(BATCH_SPECS):
        cols = list(range(m)) if dims == (64, 64, 64) else [0]
        if dims == (256, 192, 192) and level != "full":
            continue
        op = gen.channel(*dims)
        B = gen.rhs_normal(op.n, m, 10622 + 40 + i, zero_mean=True)[:, cols]
        t0 = time.perf_counter()
        H = oracle.AMG(op)
        X, it, rr, st = oracle.solve_block(op, np.ascontiguousarray(B), 1e-12, precond="amg", amg=H, parallel=par)
        H.close()
        batch["x".join(map(str, dims))] = {"X": X, "cols": cols, "tol": 1e-12, "precond": "amg", "status": st.tolist(),
                                           "seconds": time.perf_counter() - t0}
    out["batch"] = batch
    ops = gen.serving_operators()
    serving = {}
    for k, (name, B) in serving_samples(ops).items():
        op = ops[name]
        t0 = time.perf_counter()
        H = oracle.AMG(op)
        X, it, rr, st = oracle.solve_block(op, B, 1e-12, precond="amg", amg=H, parallel=par)
        H.close()
        serving[k] = {"X": X, "op": name, "tol": 1e-12, "status": st.tolist(), "seconds": time.perf_counter() - t0}
    out["serving"] = serving
    out["threads"] = oracle.threads(par)
    out["seconds"] = time.perf_counter() - t_all
    return out


def rel_err_cols(X, Xref, cols) -> float:
    """max over the listed columns of ||x_l - x_ref,l|| / ||x_ref,l|| (host arrays)."""
    import numpy as np

    X = np.asarray(X)[:, cols]
    return float((np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)).max())


TIGHT_TOL = 3e-10


def solve_metrics(reps: int = 2, keep: dict | None = None):
    """RHS-solves/s of the block solver against the one-RHS-at-a-time solver (the same library,
    m = 1, looped over the columns) on the configured solve workloads: against FP64 with the plain
    preconditioner, and like for like (same preconditioner and precision). Each solve is timed end to
    end around the synchronous ens_solve_block call (inputs resident on the GPU). The solutions are
    kept (host copies in `keep`) for the error against the oracle, attached once the oracle's
    references are in. The cube workload also runs at tol TIGHT_TOL (keys ending in "_tight"), where
    every solution error meets the 1e-6 bar (at 1e-8 the operator's conditioning leaves errors up to
    ~1e-5; at 1e-9 the float64 Chebyshev solve still measured 1.1e-6)."""
    import torch

    import gen
    import paper_1711_10622_gb300 as ens

    cases = [
        ("dirichlet32_m4", gen.WORKLOADS["dirichlet32_m4"], 4, "none"),
        ("cubes192x128x96_m8", gen.WORKLOADS["cubes192x128x96_m8"], 8, "chebyshev"),
    ]
    keep = {} if keep is None else keep
    out = {}
    for name, w, m, pre in cases:
        op = w["op"]()
        B = torch.from_numpy(w["rhs"](op.n, m)).cuda()
        tol = w["tol"]
        A = ens.Matrix.from_operator(op)
        kept = keep.setdefault(name, {})

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                t0 = time.perf_counter()
                r = fn()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None or dt < best else best
            return best, r

        res = {}

        def record(key, t, X, st, tol_used):
            kept[key] = X.cpu().numpy()
            res[key] = {
                "solves_per_s": m / t,
                "seconds": t,
                "tol": tol_used,
                "max_relres": float(st["relres"].max()),
                "converged": int((st["status"] == 0).sum()),
                "iters": st["iters"].tolist(),
                "outer": st["outer"].tolist(),
            }

        tols = (tol, TIGHT_TOL) if pre == "chebyshev" else (tol,)
        for tl in tols:
            sfx = "" if tl == tol else "_tight"
            for prec in ("f64", "mixed"):
                t, (X, st) = timed(lambda: ens.solve_block(A, B, tol=tl, precond=pre, precision=prec))
                record(prec + sfx, t, X, st, tl)
        if pre == "chebyshev":  # the same solves with the aggregation multigrid V-cycle instead
            t_setup = time.perf_counter()
            levels = A.amg_setup()
            t_setup = time.perf_counter() - t_setup
            for tl in tols:
                sfx = "" if tl == tol else "_tight"
                for prec in ("f64", "mixed"):
                    t, (X, st) = timed(lambda: ens.solve_block(A, B, tol=tl, precond="amg", precision=prec))
                    record(prec + "_amg" + sfx, t, X, st, tl)
            res["amg_setup_s"] = t_setup
            res["amg_levels"] = levels
        # the coupled block-Krylov variant (one Krylov space for all m columns, float64)
        for cp in ((pre, "amg") if pre == "chebyshev" else (pre,)):
            t, (X, st) = timed(lambda: ens.solve_block_coupled(A, B, tol=tol, precond=cp))
            record("coupled_f64" + ("" if cp == pre else "_" + cp), t, X, st, tol)
        # one-RHS-at-a-time baselines: the same solver with m = 1 looped over the columns, for every
        # preconditioner and precision above (like for like), and FP64 with the plain preconditioner
        cols = [B[:, l : l + 1].contiguous() for l in range(m)]
        for key in [k for k in ("f64", "mixed", "f64_amg", "mixed_amg") if k in res]:
            prec, _, p1 = key.partition("_")
            t1, outs = timed(lambda: [ens.solve_block(A, c, tol=tol, precond=p1 or pre, precision=prec) for c in cols])
            kept["one_rhs_" + key] = torch.cat([o[0] for o in outs], dim=1).cpu().numpy()
            res["one_rhs_" + key] = {"solves_per_s": m / t1, "seconds": t1, "iters": [int(o[1]["iters"][0]) for o in outs]}
            res[key]["speedup_vs_one_rhs_same"] = res[key]["solves_per_s"] / res["one_rhs_" + key]["solves_per_s"]
        base = res["one_rhs_f64"]["solves_per_s"]
        for prec in ("f64", "mixed", "f64_amg", "mixed_amg", "coupled_f64", "coupled_f64_amg"):
            if prec in res:
                res[prec]["speedup_vs_one_rhs_f64"] = res[prec]["solves_per_s"] / base
        res["tol"] = tol
        res["precond"] = pre
        out[name] = res
        A.close()
    return out


def attach_oracle_errors(section: dict, keep: dict, refs: dict, sol_bar: float = 1e-6):
    """Add max_rel_err_vs_oracle to every kept result of `section` (per workload) from the oracle's
    references; meets_1e-6 says whether the solution-error bar holds for that result."""
    for name, kept in keep.items():
        ref = refs.get(name)
        if ref is None or name not in section:
            continue
        for key, X in kept.items():
            err = rel_err_cols(X, ref["X"], ref["cols"])
            entry = section[name].setdefault(key, {})
            entry["max_rel_err_vs_oracle"] = err
            entry["meets_1e-6"] = err <= sol_bar
        section[name]["oracle_reference"] = {"tol": ref["tol"], "precond": ref["precond"], "columns": ref["cols"],
                                             "host_seconds": ref["seconds"]}


# cuSPARSE generic-API constants (cusparse.h, library_types.h)
_CUSPARSE_INDEX_32I, _CUSPARSE_BASE_ZERO, _CUSPARSE_NON_TRANSPOSE, _CUSPARSE_ORDER_ROW, _CUDA_R_64F = 2, 0, 0, 2, 1
_CUSPARSE_SPMM_ALGS = {"default": 0, "csr_alg1": 4, "csr_alg2": 6, "csr_alg3": 12}
_CUSPARSE_SPMV_ALGS = {"default": 0, "csr_alg1": 2, "csr_alg2": 3}


def _load_cusparse():
    import ctypes

    for name in ("libcusparse.so", "libcusparse.so.13", "libcusparse.so.12", "/usr/local/cuda/lib64/libcusparse.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def cusparse_comparator(op, Xs, per_m_us, stream, reps: int = 20):
    """External comparator only (never dispatched to): the vendor library's CSR x dense product on the
    same operator and the same row-interleaved inputs, FP64, int32 indices, called directly through
    cuSPARSE's generic API (SpMV at m = 1, SpMM with row-major dense blocks otherwise). Every
    algorithm the library offers for the case is timed (CUDA events over `reps` calls after 3 warm-up
    calls, work buffer and preprocessing outside the timed region) and the fastest is reported, with
    its algorithmic GB/s, this library's speed-up over it and the largest element-wise difference of
    the two Y relative to |A||X|."""
    import ctypes

    import numpy as np
    import torch

    lib = _load_cusparse()
    if lib is None:
        return {"unavailable": "libcusparse not found"}
    vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER(vp)
    lib.cusparseCreate.argtypes = [P]
    lib.cusparseSetStream.argtypes = [vp, vp]
    lib.cusparseCreateCsr.argtypes = [P, i64, i64, i64, vp, vp, vp, ci, ci, ci, ci]
    lib.cusparseCreateDnMat.argtypes = [P, i64, i64, i64, vp, ci, ci]
    lib.cusparseCreateDnVec.argtypes = [P, i64, vp, ci]
    lib.cusparseSpMM_bufferSize.argtypes = [vp, ci, ci, vp, vp, vp, vp, vp, ci, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.cusparseSpMM_preprocess.argtypes = [vp, ci, ci, vp, vp, vp, vp, vp, ci, ci, vp]
    lib.cusparseSpMM.argtypes = [vp, ci, ci, vp, vp, vp, vp, vp, ci, ci, vp]
    lib.cusparseSpMV_bufferSize.argtypes = [vp, ci, vp, vp, vp, vp, vp, ci, ci, ctypes.POINTER(ctypes.c_size_t)]
    lib.cusparseSpMV.argtypes = [vp, ci, vp, vp, vp, vp, vp, ci, ci, vp]
    for f in ("cusparseDestroy", "cusparseDestroySpMat", "cusparseDestroyDnMat", "cusparseDestroyDnVec"):
        getattr(lib, f).argtypes = [vp]

    def ck(status, what):
        if status != 0:
            raise RuntimeError(f"{what}: cuSPARSE status {status}")

    h, A = vp(), vp()
    ck(lib.cusparseCreate(ctypes.byref(h)), "cusparseCreate")
    ck(lib.cusparseSetStream(h, vp(stream.cuda_stream)), "cusparseSetStream")
    rp = torch.from_numpy(op.row_ptr.astype(np.int32)).cuda()
    cols = torch.from_numpy(op.col_idx.astype(np.int32)).cuda()
    vals = torch.from_numpy(op.val).cuda()
    ck(lib.cusparseCreateCsr(ctypes.byref(A), op.n, op.n, op.nnz, vp(rp.data_ptr()), vp(cols.data_ptr()),
                             vp(vals.data_ptr()), _CUSPARSE_INDEX_32I, _CUSPARSE_INDEX_32I, _CUSPARSE_BASE_ZERO,
                             _CUDA_R_64F), "cusparseCreateCsr")
    alpha, beta = ctypes.c_double(1.0), ctypes.c_double(0.0)
    pa, pb = ctypes.cast(ctypes.byref(alpha), vp), ctypes.cast(ctypes.byref(beta), vp)
    absA = torch.sparse_csr_tensor(rp, cols, vals.abs(), size=(op.n, op.n))
    out = {}
    for m, X in Xs.items():
        Y = torch.empty_like(X)
        dx, dy = vp(), vp()
        if m == 1:
            ck(lib.cusparseCreateDnVec(ctypes.byref(dx), op.n, vp(X.data_ptr()), _CUDA_R_64F), "DnVec")
            ck(lib.cusparseCreateDnVec(ctypes.byref(dy), op.n, vp(Y.data_ptr()), _CUDA_R_64F), "DnVec")
            algs = _CUSPARSE_SPMV_ALGS
        else:
            ck(lib.cusparseCreateDnMat(ctypes.byref(dx), op.n, m, m, vp(X.data_ptr()), _CUDA_R_64F, _CUSPARSE_ORDER_ROW), "DnMat")
            ck(lib.cusparseCreateDnMat(ctypes.byref(dy), op.n, m, m, vp(Y.data_ptr()), _CUDA_R_64F, _CUSPARSE_ORDER_ROW), "DnMat")
            algs = _CUSPARSE_SPMM_ALGS
        per_alg, best, best_y = {}, None, None
        for name, alg in algs.items():
            try:
                size = ctypes.c_size_t(0)
                if m == 1:
                    ck(lib.cusparseSpMV_bufferSize(h, _CUSPARSE_NON_TRANSPOSE, pa, A, dx, pb, dy, _CUDA_R_64F, alg,
                                                   ctypes.byref(size)), "SpMV_bufferSize")
                else:
                    ck(lib.cusparseSpMM_bufferSize(h, _CUSPARSE_NON_TRANSPOSE, _CUSPARSE_NON_TRANSPOSE, pa, A, dx, pb, dy,
                                                   _CUDA_R_64F, alg, ctypes.byref(size)), "SpMM_bufferSize")
                buf = torch.empty(max(int(size.value), 16), dtype=torch.uint8, device="cuda")
                bp = vp(buf.data_ptr())
                if m == 1:
                    def call():
                        ck(lib.cusparseSpMV(h, _CUSPARSE_NON_TRANSPOSE, pa, A, dx, pb, dy, _CUDA_R_64F, alg, bp), "SpMV")
                else:
                    lib.cusparseSpMM_preprocess(h, _CUSPARSE_NON_TRANSPOSE, _CUSPARSE_NON_TRANSPOSE, pa, A, dx, pb, dy,
                                                _CUDA_R_64F, alg, bp)  # optional; only some algorithms use it

                    def call():
                        ck(lib.cusparseSpMM(h, _CUSPARSE_NON_TRANSPOSE, _CUSPARSE_NON_TRANSPOSE, pa, A, dx, pb, dy,
                                            _CUDA_R_64F, alg, bp), "SpMM")
                for _ in range(3):
                    call()
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                s.record(stream)
                for _ in range(reps):
                    call()
                e.record(stream)
                torch.cuda.synchronize()
                us = s.elapsed_time(e) / reps * 1e3
                per_alg[name] = {"us": us}
                if best is None or us < per_alg[best]["us"]:
                    best = name
                    best_y = Y.clone()  # the fastest algorithm's output, for the element-wise check
            except RuntimeError as exc:
                per_alg[name] = {"unavailable": str(exc)}
        lib.cusparseDestroyDnMat(dx) if m > 1 else lib.cusparseDestroyDnVec(dx)
        lib.cusparseDestroyDnMat(dy) if m > 1 else lib.cusparseDestroyDnVec(dy)
        if best is None:
            out[str(m)] = {"unavailable": per_alg}
            continue
        us = per_alg[best]["us"]
        scale = torch.mm(absA, X.abs()) if m > 1 else torch.mv(absA, X.abs().reshape(-1)).reshape(-1, 1)
        out[str(m)] = {
            "us": us,
            "algorithm": ("spmv_" if m == 1 else "spmm_") + best,
            "us_per_algorithm": {k: v.get("us") for k, v in per_alg.items()},
            "gbs": alg_bytes(op.n, op.nnz, m) / (us * 1e-6) / 1e9,
            "ours_speedup": us / per_m_us[m],
            "Y": best_y,
            "scale": scale,
        }
    lib.cusparseDestroySpMat(A)
    lib.cusparseDestroy(h)
    return out


def cubes_gspmv_metrics(reps: int = 20):
    """FP64 GSpMV on the wall-mounted-cube operator 192 x 128 x 96 (rows of 5-7 nonzeros) for
    m = 1..32, each width autotuned: device time per launch (CUDA events around `reps` launches
    after 3 warm-up launches, inputs resident) and algorithmic GB/s."""
    import torch

    import gen
    import paper_1711_10622_gb300 as ens

    op = gen.WORKLOADS["cubes192x128x96_m8"]["op"]()
    A = ens.Matrix.from_operator(op)
    sweep = {}
    for m in M_SWEEP:
        tuned = A.autotune(m, "f64")
        X = torch.from_numpy(gen.rhs_normal(op.n, m, 20100 + m)).cuda()
        Y = torch.empty_like(X)
        for _ in range(3):
            ens.gspmv(A, X, Y)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        for _ in range(reps):
            ens.gspmv(A, X, Y)
        e.record()
        torch.cuda.synchronize()
        us = s.elapsed_time(e) / reps * 1e3
        b = alg_bytes(op.n, op.nnz, m)
        sweep[str(m)] = {"us": us, "alg_mb": b / 1e6, "gbs": b / (us * 1e-6) / 1e9, "tuned": tuned}
        del X, Y
    A.close()
    return {"workload": "cubes192x128x96", "n": op.n, "nnz": op.nnz, "sweep": sweep}


BATCH_SPECS = [((256, 192, 192), 16), ((64, 64, 64), 4), ((128, 128, 128), 8), ((96, 160, 96), 32)]


def batch_metrics(precond: str = "amg", keep: dict | None = None):
    """The batching workload: channel 256x192x192 (m = 16), 64^3 (m = 4), 128^3 (m = 8) and
    96x160x96 (m = 32) in ONE ens_solve_batch launch, FP32 inner / FP64 refinement to 1e-10.
    RHS-solves/s of the batch (set-up of the preconditioner excluded) against the one-RHS-at-a-time
    solver on the same systems (every column solved alone, same preconditioner and precision, one
    after the other), per-system iterations; the solutions are kept in `keep` for the error against
    the oracle's references."""
    import numpy as np
    import torch

    import gen
    import paper_1711_10622_gb300 as ens

    keep = {} if keep is None else keep
    mats, Bs = [], []
    try:
        for i, (dims, m) in enumerate(BATCH_SPECS):
            op = gen.channel(*dims)
            A = ens.Matrix.from_operator(op)
            if precond == "amg":
                A.amg_setup()
            mats.append(A)
            Bs.append(torch.from_numpy(gen.rhs_normal(op.n, m, 10622 + 40 + i, zero_mean=True)).cuda())
        items = [(A, B, None, 1e-10) for A, B in zip(mats, Bs)]
        ens.solve_batch(items, precond=precond, precision="mixed")  # warm: graph code paths, pools
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ens.solve_batch(items, precond=precond, precision="mixed")
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        systems = []
        for (dims, m), A, B, (X, st) in zip(BATCH_SPECS, mats, Bs, res):
            g = "x".join(map(str, dims))
            keep[g] = X.cpu().numpy()
            systems.append({"grid": g, "m": m, "converged": int((st["status"] == 0).sum()),
                            "max_relres": float(np.max(st["relres"])), "iters_max": int(np.max(st["iters"])),
                            "outer_max": int(np.max(st["outer"]))})
        # one right-hand side at a time: every column of every system alone, one after the other
        for A, B in zip(mats, Bs):  # warm the m = 1 code paths
            ens.solve_block(A, B[:, :1].contiguous(), tol=1e-10, precond=precond, precision="mixed")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for A, B in zip(mats, Bs):
            for l in range(B.shape[1]):
                ens.solve_block(A, B[:, l : l + 1].contiguous(), tol=1e-10, precond=precond, precision="mixed")
        torch.cuda.synchronize()
        t1 = time.perf_counter() - t1
    finally:
        for A in mats:
            A.close()
    rhs = sum(m for _, m in BATCH_SPECS)
    return {"precond": precond, "precision": "mixed", "tol": 1e-10, "rhs": rhs, "seconds": t, "rhs_solves_per_s": rhs / t,
            "one_rhs": {"seconds": t1, "rhs_solves_per_s": rhs / t1, "how": "ens_solve_block with m = 1 per column, same systems, precond and precision"},
            "speedup_vs_one_rhs": t1 / t, "systems": systems}


def attach_batch_errors(batch: dict, keep: dict, refs: dict, sol_bar: float = 1e-6):
    for sysd in batch["systems"]:
        ref = refs.get(sysd["grid"])
        if ref is None:
            sysd["max_rel_err_vs_oracle"] = None
            sysd["oracle_columns"] = "not compared: the oracle needs minutes on the host for one column of this system"
            continue
        err = rel_err_cols(keep[sysd["grid"]], ref["X"], ref["cols"])
        sysd["max_rel_err_vs_oracle"] = err
        sysd["meets_1e-6"] = err <= sol_bar
        sysd["oracle_columns"] = ref["cols"]


def fp64_peak_ops(sm_mhz=None):
    """FP64 pipe ceiling in operations per second: 2 DFMA/DADD/DMUL per clock per SM (the peak
    the profiler reports for this part) x 152 SMs x the SM clock (sampled, else the 2070 MHz max)."""
    mhz = sm_mhz or 2070.0
    return 2.0 * 152 * mhz * 1e6


def projection_metrics(m: int = 8, reps: int = 20):
    """The projection step around the solve (Section 2.2, Eqs. eq2/eq3) on the 256 x 128 x 128
    channel grid at m states: device time of ens_divergence and ens_grad_correct, their
    algorithmic bytes (every face value, pressure and divergence touched once) and FP64 operation
    counts. Inputs resident; every launch streams > 1 GB (> L2)."""
    import numpy as np
    import torch

    import gen
    import paper_1711_10622_gb300 as ens

    op = gen.channel(256, 128, 128)
    g = gen.grid_of(op)
    U, V, W = (torch.from_numpy(c).cuda() for c in gen.predictor_velocity(g, m, 400, noise=0.1))
    P = torch.from_numpy(np.random.default_rng(9).standard_normal((op.n, m))).cuda()
    G = ens.Grid.from_grid(g)
    D = torch.empty(op.n, m, dtype=torch.float64, device="cuda")
    faces = sum(G.nfaces)

    def timed(fn):
        for _ in range(3):
            fn()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps * 1e3

    t_div = timed(lambda: ens.divergence(G, U, V, W, scale=-1.0, D=D))
    t_cor = timed(lambda: ens.grad_correct(G, P, U, V, W, 1e-9))
    G.close()
    b_div = 8 * m * (faces + op.n) + op.n  # faces read, D written, open-face mask
    b_cor = 8 * m * (2 * faces + op.n) + op.n  # faces read and written, P read, mask
    ops_div = 7 * op.n * m  # 6 DFMA + 1 DMUL per cell and state (face areas are tabulated)
    # per owned face and state a difference and an update, plus one tau * inv_dist product per face
    # shared by the 4 states a thread carries (m = 8)
    ops_cor = int((6 + 3 / 4) * op.n * m)
    return {
        "workload": "channel256x128x128",
        "m": m,
        "divergence": {"us": t_div, "alg_bytes": b_div, "gbs": b_div / (t_div * 1e-6) / 1e9, "fp64_ops": ops_div,
                       "fp64_gops": ops_div / (t_div * 1e-6) / 1e9},
        "grad_correct": {"us": t_cor, "alg_bytes": b_cor, "gbs": b_cor / (t_cor * 1e-6) / 1e9, "fp64_ops": ops_cor,
                         "fp64_gops": ops_cor / (t_cor * 1e-6) / 1e9},
    }


SERVING_SEED = 5


def serving_plan(ops, count: int, seed: int = SERVING_SEED):
    """The serving stream's requests in arrival order: (operator name, m, first column of the block
    taken from that operator's 64-column right-hand-side pool). Request k is the same whatever the
    count (both draws are sequential)."""
    import numpy as np

    import gen

    reqs = gen.serving_requests(count, ops, seed)
    rng = np.random.default_rng(seed + 2)
    return [(name, m, int(rng.integers(0, 64 - m + 1))) for name, m, _ in reqs]


def serving_pool(ops, name: str):
    """64 zero-mean N(0, 1) right-hand sides for one serving operator (seed by operator)."""
    import gen

    k = sorted(ops).index(name)
    return gen.rhs_normal(ops[name].n, 64, 10622 + 500 + k, zero_mean=True)


def serving_samples(ops, scan: int = 200, count: int = 4):
    """Requests whose result is compared with the oracle: the first `count` of the stream on the 64^3
    operators with m <= 4 (request index -> (operator, B))."""
    import numpy as np

    out = {}
    for k, (name, m, c0) in enumerate(serving_plan(ops, scan)):
        if name.endswith("64") and m <= 4:
            out[k] = (name, np.ascontiguousarray(serving_pool(ops, name)[:, c0 : c0 + m]))
            if len(out) == count:
                break
    return out


def serving_metrics(count: int, loads=(0.7, 1.0), seed: int = SERVING_SEED, budget: float = 120e9, slots: int = 6,
                    keep: dict | None = None):
    """One Poisson stream of `count` solve requests (grids 64^3..192^3, channel and cube operators, m
    drawn from {1, 2, 4, 8, 16, 32}, FP32 inner + FP64 refinement to 1e-8, AMG-lite preconditioner)
    through the continuous-batching server under an HBM budget. The stream is cut into len(loads)
    consecutive parts of equal size; part k arrives at loads[k] times the capacity measured by a
    saturated burst of the first 16 requests. Latency = arrival to result on the host, summarised per
    part (the first part is the top level; every part under "loads"). The sampled requests
    (serving_samples) are kept for the error against the oracle."""
    import numpy as np
    import torch

    import gen
    from paper_1711_10622_gb300.serving import Request, Server, latency_summary

    keep = {} if keep is None else keep
    ops = gen.serving_operators()
    plan = serving_plan(ops, count, seed)
    pools = {name: serving_pool(ops, name) for name in sorted(ops)}
    samples = set(serving_samples(ops))

    def make(k):
        # a view of the pool's columns (the server copies a batch's columns when it runs); only the
        # sampled requests keep their solution on the host
        name, m, c0 = plan[k]
        return Request(name, pools[name][:, c0 : c0 + m], 1e-8, keep_x=k in samples)

    out = []
    with Server(ops, budget_bytes=budget, slots=slots, max_cols=32, precond="amg") as srv:
        burst_n = min(16, count)
        burst = [srv.submit(make(k)) for k in range(burst_n)]
        for r in burst:
            r.done.wait(600)
        span = max(r.end for r in burst) - min(r.arrival for r in burst)
        cap_rps = burst_n / span
        # arrival times: part k's gaps are exponential with rate loads[k] * capacity
        cuts = np.linspace(0, count, len(loads) + 1).astype(int)
        gaps = np.random.default_rng(seed + 1).exponential(1.0, size=count)
        for k, load in enumerate(loads):
            gaps[cuts[k] : cuts[k + 1]] /= load * cap_rps
        arrivals = np.cumsum(gaps)
        pending = [make(k) for k in range(count)]
        srv.sched.reset_peak()
        t0 = time.perf_counter()
        for r, ta in zip(pending, arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            srv.submit(r)
        for r in pending:
            r.done.wait(1800)
        for k in samples:
            if k < count and pending[k].done.is_set() and pending[k].X is not None:
                keep[k] = pending[k].X
        torch.cuda.synchronize()
        free, total = torch.cuda.mem_get_info()
        peak = srv.sched.peak_in_flight + srv.sched.resident
        for k, load in enumerate(loads):
            part = [r for r in pending[cuts[k] : cuts[k + 1]] if r.done.is_set()]
            s = latency_summary(part)
            s.update(
                {
                    "arrival_rate_per_s": load * cap_rps,
                    "load_vs_measured_capacity": load,
                    "capacity_requests_per_s": cap_rps,
                    "stream_requests": count,
                    "part": [int(cuts[k]), int(cuts[k + 1])],
                    "budget_gb": budget / 1e9,
                    "peak_admitted_gb": peak / 1e9,
                    "pool_gb": srv.sched.pool.size / 1e9,
                    "device_used_gb": (total - free) / 1e9,
                    "slots": slots,
                    "grids": sorted(ops),
                    "tol": 1e-8,
                    "precision": "mixed",
                    "precond": "amg",
                    "converged_all": all((r.stats is not None and (r.stats["status"] == 0).all()) for r in part),
                    "unfinished": int((cuts[k + 1] - cuts[k]) - len(part)),
                }
            )
            out.append(s)
        model = srv.model.summary()
        model["how"] = ("alpha: drop of free device memory when the operator's matrix and AMG hierarchy are created; "
                        "beta + gamma m: least-squares line through the workspace bytes the library reports for probe "
                        "solves at m = 1, 4, 16, 32 (ens_last_workspace_bytes), in the solver's padded width")
    done_all = [r for r in pending if r.done.is_set()]
    top = dict(out[0])
    top["requests_total"] = count
    top["whole_stream"] = {k: v for k, v in latency_summary(done_all).items() if k != "p99_request"}
    top["memory_model"] = model
    top["loads"] = {str(s["load_vs_measured_capacity"]): {k: s[k] for k in ("requests", "part", "p50_ms", "p99_ms", "mean_ms", "wait_p50_ms", "wait_p99_ms", "service_p50_ms", "service_p99_ms", "p99_request", "requests_per_s", "rhs_solves_per_s", "arrival_rate_per_s", "peak_admitted_gb", "errors", "converged_all", "unfinished", "mean_batch_requests", "merged_fraction", "batch_cols_hist") if k in s} for s in out}
    return top


def attach_serving_errors(serving: dict, keep: dict, refs: dict, sol_bar: float = 1e-6):
    errs = {}
    for k, X in keep.items():
        ref = refs.get(k)
        if ref is None:
            continue
        errs[str(k)] = {"op": ref["op"], "m": int(X.shape[1]), "max_rel_err_vs_oracle": rel_err_cols(X, ref["X"], list(range(X.shape[1])))}
    serving["oracle_samples"] = errs
    serving["max_rel_err_vs_oracle"] = max((e["max_rel_err_vs_oracle"] for e in errs.values()), default=None)
    if serving["max_rel_err_vs_oracle"] is not None:
        serving["meets_1e-6"] = serving["max_rel_err_vs_oracle"] <= sol_bar


def run_reference(args):
    """The CPU oracle as it stands, on the host cores, on the same workload as the GPU arm: each step
    is one FP64 GSpMV per m on the full channel operator. The OpenMP build of the oracle source
    (rows split over all host cores, the columns of a row together as in Fig. GSpMV; the same bits
    as the serial oracle) when the compiler has OpenMP, else the serial build column by column."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gen
    import oracle

    op = gen.channel(256, 128, 128)
    Xs = {m: gen.rhs_normal(op.n, m, 20000 + m) for m in M_SWEEP}
    par = oracle.lib_omp() is not None
    fn = (lambda X: oracle.gspmv_rowwise(op, X, parallel=True)) if par else (lambda X: oracle.gspmv(op, X))

    def step():
        for m in M_SWEEP:
            fn(Xs[m])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    bytes_step = sum(alg_bytes(op.n, op.nnz, m) for m in M_SWEEP)
    value = bytes_step * args.steps / dt / 1e9
    threads = oracle.threads(par)
    how = (f"OpenMP build of the C oracle on {threads} threads, rows split, the columns of a row together" if par
           else "serial C oracle on 1 core, column by column")
    sample = f"the full {WORKLOAD} operator, one FP64 GSpMV per m in {list(M_SWEEP)} per step ({how})"
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "GB/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} GSpMV sweep m={list(M_SWEEP)}", "n": op.n, "nnz": op.nnz},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_profile(args):
    """Launch-only mode for ncu captures: W + K GSpMV launches per (m, arithmetic) on a channel
    operator of the requested size, no timing output; with --profile-modes projection, W + K
    divergence + correction pairs on that channel's grid instead; with solve-amg / solve-chebyshev,
    K BiCGStab iterations of the cube workload (192 x 128 x 96, m = 8, host-driven loop) instead
    (solve-amg-mixed / solve-chebyshev-mixed: one outer step of the mixed solve, K FP32 inner
    iterations).
    Sizes: 'full' = 256 x 128 x 128,
    'half' = 128 x 128 x 128 (inputs still larger than L2, a few GB on the device at most)."""
    import torch

    import gen
    from paper_1711_10622_gb300 import build as ens_build

    ens_build.build()
    import paper_1711_10622_gb300 as ens

    dims = {"full": (256, 128, 128), "half": (128, 128, 128)}[args.profile_size]
    op = gen.channel(*dims)
    ms = [int(v) for v in args.profile_m.split(",")]
    modes = args.profile_modes.split(",")
    if modes[0].startswith("coupled-"):  # K iterations of the coupled block solver, cubes m = 8
        precond = modes[0][len("coupled-"):]
        cop = gen.WORKLOADS["cubes192x128x96_m8"]["op"]()
        A = ens.Matrix.from_operator(cop)
        if precond == "amg":
            A.amg_setup()
        B = torch.from_numpy(gen.rhs_normal(cop.n, 8, 7, zero_mean=True)).cuda()
        ens.solve_block_coupled(A, B, tol=1e-8, precond=precond, max_iter=2)  # warm
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        t0 = time.perf_counter()
        ens.solve_block_coupled(A, B, tol=1e-30, precond=precond, max_iter=args.steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        t1 = time.perf_counter()
        ens.solve_block(A, B, tol=1e-30, precond=precond, max_iter=args.steps, use_graph=0)
        torch.cuda.synchronize()
        wall_ind = time.perf_counter() - t1
        A.close()
        print(json.dumps({"profile": "coupled", "precond": precond, "workload": "cubes192x128x96", "m": 8, "iterations": args.steps,
                          "coupled_ms_per_iter": wall / args.steps * 1e3, "independent_ms_per_iter": wall_ind / args.steps * 1e3}))
        return 0
    if modes[0].startswith("solve-"):  # a short block solve (cubes 192x128x96, m = 8) in the range
        # solve-amg | solve-chebyshev (FP64), or with "-mixed": one outer step of the mixed-precision
        # solve whose FP32 inner solve runs K iterations; host-driven loop
        precond, _, mixed = modes[0][len("solve-"):].partition("-")
        cop = gen.WORKLOADS["cubes192x128x96_m8"]["op"]()
        A = ens.Matrix.from_operator(cop)
        if precond == "amg":
            A.amg_setup()
        B = torch.from_numpy(gen.rhs_normal(cop.n, 8, 7, zero_mean=True)).cuda()
        prec = "mixed" if mixed == "mixed" else "f64"
        ens.solve_block(A, B, tol=1e-8, precond=precond, precision=prec)  # warm: workspace pools, code loaded
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        if prec == "mixed":
            ens.solve_block(A, B, tol=1e-30, precond=precond, precision="mixed", max_outer=1, inner_tol=1e-30,
                            inner_max_iter=args.steps, use_graph=0)
        else:
            ens.solve_block(A, B, tol=1e-30, precond=precond, max_iter=args.steps, use_graph=0)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        A.close()
        print(json.dumps({"profile": "solve", "precond": precond, "precision": prec, "workload": "cubes192x128x96", "m": 8, "iterations": args.steps}))
        return 0
    if modes == ["projection"]:  # ens_divergence + ens_grad_correct, inside the NVTX range "profiled"
        import numpy as np

        g = gen.grid_of(op)
        G = ens.Grid.from_grid(g)
        for m in ms:
            U, V, W = (torch.from_numpy(c).cuda() for c in gen.predictor_velocity(g, m, 400, noise=0.1))
            P = torch.from_numpy(np.random.default_rng(9).standard_normal((op.n, m))).cuda()
            D = torch.empty(op.n, m, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profiled")
            for _ in range(args.warmup + args.steps):
                ens.divergence(G, U, V, W, scale=-1.0, D=D)
                ens.grad_correct(G, P, U, V, W, 1e-9)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            del U, V, W, P, D
            torch.cuda.empty_cache()
        G.close()
        print(json.dumps({"profile": "projection", "size": dims, "m": ms, "launches_per_case": 2 * (args.warmup + args.steps)}))
        return 0
    A = ens.Matrix.from_operator(op)
    for m in ms:
        X = torch.from_numpy(gen.rhs_normal(op.n, m, 20000 + m)).to("cuda")
        for mode in modes:
            Xin = X.float() if mode == "f32" else X
            Y = torch.empty_like(Xin)
            if mode == "tuned":  # the bench's own configuration: autotuner choice for this width
                A.set_f64_mode("auto")
                A.autotune(m, "f64")
            elif mode != "f32":
                A.set_f64_mode(mode)
                ens.api.N.check(ens.api.N.lib().ens_set_native_share(A.handle, args.profile_share if mode == "split" else -1))
            torch.cuda.synchronize()
            # launches to capture are inside the NVTX range "profiled" (ncu --nvtx --nvtx-include profiled/)
            torch.cuda.nvtx.range_push("profiled")
            for _ in range(args.warmup + args.steps):
                ens.gspmv(A, Xin, Y)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            del Y, Xin
        del X
        torch.cuda.empty_cache()
    A.close()
    print(json.dumps({"profile": "gspmv", "size": dims, "m": ms, "modes": modes, "launches_per_case": args.warmup + args.steps}))
    return 0


def run_sweep(args):
    """Arithmetic sweep of the float64 GSpMV on the channel operator: microseconds per launch for
    native DFMA, split-float with native shares 0..24/32, the column hybrid, the autotuned choice
    and float32 (CUDA events around 20 launches after 3 warm-up launches, inputs resident). One
    JSON line; the basis of the arithmetic tables in the tuning notes."""
    import torch

    import gen
    from paper_1711_10622_gb300 import build as ens_build

    ens_build.build()
    import paper_1711_10622_gb300 as ens

    dims = {"full": (256, 128, 128), "half": (128, 128, 128)}[args.profile_size]
    op = gen.channel(*dims)
    A = ens.Matrix.from_operator(op)
    lib = ens.api.N.lib()

    def timed(X, Y, reps=20):
        for _ in range(3):
            ens.gspmv(A, X, Y)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record()
        for _ in range(reps):
            ens.gspmv(A, X, Y)
        e.record()
        torch.cuda.synchronize()
        return round(s.elapsed_time(e) / reps * 1e3, 1)

    rows = {}
    for m in [int(v) for v in args.profile_m.split(",")]:
        X = torch.from_numpy(gen.rhs_normal(op.n, m, 20000 + m)).to("cuda")
        Y = torch.empty_like(X)
        r = {}
        A.set_f64_mode("native")
        r["native"] = timed(X, Y)
        A.set_f64_mode("split")
        for share in (0, 4, 8, 12, 16, 20, 24):
            ens.api.N.check(lib.ens_set_native_share(A.handle, share))
            r[f"split{share}"] = timed(X, Y)
        ens.api.N.check(lib.ens_set_native_share(A.handle, -1))
        if m % 2 == 0:
            A.set_f64_mode("hybrid")
            r["hybrid"] = timed(X, Y)
        A.set_f64_mode("auto")
        r["tuned_cfg"] = A.autotune(m, "f64")
        r["tuned"] = timed(X, Y)
        X32, Y32 = X.float(), torch.empty(op.n, m, dtype=torch.float32, device="cuda")
        r["f32"] = timed(X32, Y32)
        best = min((v, k) for k, v in r.items() if k not in ("f32", "tuned_cfg"))
        r["best_f64_gbs"] = round(alg_bytes(op.n, op.nnz, m) / (best[0] * 1e-6) / 1e9)
        r["best_f64"] = best[1]
        r["f32_gbs"] = round(alg_bytes(op.n, op.nnz, m, sv=4, sx=4) / (r["f32"] * 1e-6) / 1e9)
        rows[m] = r
        del X, Y, X32, Y32
        torch.cuda.empty_cache()
    A.close()
    print(json.dumps({"sweep": "gspmv_f64_arithmetic", "workload": "channel%dx%dx%d" % dims, "n": op.n, "nnz": op.nnz, "us": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--f64-mode", default="auto", choices=["auto", "native", "split"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solves", action="store_true", help="skip the solve-throughput section")
    ap.add_argument("--serving-requests", type=int, default=2000, help="requests of the serving stream (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--profile", action="store_true", help="launch-only mode for ncu captures")
    ap.add_argument("--profile-size", default="half", choices=["half", "full"])
    ap.add_argument("--profile-m", default="1,8,32")
    ap.add_argument("--profile-modes", default="split,native,f32")
    ap.add_argument("--profile-share", type=int, default=-1, help="native-DFMA share (32nds) for split mode")
    ap.add_argument("--sweep", action="store_true", help="float64 arithmetic sweep (uses --profile-size/--profile-m)")
    ap.add_argument("--oracle-refs", default="default", choices=["default", "full", "none"],
                    help="oracle solutions for the error of every solve (full: also the 9.4M-row batch system)")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.sweep:
        return run_sweep(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import gen
    from paper_1711_10622_gb300 import build as ens_build

    ens_build.build()
    import paper_1711_10622_gb300 as ens

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    op = gen.channel(256, 128, 128)
    n, nnz = op.n, op.nnz
    A = ens.Matrix.from_operator(op)
    A.set_f64_mode(args.f64_mode)
    stream = torch.cuda.current_stream()
    Xs, Ys = {}, {}
    for m in M_SWEEP:
        Xs[m] = torch.from_numpy(gen.rhs_normal(n, m, 20000 + m)).to("cuda")
        Ys[m] = torch.empty_like(Xs[m])
    # launch configuration per width picked by the library's autotuner (set-up, not timed)
    tuned = {m: A.autotune(m, "f64") for m in M_SWEEP} if args.f64_mode == "auto" else {}

    def step(evs=None):
        for m in M_SWEEP:
            if evs is not None:
                evs[m][0].record(stream)
            ens.gspmv(A, Xs[m], Ys[m], stream=stream)
            if evs is not None:
                evs[m][1].record(stream)

    for _ in range(args.warmup):
        step()
    K = args.steps
    evs = [{m: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for m in M_SWEEP} for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.25)
    torch.cuda.nvtx.range_push("timed")  # the launch-list capture selects these launches
    start.record(stream)
    for k in range(K):
        step(evs[k])
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per_m_all = {m: [1e3 * e[m][0].elapsed_time(e[m][1]) for e in evs] for m in M_SWEEP}
    per_m_us = {m: statistics.fmean(v) for m, v in per_m_all.items()}
    bytes_step = sum(alg_bytes(n, nnz, m) for m in M_SWEEP)
    sec, bps = replica_throughput(dist, start.elapsed_time(end) * 1e-3, bytes_step, K)
    ms, value = sec * 1e3, bps / 1e9
    peak, peak_kind = hbm_peak()

    # Dominant kernel: the m = 32 launch (largest share of the step).
    dom_m = max(M_SWEEP, key=lambda m: per_m_us[m])
    achieved = alg_bytes(n, nnz, dom_m) / (per_m_us[dom_m] * 1e-6) / 1e9
    traffic = profiled_traffic() if dom_m == 32 else None
    roofline = {
        "bound": "hbm",
        "achieved": achieved,
        "peak": peak,
        "unit": "GB/s",
        "frac": achieved / peak,
        "traffic": traffic,
        "kernel": f"gspmv m={dom_m} FP64 ({args.f64_mode})",
        "peak_kind": peak_kind,
    }
    sweep = {
        str(m): {
            "us": per_m_us[m],
            "us_median": statistics.median(per_m_all[m]),
            "us_min": min(per_m_all[m]),
            "gbs": alg_bytes(n, nnz, m) / (per_m_us[m] * 1e-6) / 1e9,
            "frac_of_measured_peak": alg_bytes(n, nnz, m) / (per_m_us[m] * 1e-6) / 1e9 / peak,
            "alg_mb": alg_bytes(n, nnz, m) / 1e6,
            "paper_sigma_mb": paper_traffic(n, nnz, m) / 1e6,
            "gain_vs_m1": m * per_m_us[1] / per_m_us[m],
            "tuned": tuned.get(m),
        }
        for m in M_SWEEP
    }

    # End to end through the C ABI with host buffers (copies inside the timed region).
    KE = max(1, min(args.e2e_steps, K))
    hx = {m: torch.from_numpy(gen.rhs_normal(n, m, 30000 + m)).pin_memory().numpy() for m in M_SWEEP}
    hy = {m: torch.empty((n, m), dtype=torch.float64).pin_memory().numpy() for m in M_SWEEP}
    for m in M_SWEEP:  # warm the staging buffers
        ens.gspmv_host(A, hx[m], hy[m], stream=stream)
    barrier()
    e2e_ms = {m: 0.0 for m in M_SWEEP}
    e2e_steps = []
    t0 = time.perf_counter()
    for _ in range(KE):
        ts = time.perf_counter()
        for m in M_SWEEP:
            tm = time.perf_counter()
            ens.gspmv_host(A, hx[m], hy[m], stream=stream)
            e2e_ms[m] += (time.perf_counter() - tm) * 1e3 / KE
        e2e_steps.append((time.perf_counter() - ts) * 1e3)
    torch.cuda.synchronize()
    te, e2e_bps = replica_throughput(dist, time.perf_counter() - t0, bytes_step, KE)
    io_bytes = sum(8 * n * m for m in M_SWEEP)
    e2e = {
        "value": e2e_bps / 1e9,
        "unit": "GB/s",
        "h2d_bytes_per_step": io_bytes,
        "d2h_bytes_per_step": io_bytes,
        "steps": KE,
        "ms_per_m": {str(m): e2e_ms[m] for m in M_SWEEP},
        # the value above is the mean over all steps; the median step shows the pipeline's own rate
        # when a few steps are slowed by other work on the shared host
        "median_step_ms": statistics.median(e2e_steps),
        "max_step_ms": max(e2e_steps),
        "median_value": bytes_step / (statistics.median(e2e_steps) * 1e-3) / 1e9,
        "api": "ens_gspmv_host (pinned host X/Y)",
    }

    # The oracle's reference solutions (for the error of every solve result) are computed on the host
    # cores in a spawned process while the GPU sections below run. It starts only now: its
    # all-core sweeps compete with the pinned copies of the end-to-end section for host memory
    # bandwidth (a spawned process is safe to start after the first GPU call).
    refs_future, refs_pool = None, None
    if rank == 0 and not args.no_solves and args.oracle_refs != "none":
        import concurrent.futures as cf
        import multiprocessing as mp

        refs_pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        refs_future = refs_pool.submit(oracle_references, args.oracle_refs)

    # cuSPARSE SpMM on the same operator and inputs: context only, outside the timed region
    comparator = cusparse_comparator(op, Xs, per_m_us, stream) if rank == 0 else None
    if comparator is not None and "unavailable" not in comparator:
        for m in M_SWEEP:
            c = comparator.get(str(m))
            if not c or "Y" not in c:
                continue
            ens.gspmv(A, Xs[m], Ys[m], stream=stream)
            diff = ((c.pop("Y") - Ys[m]).abs() / c.pop("scale").clamp_min(1e-300)).max().item()
            c["max_rel_diff_vs_ours"] = diff
        torch.cuda.empty_cache()

    keep_solves, keep_batch, keep_serving = {}, {}, {}
    solves = None if args.no_solves else solve_metrics(keep=keep_solves)
    projection = None if args.no_solves else projection_metrics()
    cubes = None if args.no_solves else cubes_gspmv_metrics()
    batch = None if args.no_solves else batch_metrics(keep=keep_batch)
    if cubes is not None:
        for v in cubes["sweep"].values():
            v["frac_of_measured_peak"] = v["gbs"] / peak
    if projection is not None:
        ceiling = fp64_peak_ops(clocks.get("sm_mhz") if isinstance(clocks, dict) else None) / 1e9
        for k in ("divergence", "grad_correct"):
            projection[k]["fp64_frac"] = projection[k]["fp64_gops"] / ceiling
            projection[k]["hbm_frac"] = projection[k]["gbs"] / peak
        projection["fp64_ceiling_gops"] = ceiling
    serving = None if args.serving_requests <= 0 else serving_metrics(args.serving_requests, keep=keep_serving)
    from paper_1711_10622_gb300 import report

    estimate = report.estimate_table(per_m_us, n, nnz)

    oracle_refs = None
    if refs_future is not None:
        t_wait = time.perf_counter()
        refs = refs_future.result()
        refs_pool.shutdown()
        oracle_refs = {"host_seconds": refs["seconds"], "threads": refs["threads"],
                       "waited_s": time.perf_counter() - t_wait, "level": args.oracle_refs}
        if solves is not None:
            attach_oracle_errors(solves, keep_solves, refs)
        if batch is not None:
            attach_batch_errors(batch, keep_batch, refs["batch"])
        if serving is not None:
            attach_serving_errors(serving, keep_serving, refs["serving"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sweep(op)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "GB/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": ms / K,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {
                "workload": f"{WORKLOAD} GSpMV sweep m={list(M_SWEEP)}",
                "n": n,
                "nnz": nnz,
                "f64_arithmetic": args.f64_mode,
                "l2": "no flush: every launch streams >= 435 MB (> 129 MB L2)",
                "parallelism": f"{world} independent replica(s)",
            },
            "roofline": roofline,
            "sweep": sweep,
            "e2e": e2e,
            "cusparse_spmm": comparator,
            "solves": solves,
            "projection": projection,
            "cubes_gspmv": cubes,
            "batch": batch,
            "serving": serving,
            "paper_estimate": estimate,
            "cpu_baseline": cpu,
            "oracle_references": oracle_refs,
            "clocks": clocks,
            "gpu_launches": K * len(M_SWEEP),
        }
        print(json.dumps(line))
    A.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
