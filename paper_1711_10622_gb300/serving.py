"""Serving: continuous batching of pressure-Poisson solve requests on one GPU.

A request is a block of m right-hand sides for one of the server's operators (Section 2.2: every
realization's pressure solve shares the matrix, only the right-hand side differs). The server
keeps every matrix resident, admits requests as they arrive and runs them in concurrent slots
(one CUDA stream and one host worker each):

* continuous admission: a request that arrives while others run starts as soon as a slot and
  enough memory are free; it does not wait for the running work to finish;
* batching: when a slot takes work it merges the oldest queued request with other queued requests
  for the same operator and tolerance into one block solve of up to `max_cols` columns (one GSpMV
  per iteration serves all of them), then splits the result per request;
* memory: the paper's per-process model M = alpha + gamma m (Section 4.2, Tables 6/7), fitted on the
  device when the server starts. alpha(op) = the device memory its matrix (and its multigrid
  hierarchy) holds, measured as the drop of free device memory when it is created; a solve of m
  columns takes beta(op) + gamma(op) m bytes of workspace, fitted by least squares to the bytes the
  library reports for probe solves at several m (ens_last_workspace_bytes). The whole budget minus
  the alphas is reserved ONCE as a device pool; every batch runs in a piece of it (the solver's
  Krylov state lives there, nothing is allocated per request) and is admitted only when the
  model's bytes for it can be placed in the pool.

Results do not depend on the mix: columns of a block solve run independent recurrences, so a
request gets the same answer alone or merged with others, within the solver tolerance (bit for bit
when the block width is the same). Latency is measured from arrival to the result being on the
host; each request also records its queue wait and its service time.
"""

from __future__ import annotations

import bisect
import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

ALIGN = 256


@dataclass(eq=False)
class Request:
    op: str
    B: np.ndarray  # host, (n, m) float64
    tol: float = 1e-8
    rid: int = -1
    arrival: float = 0.0
    start: float = 0.0
    end: float = 0.0
    X: np.ndarray | None = None
    stats: dict | None = None
    error: str | None = None
    batch_size: int = 0
    batch_cols: int = 0
    workspace_bytes: int = 0
    keep_x: bool = True  # False: the solution is not kept on the host (stats only; long streams)
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def m(self) -> int:
        return int(self.B.shape[1])

    @property
    def latency(self) -> float:
        return self.end - self.arrival


# ----------------------------------------------------------------------------- memory model
def fit_linear(ms, sizes):
    """Least-squares fit sizes ~ beta + gamma m; returns (beta, gamma, max relative residual)."""
    ms = np.asarray(ms, dtype=np.float64)
    y = np.asarray(sizes, dtype=np.float64)
    A = np.stack([np.ones_like(ms), ms], axis=1)
    (beta, gamma), *_ = np.linalg.lstsq(A, y, rcond=None)
    pred = beta + gamma * ms
    res = float(np.max(np.abs(pred - y) / np.maximum(y, 1.0))) if y.size else 0.0
    return float(beta), float(gamma), res


@dataclass
class MemoryModel:
    """M(op, m) = alpha[op] (resident) + beta[op] + gamma[op] m (one solve's workspace)."""

    alpha: dict
    beta: dict
    gamma: dict
    rows: dict  # op -> n
    residual: float = 0.0
    samples: dict = field(default_factory=dict)  # op -> [(m, bytes)]

    @staticmethod
    def width(m: int) -> int:
        """The solver's internal block width: m rounded up to even (m = 1 stays 1)."""
        return m if m == 1 else (m + 1) // 2 * 2

    def cost(self, op: str, m: int) -> int:
        """Workspace bytes admitted for a solve of m columns: the fit at the padded width, with 1 %
        plus 64 KiB of headroom for the 256-byte rounding of every block."""
        c = self.beta[op] + self.gamma[op] * self.width(m)
        return int((c * 1.01 + 65536 + ALIGN - 1) // ALIGN * ALIGN)

    @property
    def resident(self) -> int:
        return int(sum(self.alpha.values()))

    def fit_residual_ok(self, tol: float = 0.01) -> bool:
        return self.residual <= tol

    def gamma_per_row_col(self) -> float:
        """gamma / n averaged over the operators: bytes per row and right-hand side."""
        return float(np.mean([self.gamma[o] / self.rows[o] for o in self.gamma]))

    def summary(self) -> dict:
        return {
            "alpha_gb": {o: a / 1e9 for o, a in self.alpha.items()},
            "beta_mb": {o: b / 1e6 for o, b in self.beta.items()},
            "gamma_mb_per_rhs": {o: g / 1e6 for o, g in self.gamma.items()},
            "gamma_bytes_per_row_rhs": self.gamma_per_row_col(),
            "fit_max_rel_residual": self.residual,
        }

    @classmethod
    def fit(cls, alpha: dict, rows: dict, samples: dict):
        """samples: op -> [(m, workspace bytes)]; the line is fitted in the padded width."""
        beta, gamma, res = {}, {}, 0.0
        for op, pts in samples.items():
            b, g, r = fit_linear([cls.width(p[0]) for p in pts], [p[1] for p in pts])
            beta[op], gamma[op], res = b, g, max(res, r)
        return cls(dict(alpha), beta, gamma, dict(rows), res, {k: list(v) for k, v in samples.items()})


class PoolAllocator:
    """First-fit allocator of byte ranges [0, size) with ALIGN-byte offsets (host bookkeeping of the
    device pool)."""

    def __init__(self, size: int):
        self.size = int(size) // ALIGN * ALIGN
        self.free_list = [(0, self.size)] if self.size > 0 else []  # sorted (offset, length)
        self.used = {}
        self.in_use = 0
        self.peak = 0

    def alloc(self, nbytes: int):
        need = (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN
        for k, (off, ln) in enumerate(self.free_list):
            if ln >= need:
                if ln == need:
                    self.free_list.pop(k)
                else:
                    self.free_list[k] = (off + need, ln - need)
                self.used[off] = need
                self.in_use += need
                self.peak = max(self.peak, self.in_use)
                return off
        return None

    def free(self, off: int):
        ln = self.used.pop(off)
        self.in_use -= ln
        k = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(k, (off, ln))
        # merge with the neighbours
        if k + 1 < len(self.free_list) and off + ln == self.free_list[k + 1][0]:
            self.free_list[k] = (off, ln + self.free_list[k + 1][1])
            self.free_list.pop(k + 1)
        if k > 0 and self.free_list[k - 1][0] + self.free_list[k - 1][1] == self.free_list[k][0]:
            self.free_list[k - 1] = (self.free_list[k - 1][0], self.free_list[k - 1][1] + self.free_list[k][1])
            self.free_list.pop(k)

    def largest_free(self) -> int:
        return max((ln for _, ln in self.free_list), default=0)


class Scheduler:
    """Admission and batching policy (host logic, no GPU): a FIFO queue, per-operator merging up to
    max_cols columns, and a batch is admitted only when the memory model's bytes for it can be
    placed in the pool."""

    def __init__(self, model: MemoryModel, pool_bytes: int, max_cols: int):
        self.model = model
        self.max_cols = int(max_cols)
        self.pool = PoolAllocator(pool_bytes)
        self.queue: collections.deque = collections.deque()

    @property
    def resident(self) -> int:
        return self.model.resident

    @property
    def peak_in_flight(self) -> int:
        return self.pool.peak

    def reset_peak(self):
        self.pool.peak = self.pool.in_use

    def check(self, req: Request):
        if req.op not in self.model.rows:
            raise KeyError(f"unknown operator {req.op!r}")
        if req.m < 1 or req.m > self.max_cols:
            raise ValueError(f"request width {req.m} outside [1, {self.max_cols}]")
        if self.model.cost(req.op, req.m) > self.pool.size:
            raise MemoryError("request does not fit the HBM budget even alone")

    def take(self):
        """(batch, offset, bytes) for the next batch that fits, or None: the oldest request plus, in
        arrival order, every queued request for the same operator and tolerance that keeps the batch
        within max_cols columns and its workspace within the largest free piece of the pool."""
        if not self.queue:
            return None
        head = self.queue[0]
        room = self.pool.largest_free()
        if self.model.cost(head.op, head.m) > room:
            return None  # first in, first out: nothing overtakes a request that is waiting for memory
        batch, cols = [head], head.m
        for r in list(self.queue)[1:]:
            if (r.op == head.op and r.tol == head.tol and cols + r.m <= self.max_cols
                    and self.model.cost(head.op, cols + r.m) <= room):
                batch.append(r)
                cols += r.m
        nbytes = self.model.cost(head.op, cols)
        off = self.pool.alloc(nbytes)  # first fit succeeds: nbytes <= the largest free piece
        for r in batch:
            self.queue.remove(r)
        return batch, off, nbytes

    def release(self, off: int):
        self.pool.free(off)


class Server:
    """Continuous-batching solve server on one GPU (see the module docstring).

    solve_fn(op_name, B_device, tol, stream, workspace) -> (X_device, stats) may replace the library
    call (tests of the host logic; workspace = (device pointer or None, bytes)); then `model` must be
    given. By default the library's solve_block runs on the op's Matrix with the batch's workspace.
    precond: 'chebyshev', 'none' or 'amg' (the aggregation hierarchy of every operator is built when
    the server starts and counted in its alpha).
    """

    PROBE_WIDTHS = (1, 4, 16, 32)

    def __init__(
        self,
        operators: dict,
        budget_bytes: float = 120e9,
        slots: int = 4,
        max_cols: int = 32,
        precision: str = "mixed",
        precond: str = "chebyshev",
        solve_fn=None,
        device_io: bool = True,
        model: MemoryModel | None = None,
    ):
        self.precision, self.precond = precision, precond
        self.device_io = device_io
        self.mats = {}
        self.pool_tensor = None
        self.pool_ptr = None
        self.budget = float(budget_bytes)
        if solve_fn is None:
            model = self._measure(operators, max_cols) if model is None else model
            pool_bytes = self._reserve_pool(model)
        else:
            if model is None:
                raise ValueError("a custom solve_fn needs an explicit memory model")
            pool_bytes = int(self.budget - model.resident)
        self.model = model
        self.solve_fn = solve_fn or self._library_solve
        self.sched = Scheduler(model, pool_bytes, max_cols)
        self.cv = threading.Condition()
        self.stopping = False
        self.next_id = 0
        self.completed = []
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for w in self.workers:
            w.start()

    # ------------------------------------------------------------------ start-up measurements
    def _measure(self, operators, max_cols) -> MemoryModel:
        """alpha per operator from free device memory before and after creating its matrix (and
        hierarchy); beta, gamma per operator from the workspace bytes of probe solves."""
        import torch

        from .api import Matrix, solve_block
        from . import _native as N

        alpha, rows, samples = {}, {}, {}
        for name, op in operators.items():
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            A = Matrix.from_operator(op)
            if self.precond == "amg":
                A.amg_setup()
            torch.cuda.synchronize()
            alpha[name] = max(0, free0 - torch.cuda.mem_get_info()[0])
            self.mats[name] = A
            rows[name] = op.n
            pts = []
            for m in sorted({w for w in self.PROBE_WIDTHS if w <= max_cols} | {max_cols}):
                B = torch.zeros((op.n, m), dtype=torch.float64, device="cuda")
                # b = 0: every column finishes at the start; the call still sets up its full workspace
                solve_block(A, B, None, tol=1e-8, precond=self.precond, precision=self.precision, max_iter=1,
                            max_outer=1, inner_max_iter=0)
                pts.append((m, int(N.lib().ens_last_workspace_bytes())))
                del B
            samples[name] = pts
        torch.cuda.empty_cache()
        return MemoryModel.fit(alpha, rows, samples)

    def _reserve_pool(self, model: MemoryModel) -> int:
        import torch

        want = int(self.budget - model.resident)
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        # leave room for the per-request B/X copies (torch's caching allocator) and the graphs
        room = 4 << 30
        size = max(0, min(want, free - room)) // ALIGN * ALIGN
        if size <= 0:
            raise MemoryError("no device memory left for the solve pool")
        self.pool_tensor = torch.empty(size, dtype=torch.uint8, device="cuda")
        self.pool_ptr = self.pool_tensor.data_ptr()
        return size

    # ------------------------------------------------------------------ client side
    def submit(self, req: Request) -> Request:
        self.sched.check(req)
        with self.cv:
            req.rid = self.next_id
            self.next_id += 1
            req.arrival = time.perf_counter()
            self.sched.queue.append(req)
            self.cv.notify_all()
        return req

    def close(self):
        """Finish every queued request, then stop the workers and free the matrices and the pool."""
        with self.cv:
            self.stopping = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()
        for A in self.mats.values():
            A.close()
        self.mats = {}
        self.pool_tensor = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ workers
    def _library_solve(self, op, B, tol, stream, workspace):
        from .api import solve_block

        ptr, nbytes = workspace
        return solve_block(self.mats[op], B, None, tol=tol, precond=self.precond, precision=self.precision, stream=stream,
                           workspace=ptr, workspace_bytes=nbytes)

    def _worker(self, slot: int):
        stream = None
        if self.device_io:
            import torch

            stream = torch.cuda.Stream()
        while True:
            with self.cv:
                while True:
                    got = self.sched.take()
                    if got is not None:
                        break
                    if self.stopping and not self.sched.queue:
                        return  # drained
                    self.cv.wait()
            batch, off, nbytes = got
            try:
                self._run(batch, stream, off, nbytes)
            except Exception as exc:  # report, never lose a request
                for r in batch:
                    r.error = repr(exc)
            finally:
                with self.cv:
                    self.sched.release(off)
                    now = time.perf_counter()
                    cols = sum(r.m for r in batch)
                    for r in batch:
                        r.end = now
                        r.batch_size = len(batch)
                        r.batch_cols = cols
                        r.workspace_bytes = nbytes
                        self.completed.append(r)
                        r.done.set()
                    self.cv.notify_all()

    def _run(self, batch, stream, off, nbytes):
        t0 = time.perf_counter()
        for r in batch:
            r.start = t0
        Bh = np.ascontiguousarray(np.concatenate([r.B for r in batch], axis=1)) if len(batch) > 1 else np.ascontiguousarray(batch[0].B)
        ws = (None if self.pool_ptr is None else self.pool_ptr + off, nbytes)
        if self.device_io:
            import torch

            with torch.cuda.stream(stream):
                Bd = torch.from_numpy(Bh).to("cuda", non_blocking=False)
                X, st = self.solve_fn(batch[0].op, Bd, batch[0].tol, stream, ws)
                Xh = X.cpu().numpy()
        else:
            X, st = self.solve_fn(batch[0].op, Bh, batch[0].tol, stream, ws)
            Xh = np.asarray(X)
        c = 0
        for r in batch:
            r.X = Xh[:, c : c + r.m].copy() if r.keep_x else None
            r.stats = {k: np.asarray(v)[c : c + r.m].copy() for k, v in st.items()}
            c += r.m


def latency_summary(reqs) -> dict:
    """Latency percentiles, throughput, the split of latency into queue wait and service, and how
    often requests were merged."""
    lat = np.array([r.latency for r in reqs])
    wait = np.array([r.start - r.arrival for r in reqs])
    service = np.array([r.end - r.start for r in reqs])
    cols = sum(r.m for r in reqs)
    span = max(r.end for r in reqs) - min(r.arrival for r in reqs)
    k99 = int(np.argsort(lat)[min(len(lat) - 1, int(np.ceil(0.99 * len(lat))) - 1)])
    tail = reqs[k99]
    widths = collections.Counter(int(r.batch_cols) for r in reqs)
    return {
        "requests": len(reqs),
        "rhs": cols,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "wait_p50_ms": float(np.percentile(wait, 50) * 1e3),
        "wait_p99_ms": float(np.percentile(wait, 99) * 1e3),
        "service_p50_ms": float(np.percentile(service, 50) * 1e3),
        "service_p99_ms": float(np.percentile(service, 99) * 1e3),
        "p99_request": {"op": tail.op, "m": tail.m, "wait_ms": (tail.start - tail.arrival) * 1e3,
                        "service_ms": (tail.end - tail.start) * 1e3, "batch_cols": int(tail.batch_cols)},
        "rhs_solves_per_s": cols / span,
        "requests_per_s": len(reqs) / span,
        "mean_batch_requests": float(np.mean([r.batch_size for r in reqs])),
        "merged_fraction": float(np.mean([r.batch_size > 1 for r in reqs])),
        "batch_cols_hist": {str(k): v for k, v in sorted(widths.items())},
        "errors": sum(1 for r in reqs if r.error),
    }
