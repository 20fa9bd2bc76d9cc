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
* memory: the paper's per-process model M = alpha + gamma * m (Section 4.2, Tables 6/7) is applied
  to HBM: alpha = the resident matrices, gamma = the working set of one right-hand side of a solve
  (n rows times the bytes per row and column of the solver's blocks); a batch is admitted only if
  the working sets in flight plus its own stay within the budget.

Results do not depend on the mix: columns of a block solve run independent recurrences, so a
request gets the same answer alone or merged with others, within the solver tolerance (bit for bit
when the block width is the same). Latency is measured from arrival to the result being on the
host.
"""

from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

# Bytes per (row, right-hand side) of a solve's working set, by precision: internal b, x (+ r) in
# float64, the Krylov blocks (13 with Chebyshev) in float64 or float32, the caller's B and X.
WORKSET_BYTES_PER_ROW_COL = {"f64": 8 * (2 + 11) + 16, "mixed": 8 * 3 + 4 * 13 + 16}


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
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def m(self) -> int:
        return int(self.B.shape[1])

    @property
    def latency(self) -> float:
        return self.end - self.arrival


class Scheduler:
    """Admission and batching policy (host logic, no GPU): a FIFO queue, per-operator merging up to
    max_cols columns and an HBM budget on the working sets in flight."""

    def __init__(self, sizes: dict, resident_bytes: int, budget_bytes: float, max_cols: int, precision: str):
        self.sizes = sizes  # operator name -> n
        self.budget = float(budget_bytes)
        self.resident = int(resident_bytes)
        self.max_cols = int(max_cols)
        self.gamma = WORKSET_BYTES_PER_ROW_COL[precision]
        self.queue: collections.deque = collections.deque()
        self.in_flight = 0
        self.peak_in_flight = 0

    def cost(self, op: str, m: int) -> int:
        return self.gamma * self.sizes[op] * m

    def check(self, req: Request):
        if req.op not in self.sizes:
            raise KeyError(f"unknown operator {req.op!r}")
        if req.m < 1 or req.m > self.max_cols:
            raise ValueError(f"request width {req.m} outside [1, {self.max_cols}]")
        if self.resident + self.cost(req.op, req.m) > self.budget:
            raise MemoryError("request does not fit the HBM budget even alone")

    def take(self):
        """The next batch that fits, or None: the oldest request plus queued requests for the same
        operator and tolerance, in arrival order, while the width and the budget allow."""
        if not self.queue:
            return None
        head = self.queue[0]
        if self.resident + self.in_flight + self.cost(head.op, head.m) > self.budget:
            return None
        batch, cols = [head], head.m
        for r in list(self.queue)[1:]:
            if r.op == head.op and r.tol == head.tol and cols + r.m <= self.max_cols:
                if self.resident + self.in_flight + self.cost(head.op, cols + r.m) <= self.budget:
                    batch.append(r)
                    cols += r.m
        for r in batch:
            self.queue.remove(r)
        self.in_flight += self.cost(head.op, cols)
        self.peak_in_flight = max(self.peak_in_flight, self.in_flight)
        return batch

    def release(self, batch):
        self.in_flight -= self.cost(batch[0].op, sum(r.m for r in batch))


class Server:
    """Continuous-batching solve server on one GPU (see the module docstring).

    solve_fn(op_name, B_device, tol, stream) -> (X_device, stats) may replace the library call (tests
    of the host logic); by default it is paper_1711_10622_gb300.solve_block on the op's Matrix.
    precond: 'chebyshev', 'none' or 'amg' (the aggregation hierarchy of every operator is built when
    the server starts and counted in the resident memory).
    """

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
    ):
        self.precision, self.precond = precision, precond
        self.device_io = device_io
        self.mats = {}
        resident = 0
        if solve_fn is None:
            from .api import Matrix

            for name, op in operators.items():
                A = Matrix.from_operator(op)
                self.mats[name] = A
                levels = A.amg_setup() if precond == "amg" else [(op.n, op.nnz)]
                # matrix copies held by the library per level (the fine one and, with AMG, the coarse
                # ones): row_ptr, col, f64/f32/split values, inverse diagonals, aggregate maps
                for k, (n_l, nnz_l) in enumerate(levels):
                    copies = 2 if precond == "amg" and k < len(levels) - 1 else 1  # smoothed levels: + A D^-1
                    resident += copies * (4 * (n_l + 1) + nnz_l * (4 + 8 + 4 + 8) + 12 * n_l) + (8 * n_l if precond == "amg" else 0)
        self.solve_fn = solve_fn or self._library_solve
        self.sched = Scheduler({k: op.n for k, op in operators.items()}, resident, budget_bytes, max_cols, precision)
        self.cv = threading.Condition()
        self.stopping = False
        self.next_id = 0
        self.completed = []
        self.workers = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(slots)]
        for w in self.workers:
            w.start()

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
        """Finish every queued request, then stop the workers and free the matrices."""
        with self.cv:
            self.stopping = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()
        for A in self.mats.values():
            A.close()
        self.mats = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ workers
    def _library_solve(self, op, B, tol, stream):
        from .api import solve_block

        return solve_block(self.mats[op], B, None, tol=tol, precond=self.precond, precision=self.precision, stream=stream)

    def _worker(self, slot: int):
        stream = None
        if self.device_io:
            import torch

            stream = torch.cuda.Stream()
        while True:
            with self.cv:
                while True:
                    batch = self.sched.take()
                    if batch is not None:
                        break
                    if self.stopping and not self.sched.queue:
                        return  # drained
                    self.cv.wait()
            try:
                self._run(batch, stream)
            except Exception as exc:  # report, never lose a request
                for r in batch:
                    r.error = repr(exc)
            finally:
                with self.cv:
                    self.sched.release(batch)
                    now = time.perf_counter()
                    for r in batch:
                        r.end = now
                        r.batch_size = len(batch)
                        self.completed.append(r)
                        r.done.set()
                    self.cv.notify_all()

    def _run(self, batch, stream):
        t0 = time.perf_counter()
        for r in batch:
            r.start = t0
        Bh = np.ascontiguousarray(np.concatenate([r.B for r in batch], axis=1)) if len(batch) > 1 else np.ascontiguousarray(batch[0].B)
        if self.device_io:
            import torch

            with torch.cuda.stream(stream):
                Bd = torch.from_numpy(Bh).to("cuda", non_blocking=False)
                X, st = self.solve_fn(batch[0].op, Bd, batch[0].tol, stream)
                Xh = X.cpu().numpy()
        else:
            X, st = self.solve_fn(batch[0].op, Bh, batch[0].tol, stream)
            Xh = np.asarray(X)
        c = 0
        for r in batch:
            r.X = Xh[:, c : c + r.m].copy()
            r.stats = {k: np.asarray(v)[c : c + r.m].copy() for k, v in st.items()}
            c += r.m


def latency_summary(reqs) -> dict:
    lat = np.array([r.latency for r in reqs])
    cols = sum(r.m for r in reqs)
    span = max(r.end for r in reqs) - min(r.arrival for r in reqs)
    return {
        "requests": len(reqs),
        "rhs": cols,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "rhs_solves_per_s": cols / span,
        "requests_per_s": len(reqs) / span,
        "mean_batch_requests": float(np.mean([r.batch_size for r in reqs])),
        "errors": sum(1 for r in reqs if r.error),
    }
