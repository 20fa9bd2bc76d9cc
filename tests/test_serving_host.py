"""Host logic of the serving layer (admission, batching, budget, continuous admission) with a fake
solver, on CPU threads (no GPU)."""

import threading
import time

import numpy as np
import pytest

from paper_1711_10622_gb300.serving import Request, Scheduler, Server, latency_summary


class _Op:
    def __init__(self, n):
        self.n = n
        self.nnz = 7 * n


def _fake_solver(delay, log):
    def solve(op, B, tol, stream):
        t0 = time.perf_counter()
        time.sleep(delay)
        log.append((op, B.shape[1], t0, time.perf_counter()))
        return 2.0 * B, {"iters": np.arange(B.shape[1]), "status": np.zeros(B.shape[1], dtype=np.int32)}

    return solve


def test_batches_merge_same_operator_in_arrival_order():
    s = Scheduler({"a": 100, "b": 100}, 0, 1e12, max_cols=8, precision="mixed")
    reqs = [Request("a", np.zeros((100, 3))), Request("b", np.zeros((100, 2))), Request("a", np.zeros((100, 4))), Request("a", np.zeros((100, 2)))]
    for r in reqs:
        s.queue.append(r)
    batch = s.take()
    assert [r.op for r in batch] == ["a", "a"] and sum(r.m for r in batch) == 7  # 3 + 4; the 2 would exceed 8
    assert [r.m for r in s.take()] == [2]  # b
    assert [r.m for r in s.take()] == [2]  # the last a
    assert s.take() is None


def test_budget_limits_work_in_flight():
    gamma = Scheduler({"a": 10}, 0, 1e12, 8, "mixed").gamma
    s = Scheduler({"a": 10}, 0, budget_bytes=gamma * 10 * 4, max_cols=8, precision="mixed")
    for m in (3, 3, 1):
        s.queue.append(Request("a", np.zeros((10, m))))
    b1 = s.take()
    assert sum(r.m for r in b1) == 4  # 3 + 1 fit in 4 columns' worth, the second 3 does not
    assert s.take() is None  # budget exhausted while b1 runs
    s.release(b1)
    assert sum(r.m for r in s.take()) == 3
    with pytest.raises(MemoryError):
        s.check(Request("a", np.zeros((10, 5))))


def test_continuous_admission_and_results_per_request():
    log = []
    ops = {"a": _Op(50), "b": _Op(60)}
    with Server(ops, budget_bytes=1e12, slots=2, max_cols=8, solve_fn=_fake_solver(0.2, log), device_io=False) as srv:
        r1 = srv.submit(Request("a", np.ones((50, 2))))
        time.sleep(0.05)  # r1 is running when r2 arrives
        r2 = srv.submit(Request("b", 3 * np.ones((60, 1))))
        for r in (r1, r2):
            assert r.done.wait(5)
        # r2 did not wait for r1 to finish
        assert r2.start < r1.end
        np.testing.assert_array_equal(r1.X, 2 * np.ones((50, 2)))
        np.testing.assert_array_equal(r2.X, 6 * np.ones((60, 1)))
        # queued requests for one operator are merged and split back in order
        blocker = srv.submit(Request("b", np.ones((60, 1))))
        blocker2 = srv.submit(Request("b", np.ones((60, 1))))
        rs = [srv.submit(Request("a", (k + 1) * np.ones((50, 1)))) for k in range(3)]
        for r in rs + [blocker, blocker2]:
            assert r.done.wait(5)
        for k, r in enumerate(rs):
            np.testing.assert_array_equal(r.X, 2 * (k + 1) * np.ones((50, 1)))
        assert max(r.batch_size for r in rs) >= 2
        summ = latency_summary(rs)
        assert summ["requests"] == 3 and summ["errors"] == 0 and summ["p99_ms"] >= summ["p50_ms"]


def test_solver_errors_are_reported_not_lost():
    def bad(op, B, tol, stream):
        raise RuntimeError("boom")

    with Server({"a": _Op(10)}, slots=1, solve_fn=bad, device_io=False) as srv:
        r = srv.submit(Request("a", np.ones((10, 1))))
        assert r.done.wait(5) and "boom" in r.error
