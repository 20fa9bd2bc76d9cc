"""Host logic of the serving layer (memory-model fit, pool allocator, admission, batching,
continuous admission) with a fake solver, on CPU threads (no GPU)."""

import time

import numpy as np
import pytest

from paper_1711_10622_gb300.serving import MemoryModel, PoolAllocator, Request, Scheduler, Server, fit_linear, latency_summary


class _Op:
    def __init__(self, n):
        self.n = n
        self.nnz = 7 * n


def _model(rows, gamma_per_row=100, beta=1 << 20, alpha=1 << 24):
    return MemoryModel(alpha={k: alpha for k in rows}, beta={k: beta for k in rows},
                       gamma={k: gamma_per_row * n for k, n in rows.items()}, rows=dict(rows))


def _fake_solver(delay, log):
    def solve(op, B, tol, stream, workspace):
        t0 = time.perf_counter()
        time.sleep(delay)
        log.append((op, B.shape[1], t0, time.perf_counter(), workspace))
        return 2.0 * B, {"iters": np.arange(B.shape[1]), "status": np.zeros(B.shape[1], dtype=np.int32)}

    return solve


def test_fit_recovers_a_planted_linear_model():
    rng = np.random.default_rng(3)
    for _ in range(20):
        beta, gamma = float(rng.integers(1, 1 << 30)), float(rng.integers(1, 1 << 26))
        ms = [1, 4, 16, 32]
        b, g, res = fit_linear(ms, [beta + gamma * m for m in ms])
        assert abs(b - beta) <= 1e-6 * (beta + gamma) and abs(g - gamma) <= 1e-9 * gamma and res <= 1e-12
    # the model fits in the padded width: odd m costs what m + 1 costs
    rows = {"a": 1000}
    M = MemoryModel.fit({"a": 5}, rows, {"a": [(1, 1000 + 10**6 * 1), (4, 1000 + 10**6 * 4), (16, 1000 + 10**6 * 16)]})
    assert M.cost("a", 3) == M.cost("a", 4) > M.cost("a", 2)
    assert M.cost("a", 4) >= 1000 + 4 * 10**6 and M.resident == 5 and M.fit_residual_ok(1e-9)


def test_pool_allocator_first_fit_and_merging():
    P = PoolAllocator(10 * 256)
    a, b, c = P.alloc(256), P.alloc(300), P.alloc(256)  # 300 rounds up to 512
    assert (a, b, c) == (0, 256, 768) and P.in_use == 1024 and P.peak == 1024
    assert P.alloc(7 * 256) is None and P.largest_free() == 6 * 256
    P.free(b)
    assert P.alloc(512) == 256  # first fit reuses the hole
    P.free(256)
    P.free(a)
    P.free(c)
    assert P.free_list == [(0, 10 * 256)] and P.in_use == 0 and P.peak == 1024


def test_batches_merge_same_operator_in_arrival_order():
    rows = {"a": 100, "b": 100}
    s = Scheduler(_model(rows), pool_bytes=1 << 40, max_cols=8)
    reqs = [Request("a", np.zeros((100, 3))), Request("b", np.zeros((100, 2))), Request("a", np.zeros((100, 4))), Request("a", np.zeros((100, 2)))]
    for r in reqs:
        s.queue.append(r)
    batch, off, nbytes = s.take()
    assert [r.op for r in batch] == ["a", "a"] and sum(r.m for r in batch) == 7  # 3 + 4; the 2 would exceed 8
    assert nbytes == s.model.cost("a", 7)
    assert [r.m for r in s.take()[0]] == [2]  # b
    assert [r.m for r in s.take()[0]] == [2]  # the last a
    assert s.take() is None


def test_budget_limits_work_in_flight():
    rows = {"a": 10}
    M = _model(rows, gamma_per_row=1 << 16, beta=0)
    s = Scheduler(M, pool_bytes=M.cost("a", 4) + 256, max_cols=8)
    for m in (3, 3, 1):
        s.queue.append(Request("a", np.zeros((10, m))))
    b1, off1, _ = s.take()
    assert [r.m for r in b1] == [3, 1]  # the second 3 would need a 6-column workspace
    assert s.take() is None  # the rest of the pool cannot hold a 3-column solve (padded to 4)
    s.release(off1)
    b2, off2, _ = s.take()
    assert sum(r.m for r in b2) == 3
    with pytest.raises(MemoryError):
        Scheduler(M, pool_bytes=M.cost("a", 2), max_cols=8).check(Request("a", np.zeros((10, 5))))


def test_continuous_admission_and_results_per_request():
    log = []
    ops = {"a": _Op(50), "b": _Op(60)}
    M = _model({"a": 50, "b": 60})
    with Server(ops, budget_bytes=1e12, slots=2, max_cols=8, solve_fn=_fake_solver(0.2, log), device_io=False, model=M) as srv:
        r1 = srv.submit(Request("a", np.ones((50, 2))))
        time.sleep(0.05)  # r1 is running when r2 arrives
        r2 = srv.submit(Request("b", 3 * np.ones((60, 1))))
        for r in (r1, r2):
            assert r.done.wait(5)
        # r2 did not wait for r1 to finish
        assert r2.start < r1.end
        np.testing.assert_array_equal(r1.X, 2 * np.ones((50, 2)))
        np.testing.assert_array_equal(r2.X, 6 * np.ones((60, 1)))
        # every solve got its own piece of the pool, of the model's size
        assert all(ws[1] == M.cost(op, m) for op, m, _, _, ws in log)
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
        assert summ["merged_fraction"] > 0 and sum(summ["batch_cols_hist"].values()) == 3
        assert abs(summ["wait_p50_ms"] + summ["service_p50_ms"] - summ["p50_ms"]) < 250
    assert srv.sched.pool.in_use == 0


def test_solver_errors_are_reported_not_lost():
    def bad(op, B, tol, stream, workspace):
        raise RuntimeError("boom")

    with Server({"a": _Op(10)}, slots=1, solve_fn=bad, device_io=False, model=_model({"a": 10})) as srv:
        r = srv.submit(Request("a", np.ones((10, 1))))
        assert r.done.wait(5) and "boom" in r.error
