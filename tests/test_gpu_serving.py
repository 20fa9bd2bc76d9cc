"""The serving layer on the GPU: continuous batching of solve requests.

A request's result is the same alone and in the mix (within the solver tolerance: residual at or
below tol, solution within 1e-6 relative of the request solved alone, checked at tol = 1e-10); work
of different requests overlaps on the device; merged requests are split back correctly (each
result's residual is recomputed by the oracle's SpMV)."""

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ens():
    from paper_1711_10622_gb300 import build

    build.build()
    import paper_1711_10622_gb300 as ens

    return ens


@pytest.mark.parametrize("precond", ["chebyshev", "amg"])
def test_alone_vs_in_the_mix_with_overlap(ens, precond):
    from paper_1711_10622_gb300.serving import Request, Server, latency_summary

    ops = {"cubes": gen.cubes(48, 32, 24, size=4), "chan": gen.channel(32, 24, 16), "box": gen.dirichlet_box(16)}
    tol = 1e-10

    def rhs(name, m, seed):
        return gen.rhs_normal(ops[name].n, m, seed, zero_mean=ops[name].singular)

    target = rhs("cubes", 3, 1)
    with Server(ops, budget_bytes=16e9, slots=3, max_cols=16, precond=precond) as srv:
        alone = srv.submit(Request("cubes", target.copy(), tol))
        assert alone.done.wait(120) and alone.error is None
        mix = [
            Request("chan", rhs("chan", 4, 2), tol),
            Request("cubes", rhs("cubes", 2, 3), tol),
            Request("cubes", target.copy(), tol),
            Request("box", rhs("box", 8, 4), tol),
            Request("cubes", rhs("cubes", 5, 5), tol),
            Request("chan", rhs("chan", 1, 6), tol),
            Request("box", rhs("box", 2, 7), tol),
        ]
        for r in mix:
            srv.submit(r)
        for r in mix:
            assert r.done.wait(300) and r.error is None, r.error
    same = mix[2]
    for l in range(3):
        assert np.linalg.norm(same.X[:, l] - alone.X[:, l]) <= 1e-6 * np.linalg.norm(alone.X[:, l])
    for r in [alone] + mix:
        assert (r.stats["status"] == 0).all() and np.all(r.stats["relres"] <= 1.05 * tol)
        R = r.B - oracle.gspmv(ops[r.op], r.X)
        assert np.all(np.linalg.norm(R, axis=0) <= 1.05 * tol * np.linalg.norm(r.B, axis=0))
    # merged: the three cube requests queued together share at least one block solve
    assert max(r.batch_size for r in mix if r.op == "cubes") >= 2
    # overlapped: some two requests were on the GPU at the same time
    iv = sorted((r.start, r.end) for r in mix)
    assert any(iv[k + 1][0] < iv[k][1] for k in range(len(iv) - 1))
    s = latency_summary(mix)
    assert s["errors"] == 0 and s["p99_ms"] >= s["p50_ms"] > 0
