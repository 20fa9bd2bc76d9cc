"""The serving layer on the GPU: continuous batching of solve requests.

A request's result is the same alone and in the mix (within the solver tolerance: residual at or
below tol, solution within 1e-6 relative of the request solved alone, checked at tol = 1e-10); work
of different requests overlaps on the device; merged requests are split back correctly (each
result's residual is recomputed by the oracle's SpMV). Solves run in caller-provided workspaces
carved from one pool, sized by the memory model M = alpha + gamma m (Section 4.2) fitted on the
device at start-up."""

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


def test_solve_in_a_caller_workspace(ens):
    """ens_solve_opts.workspace: the solve takes all its scratch from caller memory (nothing is
    allocated), gives the same bits as with stream-ordered scratch, reports the bytes it took, and a
    workspace one block too small is rejected with ENS_ERR_BUDGET."""
    from paper_1711_10622_gb300 import _native as N

    op = gen.cubes(48, 32, 24, size=4)
    B = torch.from_numpy(gen.rhs_normal(op.n, 5, 31, zero_mean=True)).cuda()
    with ens.Matrix.from_operator(op) as A:
        A.amg_setup()
        for kw in (dict(precond="chebyshev"), dict(precond="amg", precision="mixed")):
            X0, st0 = ens.solve_block(A, B, tol=1e-9, **kw)
            need = int(N.lib().ens_last_workspace_bytes())
            assert need > 5 * op.n * 8
            pool = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            X1, st1 = ens.solve_block(A, B, tol=1e-9, workspace=pool.data_ptr(), workspace_bytes=need, **kw)
            torch.cuda.synchronize()
            assert int(N.lib().ens_last_workspace_bytes()) == need
            np.testing.assert_array_equal(X1.cpu().numpy(), X0.cpu().numpy())
            np.testing.assert_array_equal(st1["iters"], st0["iters"])
            assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)  # only X's tensor, no scratch
            with pytest.raises(ens.EnsError, match="ENS_ERR_BUDGET"):
                ens.solve_block(A, B, tol=1e-9, workspace=pool.data_ptr(), workspace_bytes=need - 256, **kw)
            # the batched launch takes its scratch from the workspace too
            (Xb, stb), = ens.solve_batch([(A, B, None, 1e-9)], workspace=pool.data_ptr(), workspace_bytes=need + 4096, **kw)
            assert (stb["status"] == 0).all()


def test_memory_model_fitted_on_the_device(ens):
    """alpha from free-memory drops, beta + gamma m from the library's workspace bytes: the fit is
    linear to 1 %, gamma per row and right-hand side is the solver's per-row block count, and every
    request of a served stream ran inside the pool without a budget error."""
    from paper_1711_10622_gb300.serving import Request, Server

    ops = {"cubes": gen.cubes(48, 32, 24, size=4), "chan": gen.channel(32, 24, 16)}
    with Server(ops, budget_bytes=8e9, slots=2, max_cols=16, precond="amg") as srv:
        M = srv.model
        assert M.residual <= 0.01, M.samples
        for name, op in ops.items():
            assert M.alpha[name] >= 0 and M.gamma[name] > 0
            # mixed precision + AMG: 3 float64 and at least 8 float32 blocks per column and row
            assert 8 * 3 + 4 * 8 <= M.gamma[name] / op.n <= 8 * 3 + 4 * 30, M.gamma[name] / op.n
        reqs = [srv.submit(Request(name, gen.rhs_normal(op.n, m, 50 + m, zero_mean=True), 1e-8))
                for m in (1, 3, 8, 16) for name, op in ops.items()]
        for r in reqs:
            assert r.done.wait(300) and r.error is None, r.error
            assert (r.stats["status"] == 0).all()
            assert r.workspace_bytes == M.cost(r.op, r.batch_cols)
        assert srv.sched.pool.in_use == 0 and srv.sched.pool.peak > 0
