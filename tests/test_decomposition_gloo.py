"""Multi-GPU decomposition (Section 3's geometric decomposition; the ensemble split of Section 2.2)
tested on CPU ranks: real data split over world-size 2 and 3 gloo process groups, compared with the
single-process oracle.

* Partition host logic: z-slab bounds, halo lists, send lists and the renumbered row blocks; the
  local products of every rank reproduce the global product's rows exactly.
* Row split, GSpMV with halo exchange: every rank's rows equal the oracle's global product bit for
  bit (each row is summed in the same order).
* Row split, BiCGStab (unpreconditioned, per-column scalars from allreduced dots): statuses equal
  the oracle's, iterations within 25 % + 2, solutions within 1e-6 (the dots are summed in another
  order, so iterates differ by rounding), on a non-singular box and a singular channel; the exact
  breakdown inputs give the oracle's breakdowns exactly.
* Ensemble split: each rank solves its share of the columns with no communication; the gathered
  solution equals the single-process oracle solve bit for bit (columns are independent).
The device work of a rank runs in tests/dist_cpu_ops.py (oracle products, torch CPU vector ops).
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402
from gen.breakdown import breakdown_system  # noqa: E402
from paper_1711_10622_gb300 import decomposition as dc  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ----------------------------------------------------------------------------- host logic
def test_slab_bounds_follow_planes():
    assert dc.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    b = dc.slab_bounds(16 * 8 * 6, 4, plane=16 * 8)
    assert b[0][0] == 0 and b[-1][1] == 16 * 8 * 6 and all(r0 % 128 == 0 for r0, _ in b)
    assert dc.column_shares(5, 2) == [(0, 3), (3, 5)] and dc.column_shares(1, 3) == [(0, 1), (1, 1), (1, 1)]


@pytest.mark.parametrize("size", [2, 3])
def test_row_blocks_reproduce_the_global_product(size):
    op = gen.channel(16, 8, 6)  # periodic z: the first and last slab are neighbours
    bounds = dc.slab_bounds(op.n, size, plane=16 * 8)
    X = gen.rhs_normal(op.n, 3, 5)
    ref = oracle.gspmv(op, X)
    for rank in range(size):
        rb = dc.row_block(op.row_ptr, op.col_idx, op.val, bounds, rank)
        assert rb.n_loc == bounds[rank][1] - bounds[rank][0]
        assert sorted(rb.glob.tolist()) == list(range(*bounds[rank]))
        # one message per neighbour, one grid plane per neighbouring face (7-point stencil, z-slabs;
        # with two ranks and periodic z the one neighbour borders both faces)
        assert len(rb.recv) == min(2, size - 1)
        assert all(cnt == 16 * 8 * (2 if size == 2 else 1) for _, cnt in rb.recv.values())
        assert sum(c for _, c in rb.recv.values()) == rb.halo.shape[0]
        Xe = np.concatenate([X[rb.glob], X[rb.halo]])
        Yi = oracle.gspmv_csr(rb.A_int, Xe) if rb.n_int else np.zeros((0, 3))
        Yb = oracle.gspmv_csr(rb.A_bnd, Xe)
        np.testing.assert_array_equal(np.concatenate([Yi, Yb]), ref[rb.glob])
        # send lists are the neighbours' halo rows owned here
        for q, ix in rb.send.items():
            qb = dc.row_block(op.row_ptr, op.col_idx, op.val, bounds, q)
            off, cnt = qb.recv[rank]
            np.testing.assert_array_equal(rb.glob[ix], qb.halo[off : off + cnt])


# ----------------------------------------------------------------------------- gloo ranks
def _case(name):
    if name == "dirichlet":
        op = gen.dirichlet_box(12)
        return op, gen.rhs_uniform(op.n, 3, 71), 1e-9, 12 * 12
    if name == "channel":
        op = gen.channel(16, 12, 10)
        return op, gen.rhs_normal(op.n, 2, 72, zero_mean=True), 1e-9, 16 * 12
    op, B = breakdown_system(patterns=64)
    return op, B, 1e-10, None


def _rank_main(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from dist_cpu_ops import CpuOps

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = dc.TorchComm()
        ops = CpuOps()
        op, B, tol, plane = _case(case)
        bounds = dc.slab_bounds(op.n, world, plane=plane)
        rb = dc.row_block(op.row_ptr, op.col_idx, op.val, bounds, rank)
        # halo-exchange product
        X = gen.rhs_normal(op.n, B.shape[1], 90)
        D = dc.DistMatrix(rb, ops, B.shape[1])
        Xe = ops.zeros(rb.n_ext, B.shape[1])
        Xe[: rb.n_loc] = torch.from_numpy(X[rb.glob])
        Y = ops.zeros(rb.n_loc, B.shape[1])
        D.gspmv(comm, Xe, Y)
        # distributed BiCGStab
        res = dc.dist_bicgstab(comm, ops, rb, torch.from_numpy(np.ascontiguousarray(B[rb.glob])), tol, singular=op.singular)
        # ensemble split with the oracle as the per-rank solver
        Xs, _, share = dc.solve_ensemble_split(
            comm, torch.from_numpy(B), lambda Bs: (torch.from_numpy(oracle.solve_block(op, Bs.numpy(), tol)[0]), {})
        )
        q.put((rank, rb.glob, Y.numpy(), X, res.X_loc.numpy(), res.status, res.iters, res.relres, res.allreduces,
               Xs.numpy() if rank == 0 else None, None))
    except Exception as exc:  # report to the parent instead of hanging it
        q.put((rank, None, None, None, None, None, None, None, None, None, repr(exc)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(case, world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for o in out:
        assert o[-1] is None, o[-1]
    return out


@pytest.mark.parametrize("case,world", [("dirichlet", 2), ("channel", 3), ("breakdown", 2)])
def test_row_and_ensemble_split_match_the_oracle(case, world):
    op, B, tol, _ = _case(case)
    out = _run(case, world)
    n, m = B.shape
    Y = np.zeros((n, m))
    Xd = np.zeros((n, m))
    for rank, glob, Yr, X, Xr, st, it, rr, nred, Xs, _ in out:
        Y[glob] = Yr
        Xd[glob] = Xr
    np.testing.assert_array_equal(Y, oracle.gspmv(op, out[0][3]))  # halo exchange: exact rows
    Xo, it_o, rr_o, st_o = oracle.solve_block(op, B, tol)
    st, it, rr = out[0][5], out[0][6], out[0][7]
    for o in out[1:]:  # every rank holds the same per-column outcome
        np.testing.assert_array_equal(o[5], st)
        np.testing.assert_array_equal(o[6], it)
    np.testing.assert_array_equal(st, st_o)
    if case == "breakdown":
        np.testing.assert_array_equal(it[:3], it_o[:3])
        np.testing.assert_array_equal(Xd[:, :3], Xo[:, :3])
    assert np.all(np.abs(it - it_o) <= 0.25 * it_o + 2), (it, it_o)
    conv = st_o == 0
    for l in np.nonzero(conv)[0]:
        assert rr[l] <= tol * 1.05
        assert np.linalg.norm(Xd[:, l] - Xo[:, l]) <= 1e-6 * np.linalg.norm(Xo[:, l]), l
    if op.singular:
        np.testing.assert_allclose(Xd.sum(axis=0), 0.0, atol=1e-9 * np.abs(Xd).max() * n)
    # ensemble split: independent columns, identical bits to the single-process oracle solve
    np.testing.assert_array_equal(out[0][9], Xo)
