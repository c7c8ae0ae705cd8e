"""The row-block split of SP2 (shard.row_block_sp2) as world-size 2 and 3 gloo process
groups on the CPU, each rank purifying its block of rows with the oracle: the halo
exchange, the traces summed in rank order and the per-block products must reproduce the
single-process oracle run bit for bit (iterations, branches, traces, every row of D)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from paper_2102_08505_gb300 import shard


class OracleBlockOps:
    """Per-block operations of the row-block split done by the oracle (test
    infrastructure): the product of the block's rows is the oracle's product restricted to
    those rows of a matrix holding only the block's rows and its halo; tr X^2 is the
    diagonal of that unthresholded product, as in the oracle's SP2."""

    def __init__(self, H_full):
        self.H = H_full
        self.P = None

    def bounds(self, H_blk, r0):
        return O.gershgorin(self.H)

    def x0(self, H_blk, r0, lo, hi, tau):
        X = O.x0(self.H, lo, hi, tau)
        r1 = r0 + H_blk.n
        return O.Ell(X.idx[r0:r1], X.val[r0:r1], X.nnz[r0:r1])

    def width(self, X):
        return X.w

    def widen(self, X, w):
        if X.w >= w:
            return X
        idx = np.zeros((X.n, w), np.int32)
        val = np.full((X.n, w), np.nan)
        idx[:, :X.w] = X.idx
        val[:, :X.w] = X.val
        return O.Ell(idx, val, X.nnz)

    def arrays(self, X):
        return torch.from_numpy(X.idx), torch.from_numpy(X.val), torch.from_numpy(X.nnz)

    def halo_requests(self, X, r0, r1, bounds):
        return shard.halo_requests(X.idx, X.nnz, r0, r1, bounds)

    def extended(self, X, r0, n, halo):
        rows, hi, hv, hn = (t.numpy() for t in halo)
        B = O.Ell.empty(n, X.w)
        B.val[:] = np.nan
        B.idx[r0:r0 + X.n], B.val[r0:r0 + X.n], B.nnz[r0:r0 + X.n] = X.idx, X.val, X.nnz
        B.idx[rows], B.val[rows], B.nnz[rows] = hi, hv, hn
        return B

    def trace_parts(self, X, r0, B):
        rows = np.arange(r0, r0 + X.n, dtype=np.int32)
        self.P = O.spgemm(B, B, None, 1.0, 0.0, 0.0, rows=rows)

        def diag(E):
            out = []
            for i in range(E.n):
                c, v = E.row(i)
                hit = np.nonzero(c == r0 + i)[0]
                out += [float(v[h]) for h in hit]
            return out
        return [diag(X), diag(self.P)]

    def update(self, X, r0, B, up, tau):
        if not up:
            return O.drop(self.P, tau)
        # the oracle's add takes n x n matrices: the block's rows at their global positions
        n = B.n

        def full(E):
            F = O.Ell.empty(n, E.w)
            F.idx[r0:r0 + E.n], F.val[r0:r0 + E.n], F.nnz[r0:r0 + E.n] = E.idx, E.val, E.nnz
            return F
        S = O.add(full(self.P), full(X), -1.0, 2.0, tau)
        return O.Ell(S.idx[r0:r0 + X.n], S.val[r0:r0 + X.n], S.nnz[r0:r0 + X.n])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(name):
    if name == "banded":
        return O.Ell(*I.banded(240, band=6, seed=4, delta=10.0)), 120, 1e-4
    return O.Ell(*I.tight_binding(1200, seed=5, delta=10.0)), 600, 1e-4


def _worker(rank, world, port, name, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H, nocc, tau = _case(name)
        bounds = shard.block_bounds(H.n, world)
        r0, r1 = bounds[rank], bounds[rank + 1]
        Hb = O.Ell(H.idx[r0:r1], H.val[r0:r1], H.nnz[r0:r1])
        D, st = shard.row_block_sp2(shard.DistComm(), bounds, Hb, nocc, 1e-10, tau, OracleBlockOps(H))
        q.put((rank, D.idx, D.val, D.nnz, st))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name", [(2, "banded"), (3, "tight_binding")])
def test_row_block_sp2_matches_single_process_oracle(world, name):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    H, nocc, tau = _case(name)
    D, so = O.sp2(H, nocc, 1e-10, tau)
    bounds = shard.block_bounds(H.n, world)
    for rank, idx, val, nnz, st in res:
        assert st["iterations"] == so["iterations"]
        assert st["branch"] == so["branch"]
        assert st["status"] == so["status"]
        assert np.array_equal(np.array(st["trX"]), so["trX"])    # bitwise: traces summed in row order
        assert np.array_equal(np.array(st["trX2"]), so["trX2"])
        r0 = bounds[rank]
        for i in range(len(nnz)):
            c, v = D.row(r0 + i)
            assert np.array_equal(idx[i, :nnz[i]], c)
            assert np.array_equal(val[i, :nnz[i]].view(np.int64), v.view(np.int64))
        assert sum(st["halo_rows"]) > 0  # the blocks did exchange rows
    assert "X2" in so["branch"] and "2X-X2" in so["branch"]


def test_halo_requests_and_owners():
    bounds = shard.block_bounds(10, 3)
    assert bounds == [0, 3, 6, 10]
    assert shard.owners([0, 2, 3, 5, 6, 9], bounds).tolist() == [0, 0, 1, 1, 2, 2]
    idx = np.array([[0, 4, 9, 0], [3, 5, 7, 8]], np.int32)
    nnz = np.array([3, 2], np.int32)  # row 1 stores only 3 and 5 (7, 8 are padding)
    req = shard.halo_requests(idx, nnz, 3, 6, bounds)
    assert {k: v.tolist() for k, v in req.items()} == {0: [0], 2: [9]}
    with pytest.raises(ValueError):
        shard.block_bounds(2, 3)


def test_local_comm_ranks_as_threads_match_oracle():
    """The same driver with ranks as threads of one process (the in-memory exchange used to
    run the split on one GPU)."""
    import threading
    H, nocc, tau = _case("banded")
    world = 3
    bounds = shard.block_bounds(H.n, world)
    hub = shard.LocalComm.Hub(world)
    out, errs = {}, []

    def run(rank):
        try:
            r0, r1 = bounds[rank], bounds[rank + 1]
            Hb = O.Ell(H.idx[r0:r1], H.val[r0:r1], H.nnz[r0:r1])
            out[rank] = shard.row_block_sp2(shard.LocalComm(hub, rank), bounds, Hb, nocc, 1e-10, tau,
                                            OracleBlockOps(H))
        except Exception as e:  # reported below
            errs.append(e)
    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    D, so = O.sp2(H, nocc, 1e-10, tau)
    for rank in range(world):
        Db, st = out[rank]
        assert st["branch"] == so["branch"] and np.array_equal(np.array(st["trX2"]), so["trX2"])
        for i in range(Db.n):
            c, v = D.row(bounds[rank] + i)
            assert np.array_equal(Db.row(i)[0], c) and np.array_equal(Db.row(i)[1], v)
