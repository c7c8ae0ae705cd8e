"""The row-block split of SP2 through the CUDA library on one GPU: ranks run as threads of
one process (their exchanges pass through host memory, so no kernel ever waits on another
rank), each with its block of rows and the halo it fetches.  The result must be the
single-GPU sp2_purify run row for row (same iterations and branches, bitwise the same D:
the block products sum in the same order as whole products) and the oracle's D (GPU)."""
import threading

import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from paper_2102_08505_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [1, 2, 3])
def test_row_block_sp2_matches_whole_run(gpu, world):
    S = gpu
    n, tau, tol = 4000, 1e-5, 1e-10
    idx, val, nnz = I.tight_binding(n, seed=11, delta=10.0)
    H = S.Ellpack.from_numpy(idx, val, nnz)
    Dw, sw = S.sp2_purify(H, n / 2, tol, S.sp2_options_default(tau=tau))
    wi, wv, wn = Dw.to_numpy()
    bounds = shard.block_bounds(n, world)
    hub = shard.LocalComm.Hub(world)
    out, errs = {}, []

    def run(rank):
        try:
            import torch
            torch.cuda.set_device(0)
            r0, r1 = bounds[rank], bounds[rank + 1]
            Hb = S.Ellpack.from_numpy(idx[r0:r1], val[r0:r1], nnz[r0:r1])
            out[rank] = shard.row_block_sp2(shard.LocalComm(hub, rank), bounds, Hb, n / 2, tol, tau,
                                            shard.GPUBlockOps())
        except Exception as e:  # reported below
            errs.append(e)
    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=600)
    assert not errs, errs
    Do, so = O.sp2(O.Ell(idx, val, nnz), n / 2, tol, tau)
    Dd = Do.to_dense()
    for rank in range(world):
        Db, st = out[rank]
        assert st["iterations"] == sw["iterations"] == so["iterations"]
        assert st["branch"] == sw["branch"] == so["branch"]
        assert st["status"] == sw["status"]
        assert np.allclose(st["trX"], sw["trX"], rtol=1e-13, atol=0) and np.allclose(st["trX2"], sw["trX2"], rtol=1e-13)
        if world > 1:
            assert sum(st["halo_rows"]) > 0
        bi, bv, bn = Db.to_numpy()
        r0 = bounds[rank]
        assert np.array_equal(bn, wn[r0:r0 + Db.n])
        for i in range(Db.n):
            k = bn[i]
            assert np.array_equal(bi[i, :k], wi[r0 + i, :k])
            assert np.array_equal(bv[i, :k].view(np.int64), wv[r0 + i, :k].view(np.int64))
            row = np.zeros(n)
            row[bi[i, :k]] = bv[i, :k]
            assert np.max(np.abs(row - Dd[r0 + i])) < 1e-10
