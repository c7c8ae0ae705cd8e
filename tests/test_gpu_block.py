"""The row-block product (ellpack_multiply_block) behind the row-block split of SP2 across
GPUs, on one GPU: each block of rows, multiplied against a B that holds only the rows the
block names (its own rows and the halo), is bitwise the same rows of the whole product,
its trace and squared-norm shares sum to the whole product's, and the oracle agrees
element by element (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_spgemm

pytestmark = pytest.mark.gpu


def x_of_tight_binding(n, seed, tau):
    H = O.Ell(*I.tight_binding(n, seed=seed, delta=10.0))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, tau)
    return O.spgemm(X0, X0, None, 1.0, 0.0, tau)


def rows_of(E, r0, r1, width=None):
    w = E.w if width is None else width
    idx = np.zeros((r1 - r0, w), np.int32)
    val = np.full((r1 - r0, w), np.nan)
    idx[:, :E.w] = E.idx[r0:r1]
    val[:, :E.w] = E.val[r0:r1]
    return O.Ell(idx, val, E.nnz[r0:r1].copy())


def dev(S, E, dt, width=None):
    """E on the GPU (padded to `width` columns: index 0, value NaN)."""
    w = E.w if width is None else width
    idx = np.zeros((E.n, w), np.int32)
    val = np.full((E.n, w), np.nan)
    idx[:, :E.w] = E.idx
    val[:, :E.w] = E.val
    return S.Ellpack.from_numpy(idx, val, E.nnz, dt)


def halo_only(E, r0, r1):
    """E with every row emptied except the block's rows and the rows they name."""
    need = set(range(r0, r1))
    for i in range(r0, r1):
        need.update(int(k) for k in E.row(i)[0])
    keep = np.zeros(E.n, bool)
    keep[sorted(need)] = True
    idx = np.where(keep[:, None], E.idx, 0).astype(np.int32)
    val = np.where(keep[:, None], E.val, np.nan)
    return O.Ell(idx, val, np.where(keep, E.nnz, 0).astype(np.int32)), int(keep.sum())


@pytest.mark.parametrize("ab", [(1.0, 0.0), (-1.0, 2.0)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_blocks_are_rows_of_the_whole_product(gpu, ab, dtype):
    S = gpu
    alpha, beta = ab
    n, tau = 6000, 1e-5
    X = x_of_tight_binding(n, 7, tau)
    if dtype == "f32":
        X = O.Ell(X.idx, X.val.astype(np.float32).astype(np.float64), X.nnz)
    dt = S.SP2_F64 if dtype == "f64" else S.SP2_F32
    ref = O.spgemm(X, X, X if beta else None, alpha, beta, tau)
    w = ((int(ref.nnz.max()) + 31) // 32) * 32
    dX = dev(S, X, dt)
    whole = dev(S, X, dt, width=w)  # the addend, overwritten by the product
    S.ellpack_multiply(dX, dX, whole, alpha, beta, tau)
    tr_whole = S.ellpack_trace(whole)
    fro_whole = S.ellpack_frobenius2(whole)
    gi, gv, gn = whole.to_numpy()
    bounds = [0, 1700, 1701, 4100, n]  # ragged blocks, one of a single row
    tr_sum = fro_sum = 0.0
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        Bh, kept = halo_only(X, r0, r1)
        assert kept < n  # the block sees only its rows and its halo
        dA = dev(S, rows_of(X, r0, r1), dt)
        dB = dev(S, Bh, dt)
        dC = dev(S, rows_of(X, r0, r1), dt) if beta else None
        out = S.Ellpack.empty(r1 - r0, w, dt)
        _, req, tr, fro = S.ellpack_multiply_block(dA, r0, dB, dC, out, alpha, beta, tau)
        bi, bv, bn = out.to_numpy()
        assert np.array_equal(bn, gn[r0:r1])
        for i in range(r1 - r0):
            k = bn[i]
            assert np.array_equal(bi[i, :k], gi[r0 + i, :k])
            assert np.array_equal(bv[i, :k].view(np.int64 if dtype == "f64" else np.int32),
                                  gv[r0 + i, :k].view(np.int64 if dtype == "f64" else np.int32))
        tr_sum += tr
        fro_sum += fro
    assert tr_sum == pytest.approx(tr_whole, rel=1e-13, abs=1e-13)
    assert fro_sum == pytest.approx(fro_whole, rel=1e-13)
    compare_spgemm((gi, gv, gn), X, X, X if beta else None, alpha, beta, tau, fp32=dtype == "f32",
                   rows=np.arange(0, n, 7))


def test_block_overflow_reports_width(gpu):
    S = gpu
    n, tau = 3000, 1e-5
    X = x_of_tight_binding(n, 8, tau)
    r0, r1 = 1000, 2000
    Bh, _ = halo_only(X, r0, r1)
    dA = dev(S, rows_of(X, r0, r1), S.SP2_F64)
    dB = dev(S, Bh, S.SP2_F64)
    small = S.Ellpack.empty(r1 - r0, 32)
    rc, req, _, _ = S.ellpack_multiply_block(dA, r0, dB, None, small, 1.0, 0.0, tau, raise_on_overflow=False)
    ref = O.spgemm(X, X, None, 1.0, 0.0, tau, rows=np.arange(r0, r1))
    assert rc == S.SP2E_OVERFLOW and req == int(ref.nnz.max())


def test_block_argument_checks(gpu):
    S = gpu
    X = x_of_tight_binding(500, 9, 1e-5)
    dX = dev(S, X, S.SP2_F64)
    blk = dev(S, rows_of(X, 400, 500), S.SP2_F64)
    out = S.Ellpack.empty(100, 256)
    for bad_row0 in (-1, 401):  # rows outside B
        with pytest.raises(S.Sp2Error) as e:
            S.ellpack_multiply_block(blk, bad_row0, dX, None, out, 1.0, 0.0, 1e-5)
        assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:  # beta != 0 needs the addend rows
        S.ellpack_multiply_block(blk, 400, dX, None, out, -1.0, 2.0, 1e-5)
    assert e.value.code == S.SP2E_ARG


def test_halo_rows_match_the_pattern(gpu):
    """ellpack_halo_rows: the distinct columns a block's entries name outside the block,
    ascending, against the same set taken from the pattern on the host."""
    S = gpu
    from paper_2102_08505_gb300 import shard
    n = 6000
    X = x_of_tight_binding(n, 10, 1e-5)
    for r0, r1 in ((0, 1500), (1500, 1501), (2999, 6000)):
        blk = rows_of(X, r0, r1)
        got = S.ellpack_halo_rows(dev(S, blk, S.SP2_F64), r0, n).cpu().numpy()
        want = np.concatenate(list(shard.halo_requests(blk.idx, blk.nnz, r0, r1, [0, r0, r1, n]).values()) or
                              [np.zeros(0, np.int64)])
        assert np.array_equal(got, np.sort(want)), (r0, r1)
        assert len(got) > 0
    with pytest.raises(S.Sp2Error):
        S.ellpack_halo_rows(dev(S, rows_of(X, 0, 10), S.SP2_F64), n - 5, n)  # block outside 0 .. n-1
