"""Standalone ELLPACK operations on the GPU against the oracle's definitions: transpose,
norms, drop threshold, scale, dense conversion (GPU).  Index work is compared bit for
bit; values are exact copies or single roundings, so they are compared exactly too,
except the norms' sums (1e-14 relative)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rows_equal(g, E, fp32=False):
    gi, gv, gn = g
    assert np.array_equal(gn, E.nnz)
    for i in range(E.n):
        k = E.nnz[i]
        assert np.array_equal(gi[i, :k], E.idx[i, :k]), i
        ref = E.val[i, :k].astype(np.float32).astype(np.float64) if fp32 else E.val[i, :k]
        assert np.array_equal(gv[i, :k], ref), i


def _cases():
    return [
        ("random_ragged", O.Ell(*I.random_sparse(3000, seed=1, min_nnz=0, max_nnz=40, width=64,
                                                 full_rows=(5, 2999), empty_rows=(0, 7)))),
        ("tight_binding", O.Ell(*I.tight_binding(4000, seed=2))),
        # one column gathers 700 entries (a long row of A^T, beyond the shared-memory sort)
        ("hub_column", _hub(1500)),
    ]


def _hub(n):
    idx = np.zeros((n, 2), np.int32)
    val = np.full((n, 2), np.nan)
    nnz = np.ones(n, np.int32)
    idx[:, 0] = np.arange(n)
    val[:, 0] = 1.0 + np.arange(n) / n
    for i in range(1, 701):
        idx[i] = sorted([0, i])
        val[i] = [0.5, 1.0] if idx[i, 0] == 0 else [1.0, 0.5]
        nnz[i] = 2
    return O.Ell(idx, val, nnz)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_transpose(gpu, dtype):
    S = gpu
    dt = S.SP2_F64 if dtype == "f64" else S.SP2_F32
    for name, A in _cases():
        ref = O.transpose(A)
        dA = S.Ellpack.from_numpy(A.idx, A.val, A.nnz, dt)
        small = S.Ellpack.empty(A.n, 1, dt)
        if ref.w > 1:
            rc, w = S.ellpack_transpose(dA, small, raise_on_overflow=False)
            assert rc == S.SP2E_OVERFLOW and w == ref.w
        At = S.Ellpack.empty(A.n, ((ref.w + 31) // 32) * 32, dt)
        assert S.ellpack_transpose(dA, At) == int(np.bincount(A.idx[np.arange(A.w)[None, :] < A.nnz[:, None]],
                                                              minlength=A.n).max())
        _rows_equal(At.to_numpy(), ref, fp32=dt == S.SP2_F32)


def test_norms_threshold_scale(gpu):
    S = gpu
    for name, A in _cases():
        dA = S.Ellpack.from_numpy(A.idx, A.val, A.nnz)
        mx, inf, fro = S.ellpack_norms(dA)
        rmx, rinf, rfro = O.norms(A)
        assert mx == rmx
        assert inf == pytest.approx(rinf, rel=1e-14) and fro == pytest.approx(rfro, rel=1e-14)
        S.ellpack_scale(dA, -0.75)
        _rows_equal(dA.to_numpy(), O.scale(A, -0.75))
        S.ellpack_threshold(dA, 0.2)
        _rows_equal(dA.to_numpy(), O.threshold(O.scale(A, -0.75), 0.2))
    with pytest.raises(S.Sp2Error):
        S.ellpack_threshold(dA, -1.0)
    bad = A.val.copy()
    bad[1, 0] = np.inf
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_norms(S.Ellpack.from_numpy(A.idx, bad, A.nnz))
    assert e.value.code == S.SP2E_NONFINITE


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_dense_round_trip(gpu, dtype):
    import torch
    S = gpu
    dt = S.SP2_F64 if dtype == "f64" else S.SP2_F32
    A = O.Ell(*I.random_sparse(700, seed=3, min_nnz=0, max_nnz=30, width=32, empty_rows=(3,)))
    dA = S.Ellpack.from_numpy(A.idx, A.val, A.nnz, dt)
    D = S.ellpack_to_dense(dA)
    ref = A.to_dense()
    if dt == S.SP2_F32:
        ref = ref.astype(np.float32)
    assert np.array_equal(D.cpu().numpy(), ref)
    B = S.Ellpack.empty(A.n, 32, dt)
    assert S.ellpack_from_dense(D, B) == int(A.nnz.max())
    _rows_equal(B.to_numpy(), A, fp32=dt == S.SP2_F32)
    C = S.Ellpack.empty(A.n, 32, dt)
    S.ellpack_from_dense(D, C, tau=0.5)
    _rows_equal(C.to_numpy(), O.from_dense_tau(D.double().cpu().numpy(), 0.5, width=32), fp32=False)
    narrow = S.Ellpack.empty(A.n, 8, dt)
    rc, w = S.ellpack_from_dense(D, narrow, raise_on_overflow=False)
    assert rc == S.SP2E_OVERFLOW and w == int(A.nnz.max())
    # an ld larger than n (padding columns are never read as entries beyond n)
    Dp = torch.zeros((A.n, A.n + 5), dtype=D.dtype, device="cuda")
    Dp[:, :A.n] = D
    Dp[:, A.n:] = 7.0
    E = S.Ellpack.empty(A.n, 32, dt)
    S.ellpack_from_dense(Dp, E)
    _rows_equal(E.to_numpy(), A, fp32=dt == S.SP2_F32)


def test_download_async_matches_download(gpu):
    import torch
    S = gpu
    A = O.Ell(*I.random_sparse(500, seed=9, min_nnz=0, max_nnz=20, width=32))
    dA = S.Ellpack.from_numpy(A.idx, A.val, A.nnz)
    bufs = [(torch.empty((500, 32), dtype=torch.int32).pin_memory(), torch.empty((500, 32), dtype=torch.float64).pin_memory(),
             torch.empty(500, dtype=torch.int32).pin_memory()) for _ in range(2)]
    s = torch.cuda.Stream()
    (i1, v1, n1), (i2, v2, n2) = bufs
    S._check(S.lib.ellpack_download(S._d(dA), i1.data_ptr(), v1.data_ptr(), n1.data_ptr(), S._stream(s)))
    S._check(S.lib.ellpack_download_async(S._d(dA), i2.data_ptr(), v2.data_ptr(), n2.data_ptr(), S._stream(s)))
    s.synchronize()
    assert torch.equal(n1, n2) and np.array_equal(n2.numpy(), A.nnz)
    live = np.arange(32)[None, :] < A.nnz[:, None]
    assert np.array_equal(np.where(live, i2.numpy(), 0), np.where(live, A.idx, 0))
    assert np.array_equal(np.where(live, v2.numpy(), 0), np.where(live, A.val, 0))
