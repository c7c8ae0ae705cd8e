"""The library's entry points reject bad arguments on the host, before any device call:
sp2_purify and sp2_purify_batched with out-of-range options return SP2E_ARG and say which
argument (CPU).  The matrices here are host buffers posing as device arrays, so these calls
must never get as far as a launch: the test runs only where no GPU is visible."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host buffers posing as device arrays: checked only without a GPU")


@pytest.fixture(scope="module")
def S():
    import os
    import shutil
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    from paper_2102_08505_gb300 import build
    build.build()
    from paper_2102_08505_gb300 import sp2ell
    return sp2ell


def fake_matrix(S, n=8, w=32, keep=None):
    idx = np.zeros(n * w, np.int32)
    val = np.zeros(n * w, np.float64)
    nnz = np.zeros(n, np.int32)
    keep.extend([idx, val, nnz])
    e = S.ellpack_t()
    e.n, e.width, e.dtype, e.owner = n, w, S.SP2_F64, 0
    e.idx, e.val, e.nnz = idx.ctypes.data, val.ctypes.data, nnz.ctypes.data
    return e


BAD_OPTIONS = [
    (dict(stall_ratio=0.0), "stall_ratio"),
    (dict(stall_ratio=1.5), "stall_ratio"),
    (dict(stall_ratio=float("nan")), "stall_ratio"),
    (dict(stall_arm=0.0), "stall_arm"),
    (dict(tau=-1.0), "tau"),
    (dict(tau=float("inf")), "tau"),
    (dict(precision=7), "precision"),
    (dict(spgemm_path=9), "spgemm_path"),
    (dict(spgemm_path=5), "spgemm_path"),
    (dict(max_iter=-1), "max_iter"),
    (dict(max_iter=100000), "max_iter"),
    (dict(n_fp64_tail=-1), "n_fp64_tail"),
]


@pytest.mark.parametrize("bad,word", BAD_OPTIONS + [(dict(sizing=3), "sizing"), (dict(sizing=2), "predictor"),
                                                    (dict(switch_tol=-1.0), "switch_tol")])
def test_purify_rejects_bad_options(S, bad, word):
    keep = []
    H = fake_matrix(S, keep=keep)
    D = S.ellpack_t()
    st = S.sp2_stats()
    opt = S.sp2_options_default(**bad)
    rc = S.lib.sp2_purify(ctypes.byref(H), 4.0, 1e-10, ctypes.byref(opt), ctypes.byref(D), ctypes.byref(st), None)
    assert rc == S.SP2E_ARG
    assert word.encode() in S.lib.sp2_last_error_string()


@pytest.mark.parametrize("nocc,tol,word", [(0.0, 1e-10, b"nocc"), (8.0, 1e-10, b"nocc"), (4.0, 0.0, b"tol"),
                                           (4.0, float("nan"), b"tol")])
def test_purify_rejects_bad_scalars(S, nocc, tol, word):
    keep = []
    H = fake_matrix(S, keep=keep)
    D = S.ellpack_t()
    rc = S.lib.sp2_purify(ctypes.byref(H), nocc, tol, None, ctypes.byref(D), None, None)
    assert rc == S.SP2E_ARG and word in S.lib.sp2_last_error_string()


def test_purify_rejects_bad_matrices(S):
    keep = []
    D = S.ellpack_t()
    for field, value, word in (("n", 0, b"n = 0"), ("width", 0, b"width"), ("dtype", 5, b"dtype"),
                               ("idx", None, b"null")):
        H = fake_matrix(S, keep=keep)
        setattr(H, field, value)
        rc = S.lib.sp2_purify(ctypes.byref(H), 4.0, 1e-10, None, ctypes.byref(D), None, None)
        assert rc == S.SP2E_ARG and word in S.lib.sp2_last_error_string(), field


@pytest.mark.parametrize("bad,word", BAD_OPTIONS)
def test_batched_rejects_bad_options(S, bad, word):
    keep = []
    Hs = (S.ellpack_t * 2)(fake_matrix(S, keep=keep), fake_matrix(S, n=16, keep=keep))
    Ds = (S.ellpack_t * 2)()
    noccs = (ctypes.c_double * 2)(4.0, 8.0)
    sts = (S.sp2_stats * 2)()
    opt = S.sp2_options_default(**bad)
    rc = S.lib.sp2_purify_batched(Hs, noccs, 2, 1e-10, ctypes.byref(opt), Ds, sts, None)
    assert rc == S.SP2E_ARG
    assert word.encode() in S.lib.sp2_last_error_string()


def test_batched_rejects_bad_counts_and_occupations(S):
    keep = []
    Hs = (S.ellpack_t * 2)(fake_matrix(S, keep=keep), fake_matrix(S, n=16, keep=keep))
    Ds = (S.ellpack_t * 2)()
    rc = S.lib.sp2_purify_batched(Hs, (ctypes.c_double * 2)(4.0, 8.0), 0, 1e-10, None, Ds, None, None)
    assert rc == S.SP2E_ARG and b"count" in S.lib.sp2_last_error_string()
    rc = S.lib.sp2_purify_batched(Hs, (ctypes.c_double * 2)(4.0, 16.0), 2, 1e-10, None, Ds, None, None)
    assert rc == S.SP2E_ARG and b"nocc[1]" in S.lib.sp2_last_error_string()
