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
    (dict(spgemm_path=13), "spgemm_path"),
    (dict(spgemm_path=5), "spgemm_path"),
    (dict(max_iter=-1), "max_iter"),
    (dict(max_iter=100000), "max_iter"),
    (dict(n_fp64_tail=-1), "n_fp64_tail"),
    (dict(route_rows=2), "route_rows"),
]
PURIFY_ONLY_BAD = [(dict(small_path=2), "small_path")]


@pytest.mark.parametrize("bad,word", BAD_OPTIONS + PURIFY_ONLY_BAD + [(dict(sizing=3), "sizing"), (dict(sizing=2), "predictor"),
                                                    (dict(switch_tol=-1.0), "switch_tol"),
                                                    (dict(level_up_frac=0.0), "level_up_frac"),
                                                    (dict(level_up_frac=float("nan")), "level_up_frac")])
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


def test_multiply_add_and_step_reject_bad_arguments(S):
    """ellpack_multiply, ellpack_add and sp2_step: size, dtype, aliasing, tolerance, scalar and
    path errors come back as SP2E_ARG before any device call."""
    keep = []
    A, B, C = fake_matrix(S, keep=keep), fake_matrix(S, keep=keep), fake_matrix(S, keep=keep)
    big = fake_matrix(S, n=16, keep=keep)
    f32 = fake_matrix(S, keep=keep)
    f32.dtype = S.SP2_F32
    w = ctypes.c_int32()
    mul = lambda a, b, c, al=1.0, be=0.0, tau=0.0: S.lib.sp2_last_error_string() if S.lib.ellpack_multiply(
        ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), al, be, tau, None, ctypes.byref(w)) == S.SP2E_ARG else None
    assert b"sizes differ" in mul(A, B, big)
    assert b"dtypes differ" in mul(A, B, f32)
    assert b"aliases" in mul(A, B, A)
    assert b"aliases" in mul(A, B, B)
    assert b"tau" in mul(A, B, C, tau=-1.0)
    assert b"not finite" in mul(A, B, C, al=float("inf"))
    add = lambda a, b, al=1.0, be=1.0, tau=0.0: S.lib.sp2_last_error_string() if S.lib.ellpack_add(
        ctypes.byref(a), ctypes.byref(b), al, be, tau, None, ctypes.byref(w)) == S.SP2E_ARG else None
    assert b"sizes differ" in add(A, big)
    assert b"dtypes differ" in add(A, f32)
    assert b"alias" in add(A, A)
    assert b"not finite" in add(A, B, be=float("nan"))
    info = S.sp2_step_info()

    def step(x, xn, nocc=4.0, tau=1e-5, path=0, inf=True):
        info.spgemm_path = path
        rc = S.lib.sp2_step(ctypes.byref(x), ctypes.byref(xn), nocc, tau, ctypes.byref(info) if inf else None, None)
        return S.lib.sp2_last_error_string() if rc == S.SP2E_ARG else None
    assert b"info" in step(A, B, inf=False)
    assert b"differ" in step(A, big)
    assert b"differ" in step(A, f32)
    assert b"aliases" in step(A, A)
    assert b"tau" in step(A, B, tau=float("nan"))
    assert b"nocc" in step(A, B, nocc=float("inf"))
    assert b"spgemm_path" in step(A, B, path=6)
    info.compact_level = 3
    assert b"compact_level" in step(A, B)
    info.compact_level = -1
    assert b"compact_level" in step(A, B)
    info.compact_level = 0


def test_multiply_block_rejects_bad_arguments(S):
    """ellpack_multiply_block: a row block outside B, blocks of different lengths, a missing
    addend, dtypes, aliasing and scalars come back as SP2E_ARG before any device call."""
    keep = []
    n = 16
    Bfull = fake_matrix(S, n=n, keep=keep)
    A, C, Out = fake_matrix(S, n=8, keep=keep), fake_matrix(S, n=8, keep=keep), fake_matrix(S, n=8, keep=keep)
    short = fake_matrix(S, n=4, keep=keep)
    f32 = fake_matrix(S, n=8, keep=keep)
    f32.dtype = S.SP2_F32
    w = ctypes.c_int32()

    def blk(a, row0, b, c, out, al=1.0, be=0.0, tau=0.0):
        rc = S.lib.ellpack_multiply_block(ctypes.byref(a), row0, ctypes.byref(b),
                                          ctypes.byref(c) if c is not None else None, ctypes.byref(out),
                                          al, be, tau, ctypes.byref(w), None, None, None)
        return S.lib.sp2_last_error_string() if rc == S.SP2E_ARG else None
    assert b"not rows of B" in blk(A, 9, Bfull, None, Out)
    assert b"not rows of B" in blk(A, -1, Bfull, None, Out)
    assert b"same rows" in blk(A, 0, Bfull, None, short)
    assert b"same rows" in blk(A, 0, Bfull, short, Out, be=2.0)
    assert b"NULL" in blk(A, 0, Bfull, None, Out, be=2.0)
    assert b"dtypes differ" in blk(A, 0, Bfull, None, f32)
    assert b"aliases" in blk(A, 0, Bfull, None, A)
    assert b"aliases" in blk(A, 0, Bfull, C, C, be=2.0)
    assert b"tau" in blk(A, 0, Bfull, None, Out, tau=-1.0)
    assert b"not finite" in blk(A, 0, Bfull, None, Out, al=float("nan"))


def test_block_setup_calls_reject_bad_arguments(S):
    """ellpack_halo_rows, ellpack_gershgorin_block, sp2_x0_block and ellpack_stats_block:
    rows outside the matrix, missing outputs and bad bounds come back as SP2E_ARG before
    any device call."""
    keep = []
    X = fake_matrix(S, n=8, keep=keep)
    X0 = fake_matrix(S, n=8, w=64, keep=keep)
    rows = np.zeros(16, np.int32)
    cnt = ctypes.c_int32()
    d1, d2 = ctypes.c_double(), ctypes.c_double()
    err = lambda rc: S.lib.sp2_last_error_string() if rc == S.SP2E_ARG else None
    assert b"outside" in err(S.lib.ellpack_halo_rows(ctypes.byref(X), 9, 16, rows.ctypes.data, ctypes.byref(cnt), None))
    assert b"outside" in err(S.lib.ellpack_halo_rows(ctypes.byref(X), -1, 16, rows.ctypes.data, ctypes.byref(cnt), None))
    assert b"null" in err(S.lib.ellpack_halo_rows(ctypes.byref(X), 0, 16, None, ctypes.byref(cnt), None))
    assert b"row0" in err(S.lib.ellpack_gershgorin_block(ctypes.byref(X), -2, ctypes.byref(d1), ctypes.byref(d2), None))
    assert b"row0" in err(S.lib.ellpack_stats_block(ctypes.byref(X), -2, ctypes.byref(d1), ctypes.byref(d2), None))
    assert b"bounds" in err(S.lib.sp2_x0_block(ctypes.byref(X), 0, 1.0, 1.0, 1e-5, ctypes.byref(X0), None))
    assert b"tau" in err(S.lib.sp2_x0_block(ctypes.byref(X), 0, -1.0, 1.0, -1.0, ctypes.byref(X0), None))
    assert b"width" in err(S.lib.sp2_x0_block(ctypes.byref(X), 0, -1.0, 1.0, 1e-5, ctypes.byref(X), None))


def test_stats_record_conversion(S):
    """stats_dict turns the C record into arrays of the visited iterates (traces, errors, entries,
    longest rows: iterations + 1) and of the updates (branches, cascade counts, levels:
    iterations), and carries the one-launch loop's share of the updates."""
    st = S.sp2_stats()
    st.iterations, st.status, st.small_iterations = 3, 1, 2
    for t in range(4):
        st.trX[t], st.trX2[t], st.err[t] = 10.0 + t, 9.0 + t, 0.1 / (t + 1)
        st.nnz_total[t], st.max_row_nnz[t] = 100 + t, 7 + t
    for t in range(3):
        st.branch[t] = 1 + t % 2
        st.rows_level1[t], st.rows_level2[t], st.rows_deferred[t], st.rows_routed[t] = 5 + t, 2, 1, t
        st.level[t] = -1 if t < 2 else 0
    d = S.stats_dict(st)
    assert d["iterations"] == 3 and d["status"] == "stalled" and d["small_iterations"] == 2
    assert list(d["trX"]) == [10.0, 11.0, 12.0, 13.0] and list(d["max_row_nnz"]) == [7, 8, 9, 10]
    assert d["branch"] == ["X2", "2X-X2", "X2"]
    assert list(d["rows_level1"]) == [5, 6, 7] and list(d["rows_routed"]) == [0, 1, 2]
    assert list(d["level"]) == [-1, -1, 0]
