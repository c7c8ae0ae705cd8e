"""The allocation-free trace entry point, for callers that cannot allocate device memory
(their memory is entirely reserved by their own pool, or an allocation call is not
acceptable on their path).  It must give the same results as ellpack_trace and
ellpack_frobenius2 on consecutive calls, and refuse sizes beyond its fixed scratch.

This file is collected last on purpose: the fixed scratch is shared process-wide, and
the test must pass both alone in a fresh process and after every other test."""
import numpy as np
import pytest

from paper_2102_08505_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_trace_matches_allocating_entry_points(gpu):
    S = gpu
    cases = [
        (I.tight_binding(5000, seed=1), S.SP2_F64),
        (I.banded(S.SP2_NOALLOC_MAX_N, band=4, seed=2), S.SP2_F64),  # the largest size accepted
        (I.tight_binding(3000, seed=3), S.SP2_F32),
    ]
    for (idx, val, nnz), dt in cases:
        A = S.Ellpack.from_numpy(idx, val, nnz, dt)
        want_tr = S.ellpack_trace(A)
        want_fro = S.ellpack_frobenius2(A)
        for _ in range(2):  # two calls in a row reuse the same scratch
            tr, fro = S.ellpack_trace_noalloc(A)
            assert tr == pytest.approx(want_tr, rel=1e-13, abs=1e-13)
            assert fro == pytest.approx(want_fro, rel=1e-13)


def test_noalloc_rejects_sizes_beyond_scratch(gpu):
    S = gpu
    n = S.SP2_NOALLOC_MAX_N + 1
    idx, val, nnz = I.banded(n, band=1, seed=4)
    A = S.Ellpack.from_numpy(idx, val, nnz)
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_trace_noalloc(A)
    assert e.value.code == S.SP2E_ARG and "exceeds" in str(e.value)


def test_noalloc_outputs_follow_their_allocating_counterparts(gpu):
    """Entries near 1e200: the trace is finite but the squares overflow.  ellpack_trace
    succeeds and ellpack_frobenius2 fails; the allocation-free call does the same for each
    output it is asked for (a trace-only call succeeds)."""
    S = gpu
    idx, val, nnz = I.banded(300, band=3, seed=5)
    val = np.where(np.isnan(val), val, val * 1e200)
    A = S.Ellpack.from_numpy(idx, val, nnz)
    want_tr = S.ellpack_trace(A)
    assert np.isfinite(want_tr)
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_frobenius2(A)
    assert e.value.code == S.SP2E_NONFINITE
    for _ in range(2):
        tr, fro = S.ellpack_trace_noalloc(A, frobenius=False)
        assert fro is None
        assert tr == pytest.approx(want_tr, rel=1e-13)
        with pytest.raises(S.Sp2Error) as e:
            S.ellpack_trace_noalloc(A)
        assert e.value.code == S.SP2E_NONFINITE
