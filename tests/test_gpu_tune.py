"""The SpGEMM autotuner on the GPU: every variant timed on a real product, the product
it leaves is right, and SP2 (single and batched) under the tuned choice matches the
default run and tunes each class once (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_spgemm, dense_of

pytestmark = pytest.mark.gpu


def _x0(n, seed, tau=1e-5):
    H = O.Ell(*I.tight_binding(n, seed=seed, delta=10.0))
    lo, hi = O.gershgorin(H)
    return O.x0(H, lo, hi, tau)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_tune_spgemm_times_every_variant(gpu, dtype):
    S = gpu
    S.sp2_tune_clear()
    dt = S.SP2_F64 if dtype == "f64" else S.SP2_F32
    X = _x0(20000, 7)
    dX = S.Ellpack.from_numpy(X.idx, X.val, X.nnz, dt)
    ref = O.spgemm(X, X, X, -1.0, 2.0, 1e-5)
    Out = S.Ellpack.empty(X.n, ((int(ref.nnz.max()) + 31) // 32) * 32, dt)
    best, times = S.sp2_tune_spgemm(dX, dX, dX, Out, -1.0, 2.0, 1e-5, reps=2)
    assert best in S.TUNE_CANDIDATES and set(times) == set(S.TUNE_CANDIDATES)
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    if dt == S.SP2_F64:
        compare_spgemm(Out.to_numpy(), X, X, X, -1.0, 2.0, 1e-5)
    else:
        compare_spgemm(Out.to_numpy(), X, X, X, -1.0, 2.0, 1e-5, fp32=True)
    mean = float(X.nnz.mean())
    assert S.sp2_tune_lookup(0, dt, X.n, mean) == best
    print("tune %s n=%d: best %d, ms %s" % (dtype, X.n, best, {k: round(v, 3) for k, v in times.items()}))


def test_sp2_tuned_matches_default_and_tunes_once(gpu):
    S = gpu
    S.sp2_tune_clear()
    n, tau, tol = 4096, 1e-5, 1e-10
    H = O.Ell(*I.tight_binding(n, seed=31, delta=10.0))
    dH = S.Ellpack.from_numpy(H.idx, H.val, H.nnz)
    D0, s0 = S.sp2_purify(dH, n // 2, tol, S.sp2_options_default(tau=tau))
    D1, s1 = S.sp2_purify(dH, n // 2, tol, S.sp2_options_default(tau=tau, spgemm_path=S.SP2_PATH_TUNED))
    assert s1["tuned"] >= 1 and s0["tuned"] == 0
    assert s1["iterations"] == s0["iterations"] and s1["branch"] == s0["branch"]
    d0, d1 = dense_of(*D0.to_numpy(), n), dense_of(*D1.to_numpy(), n)
    assert np.linalg.norm(d1 - d0) / np.sqrt(n) < 1e-10
    D2, s2 = S.sp2_purify(dH, n // 2, tol, S.sp2_options_default(tau=tau, spgemm_path=S.SP2_PATH_TUNED))
    assert s2["tuned"] == 0  # every class is in the table now
    assert np.array_equal(dense_of(*D2.to_numpy(), n), d1)
    # one step under the tuned choice reports the variant that ran
    X = S.Ellpack.empty(n, H.w + 32)
    S.sp2_x0(dH, X, tau)
    Xn = S.Ellpack.empty(n, 512)
    info = S.sp2_step(X, Xn, n / 2, tau, spgemm_path=S.SP2_PATH_TUNED)
    assert info.spgemm_path_used in S.TUNE_CANDIDATES


def test_batched_tuned_matches_default(gpu):
    S = gpu
    S.sp2_tune_clear()
    sizes = [600, 1500, 900]
    Hs = [S.Ellpack.from_numpy(*I.tight_binding(m, seed=40 + k, delta=10.0, periodic=False))
          for k, m in enumerate(sizes)]
    noccs = [m // 2 for m in sizes]
    for prec in (S.SP2_PREC_F64, S.SP2_PREC_MIXED):
        S.sp2_tune_clear()
        D0, s0 = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(tau=1e-5, precision=prec))
        D1, s1 = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(tau=1e-5, precision=prec,
                                                                              spgemm_path=S.SP2_PATH_TUNED))
        assert s1[0]["tuned"] == (2 if prec == S.SP2_PREC_MIXED else 1)
        for m, n in enumerate(sizes):
            assert s1[m]["iterations"] == s0[m]["iterations"]
            d0, d1 = dense_of(*D0[m].to_numpy(), n), dense_of(*D1[m].to_numpy(), n)
            assert np.linalg.norm(d1 - d0) / np.sqrt(n) < (1e-10 if prec == S.SP2_PREC_F64 else 1e-6)
    with pytest.raises(S.Sp2Error):
        S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(spgemm_path=13))
    S.sp2_tune_clear()
