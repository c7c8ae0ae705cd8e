"""SP2 purification on the GPU against the CPU oracle and the exact projector (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_density, compare_spgemm, dense_of

pytestmark = pytest.mark.gpu


def ell(t):
    return O.Ell(*t)


def dev(S, E, dtype=None):
    return S.Ellpack.from_numpy(E.idx, E.val, E.nnz, S.SP2_F64 if dtype is None else dtype)


def dense_D(D):
    idx, val, nnz = D.to_numpy()
    return dense_of(idx, val, nnz, D.n)


def test_sp2_tau0_matches_eigen_projector(gpu):
    S = gpu
    n = 512
    H = ell(I.banded(n, band=16, seed=1, delta=10.0))
    D, st = S.sp2_purify(dev(S, H), n // 2, 1e-12, S.sp2_options_default(tau=0.0))
    c = O.checks(H.to_dense(), dense_D(D), n // 2)
    assert st["status"] == "converged"
    assert c["proj_err"] < 1e-10 and c["trace_err"] < 1e-8 and c["idem_err"] < 1e-8 and c["comm_err"] < 1e-8


@pytest.mark.parametrize("delta", [10.0, 0.0])
def test_sp2_banded_f64_matches_oracle(gpu, delta):
    """The banded Hamiltonian (n=1024, |i-j| <= 16, tau 1e-5, tol 1e-10), gapped (A/B
    splitting 10) and as written (gapless)."""
    S = gpu
    n, nocc, tau, tol = 1024, 512, 1e-5, 1e-10
    H = ell(I.banded(n, band=16, seed=1, delta=delta))
    Do, so = O.sp2(H, nocc, tol, tau, max_iter=100)
    D, sg = S.sp2_purify(dev(S, H), nocc, tol, S.sp2_options_default(tau=tau), allow_notconv=True)
    assert sg["emin"] == pytest.approx(so["emin"], rel=1e-14) and sg["emax"] == pytest.approx(so["emax"], rel=1e-14)
    assert sg["iterations"] == so["iterations"]
    assert sg["branch"] == so["branch"]
    assert sg["status"] == so["status"]
    assert np.allclose(sg["trX"], so["trX"], rtol=1e-11, atol=1e-9)
    assert np.allclose(sg["trX2"], so["trX2"], rtol=1e-11, atol=1e-9)
    Dg, Dr = dense_D(D), Do.to_dense()
    assert np.linalg.norm(Dg - Dr) / np.sqrt(n) < 1e-10
    assert np.abs(Dg - Dr).max() < 1e-8
    # entry by entry: each within 1e-12 of its error-bound scale, column sets equal except
    # at entries within that bound of tau
    rep = compare_density(D.to_numpy(), Do, tau)
    print("banded delta %g: %s" % (delta, rep))


def test_sp2_3d_gapped_f64_and_mixed(gpu):
    """3D tight-binding with A/B splitting (n=4096, tau 1e-5): FP64 matches the oracle;
    mixed precision (FP32 loop to err < 1e-4, then >= 2 FP64 iterations) is within 1e-5
    of it (Frobenius / sqrt(n))."""
    S = gpu
    n, tau, tol = 4096, 1e-5, 1e-10
    H = ell(I.tight_binding(n, seed=11, delta=10.0))
    O.set_threads(O.max_threads())
    try:
        Do, so = O.sp2(H, n // 2, tol, tau)
    finally:
        O.set_threads(1)
    Dr = Do.to_dense()
    D64, s64 = S.sp2_purify(dev(S, H), n // 2, tol, S.sp2_options_default(tau=tau))
    assert s64["iterations"] == so["iterations"] and s64["branch"] == so["branch"]
    assert np.linalg.norm(dense_D(D64) - Dr) / np.sqrt(n) < 1e-10
    print("3d gapped fp64: %s" % compare_density(D64.to_numpy(), Do, tau))
    Dm, sm = S.sp2_purify(dev(S, H), n // 2, tol, S.sp2_options_default(tau=tau, precision=S.SP2_PREC_MIXED),
                          allow_notconv=True)
    Dmd = dense_D(Dm)
    dD = np.linalg.norm(Dmd - Dr) / np.sqrt(n)
    print("mixed: iterations %d (fp32 %d) status %s dD %.3e err %s; fp64: %d iterations, branches %s / %s" % (
        sm["iterations"], sm["fp32_iterations"], sm["status"], dD, ["%.2e" % e for e in sm["err"]],
        so["iterations"], "".join("2" if b == "2X-X2" else "1" for b in sm["branch"]),
        "".join("2" if b == "2X-X2" else "1" for b in so["branch"])))
    assert sm["status"] in ("converged", "stalled")
    assert dD <= 1e-5
    assert sm["fp32_iterations"] >= 1 and sm["iterations"] - sm["fp32_iterations"] >= 2
    assert abs(np.trace(Dmd) - n // 2) < 1e-3


def test_sp2_step_matches_oracle_product(gpu):
    S = gpu
    n = 3000
    H = ell(I.tight_binding(n, seed=2, delta=10.0))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, 1e-5)
    nocc = n / 2
    tr, tr2 = O.trace(X0), float(sum((X0.row(i)[1] ** 2).sum() for i in range(n)))
    up = abs(2 * tr - tr2 - nocc) < abs(tr2 - nocc)
    alpha, beta = (-1.0, 2.0) if up else (1.0, 0.0)
    ref = O.spgemm(X0, X0, X0, alpha, beta, 1e-5)
    w = ((int(ref.nnz.max()) + 31) // 32) * 32
    dX = dev(S, X0)
    out = S.Ellpack.empty(n, w)
    info = S.sp2_step(dX, out, nocc, 1e-5)
    assert info.branch == (2 if up else 1)
    assert info.trX == pytest.approx(tr, rel=1e-13) and info.trX2 == pytest.approx(tr2, rel=1e-13)
    compare_spgemm(out.to_numpy(), X0, X0, X0, alpha, beta, 1e-5)
    assert info.trXn == pytest.approx(O.trace(ref), rel=1e-12)
    assert info.nnz_total == int(ref.nnz.sum())
    assert info.max_row_nnz == int(ref.nnz.max())


def test_sp2_errors(gpu):
    S = gpu
    n = 64
    H = ell(I.banded(n, band=3, seed=1, delta=10.0))
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(dev(S, H), 0.0, 1e-10)
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(dev(S, H), n / 2, -1.0)
    assert e.value.code == S.SP2E_ARG
    bad = H.val.copy()
    bad[3, 0] = np.nan
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(S.Ellpack.from_numpy(H.idx, bad, H.nnz), n / 2, 1e-10)
    assert e.value.code == S.SP2E_NONFINITE
    D, st = S.sp2_purify(dev(S, H), n / 2, 1e-14, S.sp2_options_default(max_iter=3, stall_rule=0),
                         allow_notconv=True)
    assert st["status"] == "max_iter" and st["iterations"] == 3 and D.n == n
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(dev(S, H), n / 2, 1e-14, S.sp2_options_default(max_iter=3, stall_rule=0))
    assert e.value.code == S.SP2E_NOTCONV


@pytest.mark.parametrize("arm,ratio", [(1e-300, 1.0), (0.1, 1.0), (1e300, 1.0), (0.1, 0.9), (0.1, 0.5)])
def test_sp2_stall_arm_matches_oracle(gpu, arm, ratio):
    """Stall-rule variants on the gapless banded Hamiltonian (arming threshold: never armed,
    the reading's 0.1, armed from the start; ratio 1 and below): same iterations, status
    and branches as the oracle."""
    S = gpu
    n = 512
    H = ell(I.banded(n, band=8, seed=1, delta=0.0))
    Do, so = O.sp2(H, n // 2, 1e-14, 1e-5, max_iter=60, stall_arm=arm, stall_ratio=ratio)
    D, sg = S.sp2_purify(dev(S, H), n // 2, 1e-14,
                         S.sp2_options_default(tau=1e-5, max_iter=60, stall_arm=arm, stall_ratio=ratio),
                         allow_notconv=True)
    assert sg["iterations"] == so["iterations"] and sg["status"] == so["status"] and sg["branch"] == so["branch"]
    assert np.abs(dense_D(D) - Do.to_dense()).max() < 1e-8
    compare_density(D.to_numpy(), Do, 1e-5)
    with pytest.raises(S.Sp2Error):
        S.sp2_purify(dev(S, H), n // 2, 1e-10, S.sp2_options_default(stall_arm=0.0))
    with pytest.raises(S.Sp2Error):
        S.sp2_purify(dev(S, H), n // 2, 1e-10, S.sp2_options_default(stall_ratio=1.5))


def test_sp2_symmetric_mode_is_bitwise_the_full_product(gpu):
    """sp2_purify with the upper-triangle products (default) and with full rows: the same
    iterations, traces and density matrix bit for bit, in FP64 and mixed precision; a
    Hamiltonian that is not exactly symmetric is refused in symmetric mode."""
    S = gpu
    n = 4096
    H = ell(I.tight_binding(n, seed=12, delta=10.0))
    for prec in (S.SP2_PREC_F64, S.SP2_PREC_MIXED):
        Da, sa = S.sp2_purify(dev(S, H), n // 2, 1e-10, S.sp2_options_default(precision=prec, symmetric=1))
        Db, sb = S.sp2_purify(dev(S, H), n // 2, 1e-10, S.sp2_options_default(precision=prec, symmetric=0))
        assert sa["iterations"] == sb["iterations"] and sa["branch"] == sb["branch"]
        assert np.array_equal(sa["trX"], sb["trX"]) and np.array_equal(sa["nnz_total"], sb["nnz_total"])
        ia, va, na = Da.to_numpy()
        ib, vb, nb = Db.to_numpy()
        assert np.array_equal(na, nb)
        live = np.arange(ia.shape[1])[None, :] < na[:, None]
        assert np.array_equal(np.where(live, ia, 0), np.where(live, ib[:, :ia.shape[1]], 0))
        assert np.array_equal(np.where(live, va, 0), np.where(live, vb[:, :ia.shape[1]], 0))
    bad = H.val.copy()
    i0 = int(np.argmax(H.nnz > 1))
    bad[i0, 0 if H.idx[i0, 0] != i0 else 1] *= 1.0 + 1e-12
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(S.Ellpack.from_numpy(H.idx, bad, H.nnz), n // 2, 1e-10, S.sp2_options_default(symmetric=1))
    assert e.value.code == S.SP2E_ARG
    S.sp2_purify(S.Ellpack.from_numpy(H.idx, bad, H.nnz), n // 2, 1e-10, S.sp2_options_default(symmetric=0),
                 allow_notconv=True)


def _same_D(Da, Db):
    ia, va, na = Da.to_numpy()
    ib, vb, nb = Db.to_numpy()
    if not np.array_equal(na, nb):
        return False
    w = min(ia.shape[1], ib.shape[1])
    live = np.arange(w)[None, :] < na[:, None]
    return (np.array_equal(np.where(live, ia[:, :w], 0), np.where(live, ib[:, :w], 0)) and
            np.array_equal(np.where(live, va[:, :w], 0).view(np.int64), np.where(live, vb[:, :w], 0).view(np.int64)))


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_first_pass_cascade_policies_agree_bitwise(gpu, prec):
    """The cascade of first passes (tight compact, loose compact, full rows, bins) of the
    symmetric products: with and without per-row route flags, and whatever level it
    starts at, every row of every product gets the same sums in the same order, so the
    runs agree bit for bit.  The per-update counts nest (each pass takes the rows the
    previous one passed on), and on this 3D tight-binding run the tight pass does pass
    rows on, so the cascade and the route flags are exercised."""
    S = gpu
    n = 32768
    H = ell(I.tight_binding(n, seed=0, delta=10.0))
    p = S.SP2_PREC_F64 if prec == "f64" else S.SP2_PREC_MIXED
    runs = {}
    for route in (0, 1):
        for up in (0.002, 10.0):
            opt = S.sp2_options_default(precision=p, route_rows=route, level_up_frac=up)
            runs[(route, up)] = S.sp2_purify(dev(S, H), n // 2, 1e-10, opt)
    D0, s0 = runs[(0, 10.0)]
    for key, (D, st) in runs.items():
        assert st["iterations"] == s0["iterations"] and st["branch"] == s0["branch"], key
        assert np.array_equal(st["trX"], s0["trX"]) and np.array_equal(st["nnz_total"], s0["nnz_total"]), key
        assert _same_D(D, D0), key
        start0 = st["level"] == 0
        assert np.all(st["rows_level2"][start0] <= st["rows_level1"][start0]), key
        assert np.all(st["rows_deferred"] <= np.where(st["level"] <= 1, st["rows_level2"], n)), key
    assert np.all(s0["level"] == 0) and s0["rows_level1"].sum() > 0
    assert runs[(1, 10.0)][1]["rows_routed"].sum() > 0
    assert runs[(0, 10.0)][1]["rows_routed"].sum() == 0


SMALL_CASES = [
    # name, matrix, nocc, tau, tol
    ("banded gapped n=1024", lambda: I.banded(1024, band=16, seed=1, delta=10.0, width=64), 512, 1e-5, 1e-10),
    ("banded gapless n=1024 (stall rule)", lambda: I.banded(1024, band=16, seed=1, width=64), 512, 1e-5, 1e-10),
    ("banded tau=0 n=300", lambda: I.banded(300, band=5, seed=3, delta=10.0), 150, 0.0, 1e-10),
    ("open cluster n=1500", lambda: I.tight_binding(1500, seed=31, delta=10.0, periodic=False), 750, 1e-5, 1e-10),
    ("3D gapped n=2048 (the largest)", lambda: I.tight_binding(2048, seed=32, delta=10.0), 1024, 1e-5, 1e-10),
    ("n=3", lambda: I.banded(3, band=1, seed=4, delta=10.0), 1.5, 0.0, 1e-12),
]


@pytest.mark.parametrize("case", SMALL_CASES, ids=[c[0] for c in SMALL_CASES])
def test_small_path_is_the_host_stepped_loop(gpu, case):
    """sp2_purify of an FP64 matrix of at most 2048 rows runs the whole loop in one
    cooperative launch (small_path, the default).  Against the host-stepped loop
    (small_path = 0): the same iterations, branches and stop status, the same density
    matrix bit for bit (every product row is the same sum in the same order), and traces
    equal up to their summation order."""
    S = gpu
    name, make, nocc, tau, tol = case
    H = dev(S, ell(make()))
    Da, sa = S.sp2_purify(H, nocc, tol, S.sp2_options_default(tau=tau), allow_notconv=True)
    Db, sb = S.sp2_purify(H, nocc, tol, S.sp2_options_default(tau=tau, small_path=0), allow_notconv=True)
    assert sa["iterations"] == sb["iterations"] and sa["branch"] == sb["branch"] and sa["status"] == sb["status"]
    assert np.array_equal(sa["nnz_total"], sb["nnz_total"]) and np.array_equal(sa["max_row_nnz"], sb["max_row_nnz"])
    assert np.allclose(sa["trX"], sb["trX"], rtol=1e-13, atol=1e-12)
    assert np.allclose(sa["trX2"], sb["trX2"], rtol=1e-13, atol=1e-12)
    assert _same_D(Da, Db)
    k = sa["small_iterations"]
    assert k > 0 and np.all(sa["level"][:k] == -1)


def test_small_path_hands_long_rows_to_the_host_stepped_loop(gpu):
    """The gapless banded run grows rows past 64 entries: the one-launch loop hands the
    iterate to the host-stepped loop, which finishes the run; the result is the host-stepped
    loop's run bit for bit, with the iterations split between the two."""
    S = gpu
    n = 1024
    H = dev(S, ell(I.banded(n, band=16, seed=1, width=64)))
    Da, sa = S.sp2_purify(H, n / 2, 1e-10, S.sp2_options_default(tau=1e-5), allow_notconv=True)
    Db, sb = S.sp2_purify(H, n / 2, 1e-10, S.sp2_options_default(tau=1e-5, small_path=0), allow_notconv=True)
    assert 0 < sa["small_iterations"] < sa["iterations"] and sb["small_iterations"] == 0
    assert sa["max_row_nnz"][sa["small_iterations"]] > 64 and max(sa["max_row_nnz"][:sa["small_iterations"]]) <= 64
    assert sa["iterations"] == sb["iterations"] and sa["branch"] == sb["branch"] and sa["status"] == sb["status"]
    assert np.allclose(sa["trX"], sb["trX"], rtol=1e-13, atol=1e-12)
    assert _same_D(Da, Db)
