"""Batched SP2 (one device-resident loop over many Hamiltonians) against the CPU oracle,
matrix by matrix (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_density, dense_of

pytestmark = pytest.mark.gpu


def batch(seed=0):
    """Uneven sizes: gapped banded chains and gapped open 3D clusters."""
    mats = [I.banded(200, band=8, seed=seed + 1, delta=10.0),
            I.tight_binding(700, seed=seed + 2, delta=10.0, periodic=False),
            I.banded(513, band=16, seed=seed + 3, delta=10.0),
            I.tight_binding(1100, seed=seed + 4, delta=10.0, periodic=False),
            I.banded(64, band=3, seed=seed + 5, delta=8.0),
            I.tight_binding(900, seed=seed + 6, delta=10.0, periodic=False)]
    return [O.Ell(*m) for m in mats]


def dense_D(D):
    idx, val, nnz = D.to_numpy()
    return dense_of(idx, val, nnz, D.n)


@pytest.mark.parametrize("graph", [1, 0])
def test_batched_f64_matches_oracle(gpu, graph):
    S = gpu
    tau, tol = 1e-5, 1e-10
    mats = batch()
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [(m.n + 1) // 2 for m in mats]  # the lower (A) band holds ceil(n/2) states: nocc fills it
    Ds, sts = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, graph=graph))
    for m, H, D, st in zip(range(len(mats)), mats, Ds, sts):
        Do, so = O.sp2(H, noccs[m], tol, tau)
        assert st["iterations"] == so["iterations"], m
        assert st["branch"] == so["branch"], m
        assert st["status"] == so["status"], m
        assert np.allclose(st["trX"], so["trX"], rtol=1e-11, atol=1e-9)
        assert np.linalg.norm(dense_D(D) - Do.to_dense()) / np.sqrt(H.n) < 1e-10, m
        compare_density(D.to_numpy(), Do, tau)  # entry by entry


def test_batched_mixed_within_1e5_of_oracle(gpu):
    S = gpu
    tau, tol = 1e-5, 1e-10
    mats = batch(10)
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [(m.n + 1) // 2 for m in mats]  # the lower (A) band holds ceil(n/2) states: nocc fills it
    Ds, sts = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, precision=S.SP2_PREC_MIXED))
    for m, H, D, st in zip(range(len(mats)), mats, Ds, sts):
        Do, so = O.sp2(H, noccs[m], tol, tau)
        dD = np.linalg.norm(dense_D(D) - Do.to_dense()) / np.sqrt(H.n)
        assert dD <= 1e-5, (m, dD, st["iterations"], st["fp32_iterations"])
        assert st["fp32_iterations"] >= 1 and st["iterations"] - st["fp32_iterations"] >= 2


def test_batched_matches_single_matrix_runs(gpu):
    """The same matrices one by one through sp2_purify give the same iterations and D."""
    S = gpu
    tau, tol = 1e-5, 1e-10
    mats = batch(20)[:3]
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [(m.n + 1) // 2 for m in mats]  # the lower (A) band holds ceil(n/2) states: nocc fills it
    for prec in (S.SP2_PREC_F64, S.SP2_PREC_F32):
        opt = S.sp2_options_default(tau=tau, precision=prec)
        Ds, sts = S.sp2_purify_batched(Hs, noccs, tol, opt)
        for H, nocc, D, st in zip(Hs, noccs, Ds, sts):
            D1, s1 = S.sp2_purify(H, nocc, tol, opt)
            assert st["iterations"] == s1["iterations"] and st["branch"] == s1["branch"]
            assert np.allclose(dense_D(D), dense_D(D1), rtol=0, atol=1e-12 if prec == S.SP2_PREC_F64 else 1e-6)


def test_batched_regrows_when_width_is_too_small(gpu):
    S = gpu
    tau, tol = 1e-5, 1e-10
    mats = batch(30)[:2]
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [(m.n + 1) // 2 for m in mats]  # the lower (A) band holds ceil(n/2) states: nocc fills it
    Ds, sts = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, max_width=64))
    assert sts[0]["regrows"] >= 1
    for m, H, D in zip(range(2), mats, Ds):
        Do, so = O.sp2(H, noccs[m], tol, tau)
        assert np.linalg.norm(dense_D(D) - Do.to_dense()) / np.sqrt(H.n) < 1e-10


@pytest.mark.parametrize("ratio", [1.0, 0.5])
def test_batched_stall_rule_matches_oracle(gpu, ratio):
    """Gapless banded chains at tau = 1e-5 stop by the stall rule (ratio 1 and 0.5): the
    same iterations, status and branches as the oracle, matrix by matrix."""
    S = gpu
    tau, tol = 1e-5, 1e-14
    mats = [O.Ell(*I.banded(256, band=8, seed=1, delta=0.0)), O.Ell(*I.banded(384, band=6, seed=2, delta=0.0))]
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [m.n // 2 for m in mats]
    Ds, sts = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, max_iter=60, stall_ratio=ratio),
                                   allow_notconv=True)
    for m, H, D, st in zip(range(len(mats)), mats, Ds, sts):
        Do, so = O.sp2(H, noccs[m], tol, tau, max_iter=60, stall_ratio=ratio)
        assert so["status"] == "stalled", m
        assert (st["iterations"], st["status"], st["branch"]) == (so["iterations"], so["status"], so["branch"]), m
        assert np.abs(dense_D(D) - Do.to_dense()).max() < 1e-8, m


def test_batched_argument_errors(gpu):
    S = gpu
    m = batch()[0]
    H = S.Ellpack.from_numpy(m.idx, m.val, m.nnz)
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify_batched([H], [0.0], 1e-10)
    assert e.value.code == S.SP2E_ARG
    F = S.Ellpack.from_numpy(m.idx, m.val, m.nnz, S.SP2_F32)
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify_batched([F], [10.0], 1e-10)
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify_batched([H], [10.0], 1e-10, S.sp2_options_default(stall_ratio=0.0))
    assert e.value.code == S.SP2E_ARG


def test_batched_symmetric_mode_is_bitwise_the_full_product(gpu):
    S = gpu
    sizes = [700, 1300, 520]
    Hs = [S.Ellpack.from_numpy(*I.tight_binding(m, seed=60 + k, delta=10.0, periodic=False))
          for k, m in enumerate(sizes)]
    noccs = [(m + 1) // 2 for m in sizes]
    for prec in (S.SP2_PREC_F64, S.SP2_PREC_MIXED):
        Da, sa = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(precision=prec, symmetric=1))
        Db, sb = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(precision=prec, symmetric=0))
        for m in range(len(sizes)):
            assert sa[m]["iterations"] == sb[m]["iterations"] and sa[m]["branch"] == sb[m]["branch"]
            ia, va, na = Da[m].to_numpy()
            ib, vb, nb = Db[m].to_numpy()
            assert np.array_equal(na, nb)
            live = np.arange(ia.shape[1])[None, :] < na[:, None]
            assert np.array_equal(np.where(live, va, 0), np.where(live, vb[:, :ia.shape[1]], 0))


def test_batched_route_flags_agree_bitwise(gpu):
    """The captured loop runs the first-pass cascade from the tight compact level; with and
    without per-row route flags every matrix gets the same iterations and the same D bit for
    bit, and the stacked rows (above 2048) do start at the tight level."""
    S = gpu
    sizes = [4096, 700, 2600, 1500]
    Hs = [S.Ellpack.from_numpy(*I.tight_binding(m, seed=80 + k, delta=10.0, periodic=False))
          for k, m in enumerate(sizes)]
    noccs = [(m + 1) // 2 for m in sizes]
    for prec in (S.SP2_PREC_F64, S.SP2_PREC_MIXED):
        Da, sa = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(precision=prec, route_rows=1))
        Db, sb = S.sp2_purify_batched(Hs, noccs, 1e-10, S.sp2_options_default(precision=prec, route_rows=0))
        for m in range(len(sizes)):
            assert sa[m]["iterations"] == sb[m]["iterations"] and sa[m]["branch"] == sb[m]["branch"]
            assert np.all(sa[m]["level"] == 0)
            ia, va, na = Da[m].to_numpy()
            ib, vb, nb = Db[m].to_numpy()
            assert np.array_equal(na, nb)
            live = np.arange(ia.shape[1])[None, :] < na[:, None]
            assert np.array_equal(np.where(live, ia, 0), np.where(live, ib[:, :ia.shape[1]], 0))
            assert np.array_equal(np.where(live, va, 0).view(np.int64), np.where(live, vb[:, :ia.shape[1]], 0).view(np.int64))
