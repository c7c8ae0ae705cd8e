"""Learned row-length sizing on the GPU: structural counts against the oracle's tau = 0
pattern, row features and MLP gradients against the FP64 oracle, training, save/load,
and SP2 runs that give the same density matrix under every sizing mode (GPU)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _x0(n, seed, tau=1e-5):
    H = O.Ell(*I.tight_binding(n, seed=seed, delta=10.0))
    lo, hi = O.gershgorin(H)
    return O.x0(H, lo, hi, tau)


def _dev(S, E, dtype=None):
    return S.Ellpack.from_numpy(E.idx, E.val, E.nnz, S.SP2_F64 if dtype is None else dtype)


@pytest.mark.parametrize("with_c", [False, True])
def test_struct_counts_match_oracle_pattern(gpu, with_c):
    S = gpu
    X = _x0(3000, 4)
    ref = O.spgemm(X, X, X if with_c else None, 1.0, 1.0 if with_c else 0.0, 0.0)
    for dt in (S.SP2_F64, S.SP2_F32):
        dX = _dev(S, X, dt)
        c, mx = S.ellpack_struct_count(dX, dX, dX if with_c else None)
        assert np.array_equal(c.cpu().numpy(), ref.nnz)
        assert mx == int(ref.nnz.max())


def test_struct_counts_wide_row_bound(gpu):
    """Row 0 gathers 2400 column groups of 32 (more than the 2048 the count tracks): it
    reports the undeduplicated sum (4800 >= its exact 2400); the other rows are exact."""
    S = gpu
    n = 80000
    # B: rows 2q and 2q+1 (q < 60) hold the same 40 columns, one per group; other rows {i}
    bi = np.zeros((n, 64), np.int32)
    bv = np.full((n, 64), np.nan)
    bn = np.ones(n, np.int32)
    bi[:, 0] = np.arange(n)
    bv[:, 0] = 1.0
    for k in range(120):
        bi[k, :40] = 32 * (40 * (k // 2) + np.arange(40))
        bv[k, :40] = 1.0
        bn[k] = 40
    # A: row 0 gathers B rows 0..119, every other row i gathers row i
    ai = np.zeros((n, 128), np.int32)
    av = np.full((n, 128), np.nan)
    an = np.ones(n, np.int32)
    ai[:, 0] = np.arange(n)
    av[:, 0] = 1.0
    ai[0, :120] = np.arange(120)
    av[0, :120] = 0.5
    an[0] = 120
    A, B = O.Ell(ai, av, an), O.Ell(bi, bv, bn)
    ref = O.spgemm(A, B, None, 1.0, 0.0, 0.0)
    assert ref.nnz[0] == 2400
    c, mx = S.ellpack_struct_count(_dev(S, A), _dev(S, B))
    c = c.cpu().numpy()
    assert c[0] == 4800 and mx == 4800
    assert np.array_equal(c[1:], ref.nnz[1:])


@pytest.mark.parametrize("branch", [1, 2])
def test_features_match_oracle(gpu, branch):
    S = gpu
    X = _x0(3000, 5)
    for dt in (S.SP2_F64, S.SP2_F32):
        dX = _dev(S, X, dt)
        f = S.nnzpred_features(dX, 1e-5, branch).cpu().numpy().astype(np.float64)
        idx, val, nnz = dX.to_numpy()
        ref = M.features(idx, val, nnz, 1e-5, branch)
        np.testing.assert_allclose(f, ref, rtol=2e-6, atol=2e-5)


@pytest.fixture(scope="module")
def trainset(gpu):
    """Features of X0 .. X4 of a 3D-gapped SP2 run (n = 4096) with the exact lengths of
    the products they lead to."""
    from paper_2102_08505_gb300 import learned
    H = I.tight_binding(4096, seed=21, delta=10.0)
    return learned.collect([H], 1e-5, 5)


def test_training_set_counts_are_products(gpu, trainset):
    feat, counts = trainset
    assert feat.shape == (5 * 4096, 16) and counts.shape == (5 * 4096,)
    c = counts.cpu().numpy()
    assert c.min() >= 1 and (feat[:, 12].cpu().numpy() >= 0).all()


def test_stats_grad_and_predict_match_oracle(gpu, trainset):
    S = gpu
    feat, counts = trainset
    p = S.NnzPredictor(seed=3)
    p.set_stats(feat, counts)
    theta, stats = p.params()
    f64 = feat.cpu().numpy().astype(np.float64)
    c64 = counts.cpu().numpy()
    np.testing.assert_allclose(stats[:16], f64.mean(0), rtol=1e-5, atol=1e-5)
    sd = f64.std(0)
    np.testing.assert_allclose(stats[16:32], np.where(sd > 1e-6, sd, 1.0), rtol=1e-4, atol=1e-6)
    lt = np.log1p(c64.astype(np.float64))
    assert stats[32] == pytest.approx(lt.mean(), rel=1e-6) and stats[33] == pytest.approx(lt.std(), rel=1e-5)
    g, loss = p.grad(feat, counts)
    x, t = M.standardise(f64, c64, stats.astype(np.float64))
    lo, go = M.loss_and_grad(theta.astype(np.float64), x, t)
    assert loss == pytest.approx(lo, rel=1e-4)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    # block by block (W1, b1, W2, b2, w3, b3): each block's norm, and each element against its
    # block's largest entry, so that one wrong block or element cannot hide in the whole
    names = ("W1", "b1", "W2", "b2", "w3", "b3")
    for name, gb, ob in zip(names, M.unpack(g), M.unpack(go)):
        gb, ob = np.atleast_1d(gb).ravel(), np.atleast_1d(ob).ravel()
        scale = np.abs(ob).max()
        assert scale > 0, name
        assert np.linalg.norm(gb - ob) <= 1e-4 * np.linalg.norm(ob) + 1e-7 * scale, name
        assert np.abs(gb - ob).max() <= 1e-3 * scale, (name, float(np.abs(gb - ob).max() / scale))
    pred = p.predict(feat).cpu().numpy()
    ref = M.predict_counts(theta.astype(np.float64), stats.astype(np.float64), f64)
    np.testing.assert_allclose(pred, ref, rtol=2e-4, atol=1e-3)


def test_train_reduces_loss_and_save_load(gpu, trainset, tmp_path):
    S = gpu
    feat, counts = trainset
    p = S.NnzPredictor(seed=1)
    p.set_stats(feat, counts)
    _, l0 = p.grad(feat, counts)
    p.train(feat, counts, 400, 1024, 2e-3)
    _, l1 = p.grad(feat, counts)
    assert l1 < 0.25 * l0
    pred = p.predict(feat).cpu().numpy()
    c = counts.cpu().numpy()
    mae = np.mean(np.abs(np.log1p(pred) - np.log1p(c)))
    assert mae < 0.15
    path = str(tmp_path / "p.nnzpred")
    p.save(path)
    q = S.NnzPredictor(seed=99)
    q.load(path)
    assert np.array_equal(q.predict(feat).cpu().numpy(), pred)
    with pytest.raises(S.Sp2Error):
        q.load(str(tmp_path / "missing.nnzpred"))


def test_sizing_modes_give_the_same_density_matrix(gpu, trainset):
    """3D-gapped n = 8192, tau 1e-5: heuristic, exact structural and predicted widths
    give bitwise the same D and the same iteration record."""
    S = gpu
    feat, counts = trainset
    p = S.NnzPredictor(seed=2)
    p.set_stats(feat, counts)
    p.train(feat, counts, 600, 1024, 2e-3)
    H = O.Ell(*I.tight_binding(8192, seed=22, delta=10.0))
    runs = {}
    for mode in (0, 1, 2):
        kw = dict(tau=1e-5, sizing=mode)
        if mode == 2:
            kw["predictor"] = p
        D, st = S.sp2_purify(_dev(S, H), 4096, 1e-10, S.sp2_options_default(**kw), allow_notconv=True)
        runs[mode] = (D.to_numpy(), st)
    (i0, v0, n0), s0 = runs[0]
    for mode in (1, 2):
        (i1, v1, n1), s1 = runs[mode]
        assert s1["iterations"] == s0["iterations"] and s1["branch"] == s0["branch"]
        assert np.array_equal(n1, n0)
        live = np.arange(i0.shape[1])[None, :] < n0[:, None]
        w = min(i0.shape[1], i1.shape[1])
        assert np.array_equal(np.where(live[:, :w], i1[:, :w], 0), np.where(live[:, :w], i0[:, :w], 0))
        assert np.array_equal(np.where(live[:, :w], v1[:, :w], 0), np.where(live[:, :w], v0[:, :w], 0))
    assert runs[1][1]["struct_passes"] == runs[1][1]["iterations"] and runs[1][1]["regrows"] == 0
    s2 = runs[2][1]
    assert s2["struct_passes"] == 0
    assert s2["pred_log_mae"] < 0.3
    # predicted widths are tighter than the structural bound
    assert s2["width_max"] < runs[1][1]["width_max"]
    print("sizing: widths %d / %d / %d, regrows %d / %d / %d, predicted log-MAE %.3f under %.4f" % (
        s0["width_max"], runs[1][1]["width_max"], s2["width_max"], s0["regrows"], runs[1][1]["regrows"],
        s2["regrows"], s2["pred_log_mae"], s2["pred_under_frac"]))


def test_sizing_errors(gpu):
    S = gpu
    H = O.Ell(*I.banded(64, band=3, seed=1, delta=10.0))
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(_dev(S, H), 32, 1e-10, S.sp2_options_default(sizing=2))
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.sp2_purify(_dev(S, H), 32, 1e-10, S.sp2_options_default(sizing=3))
    assert e.value.code == S.SP2E_ARG


def test_predicted_width_rule(gpu, trainset):
    """nnzpred_width: the predictions from the features of X, and the width rule
    ceil(1.1 x longest) + 16 rounded up to 32."""
    S = gpu
    feat, counts = trainset
    p = S.NnzPredictor(seed=4)
    p.set_stats(feat, counts)
    p.train(feat, counts, 300, 1024, 2e-3)
    X = _dev(S, _x0(4096, 23))
    w, pred = p.width(X, 1e-5, 2)
    ref = p.predict(S.nnzpred_features(X, 1e-5, 2))
    assert torch_equal(pred, ref)
    m = float(ref.max().item())
    expect = min(4096, ((int(np.ceil(1.10 * m)) + 16 + 31) // 32) * 32)
    assert w == expect


def torch_equal(a, b):
    import torch
    return torch.equal(a, b)


def test_calibration_margin_matches_oracle(gpu, trainset):
    """The margin for quantile 0.9 is the oracle's (the 0.9 quantile of the residuals
    log1p(count) - y, in FP32 on the GPU), and with it at least 90 % of the training rows
    lie at or below their predicted length (about half do without it)."""
    S = gpu
    feat, counts = trainset
    p = S.NnzPredictor(seed=5)
    p.set_stats(feat, counts)
    p.train(feat, counts, 400, 1024, 2e-3)
    c = counts.cpu().numpy()
    under0 = np.mean(c > p.predict(feat).cpu().numpy())
    m = p.calibrate(feat, counts, 0.9)
    theta, stats = p.params()
    assert stats[34] == m and m > 0.0
    mo = M.calibration_margin(theta.astype(np.float64), stats.astype(np.float64)[:34],
                              feat.cpu().numpy().astype(np.float64), c, 0.9)
    assert m == pytest.approx(mo, abs=2e-4)
    pred = p.predict(feat).cpu().numpy()
    ref = M.predict_counts(theta.astype(np.float64), stats.astype(np.float64), feat.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(pred, ref, rtol=2e-4, atol=1e-3)
    under = np.mean(c > pred)
    print("rows above their prediction: %.3f uncalibrated, %.3f with margin %.4f" % (under0, under, m))
    assert under <= 0.1 + 1e-3 and under < under0
