"""Pins of the row-length predictor's oracle (CPU): backpropagation against central
finite differences, forward closed forms, and the 16 row features on a hand-worked
3x3 matrix."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _theta(seed):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 0.5, (M.NH, M.NIN))
    W2 = rng.normal(0, 0.3, (M.NH, M.NH))
    return M.pack(W1, rng.normal(0, 0.2, M.NH), W2, rng.normal(0, 0.2, M.NH), rng.normal(0, 0.3, M.NH), 0.1)


def test_pack_layout():
    th = np.arange(M.NPARAMS, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = M.unpack(th)
    assert M.NPARAMS == 5313
    assert W1[1, 0] == 16 and b1[0] == 1024 and W2[0, 1] == 1024 + 64 + 1
    assert b2[0] == 1024 + 64 + 4096 and w3[0] == b2[0] + 64 and b3 == M.NPARAMS - 1
    assert np.array_equal(M.pack(W1, b1, W2, b2, w3, b3), th)


def test_gradient_matches_finite_differences():
    """Every block of the analytic gradient against central differences of the loss."""
    rng = np.random.default_rng(1)
    th = _theta(2)
    x = rng.normal(0, 1, (40, 16))
    t = rng.normal(0, 1, 40)
    loss, g = M.loss_and_grad(th, x, t)
    blocks = [(0, 1024), (1024, 1088), (1088, 5184), (5184, 5248), (5248, 5312), (5312, 5313)]
    h = 1e-6
    for lo, hi in blocks:
        for i in rng.choice(np.arange(lo, hi), min(12, hi - lo), replace=False):
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            fd = (M.loss_and_grad(tp, x, t)[0] - M.loss_and_grad(tm, x, t)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])
    # the loss itself: mean of (y - t)^2 / 2
    y, _ = M.forward(th, x)
    assert loss == pytest.approx(0.5 * np.mean((y - t) ** 2), rel=1e-15)


def test_forward_closed_form():
    """A network that computes y = 1 + 6 relu(x_0) (unit 0 of each layer only)."""
    W1 = np.zeros((64, 16)); W1[0, 0] = 1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 2.0
    w3 = np.zeros(64); w3[0] = 3.0
    th = M.pack(W1, np.zeros(64), W2, np.zeros(64), w3, 1.0)
    x = np.zeros((3, 16)); x[:, 0] = [-1.0, 0.5, 2.0]; x[:, 5] = 7.0
    y, _ = M.forward(th, x)
    assert np.array_equal(y, [1.0, 4.0, 13.0])
    # a constant network (all zero but b3 = c): the gradient is mean(c - t) on b3 alone
    th = M.pack(np.zeros((64, 16)), np.zeros(64), np.zeros((64, 64)), np.zeros(64), np.zeros(64), 0.25)
    t = np.array([1.0, -0.5, 0.0, 2.0])
    loss, g = M.loss_and_grad(th, x[:1].repeat(4, 0), t)
    assert loss == pytest.approx(np.mean((0.25 - t) ** 2) / 2)
    assert g[-1] == pytest.approx(np.mean(0.25 - t)) and not g[:-1].any()


def test_standardise_and_predict_round_trip():
    """With a zero network the prediction is expm1 of the target mean."""
    stats = np.concatenate([np.full(16, 2.0), np.full(16, 4.0), [np.log1p(99.0), 0.5]])
    th = np.zeros(M.NPARAMS)
    p = M.predict_counts(th, stats, np.zeros((5, 16)))
    assert np.allclose(p, 99.0, rtol=1e-14)
    x, t = M.standardise(np.full((1, 16), 6.0), [99], stats)
    assert np.allclose(x, 1.0) and t[0] == pytest.approx(0.0, abs=1e-15)
    # a margin m multiplies 1 + prediction by e^m
    pm = M.predict_counts(th, np.concatenate([stats, [np.log(2.0)]]), np.zeros((2, 16)))
    assert np.allclose(pm, 199.0, rtol=1e-13)


def test_calibration_margin_is_the_residual_quantile():
    """With a zero network every prediction is expm1(target mean): the margin for quantile
    q is the ceil(q n)-th smallest log1p(count) minus that mean (never negative), and with
    it at least a share q of the samples lie at or below their prediction."""
    rng = np.random.default_rng(7)
    counts = rng.integers(1, 500, 101)
    stats = np.concatenate([np.zeros(16), np.ones(16), [np.log1p(120.0), 1.0]])
    th = np.zeros(M.NPARAMS)
    feat = np.zeros((len(counts), 16))
    for q in (0.5, 0.9, 1.0):
        m = M.calibration_margin(th, stats, feat, counts, q)
        srt = np.sort(np.log1p(counts.astype(np.float64)))
        assert m == pytest.approx(max(srt[int(np.ceil(q * len(counts))) - 1] - np.log1p(120.0), 0.0), abs=1e-14)
        pred = M.predict_counts(th, np.concatenate([stats, [m]]), feat)
        assert np.mean(counts <= pred * (1 + 1e-12)) >= q
    assert M.calibration_margin(th, stats, feat[:5], np.ones(5, np.int64), 0.9) == 0.0  # over-predicted: no margin


def test_features_hand_worked():
    """3x3 symmetric matrix, tau 1e-5, branch 2 (2X - X^2): every feature by hand."""
    idx = np.array([[0, 1, 0], [0, 1, 2], [1, 2, 0]], np.int32)
    val = np.array([[0.5, -0.2, np.nan], [-0.2, 0.4, 2e-4], [2e-4, 0.3, np.nan]])
    nnz = np.array([2, 3, 2], np.int32)
    f = M.features(idx, val, nnz, 1e-5, 2)
    lg = np.log10
    row0 = [np.log1p(2), np.log1p(5), np.log1p(3), np.log1p(2), lg(0.5), lg(np.sqrt(0.29)), lg(0.7), lg(0.5),
            lg(0.5 * 0.5 + 0.2 * 0.4), np.log1p(2), np.log1p(2), -5.0, 1.0, np.log1p(1.6 / 0.7), 1.0, 0.0]
    row1 = [np.log1p(3), np.log1p(7), np.log1p(3), np.log1p(2), lg(0.4), lg(np.sqrt(0.04 + 0.16 + 4e-8)),
            lg(0.6002), lg(0.4), lg(0.2 * 0.5 + 0.4 * 0.4 + 2e-4 * 0.3), np.log1p(3), np.log1p(2), -5.0, 1.0,
            np.log1p((0.2 * 2 + 0.4 * 3 + 2e-4 * 2) / 0.6002), 1.0, 0.0]
    row2 = [np.log1p(2), np.log1p(5), np.log1p(3), np.log1p(2), lg(0.3), lg(np.sqrt(0.09 + 4e-8)), lg(0.3002),
            lg(0.3), lg(2e-4 * 0.4 + 0.3 * 0.3), np.log1p(2), np.log1p(1), -5.0, 1.0,
            np.log1p((2e-4 * 3 + 0.3 * 2) / 0.3002), 1.0, 0.0]
    assert np.allclose(f, np.array([row0, row1, row2]), rtol=1e-12, atol=1e-12)
    g = M.features(idx, val, nnz, 0.0, 1)
    assert g[0, 11] == -30.0 and g[0, 12] == 0.0
