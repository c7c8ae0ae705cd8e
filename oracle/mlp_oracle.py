"""FP64 numpy oracle of the row-length predictor (test infrastructure only).

The predictor is a plain MLP 16 -> 64 -> 64 -> 1 with ReLU on the hidden layers, acting on
standardised features; its target is the standardised log1p of the post-threshold row
length, and the loss of a batch is the mean of (y - t)^2 / 2.  Parameters are packed as
W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.  The paper sizes ELLPACK rows with a
fixed width (Section "Micro-Kernel Performance Evaluation - NUMA Aware
Data") and has no learned part: the predictor is an extension that sizes
the output of each SP2 product.  This oracle writes out the standard backpropagation
equations of that network, and the features below are the plain definitions of the 16
row statistics.  Only the tests import it.
"""
import numpy as np

NIN, NH = 16, 64
NPARAMS = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(theta):
    t = np.asarray(theta, np.float64)
    o = 0
    W1 = t[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = t[o:o + NH]; o += NH
    W2 = t[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = t[o:o + NH]; o += NH
    w3 = t[o:o + NH]; o += NH
    b3 = t[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])


def standardise(feat, counts, stats):
    mean, std = stats[:16], stats[16:32]
    x = (np.asarray(feat, np.float64) - mean) / std
    t = (np.log1p(np.asarray(counts, np.float64)) - stats[32]) / stats[33]
    return x, t


def forward(theta, x):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (z1, h1, z2, h2)


def loss_and_grad(theta, x, t):
    """Mean of (y - t)^2 / 2 over the batch and its gradient (backpropagation)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    y, (z1, h1, z2, h2) = forward(theta, x)
    n = x.shape[0]
    e = y - t
    loss = 0.5 * np.mean(e * e)
    dy = e / n
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def predict_counts(theta, stats, feat):
    """Predicted row lengths: expm1 of the de-standardised output plus the calibration
    margin stats[34] (when present), floored at 0."""
    x, _ = standardise(feat, np.zeros(len(feat)), stats)
    y, _ = forward(theta, x)
    margin = stats[34] if len(stats) > 34 else 0.0
    return np.expm1(np.maximum(y * stats[33] + stats[32] + margin, 0.0))


def calibration_margin(theta, stats, feat, counts, quantile):
    """The smallest m >= 0 with at least a share `quantile` of the samples satisfying
    log1p(count) <= y + m (y the de-standardised network output): the k-th smallest
    residual log1p(count) - y, k = ceil(quantile * n)."""
    x, _ = standardise(feat, np.zeros(len(feat)), stats)
    y, _ = forward(theta, x)
    r = np.sort(np.log1p(np.asarray(counts, np.float64)) - (y * stats[33] + stats[32]))
    k = min(len(r), max(1, int(np.ceil(quantile * len(r)))))
    return max(float(r[k - 1]), 0.0)


def features(idx, val, nnz, tau, branch):
    """The 16 row features of an ELLPACK matrix (see nnzpred_features), in float64."""
    idx, val, nnz = np.asarray(idx), np.asarray(val, np.float64), np.asarray(nnz)
    n = len(nnz)
    rmax = np.array([np.max(np.abs(val[i, :nnz[i]])) if nnz[i] else 0.0 for i in range(n)])
    out = np.zeros((n, 16))
    lg = lambda v: np.log10(v + 1e-30)
    for i in range(n):
        c = idx[i, :nnz[i]]
        v = np.abs(val[i, :nnz[i]])
        nb = nnz[c].astype(np.float64) if len(c) else np.zeros(0)
        out[i, 0] = np.log1p(len(c))
        out[i, 1] = np.log1p(nb.sum())
        out[i, 2] = np.log1p(nb.max() if len(c) else 0.0)
        out[i, 3] = np.log1p(nb.min() if len(c) else 0.0)
        out[i, 4] = lg(v.max() if len(c) else 0.0)
        out[i, 5] = lg(np.sqrt((v * v).sum()))
        out[i, 6] = lg(v.sum())
        out[i, 7] = lg(v[c == i].max() if np.any(c == i) else 0.0)
        out[i, 8] = lg((v * rmax[c]).sum())
        out[i, 9] = np.log1p((v > 10 * tau).sum())
        out[i, 10] = np.log1p((v > 100 * tau).sum())
        out[i, 11] = np.log10(tau) if tau > 0 else -30.0
        out[i, 12] = 1.0 if branch == 2 else 0.0
        out[i, 13] = np.log1p((v * nb).sum() / v.sum() if v.sum() > 0 else 0.0)
        out[i, 14] = 1.0
    return out
