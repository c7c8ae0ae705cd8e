"""Training the row-length predictor on products the SP2 method itself generates.

Orchestration only: every product, feature row, gradient and optimiser step is computed
by the CUDA library (sp2_step, nnzpred_features, nnzpred_train); this module decides
which Hamiltonians and iterations feed the training set and concatenates the device
arrays the library returns.
"""
import numpy as np

from . import inputs as I
from . import sp2ell as S


def sp2_products(H, nocc, tau, steps, dtype=S.SP2_F64):
    """Runs `steps` SP2 iterations from X0 of H; yields (X, branch, Xn) per iteration:
    the features of X and the row lengths of Xn form one training batch."""
    X = S.Ellpack.empty(H.n, H.width + 32)
    S.sp2_x0(H, X, tau)
    if dtype == S.SP2_F32:
        Xf = S.Ellpack.empty(H.n, X.width, S.SP2_F32)
        S.ellpack_copy(X, Xf)
        X = Xf
    traces = None
    for _ in range(steps):
        w = min(H.n, max(64, ((4 * int(X.nnz.max().item()) + 31) // 32) * 32))
        while True:
            Xn = S.Ellpack.empty(H.n, w, dtype)
            rc, info = S.sp2_step(X, Xn, nocc, tau, traces=traces, raise_on_overflow=False)
            if rc == 0:
                break
            w = min(H.n, ((info.required_width + 31) // 32) * 32)
        yield X, info.branch, Xn
        traces = (info.trXn, info.trXn2)
        X = Xn


def collect(hamiltonians, tau, steps, rows_per_product=None, dtype=S.SP2_F64):
    """Features and exact row lengths of SP2 products of the given Hamiltonians
    ((idx, val, nnz) numpy triples).  rows_per_product: keep every k-th row so that each
    product contributes about that many rows.  Returns (feat [m,16], counts [m]) on the GPU."""
    import torch
    feats, counts = [], []
    for idx, val, nnz in hamiltonians:
        H = S.Ellpack.from_numpy(idx, val, nnz)
        for X, branch, Xn in sp2_products(H, H.n / 2, tau, steps, dtype):
            f = S.nnzpred_features(X, tau, branch)
            c = Xn.nnz
            if rows_per_product and rows_per_product < H.n:
                stride = max(1, H.n // rows_per_product)
                f, c = f[::stride], c[::stride]
            feats.append(f.contiguous())
            counts.append(c.contiguous())
    return torch.cat(feats).contiguous(), torch.cat(counts).contiguous()


def default_training_set(seed=0, rows=50000, tau=1e-5, steps=10, dtype=S.SP2_F64):
    """About `rows` rows from the first `steps` SP2 products of gapped 3D tight-binding
    Hamiltonians of 4096 .. 16384 sites (both update branches occur)."""
    sizes = [4096, 8192, 16384]
    hs = [I.tight_binding(n, seed=seed + k, delta=10.0) for k, n in enumerate(sizes)]
    per = max(1, rows // (len(sizes) * steps))
    return collect(hs, tau, steps, rows_per_product=per, dtype=dtype)


def train(feat, counts, seed=0, steps=1500, batch=2048, lr=2e-3, quantile=0.9):
    """A new predictor trained on (feat, counts) and calibrated so that a share `quantile`
    of the training rows lie at or below their predicted lengths (None: no margin);
    returns (predictor, final batch loss)."""
    p = S.NnzPredictor(seed)
    p.set_stats(feat, counts)
    loss = p.train(feat, counts, steps, batch, lr)
    if quantile is not None:
        p.calibrate(feat, counts, quantile)
    return p, loss
