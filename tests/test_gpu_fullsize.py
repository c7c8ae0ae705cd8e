"""Full-size ELLPACK X^2 case (3D tight-binding N=262144, FP64, tau 1e-6) in the launch
configuration the benchmark times (sp2_step, automatic first pass, symmetric product) and
with full rows: sampled output rows against the oracle computed row by row, plus
properties that hold at any size (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_spgemm

pytestmark = pytest.mark.gpu

N, TAU = 262144, 1e-6


@pytest.fixture(scope="module")
def x1():
    """X = one SP2 step of H, built by the oracle (not by the CUDA path)."""
    O.set_threads(O.max_threads())
    try:
        H = O.Ell(*I.tight_binding(N, seed=0))
        lo, hi = O.gershgorin(H)
        X0 = O.x0(H, lo, hi, TAU)
        live = np.arange(X0.w)[None, :] < X0.nnz[:, None]
        t, t2 = O.trace(X0), float((np.where(live, X0.val, 0.0) ** 2).sum())
        up = abs(2 * t - t2 - N / 2) < abs(t2 - N / 2)
        X1 = O.spgemm(X0, X0, X0 if up else None, -1.0 if up else 1.0, 2.0 if up else 0.0, TAU)
    finally:
        O.set_threads(1)
    live = np.arange(X1.w)[None, :] < X1.nnz[:, None]
    return X1, O.trace(X1), float((np.where(live, X1.val, 0.0) ** 2).sum())


@pytest.mark.parametrize("symmetric", [True, False])
def test_fullsize_step_sampled_rows(gpu, x1, symmetric):
    """symmetric: the upper-triangle product mirrored (the benchmark's configuration)."""
    S = gpu
    X1, tr, tr2 = x1
    nocc = N / 2
    up = abs(2 * tr - tr2 - nocc) < abs(tr2 - nocc)
    alpha, beta = (-1.0, 2.0) if up else (1.0, 0.0)
    w = ((int(X1.nnz.max()) + 31) // 32) * 32
    idx = np.zeros((N, w), np.int32)
    val = np.full((N, w), np.nan)
    idx[:, :X1.w] = X1.idx
    val[:, :X1.w] = X1.val
    dX = S.Ellpack.from_numpy(idx, val, X1.nnz)
    probe = S.Ellpack.empty(N, 32)
    rc, info = S.sp2_step(dX, probe, nocc, TAU, traces=(tr, tr2), raise_on_overflow=False, symmetric=symmetric)
    assert rc == S.SP2E_OVERFLOW
    out = S.Ellpack.empty(N, ((info.required_width + 31) // 32) * 32)
    info = S.sp2_step(dX, out, nocc, TAU, traces=(tr, tr2), symmetric=symmetric)
    assert info.branch == (2 if up else 1)
    g = out.to_numpy()
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, 1, N // 2, N - 2, N - 1], rng.choice(N, 1500, replace=False)]))
    rep = compare_spgemm(g, X1, X1, X1, alpha, beta, TAU, rows=rows)
    assert rep["entries"] > 1500 * 100
    # properties at full size: the product of a symmetric X is symmetric; sorted rows;
    # reductions agree with the stored result
    gi, gv, gn = g
    for i in rows[:300]:
        for j, v in zip(gi[i, :gn[i]][:20], gv[i, :gn[i]][:20]):
            cols = gi[j, :gn[j]]
            p = np.searchsorted(cols, i)
            assert p < len(cols) and cols[p] == i
            assert abs(gv[j, p] - v) <= 1e-12 * max(1.0, abs(v))
    assert info.nnz_total == int(gn.sum())
    assert info.max_row_nnz == int(gn.max())
    live = np.arange(gi.shape[1])[None, :] < gn[:, None]
    assert info.trXn2 == pytest.approx(float((np.where(live, gv, 0.0) ** 2).sum()), rel=1e-12)
