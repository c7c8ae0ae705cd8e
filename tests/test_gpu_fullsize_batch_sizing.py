"""The two remaining workloads at their full configuration (GPU):
  - 256 gapped open 3D clusters, N log-uniform in [512, 8192] (sum N about 7.9e5), in one
    graph-captured batched launch: FP64 matrix by matrix against the oracle (iterations,
    branches, D entry by entry), mixed precision within 1e-5 of the oracle's D;
  - the gapped 3D tight-binding H of N = 1048576 sites (input width 128) with the learned
    row-length sizing: the last FP64 update's rows, sampled, against the oracle's product
    of the previous iterate computed row by row; mixed precision with the learned sizing
    within 1e-5 of FP64, and bitwise the mixed run with heuristic sizing (the sizing moves
    no result)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_density, compare_spgemm, sparse_fro, sparse_of

pytestmark = pytest.mark.gpu


def test_batched_256_clusters_against_oracle(gpu):
    S = gpu
    tau, tol = 1e-5, 1e-10
    sizes = I.cluster_sizes(256, 512, 8192, seed=0)
    mats = [O.Ell(*I.tight_binding(int(m), seed=k, delta=10.0, periodic=False)) for k, m in enumerate(sizes)]
    Hs = [S.Ellpack.from_numpy(m.idx, m.val, m.nnz) for m in mats]
    noccs = [(m.n + 1) // 2 for m in mats]  # the A sublattice's states: the gap stays at nocc
    D64, s64 = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, graph=1))
    Dmx, smx = S.sp2_purify_batched(Hs, noccs, tol, S.sp2_options_default(tau=tau, graph=1,
                                                                         precision=S.SP2_PREC_MIXED))
    O.set_threads(O.max_threads())
    worst_mixed = 0.0
    try:
        for m, H in enumerate(mats):
            Do, so = O.sp2(H, noccs[m], tol, tau)
            st = s64[m]
            assert (st["iterations"], st["branch"], st["status"]) == (so["iterations"], so["branch"], so["status"]), m
            compare_density(D64[m].to_numpy(), Do, tau)
            ref = sparse_of(Do.idx, Do.val, Do.nnz, H.n)
            dm = sparse_fro(sparse_of(*Dmx[m].to_numpy(), H.n) - ref) / math.sqrt(H.n)
            worst_mixed = max(worst_mixed, dm)
            assert dm <= 1e-5, (m, dm)
    finally:
        O.set_threads(1)
    print("256 clusters (sum N = %d): FP64 per entry within 1e-12 of scale; mixed worst %.3e" % (
        int(sizes.sum()), worst_mixed))


def test_learned_sizing_full_size(gpu):
    S = gpu
    from paper_2102_08505_gb300 import learned
    n, tau, tol = 1048576, 1e-5, 1e-10
    feat, counts = learned.default_training_set(seed=100, rows=50000, tau=tau, dtype=S.SP2_F32)
    pred, _ = learned.train(feat, counts, seed=0, steps=1500, batch=2048, lr=2e-3)
    idx, val, nnz = I.tight_binding(n, seed=0, delta=10.0, width=128)
    H = S.Ellpack.from_numpy(idx, val, nnz)
    # FP64 with the learned sizing, and the same run stopped one update earlier
    opt = S.sp2_options_default(tau=tau, sizing=2, predictor=pred)
    D, st = S.sp2_purify(H, n / 2, tol, opt)
    K = st["iterations"]
    Xp, sp = S.sp2_purify(H, n / 2, tol, S.sp2_options_default(tau=tau, sizing=2, predictor=pred, max_iter=K - 1),
                          allow_notconv=True)
    assert sp["iterations"] == K - 1 and sp["branch"] == st["branch"][:K - 1]
    up = st["branch"][K - 1] == "2X-X2"
    xi, xv, xn = Xp.to_numpy()
    X = O.Ell(xi, xv, xn)
    rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(3).choice(n, 1500, replace=False)]))
    O.set_threads(O.max_threads())
    try:
        rep = compare_spgemm(D.to_numpy(), X, X, X if up else None, -1.0 if up else 1.0, 2.0 if up else 0.0, tau,
                             rows=rows)
    finally:
        O.set_threads(1)
    assert rep["entries"] > 0
    # mixed precision, learned and heuristic sizing
    Dml, sml = S.sp2_purify(H, n / 2, tol, S.sp2_options_default(tau=tau, sizing=2, predictor=pred,
                                                                   precision=S.SP2_PREC_MIXED))
    Dmh, smh = S.sp2_purify(H, n / 2, tol, S.sp2_options_default(tau=tau, precision=S.SP2_PREC_MIXED))
    assert sml["iterations"] == smh["iterations"] and sml["branch"] == smh["branch"]
    a, b = Dml.to_numpy(), Dmh.to_numpy()
    assert np.array_equal(a[2], b[2])
    w = int(a[2].max())  # both results hold their rows in the first w slots
    live = np.arange(w)[None, :] < a[2][:, None]
    assert np.array_equal(np.where(live, a[0][:, :w], 0), np.where(live, b[0][:, :w], 0))
    assert np.array_equal(np.where(live, a[1][:, :w], 0), np.where(live, b[1][:, :w], 0))
    ref = sparse_of(*D.to_numpy(), n)
    dm = sparse_fro(sparse_of(*a, n) - ref) / math.sqrt(n)
    print("N=%d: FP64 %d iterations, last update per entry worst ratio %.3g; mixed %d (fp32 %d), dD %.3e; "
          "widths learned %d heuristic %d" % (n, K, rep["worst_ratio"], sml["iterations"], sml["fp32_iterations"], dm,
                                              sml["width_max"], smh["width_max"]))
    assert dm <= 1e-5
    assert sml["width_max"] < smh["width_max"]  # the learned widths are the tighter ones
