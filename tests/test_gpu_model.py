"""The paper's model Hamiltonians (two-level A/B chain, Section "On the Generation of
Model Hamiltonian System Matrices"): X^2 of every parameter set against the oracle, and
SP2 of the semiconductor set, the one gapped at half filling (FP64 against the oracle;
mixed precision reported and held to 5e-3, the distance FP32 products can reach on a
chain whose gap is 1e-3 of its spectral width) (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_spgemm, dense_of

pytestmark = pytest.mark.gpu

SETS = {
    "metals": dict(d_aa=-1.0, d_bb=-1.0, k=-0.01),
    "semiconductor": dict(d_bb=-1.0, d_ab=-2.0, k=-0.01),
    "soft_matter": dict(d_bb=-1.0, d_ab=-1.0, eps_a=-10.0, k=-0.1, r=1.0),
}


@pytest.mark.parametrize("name", sorted(SETS))
def test_model_x2_matches_oracle(gpu, name):
    S = gpu
    n, tau = 1200, 1e-5
    H = O.Ell(*I.model_chain(n, seed=2, **SETS[name]))
    dH = S.Ellpack.from_numpy(H.idx, H.val, H.nnz)
    rc, req = S.ellpack_multiply(dH, dH, S.Ellpack.empty(n, 32), 1.0, 0.0, tau, raise_on_overflow=False)
    C = S.Ellpack.empty(n, ((req + 31) // 32) * 32)
    S.ellpack_multiply(dH, dH, C, 1.0, 0.0, tau)
    rows = np.unique(np.concatenate([[0, 1, n // 2, n - 1], np.random.default_rng(1).choice(n, 150, replace=False)]))
    rep = compare_spgemm(C.to_numpy(), H, H, None, 1.0, 0.0, tau, rows=rows)
    assert rep["entries"] > 0


def test_model_semiconductor_sp2(gpu):
    """The semiconductor set is the gapped one at half filling (gap 0.94 at N = 2000; the
    soft-matter and metal sets are gapless there).  SP2 stops by the stall rule.  FP64
    matches the oracle.  Mixed precision is reported, not held to 1e-5: the gap is 1e-3 of
    the spectral width, and the FP32 products of the first iterations already move D by
    ~5e-4 (a dense float32 emulation gives the same figure for every switch point), so
    this chain is outside what FP32 products can reach; the 1e-5 bar is met on the 3D
    gapped workload (test_gpu_sp2)."""
    S = gpu
    n, tau, tol = 1200, 1e-5, 1e-10
    H = O.Ell(*I.model_chain(n, seed=3, **SETS["semiconductor"]))
    O.set_threads(O.max_threads())
    try:
        Do, so = O.sp2(H, n // 2, tol, tau)
    finally:
        O.set_threads(1)
    dH = S.Ellpack.from_numpy(H.idx, H.val, H.nnz)
    D, sg = S.sp2_purify(dH, n // 2, tol, S.sp2_options_default(tau=tau), allow_notconv=True)
    assert sg["iterations"] == so["iterations"] and sg["branch"] == so["branch"] and sg["status"] == so["status"]
    Dr = Do.to_dense()
    assert np.linalg.norm(dense_of(*D.to_numpy(), n) - Dr) / np.sqrt(n) < 1e-10
    Dm, sm = S.sp2_purify(dH, n // 2, tol, S.sp2_options_default(tau=tau, precision=S.SP2_PREC_MIXED),
                          allow_notconv=True)
    dD = np.linalg.norm(dense_of(*Dm.to_numpy(), n) - Dr) / np.sqrt(n)
    print("semiconductor n=%d: fp64 %d iterations (%s), mixed %d (fp32 %d), dD %.2e" % (
        n, sg["iterations"], sg["status"], sm["iterations"], sm["fp32_iterations"], dD))
    assert dD <= 5e-3 and sm["status"] in ("converged", "stalled")
    assert abs(np.trace(dense_of(*Dm.to_numpy(), n)) - n // 2) < 1e-2
