"""The seeded input generators follow the recipes they state: ELLPACK layout, exact symmetry,
the tight-binding law (density, cutoff, hopping, onsite spread, A/B splitting, Morton order),
the two-level chain model and the cluster-size mix (CPU)."""
import math

import numpy as np
import pytest

from paper_2102_08505_gb300 import inputs as I


def check_ellpack(idx, val, nnz, n):
    w = idx.shape[1]
    assert idx.shape == val.shape == (n, w) and nnz.shape == (n,)
    assert w % 32 == 0 and nnz.max() <= w
    for i in range(n):
        c = idx[i, :nnz[i]]
        assert np.all(np.diff(c) > 0), i          # sorted, no duplicates
        assert c.min() >= 0 and c.max() < n
        assert np.all(idx[i, nnz[i]:] == 0) and np.all(np.isnan(val[i, nnz[i]:]))


def dense(idx, val, nnz, n):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, idx[i, :nnz[i]]] = val[i, :nnz[i]]
    return D


def test_banded_layout_symmetry_and_gap_splitting():
    n, band = 300, 7
    idx, val, nnz = I.banded(n, band=band, seed=3)
    check_ellpack(idx, val, nnz, n)
    D = dense(idx, val, nnz, n)
    assert np.array_equal(D, D.T)
    i, j = np.nonzero(D)
    assert np.abs(i - j).max() == band
    assert np.all((np.diag(D) >= -2.0) & (np.diag(D) <= 0.0))
    Dg = dense(*I.banded(n, band=band, seed=3, delta=10.0), n)
    shift = np.diag(Dg) - np.diag(D)
    assert np.allclose(shift[0::2], -5.0) and np.allclose(shift[1::2], 5.0)
    assert np.array_equal(Dg - np.diag(np.diag(Dg)), D - np.diag(np.diag(D)))


@pytest.mark.parametrize("periodic", [True, False])
def test_tight_binding_law(periodic):
    """Every pair closer than the cutoff is coupled by -exp(-r/1.5) (minimum image when
    periodic), no other pair is, and the sites come in Morton order."""
    n = 600
    (idx, val, nnz), pos = I.tight_binding(n, seed=5, periodic=periodic, return_positions=True)
    check_ellpack(idx, val, nnz, n)
    H = dense(idx, val, nnz, n)
    assert np.array_equal(H, H.T)
    L = (n / 0.1) ** (1.0 / 3.0)
    d = pos[:, None, :] - pos[None, :, :]
    if periodic:
        d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(axis=2))
    off = ~np.eye(n, dtype=bool)
    near = (r < 4.0) & off
    assert np.array_equal(H[off] != 0.0, near[off])
    assert np.allclose(H[near], -np.exp(-r[near] / 1.5), rtol=1e-14, atol=0)
    # Morton order of the 4 A cells
    q = np.floor(pos / 4.0).astype(np.int64)
    q -= q.min(axis=0)

    def code(x):
        c = 0
        for b in range(21):
            for a in range(3):
                c |= ((int(x[a]) >> b) & 1) << (3 * b + a)
        return c
    codes = [code(x) for x in q]
    assert all(a <= b for a, b in zip(codes, codes[1:]))


def test_tight_binding_statistics_and_splitting():
    """Mean coordination of the periodic law at density 0.1/A^3 and cutoff 4 A is
    (4/3) pi 4^3 * 0.1 = 26.8 neighbours, plus the diagonal; onsite N(0, 0.5); the A/B
    splitting moves even sites by -delta/2 and odd sites by +delta/2 and nothing else."""
    n = 8000
    idx, val, nnz = I.tight_binding(n, seed=2)
    expect = 1.0 + 4.0 / 3.0 * math.pi * 4.0 ** 3 * 0.1
    assert abs(nnz.mean() - expect) < 0.3
    diag = np.array([val[i, np.searchsorted(idx[i, :nnz[i]], i)] for i in range(n)])
    assert abs(diag.mean()) < 0.03 and abs(diag.std() - 0.5) < 0.02
    idx2, val2, nnz2 = I.tight_binding(n, seed=2, delta=10.0)
    assert np.array_equal(idx, idx2) and np.array_equal(nnz, nnz2)
    diag2 = np.array([val2[i, np.searchsorted(idx2[i, :nnz2[i]], i)] for i in range(n)])
    assert np.allclose((diag2 - diag)[0::2], -5.0) and np.allclose((diag2 - diag)[1::2], 5.0)
    mask = np.ones_like(val, dtype=bool)
    for i in range(n):
        mask[i, np.searchsorted(idx[i, :nnz[i]], i)] = False
        mask[i, nnz[i]:] = False
    assert np.array_equal(val[mask], val2[mask])


def test_generators_are_seeded():
    for make in (lambda s: I.banded(200, band=5, seed=s), lambda s: I.tight_binding(700, seed=s),
                 lambda s: I.random_sparse(100, seed=s, max_nnz=9)):
        a, b, c = make(1), make(1), make(2)
        assert all(np.array_equal(x, y, equal_nan=True) for x, y in zip(a, b))
        assert not all(np.array_equal(x, y, equal_nan=True) for x, y in zip(a, c))


def test_model_chain_couplings():
    """Without noise: onsite eps_a on even and eps_b on odd orbitals; A-A, B-B and A-B
    couplings d * exp(k |m - m'|) between chain positions m, m'; entries whose decayed
    magnitude falls below the cutoff are not stored."""
    n, k = 80, -0.5
    p = dict(eps_a=-10.0, eps_b=0.5, d_aa=-1.0, d_bb=-2.0, d_ab=-3.0, k=k, r=0.0)
    idx, val, nnz = I.model_chain(n, cutoff=1e-3, **p)
    check_ellpack(idx, val, nnz, n)
    H = dense(idx, val, nnz, n)
    assert np.array_equal(H, H.T)
    want = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            ma, mb = a // 2, b // 2
            dist = abs(ma - mb)
            if a == b:
                want[a, b] = p["eps_a"] if a % 2 == 0 else p["eps_b"]
                continue
            if a % 2 != b % 2:
                coup = p["d_ab"]
            else:
                coup = p["d_aa"] if a % 2 == 0 else p["d_bb"]
            if dist == 0 and a % 2 == b % 2:
                continue
            f = math.exp(k * dist)
            if dist > 0 and 3.0 * f < 1e-3:  # beyond the largest coupling's cutoff range
                continue
            want[a, b] = coup * f
    assert np.allclose(H, want, rtol=1e-14, atol=0)
    # noise r perturbs every parameter within param * (1 +- r)
    Hn = dense(*I.model_chain(n, cutoff=1e-3, seed=4, **dict(p, r=0.1)), n)
    nz = want != 0
    ratio = Hn[nz] / want[nz]
    assert np.all((ratio >= 0.9 - 1e-12) & (ratio <= 1.1 + 1e-12)) and np.any(ratio != 1.0)


def test_cluster_sizes_log_uniform():
    s = I.cluster_sizes(4000, 512, 8192, seed=0)
    assert s.min() >= 512 and s.max() <= 8192 and len(s) == 4000
    lg = np.log(s)
    mid = 0.5 * (math.log(512) + math.log(8192))
    assert abs(lg.mean() - mid) < 0.05
    # uniform in log: each quarter of the log range holds about a quarter of the sizes
    edges = np.linspace(math.log(512), math.log(8192), 5)
    counts = np.histogram(lg, edges)[0]
    assert np.all(np.abs(counts - 1000) < 120)
