"""Seeded synthetic inputs (Hamiltonians and random sparse matrices) in ELLPACK form.

This module holds no step of the method: it only draws matrices.  Both the CUDA path
and the CPU oracle consume what it returns (plain numpy arrays), so it is the one
module the two share.

ELLPACK arrays (row-major, the storage of the paper's allocation listing, Section
"Micro-Kernel Performance Evaluation - NUMA Aware Data"):
  idx int32[n, w], val float64[n, w], nnz int32[n]; row i holds nnz[i] entries, sorted
  by column.  Padding slots hold column 0 and a NaN value so that any reader that looks
  past nnz[i] produces visibly wrong results.

Workloads:
  banded        -- symmetric banded H: diagonal ~U(-2, 0), off-diagonals
                   exp(-|i-j|/4) * U(-1, 1) for |i-j| <= band.  With delta > 0 an A/B
                   onsite splitting (-delta/2 on even rows, +delta/2 on odd rows) opens a
                   gap, the two-level A/B mechanism of the paper's model Hamiltonians
                   (Section "On the Generation of Model Hamiltonian System Matrices").
  tight_binding -- sites uniform in a cube at a given density (periodic or open),
                   hopping -exp(-r/decay) for r < rcut, onsite ~N(0, sigma); sites are
                   ordered by the Morton code of a cubic cell grid; optional A/B onsite
                   splitting on even/odd site index.
  model_chain   -- the paper's two-level A/B chain model Hamiltonian (same section).
  random_sparse -- unstructured random square matrices for unit tests.
"""
import math

import numpy as np

PAD_VAL = float("nan")


def round_up(x, m=32):
    return max(m, ((int(x) + m - 1) // m) * m)


def coo_to_ellpack(n, rows, cols, vals, width=None, multiple=32):
    """Sorted ELLPACK arrays from COO triplets without duplicates."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    vals = np.asarray(vals, np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    nnz = np.bincount(rows, minlength=n).astype(np.int32)
    mx = int(nnz.max()) if n else 0
    w = round_up(mx, multiple) if width is None else int(width)
    if mx > w:
        raise ValueError("row with %d entries does not fit width %d" % (mx, w))
    start = np.zeros(n + 1, np.int64)
    np.cumsum(nnz, out=start[1:])
    slot = np.arange(len(rows), dtype=np.int64) - start[rows]
    idx = np.zeros((n, w), np.int32)
    val = np.full((n, w), PAD_VAL, np.float64)
    idx[rows, slot] = cols
    val[rows, slot] = vals
    return idx, val, nnz


def banded(n=1024, band=16, seed=1, delta=0.0, width=None):
    """Symmetric banded Hamiltonian (see module docstring)."""
    rng = np.random.default_rng(seed)
    diag = rng.uniform(-2.0, 0.0, n)
    if delta:
        diag = diag + np.where(np.arange(n) % 2 == 0, -0.5 * delta, 0.5 * delta)
    r, c, v = [np.arange(n)], [np.arange(n)], [diag]
    for d in range(1, band + 1):
        m = n - d
        if m <= 0:
            break
        off = math.exp(-d / 4.0) * rng.uniform(-1.0, 1.0, m)
        i = np.arange(m)
        r += [i, i + d]
        c += [i + d, i]
        v += [off, off]
    return coo_to_ellpack(n, np.concatenate(r), np.concatenate(c), np.concatenate(v), width)


def _spread_bits(x):
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton_order(pos, cell):
    """Stable permutation sorting points by the Morton code of their grid cell."""
    q = np.floor(pos / cell).astype(np.int64)
    q -= q.min(axis=0)
    code = _spread_bits(q[:, 0]) | (_spread_bits(q[:, 1]) << np.uint64(1)) | (_spread_bits(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def tight_binding(n, seed=0, density=0.1, rcut=4.0, decay=1.5, onsite_sigma=0.5, periodic=True,
                  delta=0.0, morton=True, cell=4.0, width=None, return_positions=False):
    """3D tight-binding Hamiltonian (see module docstring)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    L = (n / density) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, L, (n, 3))
    onsite = rng.normal(0.0, onsite_sigma, n)
    if periodic and L <= 2.0 * rcut:
        raise ValueError("periodic box %.2f too small for cutoff %.2f" % (L, rcut))
    if morton:
        perm = morton_order(pos, cell)
        pos, onsite = pos[perm], onsite[perm]
    if delta:
        onsite = onsite + np.where(np.arange(n) % 2 == 0, -0.5 * delta, 0.5 * delta)
    pos = np.mod(pos, L) if periodic else pos
    tree = cKDTree(pos, boxsize=L if periodic else None)
    pairs = tree.query_pairs(rcut, output_type="ndarray")
    d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    if periodic:
        d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(axis=1))
    hop = -np.exp(-r / decay)
    i, j = pairs[:, 0], pairs[:, 1]
    rows = np.concatenate([np.arange(n), i, j])
    cols = np.concatenate([np.arange(n), j, i])
    vals = np.concatenate([onsite, hop, hop])
    out = coo_to_ellpack(n, rows, cols, vals, width)
    return (out, pos) if return_positions else out


def cluster_sizes(count=256, lo=512, hi=8192, seed=0):
    """Sizes log-uniform in [lo, hi] (rounded to the nearest integer)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


def model_chain(n, eps_a=0.0, eps_b=0.0, d_aa=0.0, d_bb=0.0, d_ab=0.0, k=-0.01, r=0.0,
                seed=0, cutoff=1e-5, max_range=None, width=None):
    """The paper's two-level A/B chain: orbitals 2m (A) and 2m+1 (B) sit at chain
    position m; onsite energies eps_a / eps_b; same-type couplings d_aa / d_bb and A-B
    couplings d_ab between positions m and m', each times exp(k |m - m'|); every
    parameter is perturbed as param * (1 + r * U(-1, 1)).  Couplings whose decayed
    magnitude is below `cutoff` are not stored."""
    rng = np.random.default_rng(seed)
    npos = n // 2
    if n % 2:
        raise ValueError("n must be even (one A and one B orbital per site)")
    kmax = npos - 1
    if k < 0 and cutoff > 0:
        big = max(abs(d_aa), abs(d_bb), abs(d_ab), 1e-300)
        kmax = min(kmax, int(math.floor(math.log(cutoff / big) / k)))
    if max_range is not None:
        kmax = min(kmax, int(max_range))

    def noisy(p, size):
        return p * (1.0 + r * rng.uniform(-1.0, 1.0, size))

    rows, cols, vals = [], [], []
    m = np.arange(npos)
    onsite = np.empty(n)
    onsite[0::2] = noisy(eps_a, npos)
    onsite[1::2] = noisy(eps_b, npos)
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(onsite)
    # A-B coupling on the same site
    if d_ab:
        v = noisy(d_ab, npos)
        rows += [2 * m, 2 * m + 1]; cols += [2 * m + 1, 2 * m]; vals += [v, v]
    for dist in range(1, kmax + 1):
        mm = np.arange(npos - dist)
        f = math.exp(k * dist)
        for (p, da, db) in ((d_aa, 0, 0), (d_bb, 1, 1), (d_ab, 0, 1), (d_ab, 1, 0)):
            if not p:
                continue
            v = noisy(p, npos - dist) * f
            a, b = 2 * mm + da, 2 * (mm + dist) + db
            rows += [a, b]; cols += [b, a]; vals += [v, v]
    return coo_to_ellpack(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), width)


def random_sparse(n, seed=0, min_nnz=0, max_nnz=8, width=None, symmetric=False, full_rows=(),
                  empty_rows=(), value_scale=1.0):
    """Random square sparse matrix with a ragged row-length mix for unit tests.
    `full_rows` get exactly `width` (or max_nnz) entries, `empty_rows` none."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        if i in empty_rows:
            k = 0
        elif i in full_rows:
            k = min(n, max_nnz)
        else:
            k = int(rng.integers(min_nnz, max_nnz + 1))
        k = min(k, n)
        c = rng.choice(n, size=k, replace=False)
        rows.append(np.full(k, i))
        cols.append(c)
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = value_scale * rng.uniform(-1.0, 1.0, len(rows))
    if symmetric:
        key = {}
        for a, b, v in zip(rows, cols, vals):
            key[(int(min(a, b)), int(max(a, b)))] = v
        rr, cc, vv = [], [], []
        for (a, b), v in key.items():
            rr.append(a); cc.append(b); vv.append(v)
            if a != b:
                rr.append(b); cc.append(a); vv.append(v)
        rows, cols, vals = np.array(rr, np.int64), np.array(cc, np.int64), np.array(vv)
    return coo_to_ellpack(n, rows, cols, vals, width)
