"""Element-by-element comparison of CUDA-path results with the CPU oracle.

Tolerances (derived from the arithmetic, written here once):
  FP64: |g - o| <= 1e-12 * S_ij, S_ij = |alpha| sum_k |a_ik b_kj| + |beta c_ij|, the
        scale of the dot-product error bound; column sets identical at tau = 0; at
        tau > 0 an entry may be present on one side only if its exact value lies within
        that bound of tau.
  FP32: |g - o| <= (m_ij + 4) * 2^-23 * S_ij with m_ij the number of terms of the entry
        (rounding of the inputs to FP32 plus one rounding per FMA, doubled for margin).
"""
import numpy as np

from oracle import oracle as O

F64_REL = 1e-12
U32 = 2.0 ** -23


def sorted_rows_ok(idx, nnz):
    for i in range(len(nnz)):
        c = idx[i, :nnz[i]]
        if len(c) > 1 and not np.all(np.diff(c) > 0):
            return False
    return True


def coo(idx, val, nnz, rows=None):
    """(keys = row*n_cols_bound + col, values) over the listed rows (all if None)."""
    rows = np.arange(len(nnz)) if rows is None else np.asarray(rows)
    ks, vs = [], []
    for r_out, i in enumerate(rows):
        k = int(nnz[i])
        ks.append(np.int64(r_out) * (1 << 32) + idx[i, :k].astype(np.int64))
        vs.append(val[i, :k].astype(np.float64))
    if not ks:
        return np.zeros(0, np.int64), np.zeros(0)
    return np.concatenate(ks), np.concatenate(vs)


def _abs(E):
    return O.Ell(E.idx, np.abs(E.val), E.nnz)


def _ones(E):
    return O.Ell(E.idx, np.where(np.isnan(E.val), np.nan, 1.0), E.nnz)


def _lookup(keys, vals, q):
    pos = np.searchsorted(keys, q)
    pos = np.minimum(pos, len(keys) - 1)
    ok = len(keys) > 0 and True
    found = (keys[pos] == q) if len(keys) else np.zeros(len(q), bool)
    return found, np.where(found, vals[pos] if len(keys) else 0.0, 0.0)


def compare_spgemm(gpu, A, B, C, alpha, beta, tau, fp32=False, rows=None, report=None):
    """gpu = (idx, val, nnz) numpy arrays of the CUDA result (all rows).  A, B, C are
    oracle Ell matrices (C may be None).  rows: compare only these product rows.
    Returns a dict of statistics; raises AssertionError on a violation."""
    gidx, gval, gnnz = gpu
    use_c = C is not None and beta != 0.0
    Cc = C if use_c else None
    ref = O.spgemm(A, B, Cc, alpha, beta, tau, rows=rows)
    full = O.spgemm(A, B, Cc, alpha, beta, 0.0, rows=rows)
    scale = O.spgemm(_abs(A), _abs(B), _abs(Cc) if use_c else None, abs(alpha), abs(beta), 0.0, rows=rows)
    terms = O.spgemm(_ones(A), _ones(B), _ones(Cc) if use_c else None, 1.0, 1.0 if use_c else 0.0, 0.0, rows=rows)
    sel = np.arange(len(gnnz)) if rows is None else np.asarray(rows)
    assert sorted_rows_ok(gidx[sel], gnnz[sel]), "GPU rows not strictly sorted"
    gk, gv = coo(gidx, gval, gnnz, sel)
    rk, rv = coo(ref.idx, ref.val, ref.nnz)
    fk, fv = coo(full.idx, full.val, full.nnz)
    sk, sv = coo(scale.idx, scale.val, scale.nnz)
    tk, tv = coo(terms.idx, terms.val, terms.nnz)
    assert np.array_equal(fk, sk) and np.array_equal(fk, tk)
    bound_all = (tv + 4.0) * U32 * sv if fp32 else F64_REL * sv
    bound_all = bound_all + 1e-300
    # entries present on the GPU must be structural entries
    found, _ = _lookup(fk, fv, gk)
    assert found.all(), "GPU produced %d non-structural entries" % int((~found).sum())
    pos_g = np.searchsorted(fk, gk)
    in_ref = np.isin(gk, rk, assume_unique=True)
    # common entries: values
    common = gk[in_ref]
    cg = gv[in_ref]
    cr = rv[np.searchsorted(rk, common)]
    cb = bound_all[pos_g[in_ref]]
    diff = np.abs(cg - cr)
    bad = diff > cb
    assert not bad.any(), "%d values out of tolerance; worst ratio %.3g" % (int(bad.sum()), float((diff / cb).max()))
    # set differences: only near tau
    g_only = ~in_ref
    r_only = ~np.isin(rk, gk, assume_unique=True)
    if tau == 0.0:
        assert not g_only.any() and not r_only.any(), "column sets differ at tau = 0 (%d extra, %d missing)" % (
            int(g_only.sum()), int(r_only.sum()))
    else:
        if g_only.any():
            p = pos_g[g_only]
            assert np.all(np.abs(np.abs(fv[p]) - tau) <= bound_all[p]), "GPU kept an entry clearly below tau"
        if r_only.any():
            p = np.searchsorted(fk, rk[r_only])
            assert np.all(np.abs(np.abs(fv[p]) - tau) <= bound_all[p]), "GPU dropped an entry clearly above tau"
    worst = float((diff / cb).max()) if len(diff) else 0.0
    out = {"entries": int(len(gk)), "worst_ratio": worst, "max_abs_diff": float(diff.max()) if len(diff) else 0.0,
           "flips": int(g_only.sum() + r_only.sum())}
    if report is not None:
        report.update(out)
    return out


def dense_of(idx, val, nnz, n):
    M = np.zeros((n, n))
    for i in range(n):
        k = int(nnz[i])
        M[i, idx[i, :k]] = val[i, :k]
    return M


def sparse_of(idx, val, nnz, n):
    """scipy CSR copy of an ELLPACK matrix, for comparisons at sizes a dense copy cannot hold."""
    import scipy.sparse as sp
    live = np.arange(idx.shape[1])[None, :] < np.asarray(nnz)[:, None]
    rows = np.repeat(np.arange(n), np.asarray(nnz, dtype=np.int64))
    return sp.csr_matrix((np.asarray(val, dtype=np.float64)[live], (rows, idx[live].astype(np.int64))), shape=(n, n))


def sparse_fro(M):
    """Frobenius norm of a scipy sparse matrix."""
    return float(np.sqrt((M.multiply(M)).sum()))


def compare_density(gpu, Do, tau, rows=None, rel=F64_REL):
    """Per-entry check of an FP64 SP2 result against the oracle's D (Do, an oracle Ell).

    The scale of entry (i, j) is S_ij = (|D| |D|)_ij + |D_ij| from the oracle's D: at
    convergence D is close to the last iterate X, so S_ij is the error-bound scale of the
    last update (X^2 or 2X - X^2) at that entry.  Values of entries stored on both sides
    must agree within rel * S_ij; an entry may be stored on one side only if its magnitude
    lies within rel * S_ij of tau (the drop decision there depends on rounding).
    rows: compare only these rows (all if None).  Returns statistics."""
    gidx, gval, gnnz = gpu
    sel = np.arange(len(gnnz)) if rows is None else np.asarray(rows)
    absD = _abs(Do)
    scale = O.spgemm(absD, absD, absD, 1.0, 1.0, 0.0, rows=sel)
    gk, gv = coo(gidx, gval, gnnz, sel)
    rk, rv = coo(Do.idx, Do.val, Do.nnz, sel)
    sk, sv = coo(scale.idx, scale.val, scale.nnz)
    assert sorted_rows_ok(gidx[sel], gnnz[sel]), "GPU rows not strictly sorted"
    bound_g = rel * _lookup(sk, sv, gk)[1] + 1e-300
    found, _ = _lookup(sk, sv, gk)
    assert found.all(), "GPU stores %d entries outside the pattern of D^2 + D" % int((~found).sum())
    in_ref = np.isin(gk, rk, assume_unique=True)
    cr = rv[np.searchsorted(rk, gk[in_ref])]
    diff = np.abs(gv[in_ref] - cr)
    bad = diff > bound_g[in_ref]
    assert not bad.any(), "%d entries of D out of tolerance; worst ratio %.3g" % (
        int(bad.sum()), float((diff / bound_g[in_ref]).max()))
    g_only = ~in_ref
    r_only = ~np.isin(rk, gk, assume_unique=True)
    if tau == 0.0:
        assert not g_only.any() and not r_only.any(), "column sets of D differ at tau = 0"
    else:
        if g_only.any():
            assert np.all(np.abs(np.abs(gv[g_only]) - tau) <= bound_g[g_only]), "GPU kept an entry of D clearly below tau"
        if r_only.any():
            b = rel * _lookup(sk, sv, rk[r_only])[1] + 1e-300
            assert np.all(np.abs(np.abs(rv[r_only]) - tau) <= b), "GPU dropped an entry of D clearly above tau"
    return {"entries": int(len(gk)), "worst_ratio": float((diff / bound_g[in_ref]).max()) if len(diff) else 0.0,
            "max_abs_diff": float(diff.max()) if len(diff) else 0.0, "flips": int(g_only.sum() + r_only.sum())}
