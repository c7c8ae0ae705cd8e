"""ctypes front end of the CPU FP64 oracle, plus numpy checks.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  It shares no code with the CUDA library; its
inputs are plain numpy arrays in the ELLPACK layout (per row i: nnz[i] stored entries in
idx[i, :nnz[i]] / val[i, :nnz[i]]; the slots past nnz[i] are never read), the storage of
the paper's allocation listing (Section "Micro-Kernel Performance Evaluation - NUMA
Aware Data").

Which passage each function follows:
  spgemm     -- the thresholded ELLPACK matrix-matrix multiply ("BML ELLPACK
                matrix-matrix multiply", Section "Performance Evaluation using System
                Matrices"), as its plain definition (see sp2_oracle.c).
  add, drop  -- the "SP2 Loop Misc" update and the drop tolerance (Section "Performance
                Evaluation using an ExaSP2 Application").
  trace      -- the "SP2 Loop Norm" quantities (same section).
  gershgorin, x0, sp2 -- SP2-Basic (same section) following the published SP2 recursion
                (Niklasson 2002, cited in the Introduction).
  eigen_projector / checks -- the exact answer SP2 approximates: the projector onto the
                nocc lowest eigenvectors of H (dense eigendecomposition, as used for the
                total density of states, Section "On the Generation of Model Hamiltonian
                System Matrices").
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _OrcEll(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("w", ctypes.c_int),
                ("idx", ctypes.POINTER(ctypes.c_int)), ("val", ctypes.POINTER(ctypes.c_double)),
                ("nnz", ctypes.POINTER(ctypes.c_int))]


class _OrcStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("trX", ctypes.POINTER(ctypes.c_double)), ("trX2", ctypes.POINTER(ctypes.c_double)),
                ("err", ctypes.POINTER(ctypes.c_double)), ("branch", ctypes.POINTER(ctypes.c_int)),
                ("nnz_total", ctypes.POINTER(ctypes.c_longlong)),
                ("max_row_nnz", ctypes.POINTER(ctypes.c_int))]


def _declare(L):
    P = ctypes.POINTER
    L.orc_spgemm.argtypes = [P(_OrcEll), P(_OrcEll), P(_OrcEll), ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, P(ctypes.c_int), ctypes.c_int, P(_OrcEll),
                             P(ctypes.c_int), P(ctypes.c_double)]
    L.orc_add.argtypes = [P(_OrcEll), P(_OrcEll), ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, P(_OrcEll), P(ctypes.c_int)]
    L.orc_drop.argtypes = [P(_OrcEll), ctypes.c_double, P(_OrcEll)]
    L.orc_trace.argtypes = [P(_OrcEll)]
    L.orc_trace.restype = ctypes.c_double
    L.orc_gershgorin.argtypes = [P(_OrcEll), P(ctypes.c_double), P(ctypes.c_double)]
    L.orc_x0.argtypes = [P(_OrcEll), ctypes.c_double, ctypes.c_double, ctypes.c_double, P(_OrcEll)]
    L.orc_sp2.argtypes = [P(_OrcEll), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int, ctypes.c_double, ctypes.c_double, P(_OrcEll), P(_OrcStats)]
    L.orc_free_ell.argtypes = [P(_OrcEll)]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_get_max_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


class use_variant:
    """Context manager: run the oracle functions on another build of sp2_oracle.c (used by
    the tests that plant a mistake in a copy of the oracle to show a pin catches it)."""

    def __init__(self, path):
        self.L = _declare(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        self.prev, _lib = lib(), self.L
        return self

    def __exit__(self, *a):
        global _lib
        _lib = self.prev


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def max_threads() -> int:
    return int(lib().orc_get_max_threads())


class Ell:
    """An ELLPACK matrix held in numpy arrays (n rows, width w)."""

    def __init__(self, idx, val, nnz):
        self.idx = np.ascontiguousarray(idx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.nnz = np.ascontiguousarray(nnz, dtype=np.int32)
        assert self.idx.ndim == 2 and self.idx.shape == self.val.shape
        assert self.nnz.shape == (self.idx.shape[0],)

    @property
    def n(self):
        return self.idx.shape[0]

    @property
    def w(self):
        return self.idx.shape[1]

    @staticmethod
    def empty(n, w):
        return Ell(np.zeros((n, w), np.int32), np.zeros((n, w), np.float64), np.zeros(n, np.int32))

    def _c(self, n_rows=None):
        s = _OrcEll()
        s.n = self.n if n_rows is None else n_rows
        s.w = self.w
        s.idx = self.idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        s.val = self.val.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.nnz = self.nnz.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        return s

    def row(self, i):
        k = int(self.nnz[i])
        return self.idx[i, :k], self.val[i, :k]

    def to_dense(self):
        """Dense n x n copy (explicit zeros in the pattern become 0.0)."""
        n = self.n
        M = np.zeros((n, n))
        for i in range(n):
            c, v = self.row(i)
            M[i, c] = v
        return M

    def pattern(self):
        """Set of (i, j) stored positions."""
        out = set()
        for i in range(self.n):
            for j in self.row(i)[0]:
                out.add((i, int(j)))
        return out


def from_dense(M, width=None, keep_zeros=False):
    """ELLPACK matrix holding the nonzeros (or every entry if keep_zeros) of M, sorted."""
    n = M.shape[0]
    rows = [np.nonzero(M[i])[0] if not keep_zeros else np.arange(n) for i in range(n)]
    w = max(1, max((len(r) for r in rows), default=1)) if width is None else width
    E = Ell.empty(n, w)
    for i, r in enumerate(rows):
        E.idx[i, :len(r)] = r
        E.val[i, :len(r)] = M[i, r]
        E.nnz[i] = len(r)
    return E


ORC_NOMEM = -3


def _check(rc):
    """Raises for a negative oracle status: -3 is out of host memory, others bad arguments."""
    if rc == ORC_NOMEM:
        raise MemoryError("oracle ran out of host memory")
    if rc < 0:
        raise ValueError("oracle rejected its arguments")


def _fit(call, n_rows, w0, n_cols_cap):
    w = max(1, min(int(w0), n_cols_cap))
    cnt = np.zeros(n_rows, np.int32)
    while True:
        out = Ell.empty(n_rows, w)
        rc = call(out, cnt)
        _check(rc)
        if rc == 0:
            return out, cnt
        w = int(cnt.max())


def spgemm(A, B, C=None, alpha=1.0, beta=0.0, tau=0.0, rows=None, with_diag=False):
    """drop_tau(alpha*A*B + beta*C) for all rows, or for the listed rows (output row r =
    product row rows[r])."""
    L = lib()
    a, b = A._c(), B._c()
    c = C._c() if C is not None else None
    if rows is None:
        nr, rp = A.n, None
        rows_arr = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int32)
        nr = len(rows_arr)
        rp = rows_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    diag = np.zeros(nr) if with_diag else None
    dp = diag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if with_diag else None
    w0 = min(A.n, max(1, 2 * max(A.w, B.w)))

    def call(out, cnt):
        o = out._c()
        return L.orc_spgemm(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c) if c is not None else None,
                            float(alpha), float(beta), float(tau), rp, nr, ctypes.byref(o),
                            cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), dp)

    out, cnt = _fit(call, nr, w0, A.n)
    return (out, diag) if with_diag else out


def add(A, B, alpha, beta, tau=0.0):
    """drop_tau(alpha*A + beta*B)."""
    L = lib()
    a, b = A._c(), B._c()

    def call(out, cnt):
        o = out._c()
        return L.orc_add(ctypes.byref(a), ctypes.byref(b), float(alpha), float(beta), float(tau),
                         ctypes.byref(o), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))

    return _fit(call, A.n, min(A.n, A.w + B.w), A.n)[0]


def drop(A, tau):
    L = lib()
    out = Ell.empty(A.n, A.w)
    a, o = A._c(), out._c()
    if L.orc_drop(ctypes.byref(a), float(tau), ctypes.byref(o)) != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def trace(A):
    a = A._c()
    return float(lib().orc_trace(ctypes.byref(a)))


def gershgorin(H):
    a = H._c()
    lo, hi = ctypes.c_double(), ctypes.c_double()
    if lib().orc_gershgorin(ctypes.byref(a), ctypes.byref(lo), ctypes.byref(hi)) != 0:
        raise ValueError("oracle rejected its arguments")
    return lo.value, hi.value


def x0(H, emin, emax, tau=0.0):
    out = Ell.empty(H.n, H.w + 1)
    a, o = H._c(), out._c()
    _check(lib().orc_x0(ctypes.byref(a), float(emin), float(emax), float(tau), ctypes.byref(o)))
    return out


def sp2(H, nocc, tol, tau=0.0, max_iter=100, stall=True, stall_arm=0.1, stall_ratio=1.0):
    """SP2 purification.  Returns (D, stats) where stats is a dict with the per-iteration
    trace, trace-of-square, error and branch sequences ("X2" / "2X-X2").  The stall rule
    (stall=True) arms once |trX - trX2| < stall_arm and fires when
    err_n >= stall_ratio * err_{n-2}."""
    L = lib()
    cap = max_iter + 1
    trX, trX2, err = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    branch = np.zeros(cap, np.int32)
    nnzt = np.zeros(cap, np.int64)
    mxr = np.zeros(cap, np.int32)
    st = _OrcStats()
    st.max_iter = max_iter
    P = ctypes.POINTER
    st.trX = trX.ctypes.data_as(P(ctypes.c_double))
    st.trX2 = trX2.ctypes.data_as(P(ctypes.c_double))
    st.err = err.ctypes.data_as(P(ctypes.c_double))
    st.branch = branch.ctypes.data_as(P(ctypes.c_int))
    st.nnz_total = nnzt.ctypes.data_as(P(ctypes.c_longlong))
    st.max_row_nnz = mxr.ctypes.data_as(P(ctypes.c_int))
    h = H._c()
    d = _OrcEll()
    rc = L.orc_sp2(ctypes.byref(h), float(nocc), float(tol), float(tau), int(max_iter),
                   float(stall_arm) if stall else 0.0, float(stall_ratio), ctypes.byref(d), ctypes.byref(st))
    _check(rc)
    n, w = d.n, d.w
    idx = np.ctypeslib.as_array(d.idx, shape=(n * w,)).reshape(n, w).copy()
    val = np.ctypeslib.as_array(d.val, shape=(n * w,)).reshape(n, w).copy()
    nnz = np.ctypeslib.as_array(d.nnz, shape=(n,)).copy()
    L.orc_free_ell(ctypes.byref(d))
    it = st.iterations
    stats = {
        "iterations": it,
        "status": {0: "converged", 1: "stalled", 2: "max_iter"}.get(st.status, "error"),
        "emin": st.emin, "emax": st.emax,
        "trX": trX[:it + 1].copy(), "trX2": trX2[:it + 1].copy(), "err": err[:it + 1].copy(),
        "branch": ["X2" if b == 1 else "2X-X2" for b in branch[:it]],
        "nnz_total": nnzt[:it + 1].copy(), "max_row_nnz": mxr[:it + 1].copy(),
    }
    return Ell(idx, val, nnz), stats


# ----------------------------------------------------------------- numpy checks

def eigen_projector(Hd, nocc):
    """D_eig = V[:, :nocc] V[:, :nocc]^T from the dense symmetric eigendecomposition."""
    w, V = np.linalg.eigh(Hd)
    Vo = V[:, :int(nocc)]
    return Vo @ Vo.T, w


def checks(Hd, Dd, nocc):
    """Errors of a dense density matrix against the exact projector and invariants."""
    n = Hd.shape[0]
    Pe, w = eigen_projector(Hd, nocc)
    return {
        "proj_err": float(np.linalg.norm(Dd - Pe) / np.sqrt(n)),
        "trace_err": float(abs(np.trace(Dd) - nocc)),
        "idem_err": float(np.linalg.norm(Dd @ Dd - Dd)),
        "comm_err": float(np.linalg.norm(Hd @ Dd - Dd @ Hd)),
        "gap": float(w[int(nocc)] - w[int(nocc) - 1]) if 0 < nocc < n else float("nan"),
    }


# ---------------------------------------------------------------- standalone ELLPACK ops
# Plain definitions of the library's standalone operations (scale, drop threshold,
# norms, transpose, dense conversion) on the stored entries of an Ell matrix.

def _live(A):
    return np.arange(A.w)[None, :] < A.nnz[:, None]


def scale(A, alpha):
    """alpha * A on the stored entries (pattern unchanged)."""
    B = Ell(A.idx.copy(), A.val.copy(), A.nnz.copy())
    lv = _live(A)
    B.val[lv] = A.val[lv] * alpha
    return B


def threshold(A, tau):
    """Keeps the stored entries with |v| > tau, in their order (tau = 0 drops exact zeros)."""
    B = Ell.empty(A.n, A.w)
    for i in range(A.n):
        j, v = A.row(i)
        keep = np.abs(v) > tau
        k = int(keep.sum())
        B.idx[i, :k] = j[keep]
        B.val[i, :k] = v[keep]
        B.nnz[i] = k
    return B


def norms(A):
    """(max |a_ij|, max_i sum_j |a_ij|, sqrt(sum a_ij^2)) over the stored entries."""
    lv = _live(A)
    a = np.where(lv, np.abs(A.val), 0.0)
    return float(a.max(initial=0.0)), float(a.sum(axis=1).max(initial=0.0)), float(np.sqrt((a * a).sum()))


def transpose(A, width=None):
    """A^T with rows sorted by column: the stored entries (i, j, v) become (j, i, v)."""
    lv = _live(A)
    rows = np.repeat(np.arange(A.n), A.nnz)
    cols = A.idx[lv]
    vals = A.val[lv]
    order = np.lexsort((rows, cols))
    cols, rows, vals = cols[order], rows[order], vals[order]
    cnt = np.bincount(cols, minlength=A.n).astype(np.int32)
    w = max(1, int(cnt.max(initial=0))) if width is None else width
    T = Ell.empty(A.n, w)
    start = np.concatenate([[0], np.cumsum(cnt)])
    for j in range(A.n):
        k = cnt[j]
        T.idx[j, :k] = rows[start[j]:start[j] + k]
        T.val[j, :k] = vals[start[j]:start[j] + k]
        T.nnz[j] = k
    return T


def from_dense_tau(M, tau, width=None):
    """ELLPACK of a dense matrix keeping v != 0 (tau = 0) or |v| > tau, in column order."""
    n = M.shape[0]
    rows = [np.nonzero(M[i] != 0)[0] if tau == 0 else np.nonzero(np.abs(M[i]) > tau)[0] for i in range(n)]
    w = max(1, max((len(r) for r in rows), default=1)) if width is None else width
    E = Ell.empty(n, w)
    for i, r in enumerate(rows):
        E.idx[i, :len(r)] = r
        E.val[i, :len(r)] = M[i, r]
        E.nnz[i] = len(r)
    return E
