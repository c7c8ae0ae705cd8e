"""Thin ctypes binding of libsp2ell.so (C ABI in include/sp2ell.h).

Argument marshalling only: every step of the computation runs in the CUDA library.
Device memory comes from torch tensors (wrapped, borrowed by the library) or from the
library itself (matrices returned by sp2_purify, released when their Python owner is
garbage-collected).  If the library is missing the import of this module raises; there
is no other code path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsp2ell.so")

SP2_OK = 0
SP2E_ARG, SP2E_OVERFLOW, SP2E_NOMEM, SP2E_CUDA, SP2E_NOTCONV, SP2E_NONFINITE, SP2E_TIMEOUT = -1, -2, -3, -4, -5, -6, -7
SP2_F64, SP2_F32 = 0, 1
SP2_PREC_F64, SP2_PREC_MIXED, SP2_PREC_F32 = 0, 1, 2
SP2_STATS_CAP = 256
SP2_PATH_TUNED = -1
_CODES = {0: "SP2_OK", -1: "SP2E_ARG", -2: "SP2E_OVERFLOW", -3: "SP2E_NOMEM", -4: "SP2E_CUDA",
          -5: "SP2E_NOTCONV", -6: "SP2E_NONFINITE", -7: "SP2E_TIMEOUT"}


class Sp2Error(RuntimeError):
    def __init__(self, code, message):
        super().__init__("%s: %s" % (_CODES.get(code, code), message))
        self.code = code


class ellpack_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("width", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("owner", ctypes.c_int32), ("idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("nnz", ctypes.c_void_p)]


NNZPRED_NPARAMS, NNZPRED_NSTATS = 5313, 35


class nnzpred_t(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("stats", ctypes.c_void_p), ("steps", ctypes.c_int64)]


class sp2_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("stall_rule", ctypes.c_int32),
                ("n_fp64_tail", ctypes.c_int32), ("max_width", ctypes.c_int32), ("spgemm_path", ctypes.c_int32),
                ("tau", ctypes.c_double), ("switch_tol", ctypes.c_double), ("graph", ctypes.c_int32),
                ("sizing", ctypes.c_int32), ("predictor", ctypes.POINTER(nnzpred_t)), ("stall_arm", ctypes.c_double),
                ("symmetric", ctypes.c_int32), ("stall_ratio", ctypes.c_double), ("route_rows", ctypes.c_int32),
                ("small_path", ctypes.c_int32), ("level_up_frac", ctypes.c_double)]


class sp2_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("fp32_iterations", ctypes.c_int32),
                ("regrows", ctypes.c_int32), ("struct_passes", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("width_max", ctypes.c_int32),
                ("pred_log_mae", ctypes.c_double), ("pred_under_frac", ctypes.c_double),
                ("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("time_ms", ctypes.c_double),
                ("trX", ctypes.c_double * SP2_STATS_CAP), ("trX2", ctypes.c_double * SP2_STATS_CAP),
                ("err", ctypes.c_double * SP2_STATS_CAP), ("branch", ctypes.c_int32 * SP2_STATS_CAP),
                ("nnz_total", ctypes.c_int64 * SP2_STATS_CAP), ("max_row_nnz", ctypes.c_int32 * SP2_STATS_CAP),
                ("rows_level1", ctypes.c_int32 * SP2_STATS_CAP), ("rows_level2", ctypes.c_int32 * SP2_STATS_CAP),
                ("rows_deferred", ctypes.c_int32 * SP2_STATS_CAP), ("rows_routed", ctypes.c_int32 * SP2_STATS_CAP),
                ("level", ctypes.c_int32 * SP2_STATS_CAP), ("small_iterations", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class sp2_step_info(ctypes.Structure):
    _fields_ = [("trX", ctypes.c_double), ("trX2", ctypes.c_double), ("have_traces", ctypes.c_int32),
                ("branch", ctypes.c_int32), ("err", ctypes.c_double), ("trXn", ctypes.c_double),
                ("trXn2", ctypes.c_double), ("nnz_total", ctypes.c_int64), ("max_row_nnz", ctypes.c_int32),
                ("required_width", ctypes.c_int32), ("spgemm_path", ctypes.c_int32),
                ("rows_deferred", ctypes.c_int32), ("rows_dense", ctypes.c_int32),
                ("spgemm_path_used", ctypes.c_int32), ("symmetric", ctypes.c_int32),
                ("compact_level", ctypes.c_int32)]


SP2_PROF_CLASSES = 6
PROF_NAMES = ("spgemm", "large_rows", "reduce", "other", "symmetry", "cascade")


class sp2_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("count", ctypes.c_int32 * SP2_PROF_CLASSES),
                ("total_ms", ctypes.c_double * SP2_PROF_CLASSES)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsp2ell.so is not built (run __graft_entry__.build() or "
                          "python paper_2102_08505_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P, V, I, D = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    E = P(ellpack_t)
    sig = {
        "sp2_version": ([], ctypes.c_int),
        "sp2_last_error_string": ([], ctypes.c_char_p),
        "sp2_release_memory": ([], ctypes.c_int),
        "ellpack_create": ([I, I, I, V, E], ctypes.c_int),
        "ellpack_wrap": ([I, I, I, V, V, V, E], ctypes.c_int),
        "ellpack_destroy": ([E, V], ctypes.c_int),
        "ellpack_upload": ([E, V, V, V, V], ctypes.c_int),
        "ellpack_download": ([E, V, V, V, V], ctypes.c_int),
        "ellpack_download_async": ([E, V, V, V, V], ctypes.c_int),
        "ellpack_copy": ([E, E, V], ctypes.c_int),
        "ellpack_multiply": ([E, E, E, D, D, D, V, P(I)], ctypes.c_int),
        "ellpack_add": ([E, E, D, D, D, V, P(I)], ctypes.c_int),
        "ellpack_trace": ([E, P(D), V], ctypes.c_int),
        "ellpack_frobenius2": ([E, P(D), V], ctypes.c_int),
        "ellpack_gershgorin": ([E, P(D), P(D), V], ctypes.c_int),
        "ellpack_multiply_block": ([E, I, E, E, E, D, D, D, P(I), P(D), P(D), V], ctypes.c_int),
        "ellpack_gershgorin_block": ([E, I, P(D), P(D), V], ctypes.c_int),
        "sp2_x0_block": ([E, I, D, D, D, E, V], ctypes.c_int),
        "ellpack_stats_block": ([E, I, P(D), P(D), V], ctypes.c_int),
        "ellpack_halo_rows": ([E, I, I, V, P(I), V], ctypes.c_int),
        "sp2_fma_peak": ([I, I, P(D), V], ctypes.c_int),
        "ellpack_trace_noalloc": ([E, P(D), P(D), V], ctypes.c_int),
        "sp2_options_default": ([P(sp2_options)], None),
        "sp2_purify": ([E, D, D, P(sp2_options), E, P(sp2_stats), V], ctypes.c_int),
        "sp2_x0": ([E, D, E, P(D), P(D), V], ctypes.c_int),
        "sp2_purify_batched": ([E, P(D), I, D, P(sp2_options), E, P(sp2_stats), V], ctypes.c_int),
        "ellpack_struct_count": ([E, E, E, V, P(I), V], ctypes.c_int),
        "nnzpred_features": ([E, D, I, V, V], ctypes.c_int),
        "nnzpred_create": ([P(nnzpred_t), ctypes.c_uint64, V], ctypes.c_int),
        "nnzpred_destroy": ([P(nnzpred_t), V], ctypes.c_int),
        "nnzpred_set_stats": ([P(nnzpred_t), V, V, ctypes.c_int64, V], ctypes.c_int),
        "nnzpred_grad": ([P(nnzpred_t), V, V, ctypes.c_int64, V, P(ctypes.c_float), V], ctypes.c_int),
        "nnzpred_train": ([P(nnzpred_t), V, V, ctypes.c_int64, I, I, ctypes.c_float, P(ctypes.c_float), V],
                          ctypes.c_int),
        "nnzpred_calibrate": ([P(nnzpred_t), V, V, ctypes.c_int64, ctypes.c_float, P(ctypes.c_float), V], ctypes.c_int),
        "nnzpred_predict": ([P(nnzpred_t), V, ctypes.c_int64, V, V], ctypes.c_int),
        "nnzpred_width": ([P(nnzpred_t), E, D, I, P(I), V, V], ctypes.c_int),
        "nnzpred_save": ([P(nnzpred_t), ctypes.c_char_p, V], ctypes.c_int),
        "nnzpred_load": ([P(nnzpred_t), ctypes.c_char_p, V], ctypes.c_int),
        "sp2_profile_start": ([], ctypes.c_int),
        "sp2_profile_stop": ([P(sp2_profile)], ctypes.c_int),
        "sp2_step": ([E, E, D, D, P(sp2_step_info), V], ctypes.c_int),
        "ellpack_scale": ([E, D, V], ctypes.c_int),
        "ellpack_threshold": ([E, D, V], ctypes.c_int),
        "ellpack_norms": ([E, P(D), V], ctypes.c_int),
        "ellpack_transpose": ([E, E, P(I), V], ctypes.c_int),
        "ellpack_to_dense": ([E, V, ctypes.c_int64, V], ctypes.c_int),
        "ellpack_from_dense": ([V, ctypes.c_int64, D, E, P(I), V], ctypes.c_int),
        "sp2_tune_spgemm": ([E, E, E, E, D, D, D, I, P(I), P(ctypes.c_float), V], ctypes.c_int),
        "sp2_tune_record": ([I, I, I, D, I, ctypes.c_float], ctypes.c_int),
        "sp2_tune_lookup": ([I, I, I, D, P(I)], ctypes.c_int),
        "sp2_tune_clear": ([], ctypes.c_int),
        "sp2_tune_size": ([P(I)], ctypes.c_int),
        "sp2_tune_save": ([ctypes.c_char_p], ctypes.c_int),
        "sp2_tune_load": ([ctypes.c_char_p], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _check(rc):
    if rc != SP2_OK:
        raise Sp2Error(rc, lib.sp2_last_error_string().decode())
    return rc


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _torch_dtype(dt):
    import torch
    return torch.float64 if dt == SP2_F64 else torch.float32


class Ellpack:
    """ELLPACK matrix on the GPU: torch tensors idx int32[n, w], val f64/f32[n, w], nnz int32[n],
    exposed to the library through a borrowed ellpack_t descriptor."""

    def __init__(self, idx, val, nnz):
        import torch
        assert idx.is_cuda and val.is_cuda and nnz.is_cuda
        assert idx.dtype == torch.int32 and nnz.dtype == torch.int32
        assert val.dtype in (torch.float64, torch.float32)
        assert idx.shape == val.shape and idx.dim() == 2 and nnz.shape == (idx.shape[0],)
        self.idx, self.val, self.nnz = idx.contiguous(), val.contiguous(), nnz.contiguous()
        self.dtype = SP2_F64 if val.dtype == torch.float64 else SP2_F32
        self.desc = ellpack_t()
        _check(lib.ellpack_wrap(self.n, self.width, self.dtype, self.idx.data_ptr(), self.val.data_ptr(),
                                self.nnz.data_ptr(), ctypes.byref(self.desc)))

    @property
    def n(self):
        return self.idx.shape[0]

    @property
    def width(self):
        return self.idx.shape[1]

    @classmethod
    def empty(cls, n, width, dtype=SP2_F64, device="cuda"):
        import torch
        return cls(torch.zeros((n, width), dtype=torch.int32, device=device),
                   torch.zeros((n, width), dtype=_torch_dtype(dtype), device=device),
                   torch.zeros(n, dtype=torch.int32, device=device))

    @classmethod
    def from_numpy(cls, idx, val, nnz, dtype=SP2_F64, device="cuda"):
        import torch
        return cls(torch.as_tensor(np.ascontiguousarray(idx, np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(val), device=device).to(_torch_dtype(dtype)),
                   torch.as_tensor(np.ascontiguousarray(nnz, np.int32), device=device))

    def to_numpy(self):
        return self.idx.cpu().numpy(), self.val.double().cpu().numpy(), self.nnz.cpu().numpy()


class OwnedEllpack:
    """A matrix allocated by the library (e.g. the density matrix of sp2_purify)."""

    def __init__(self, desc):
        self.desc = desc

    @property
    def n(self):
        return self.desc.n

    @property
    def width(self):
        return self.desc.width

    @property
    def dtype(self):
        return self.desc.dtype

    def to_torch(self, stream=None):
        """Copy into a new torch-backed Ellpack (same width and dtype)."""
        out = Ellpack.empty(self.n, self.width, self.dtype)
        _check(lib.ellpack_copy(ctypes.byref(self.desc), ctypes.byref(out.desc), _stream(stream)))
        return out

    def to_numpy(self, stream=None):
        n, w = self.n, self.width
        idx = np.empty((n, w), np.int32)
        val = np.empty((n, w), np.float64 if self.dtype == SP2_F64 else np.float32)
        nnz = np.empty(n, np.int32)
        _check(lib.ellpack_download(ctypes.byref(self.desc), idx.ctypes.data, val.ctypes.data, nnz.ctypes.data,
                                    _stream(stream)))
        return idx, val.astype(np.float64), nnz

    def release(self, stream=None):
        if self.desc is not None and self.desc.owner:
            lib.ellpack_destroy(ctypes.byref(self.desc), _stream(stream) if stream is not None else None)
        self.desc = None

    def __del__(self):
        try:
            if self.desc is not None and self.desc.owner:
                lib.ellpack_destroy(ctypes.byref(self.desc), None)
        except Exception:
            pass


def _d(m):
    return ctypes.byref(m.desc)


def ellpack_create(n, width, dtype=SP2_F64, stream=None):
    d = ellpack_t()
    _check(lib.ellpack_create(n, width, dtype, _stream(stream), ctypes.byref(d)))
    return OwnedEllpack(d)


def ellpack_upload(m, idx, val, nnz, stream=None):
    """Host numpy arrays -> device matrix (asynchronous; arrays must outlive the copy)."""
    _check(lib.ellpack_upload(_d(m), idx.ctypes.data, val.ctypes.data, nnz.ctypes.data, _stream(stream)))


def ellpack_download(m, idx, val, nnz, stream=None):
    _check(lib.ellpack_download(_d(m), idx.ctypes.data, val.ctypes.data, nnz.ctypes.data, _stream(stream)))


def ellpack_copy(src, dst, stream=None):
    _check(lib.ellpack_copy(_d(src), _d(dst), _stream(stream)))


def ellpack_multiply(A, B, C, alpha=1.0, beta=0.0, tau=0.0, stream=None, raise_on_overflow=True):
    """C <- drop_tau(alpha*A*B + beta*C).  Returns the largest post-threshold row length;
    raises Sp2Error(SP2E_OVERFLOW) if C is too narrow (unless raise_on_overflow=False,
    then returns (status, required_width))."""
    req = ctypes.c_int32(0)
    rc = lib.ellpack_multiply(_d(A), _d(B), _d(C), float(alpha), float(beta), float(tau), _stream(stream),
                              ctypes.byref(req))
    if not raise_on_overflow:
        if rc not in (SP2_OK, SP2E_OVERFLOW):
            _check(rc)
        return rc, req.value
    _check(rc)
    return req.value


def ellpack_multiply_block(A, row0, B, C, Out, alpha=1.0, beta=0.0, tau=0.0, stream=None, raise_on_overflow=True):
    """Out <- drop_tau(alpha A B + beta C) for the row block held by A, C and Out (global
    rows row0 .. row0 + A.n - 1, global column indices; B has the global row count and
    holds every row A names).  Returns (status, required width, block trace, block
    squared Frobenius norm)."""
    req, tr, fro = ctypes.c_int32(0), ctypes.c_double(), ctypes.c_double()
    rc = lib.ellpack_multiply_block(_d(A), int(row0), _d(B), _d(C) if C is not None else None, _d(Out),
                                    float(alpha), float(beta), float(tau), ctypes.byref(req), ctypes.byref(tr),
                                    ctypes.byref(fro), _stream(stream))
    if rc == SP2E_OVERFLOW and not raise_on_overflow:
        return rc, req.value, None, None
    _check(rc)
    return rc, req.value, tr.value, fro.value


def ellpack_gershgorin_block(H, row0, stream=None):
    """Gershgorin bounds (emin, emax) of the discs of a row block (global rows row0 ..)."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib.ellpack_gershgorin_block(_d(H), int(row0), ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return lo.value, hi.value


def sp2_x0_block(H, row0, emin, emax, tau, X0, stream=None):
    """X0's rows of a row block from the global spectral bounds."""
    _check(lib.sp2_x0_block(_d(H), int(row0), float(emin), float(emax), float(tau), _d(X0), _stream(stream)))


def ellpack_stats_block(X, row0, stream=None):
    """(block share of tr X, block share of ||X||_F^2)."""
    tr, fro = ctypes.c_double(), ctypes.c_double()
    _check(lib.ellpack_stats_block(_d(X), int(row0), ctypes.byref(tr), ctypes.byref(fro), _stream(stream)))
    return tr.value, fro.value


def ellpack_halo_rows(X, row0, ncols, stream=None):
    """Ascending int32 device tensor of the rows outside the block (global rows row0 ..
    row0 + X.n - 1) that X's entries name."""
    import torch
    rows = torch.empty(int(ncols), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int32()
    _check(lib.ellpack_halo_rows(_d(X), int(row0), int(ncols), rows.data_ptr(), ctypes.byref(cnt), _stream(stream)))
    return rows[:cnt.value]


def ellpack_add(A, B, alpha=1.0, beta=1.0, tau=0.0, stream=None):
    req = ctypes.c_int32(0)
    _check(lib.ellpack_add(_d(A), _d(B), float(alpha), float(beta), float(tau), _stream(stream), ctypes.byref(req)))
    return req.value


def ellpack_trace(A, stream=None):
    out = ctypes.c_double()
    _check(lib.ellpack_trace(_d(A), ctypes.byref(out), _stream(stream)))
    return out.value


def ellpack_frobenius2(A, stream=None):
    out = ctypes.c_double()
    _check(lib.ellpack_frobenius2(_d(A), ctypes.byref(out), _stream(stream)))
    return out.value


SP2_NOALLOC_MAX_N = 65536


def ellpack_trace_noalloc(A, stream=None, frobenius=True):
    """(tr A, ||A||_F^2) through the entry point that allocates no device memory (its
    scratch is a fixed array inside the library; n <= SP2_NOALLOC_MAX_N).  With
    frobenius=False the squared norm is not requested (NULL) and None is returned for it."""
    tr, fro = ctypes.c_double(), ctypes.c_double()
    _check(lib.ellpack_trace_noalloc(_d(A), ctypes.byref(tr), ctypes.byref(fro) if frobenius else None,
                                     _stream(stream)))
    return tr.value, (fro.value if frobenius else None)


def ellpack_gershgorin(H, stream=None):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib.ellpack_gershgorin(_d(H), ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return lo.value, hi.value


def sp2_options_default(**kw):
    o = sp2_options()
    lib.sp2_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError("unknown sp2 option %r" % k)
        if k == "predictor":
            o._pred_ref = v  # keep the predictor alive as long as the options
            v = ctypes.pointer(v.desc)
        setattr(o, k, v)
    return o


def stats_dict(st):
    it = st.iterations
    m = min(it + 1, SP2_STATS_CAP)
    return {
        "iterations": it, "status": {0: "converged", 1: "stalled", 2: "max_iter"}.get(st.status, st.status),
        "fp32_iterations": st.fp32_iterations, "regrows": st.regrows, "struct_passes": st.struct_passes,
        "tuned": st.tuned,
        "width_max": st.width_max, "pred_log_mae": st.pred_log_mae, "pred_under_frac": st.pred_under_frac,
        "emin": st.emin, "emax": st.emax,
        "time_ms": st.time_ms,
        "trX": np.array(st.trX[:m]), "trX2": np.array(st.trX2[:m]), "err": np.array(st.err[:m]),
        "branch": ["X2" if b == 1 else "2X-X2" for b in st.branch[:min(it, SP2_STATS_CAP)]],
        "nnz_total": np.array(st.nnz_total[:m]), "max_row_nnz": np.array(st.max_row_nnz[:m]),
        "rows_level1": np.array(st.rows_level1[:min(it, SP2_STATS_CAP)]),
        "rows_level2": np.array(st.rows_level2[:min(it, SP2_STATS_CAP)]),
        "rows_deferred": np.array(st.rows_deferred[:min(it, SP2_STATS_CAP)]),
        "rows_routed": np.array(st.rows_routed[:min(it, SP2_STATS_CAP)]),
        "level": np.array(st.level[:min(it, SP2_STATS_CAP)]),
        "small_iterations": st.small_iterations,
    }


def sp2_purify(H, nocc, tol, options=None, stream=None, allow_notconv=False):
    """SP2 purification of H; returns (D as OwnedEllpack, stats dict)."""
    opt = options if options is not None else sp2_options_default()
    D = ellpack_t()
    st = sp2_stats()
    rc = lib.sp2_purify(_d(H), float(nocc), float(tol), ctypes.byref(opt), ctypes.byref(D), ctypes.byref(st),
                        _stream(stream))
    out = OwnedEllpack(D)  # owns D even when an error is raised below (freed with it)
    if rc == SP2E_NOTCONV and allow_notconv:
        return out, stats_dict(st)
    try:
        _check(rc)
    except Sp2Error as e:
        e.stats = stats_dict(st)  # the iterations recorded before the error
        raise
    return out, stats_dict(st)


def sp2_x0(H, X0, tau, stream=None):
    """X0 = drop_tau((e_max I - H)/(e_max - e_min)) into X0; returns (e_min, e_max)."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib.sp2_x0(_d(H), float(tau), _d(X0), ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return lo.value, hi.value


def sp2_step(X, Xn, nocc, tau, traces=None, spgemm_path=0, stream=None, raise_on_overflow=True, symmetric=False,
             compact_level=0):
    """One SP2 iteration X -> Xn.  traces = (trX, trX2) of X if known.  symmetric: X is
    exactly symmetric (the product's upper triangle is computed and mirrored);
    compact_level: its automatic first pass (0 tight, 1 loose, 2 full rows).  Returns
    the sp2_step_info record (and the status when raise_on_overflow=False)."""
    info = sp2_step_info()
    info.symmetric = 1 if symmetric else 0
    info.compact_level = compact_level
    if traces is not None:
        info.trX, info.trX2 = traces
        info.have_traces = 1
    info.spgemm_path = spgemm_path
    rc = lib.sp2_step(_d(X), _d(Xn), float(nocc), float(tau), ctypes.byref(info), _stream(stream))
    if not raise_on_overflow:
        if rc not in (SP2_OK, SP2E_OVERFLOW):
            _check(rc)
        return rc, info
    _check(rc)
    return info


def sp2_profile_start():
    _check(lib.sp2_profile_start())


def sp2_profile_stop():
    """Returns {"launches": L, "<class>": (count, total_ms), ...}."""
    p = sp2_profile()
    _check(lib.sp2_profile_stop(ctypes.byref(p)))
    out = {"launches": int(p.launches)}
    for i, name in enumerate(PROF_NAMES):
        out[name] = (int(p.count[i]), float(p.total_ms[i]))
    return out


def sp2_purify_batched(Hs, noccs, tol, options=None, stream=None, allow_notconv=False):
    """Batched SP2 of the matrices Hs (Ellpack, F64); returns ([D as OwnedEllpack], [stats])."""
    count = len(Hs)
    opt = options if options is not None else sp2_options_default()
    harr = (ellpack_t * count)(*[h.desc for h in Hs])
    narr = (ctypes.c_double * count)(*[float(x) for x in noccs])
    darr = (ellpack_t * count)()
    sarr = (sp2_stats * count)()
    rc = lib.sp2_purify_batched(harr, narr, count, float(tol), ctypes.byref(opt), darr, sarr, _stream(stream))
    Ds = [OwnedEllpack(darr[m]) for m in range(count)]
    for m in range(count):  # the descriptors now belong to the OwnedEllpack objects
        darr[m].owner = 0
    if not (rc == SP2E_NOTCONV and allow_notconv):
        _check(rc)
    return Ds, [stats_dict(sarr[m]) for m in range(count)]


def ellpack_struct_count(A, B, C=None, stream=None):
    """Exact structural row counts of A*B (+C): (torch int32 tensor [n], max)."""
    import torch
    counts = torch.empty(A.n, dtype=torch.int32, device="cuda")
    mx = ctypes.c_int32()
    _check(lib.ellpack_struct_count(_d(A), _d(B), _d(C) if C is not None else None, counts.data_ptr(),
                                    ctypes.byref(mx), _stream(stream)))
    return counts, mx.value


def nnzpred_features(X, tau, branch, stream=None):
    """Row features of X (torch float32 [n, 16]) for the product of an SP2 step with `branch`."""
    import torch
    feat = torch.empty((X.n, 16), dtype=torch.float32, device="cuda")
    _check(lib.nnzpred_features(_d(X), float(tau), int(branch), feat.data_ptr(), _stream(stream)))
    return feat


class NnzPredictor:
    """The row-length MLP (weights on the GPU, trained by the library's kernels)."""

    def __init__(self, seed=0, stream=None):
        self.desc = nnzpred_t()
        _check(lib.nnzpred_create(ctypes.byref(self.desc), int(seed), _stream(stream)))

    def set_stats(self, feat, counts, stream=None):
        _check(lib.nnzpred_set_stats(ctypes.byref(self.desc), feat.data_ptr(), counts.data_ptr(), feat.shape[0],
                                     _stream(stream)))

    def grad(self, feat, counts, stream=None):
        import torch
        g = torch.empty(NNZPRED_NPARAMS, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        _check(lib.nnzpred_grad(ctypes.byref(self.desc), feat.data_ptr(), counts.data_ptr(), feat.shape[0],
                                g.data_ptr(), ctypes.byref(loss), _stream(stream)))
        return g, loss.value

    def train(self, feat, counts, steps, batch=2048, lr=1e-3, stream=None):
        loss = ctypes.c_float()
        _check(lib.nnzpred_train(ctypes.byref(self.desc), feat.data_ptr(), counts.data_ptr(), feat.shape[0],
                                 int(steps), int(batch), float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def calibrate(self, feat, counts, quantile=0.9, stream=None):
        """Sets the log-space margin so that a share `quantile` of the samples' lengths lie
        at or below their predictions; returns the margin."""
        m = ctypes.c_float()
        _check(lib.nnzpred_calibrate(ctypes.byref(self.desc), feat.data_ptr(), counts.data_ptr(), feat.shape[0],
                                     float(quantile), ctypes.byref(m), _stream(stream)))
        return m.value

    def predict(self, feat, stream=None):
        import torch
        pred = torch.empty(feat.shape[0], dtype=torch.float32, device="cuda")
        _check(lib.nnzpred_predict(ctypes.byref(self.desc), feat.data_ptr(), feat.shape[0], pred.data_ptr(),
                                   _stream(stream)))
        return pred

    def width(self, X, tau, branch, stream=None):
        """(output width for the SP2 product of X, predicted row lengths [n])."""
        import torch
        pred = torch.empty(X.n, dtype=torch.float32, device="cuda")
        w = ctypes.c_int32()
        _check(lib.nnzpred_width(ctypes.byref(self.desc), _d(X), float(tau), int(branch), ctypes.byref(w),
                                 pred.data_ptr(), _stream(stream)))
        return w.value, pred

    def params(self):
        """(weights float32[NNZPRED_NPARAMS], statistics float32[NNZPRED_NSTATS]) on the host,
        read back through the library's save format."""
        import os
        import tempfile
        fd, path = tempfile.mkstemp(suffix=".nnzpred")
        os.close(fd)
        try:
            self.save(path)
            raw = np.fromfile(path, dtype=np.uint8)
            vals = raw[8:].view(np.float32)
            return vals[:NNZPRED_NPARAMS].copy(), vals[NNZPRED_NPARAMS:].copy()
        finally:
            os.remove(path)

    def save(self, path, stream=None):
        _check(lib.nnzpred_save(ctypes.byref(self.desc), path.encode(), _stream(stream)))

    def load(self, path, stream=None):
        _check(lib.nnzpred_load(ctypes.byref(self.desc), path.encode(), _stream(stream)))

    def __del__(self):
        try:
            if self.desc.params:
                lib.nnzpred_destroy(ctypes.byref(self.desc), None)
        except Exception:
            pass


# ---------------------------------------------------------------- autotuner
TUNE_CANDIDATES = (1, 2, 4, 7, 3, 8, 9, 10, 11, 12)


def sp2_tune_spgemm(A, B, C, Out, alpha=1.0, beta=0.0, tau=0.0, reps=3, stream=None):
    """Times every SpGEMM first-pass variant on Out <- drop_tau(alpha A*B + beta C) and
    records the fastest; returns (best path, {path: ms})."""
    best = ctypes.c_int32()
    times = (ctypes.c_float * len(TUNE_CANDIDATES))()
    _check(lib.sp2_tune_spgemm(_d(A), _d(B), _d(C) if C is not None else None, _d(Out), float(alpha), float(beta),
                               float(tau), int(reps), ctypes.byref(best), times, _stream(stream)))
    return best.value, dict(zip(TUNE_CANDIDATES, list(times)))


def sp2_tune_record(sms, dtype, n, mean_row_nnz, path, ms=0.0):
    _check(lib.sp2_tune_record(int(sms), int(dtype), int(n), float(mean_row_nnz), int(path), float(ms)))


def sp2_tune_lookup(sms, dtype, n, mean_row_nnz):
    """The recorded variant for the class, or -1 (sms = 0: the current device)."""
    p = ctypes.c_int32()
    _check(lib.sp2_tune_lookup(int(sms), int(dtype), int(n), float(mean_row_nnz), ctypes.byref(p)))
    return p.value


def sp2_tune_clear():
    _check(lib.sp2_tune_clear())


def sp2_tune_size():
    v = ctypes.c_int32()
    _check(lib.sp2_tune_size(ctypes.byref(v)))
    return v.value


def sp2_tune_save(path):
    _check(lib.sp2_tune_save(str(path).encode()))


def sp2_tune_load(path):
    _check(lib.sp2_tune_load(str(path).encode()))


# ---------------------------------------------------------------- standalone ops
def ellpack_scale(A, alpha, stream=None):
    _check(lib.ellpack_scale(_d(A), float(alpha), _stream(stream)))


def ellpack_threshold(A, tau, stream=None):
    _check(lib.ellpack_threshold(_d(A), float(tau), _stream(stream)))


def ellpack_norms(A, stream=None):
    """(max |a_ij|, infinity norm, Frobenius norm)."""
    out = (ctypes.c_double * 3)()
    _check(lib.ellpack_norms(_d(A), out, _stream(stream)))
    return tuple(out)


def ellpack_transpose(A, At, stream=None, raise_on_overflow=True):
    """At <- A^T; returns the longest column count of A (and the status when
    raise_on_overflow=False)."""
    w = ctypes.c_int32()
    rc = lib.ellpack_transpose(_d(A), _d(At), ctypes.byref(w), _stream(stream))
    if not raise_on_overflow:
        if rc not in (SP2_OK, SP2E_OVERFLOW):
            _check(rc)
        return rc, w.value
    _check(rc)
    return w.value


def ellpack_to_dense(A, stream=None):
    """Dense torch tensor [n, n] of A's dtype on the GPU."""
    import torch
    D = torch.empty((A.n, A.n), dtype=_torch_dtype(A.dtype), device="cuda")
    _check(lib.ellpack_to_dense(_d(A), D.data_ptr(), A.n, _stream(stream)))
    return D


def ellpack_from_dense(D, A, tau=0.0, stream=None, raise_on_overflow=True):
    """A <- entries of the dense torch tensor D (A's dtype, [n, ld]); returns the longest
    row (and the status when raise_on_overflow=False)."""
    assert D.is_cuda and D.dim() == 2 and D.is_contiguous() and D.dtype == _torch_dtype(A.dtype)
    w = ctypes.c_int32()
    rc = lib.ellpack_from_dense(D.data_ptr(), D.shape[1], float(tau), _d(A), ctypes.byref(w), _stream(stream))
    if not raise_on_overflow:
        if rc not in (SP2_OK, SP2E_OVERFLOW):
            _check(rc)
        return rc, w.value
    _check(rc)
    return w.value


def sp2_fma_peak(dtype=SP2_F64, reps=5, stream=None):
    """Measured FMA rate of the current device in TFLOP/s (DFMA for SP2_F64, FFMA for SP2_F32)."""
    out = ctypes.c_double()
    _check(lib.sp2_fma_peak(int(dtype), int(reps), ctypes.byref(out), _stream(stream)))
    return out.value
