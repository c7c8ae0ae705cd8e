"""CUDA thresholded ELLPACK SpGEMM / add / reductions against the CPU oracle (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I
from parity import compare_spgemm, dense_of, sorted_rows_ok

pytestmark = pytest.mark.gpu


def dev(S, E, dtype=None, width=None):
    dt = S.SP2_F64 if dtype is None else dtype
    idx, val, nnz = E.idx, E.val, E.nnz
    if width is not None and width > idx.shape[1]:
        pad = width - idx.shape[1]
        idx = np.pad(idx, ((0, 0), (0, pad)))
        val = np.pad(val, ((0, 0), (0, pad)), constant_values=np.nan)
    return S.Ellpack.from_numpy(idx, val, nnz, dt)


def ell(t):
    return O.Ell(*t)


def f32_input(E):
    """The oracle's input for an FP32 run: the FP64 values rounded to FP32."""
    return O.Ell(E.idx, E.val.astype(np.float32).astype(np.float64), E.nnz)


RANDOM_CASES = [
    # n, seed, min, max nnz, full rows, empty rows
    (1, 0, 0, 1, (), ()),
    (37, 1, 0, 9, (4,), (0, 5)),
    (700, 2, 0, 40, (10,), (3, 699)),
    (3000, 3, 20, 160, (7, 2999), (100,)),   # B rows above 128 entries: register tail path
]


@pytest.mark.parametrize("case", RANDOM_CASES)
@pytest.mark.parametrize("ab", [(1.0, 0.0), (-1.0, 2.0), (0.5, -1.5)])
@pytest.mark.parametrize("tau", [0.0, 2e-3])
def test_multiply_f64_random(gpu, case, ab, tau):
    S = gpu
    n, seed, lo, hi, full, empty = case
    alpha, beta = ab
    A = ell(I.random_sparse(n, seed=seed, min_nnz=lo, max_nnz=hi, full_rows=full, empty_rows=empty,
                            value_scale=0.2))
    B = ell(I.random_sparse(n, seed=seed + 7, min_nnz=lo, max_nnz=hi, full_rows=full[:1], value_scale=0.2))
    C = ell(I.random_sparse(n, seed=seed + 9, min_nnz=0, max_nnz=max(1, hi // 4)))
    ref = O.spgemm(A, B, C if beta else None, alpha, beta, tau)
    width = max(32, ((int(ref.nnz.max()) + 31) // 32) * 32)
    dA, dB = dev(S, A), dev(S, B)
    dC = dev(S, C, width=width)
    S.ellpack_multiply(dA, dB, dC, alpha, beta, tau)
    compare_spgemm(dC.to_numpy(), A, B, C, alpha, beta, tau)


@pytest.mark.parametrize("case", RANDOM_CASES[1:])
@pytest.mark.parametrize("tau", [0.0, 2e-3])
def test_multiply_f32_random(gpu, case, tau):
    S = gpu
    n, seed, lo, hi, full, empty = case
    A = f32_input(ell(I.random_sparse(n, seed=seed, min_nnz=lo, max_nnz=hi, full_rows=full, empty_rows=empty,
                                      value_scale=0.2)))
    C = f32_input(ell(I.random_sparse(n, seed=seed + 9, min_nnz=0, max_nnz=max(1, hi // 4))))
    ref = O.spgemm(A, A, C, -1.0, 2.0, tau)
    width = max(32, ((int(ref.nnz.max()) + 31) // 32) * 32)
    dA = dev(S, A, S.SP2_F32)
    dC = dev(S, C, S.SP2_F32, width=width)
    S.ellpack_multiply(dA, dA, dC, -1.0, 2.0, tau)
    compare_spgemm(dC.to_numpy(), A, A, C, -1.0, 2.0, tau, fp32=True)


def test_multiply_long_rows_use_large_row_kernel(gpu):
    """Rows with more than half a hash table of distinct columns go to the dense
    global-memory kernel; results must be the same."""
    S = gpu
    n = 2500
    A = ell(I.random_sparse(n, seed=51, min_nnz=5, max_nnz=60, full_rows=tuple(range(0, n, 97)), value_scale=0.3))
    ref = O.spgemm(A, A, None, 1.0, 0.0, 1e-4)
    assert ref.nnz.max() > 600  # some rows exceed the default table's limit
    width = ((int(ref.nnz.max()) + 31) // 32) * 32
    dA = dev(S, A)
    dC = S.Ellpack.empty(n, width)
    S.ellpack_multiply(dA, dA, dC, 1.0, 0.0, 1e-4)
    compare_spgemm(dC.to_numpy(), A, A, None, 1.0, 0.0, 1e-4)


def test_multiply_tight_binding_product(gpu):
    """Realistic pattern: X0^2 of a Morton-ordered 3D tight-binding Hamiltonian."""
    S = gpu
    n = 6000
    H = ell(I.tight_binding(n, seed=3))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, 1e-6)
    X1 = O.spgemm(X0, X0, None, 1.0, 0.0, 1e-6)
    ref = O.spgemm(X1, X1, X1, -1.0, 2.0, 1e-6)
    w = ((int(ref.nnz.max()) + 31) // 32) * 32
    d1 = dev(S, X1)
    out = S.Ellpack.empty(n, w)
    S.ellpack_multiply(d1, d1, out, 1.0, 0.0, 1e-6)
    compare_spgemm(out.to_numpy(), X1, X1, None, 1.0, 0.0, 1e-6)
    # fused update as in an SP2 step: 2X - X^2 (C holds X beforehand)
    out2 = dev(S, X1, width=w)
    S.ellpack_multiply(d1, d1, out2, -1.0, 2.0, 1e-6)
    compare_spgemm(out2.to_numpy(), X1, X1, X1, -1.0, 2.0, 1e-6)


def test_multiply_tight_binding_product_f32(gpu):
    """FP32 values on the same realistic pattern, both branches of the SP2 update."""
    S = gpu
    n = 6000
    H = ell(I.tight_binding(n, seed=4, delta=10.0))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, 1e-5)
    X1 = f32_input(O.spgemm(X0, X0, None, 1.0, 0.0, 1e-5))
    for alpha, beta in ((1.0, 0.0), (-1.0, 2.0)):
        ref = O.spgemm(X1, X1, X1 if beta else None, alpha, beta, 1e-5)
        w = ((int(ref.nnz.max()) + 31) // 32) * 32
        d1 = dev(S, X1, S.SP2_F32)
        out = dev(S, X1, S.SP2_F32, width=w) if beta else S.Ellpack.empty(n, w, S.SP2_F32)
        S.ellpack_multiply(d1, d1, out, alpha, beta, 1e-5)
        compare_spgemm(out.to_numpy(), X1, X1, X1, alpha, beta, 1e-5, fp32=True)


def test_multiply_is_deterministic(gpu):
    S = gpu
    n = 3000
    A = ell(I.random_sparse(n, seed=61, min_nnz=10, max_nnz=80, value_scale=0.2))
    dA = dev(S, A)
    need = S.ellpack_multiply(dA, dA, S.Ellpack.empty(n, 32), 1.0, 0.0, 1e-5, raise_on_overflow=False)[1]
    outs = []
    for _ in range(2):
        C = S.Ellpack.empty(n, ((need + 31) // 32) * 32)
        S.ellpack_multiply(dA, dA, C, 1.0, 0.0, 1e-5)
        outs.append(C.to_numpy())
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(np.nan_to_num(a), np.nan_to_num(b))


def test_multiply_overflow_status_and_retry(gpu):
    S = gpu
    n = 500
    A = ell(I.random_sparse(n, seed=71, min_nnz=5, max_nnz=20))
    ref = O.spgemm(A, A, None, 1.0, 0.0, 0.0)
    need = int(ref.nnz.max())
    dA = dev(S, A)
    small = S.Ellpack.empty(n, 32)
    rc, req = S.ellpack_multiply(dA, dA, small, raise_on_overflow=False)
    assert rc == S.SP2E_OVERFLOW and req == need
    big = S.Ellpack.empty(n, ((need + 31) // 32) * 32)
    assert S.ellpack_multiply(dA, dA, big) == need
    compare_spgemm(big.to_numpy(), A, A, None, 1.0, 0.0, 0.0)


def test_multiply_argument_errors(gpu):
    S = gpu
    A = dev(S, ell(I.random_sparse(10, seed=1, max_nnz=3)))
    B = dev(S, ell(I.random_sparse(11, seed=2, max_nnz=3)))
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_multiply(A, A, A)  # C aliases A
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_multiply(A, B, S.Ellpack.empty(10, 32))
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_multiply(A, A, S.Ellpack.empty(10, 32), tau=-1.0)
    assert e.value.code == S.SP2E_ARG
    with pytest.raises(S.Sp2Error) as e:
        S.ellpack_multiply(A, A, S.Ellpack.empty(10, 32, S.SP2_F32))
    assert e.value.code == S.SP2E_ARG


@pytest.mark.parametrize("ab", [(1.0, 1.0), (2.0, -1.0), (-0.5, 0.25)])
@pytest.mark.parametrize("tau", [0.0, 0.05])
def test_add(gpu, ab, tau):
    S = gpu
    alpha, beta = ab
    n = 900
    A = ell(I.random_sparse(n, seed=81, min_nnz=0, max_nnz=30, empty_rows=(0,)))
    B = ell(I.random_sparse(n, seed=82, min_nnz=0, max_nnz=30, empty_rows=(0, 1)))
    ref = O.add(A, B, alpha, beta, tau)
    dA = dev(S, A, width=64)
    dB = dev(S, B)
    S.ellpack_add(dA, dB, alpha, beta, tau)
    gi, gv, gn = dA.to_numpy()
    assert sorted_rows_ok(gi, gn)
    G = dense_of(gi, gv, gn, n)
    R = ref.to_dense()
    scale = abs(alpha) * np.abs(A.to_dense()) + abs(beta) * np.abs(B.to_dense())
    bound = 1e-15 * scale + 1e-300
    pg = np.zeros((n, n), bool)
    pr = np.zeros((n, n), bool)
    for i in range(n):
        pg[i, gi[i, :gn[i]]] = True
        pr[i, ref.row(i)[0]] = True
    if tau == 0.0:
        assert np.array_equal(pg, pr)
    both = pg & pr
    assert np.all(np.abs(G - R)[both] <= bound[both])
    flip = pg ^ pr
    exact = alpha * A.to_dense() + beta * B.to_dense()
    assert np.all(np.abs(np.abs(exact[flip]) - tau) <= bound[flip])


def test_add_long_rows(gpu):
    S = gpu
    n = 3000
    A = ell(I.random_sparse(n, seed=91, min_nnz=0, max_nnz=700, width=704))
    B = ell(I.random_sparse(n, seed=92, min_nnz=0, max_nnz=700))
    ref = O.add(A, B, 1.0, -1.0, 0.0)
    w = ((int(ref.nnz.max()) + 31) // 32) * 32
    dA = dev(S, A, width=w)
    S.ellpack_add(dA, dev(S, B), 1.0, -1.0, 0.0)
    gi, gv, gn = dA.to_numpy()
    assert np.array_equal(gn, ref.nnz)
    for i in range(0, n, 37):
        assert np.array_equal(gi[i, :gn[i]], ref.row(i)[0])
        assert np.allclose(gv[i, :gn[i]], ref.row(i)[1], rtol=0, atol=1e-15)


def test_trace_frobenius_gershgorin(gpu):
    S = gpu
    H = ell(I.tight_binding(5000, seed=5))
    dH = dev(S, H)
    tr = S.ellpack_trace(dH)
    assert tr == pytest.approx(O.trace(H), rel=1e-13, abs=1e-12)
    fro = S.ellpack_frobenius2(dH)
    want = float(sum((H.row(i)[1] ** 2).sum() for i in range(H.n)))
    assert fro == pytest.approx(want, rel=1e-13)
    lo, hi = S.ellpack_gershgorin(dH)
    olo, ohi = O.gershgorin(H)
    assert lo == pytest.approx(olo, rel=1e-13) and hi == pytest.approx(ohi, rel=1e-13)
    dF = dev(S, H, S.SP2_F32)
    assert S.ellpack_trace(dF) == pytest.approx(O.trace(H), rel=1e-6)


@pytest.mark.parametrize("tau", [0.0, 1e-2])
def test_x0(gpu, tau):
    S = gpu
    n = 2000
    H = ell(I.banded(n, band=12, seed=4))
    # knock out a few diagonal entries so that the insertion path runs
    Hd_idx, Hd_val, Hd_nnz = H.idx.copy(), H.val.copy(), H.nnz.copy()
    for i in (0, 5, 1999):
        k = Hd_nnz[i]
        cols = Hd_idx[i, :k]
        keep = cols != i
        m = int(keep.sum())
        Hd_idx[i, :m], Hd_val[i, :m] = cols[keep], Hd_val[i, :k][keep]
        Hd_nnz[i] = m
    H = O.Ell(Hd_idx, Hd_val, Hd_nnz)
    lo, hi = O.gershgorin(H)
    ref = O.x0(H, lo, hi, tau)
    dH = dev(S, H)
    X = S.Ellpack.empty(n, H.w + 32)
    glo, ghi = S.sp2_x0(dH, X, tau)
    assert glo == pytest.approx(lo, rel=1e-14) and ghi == pytest.approx(hi, rel=1e-14)
    gi, gv, gn = X.to_numpy()
    assert np.array_equal(gn, ref.nnz)
    for i in range(n):
        assert np.array_equal(gi[i, :gn[i]], ref.row(i)[0])
        assert np.allclose(gv[i, :gn[i]], ref.row(i)[1], rtol=5e-16, atol=1e-300)


@pytest.mark.parametrize("first_pass", [0, 1, 2, 3, 4, 7, 8, 9, 11])
@pytest.mark.parametrize("fp32", [False, True])
def test_first_pass_variants(gpu, first_pass, fp32):
    """Every first-pass variant (column blocks with 1, 2, 4 warps per row and the compact
    2-warp form, the two-step one-warp variant and its compact form, a per-warp hash table) on one SP2 step of a
    gapped tight-binding X; a second run is bitwise identical."""
    S = gpu
    n = 5000
    H = ell(I.tight_binding(n, seed=6, delta=10.0))
    lo, hi = O.gershgorin(H)
    X0 = O.x0(H, lo, hi, 1e-5)
    X1 = O.spgemm(X0, X0, None, 1.0, 0.0, 1e-5)
    if fp32:
        X1 = f32_input(X1)
    dt = S.SP2_F32 if fp32 else S.SP2_F64
    d1 = dev(S, X1, dt)
    probe = S.Ellpack.empty(n, 32, dt)
    rc, info = S.sp2_step(d1, probe, n / 2, 1e-5, spgemm_path=first_pass, raise_on_overflow=False)
    out = S.Ellpack.empty(n, ((info.required_width + 31) // 32) * 32, dt)
    info = S.sp2_step(d1, out, n / 2, 1e-5, spgemm_path=first_pass)
    up = info.branch == 2
    compare_spgemm(out.to_numpy(), X1, X1, X1, -1.0 if up else 1.0, 2.0 if up else 0.0, 1e-5, fp32=fp32)
    if first_pass not in (7, 8):  # the compact variants hold half a full row's blocks: long rows defer
        assert info.rows_deferred == 0
    again = S.Ellpack.empty(n, out.width, dt)
    S.sp2_step(d1, again, n / 2, 1e-5, spgemm_path=first_pass)
    for a, b in zip(out.to_numpy(), again.to_numpy()):
        assert np.array_equal(np.nan_to_num(a), np.nan_to_num(b))
    # X1 is exactly symmetric: the upper-triangle product mirrored gives the same bits
    sym = S.Ellpack.empty(n, out.width, dt)
    info_s = S.sp2_step(d1, sym, n / 2, 1e-5, spgemm_path=first_pass, symmetric=True)
    assert rows_equal(out.to_numpy(), sym.to_numpy())
    assert (info_s.trXn, info_s.nnz_total, info_s.max_row_nnz) == (info.trXn, info.nnz_total, info.max_row_nnz)
    assert info_s.trXn2 == pytest.approx(info.trXn2, rel=1e-13)


def rows_equal(g1, g2):
    """Stored entries of two ELLPACK results (idx, val, nnz) identical bit for bit."""
    i1, v1, n1 = g1
    i2, v2, n2 = g2
    if not np.array_equal(n1, n2):
        return False
    w = min(i1.shape[1], i2.shape[1])
    live = np.arange(w)[None, :] < n1[:, None]
    return (np.array_equal(np.where(live, i1[:, :w], 0), np.where(live, i2[:, :w], 0)) and
            np.array_equal(np.where(live, v1[:, :w], 0).view(np.int64), np.where(live, v2[:, :w], 0).view(np.int64)))


def hub_matrix(n, hubs, hub_nnz, other_nnz, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        k = hub_nnz if i in hubs else other_nnz
        c = rng.choice(n, size=k, replace=False)
        rows.append(np.full(k, i))
        cols.append(c)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    vals = rng.uniform(-1.0, 1.0, len(rows)) * 0.05
    return O.Ell(*I.coo_to_ellpack(n, rows, cols, vals))


@pytest.mark.parametrize("first_pass", [0, 3, 9])
def test_all_three_passes(gpu, first_pass):
    """Rows with more column groups than the block accumulator holds and a column span
    wider than the shared-memory window go to the 2^14-slot table; rows with more
    distinct columns than that go to the dense global-row pass.  Sampled rows (all hubs
    included) against the oracle (tau = 0: every structural entry is kept)."""
    S = gpu
    n = 60000
    hubs = set(range(0, n, 2000)) | {n - 1}
    X = hub_matrix(n, hubs, 1000, 40, seed=3)
    dX = dev(S, X)
    probe = S.Ellpack.empty(n, 32)
    rc, info = S.sp2_step(dX, probe, n / 2, 0.0, spgemm_path=first_pass, raise_on_overflow=False)
    out = S.Ellpack.empty(n, ((info.required_width + 31) // 32) * 32)
    info = S.sp2_step(dX, out, n / 2, 0.0, spgemm_path=first_pass)
    assert info.rows_deferred > len(hubs) and info.rows_dense >= len(hubs)
    up = info.branch == 2
    rng = np.random.default_rng(4)
    rows = np.unique(np.concatenate([sorted(hubs), rng.choice(n, 300, replace=False)]))
    compare_spgemm(out.to_numpy(), X, X, X, -1.0 if up else 1.0, 2.0 if up else 0.0, 0.0, rows=rows)


@pytest.mark.parametrize("n", [12000, 60000])
def test_symmetric_product_with_long_rows(gpu, n):
    """The upper-triangle product on a symmetric matrix with hub rows, deferred (n = 12000:
    to the window bin; n = 60000: to the 2^14-slot table and the dense pass, all in
    upper-triangle mode; lower parts longer than the shared-memory sorts): the same bits
    as full rows, and the oracle's values."""
    S = gpu
    hubs = set(range(0, n, 1500)) | {n - 1}
    X = hub_matrix(n, hubs, 700, 30, seed=5)
    Xs = O.add(X, O.transpose(X), 1.0, 1.0)  # symmetric: X + X^T
    dX = dev(S, Xs)
    probe = S.Ellpack.empty(n, 32)
    rc, info = S.sp2_step(dX, probe, n / 2, 0.0, raise_on_overflow=False)
    w = ((info.required_width + 31) // 32) * 32
    full = S.Ellpack.empty(n, w)
    info_f = S.sp2_step(dX, full, n / 2, 0.0)
    sym = S.Ellpack.empty(n, w)
    info_s = S.sp2_step(dX, sym, n / 2, 0.0, symmetric=True)
    assert info_f.rows_deferred > 0
    assert rows_equal(full.to_numpy(), sym.to_numpy())
    assert info_s.nnz_total == info_f.nnz_total and info_s.trXn == info_f.trXn
    # too narrow an output: the same overflow report as full rows
    narrow = S.Ellpack.empty(n, 64)
    rc_s, inf_s = S.sp2_step(dX, narrow, n / 2, 0.0, symmetric=True, raise_on_overflow=False)
    assert rc_s == S.SP2E_OVERFLOW and inf_s.required_width == info_f.max_row_nnz
    up = info_s.branch == 2
    rng = np.random.default_rng(6)
    rows = np.unique(np.concatenate([sorted(hubs), rng.choice(n, 200, replace=False)]))
    compare_spgemm(sym.to_numpy(), Xs, Xs, Xs, -1.0 if up else 1.0, 2.0 if up else 0.0, 0.0, rows=rows)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_window_bin_banded_long_rows(gpu, dtype):
    """A banded matrix with rows of ~3600 entries: every product row (~450 column groups)
    outgrows the block accumulator and is deferred to the dense-window bin (span ~7200
    columns).  Sampled rows against the oracle; symmetric and full products bit for bit
    equal."""
    S = gpu
    n, band = 12000, 1800
    H = ell(I.banded(n, band=band, seed=4, delta=10.0))
    dt = S.SP2_F64 if dtype == "f64" else S.SP2_F32
    Hq = f32_input(H) if dt == S.SP2_F32 else H
    dH = dev(S, Hq, dt)
    rc, info = S.sp2_step(dH, S.Ellpack.empty(n, 32, dt), n / 2, 1e-5, raise_on_overflow=False)
    w = ((info.required_width + 31) // 32) * 32
    full = S.Ellpack.empty(n, w, dt)
    info = S.sp2_step(dH, full, n / 2, 1e-5)
    assert info.rows_deferred > n // 2 and info.rows_dense == 0
    sym = S.Ellpack.empty(n, w, dt)
    S.sp2_step(dH, sym, n / 2, 1e-5, symmetric=True)
    assert rows_equal(full.to_numpy(), sym.to_numpy())
    up = info.branch == 2
    rows = np.unique(np.concatenate([[0, 1, band, n // 2, n - 1], np.random.default_rng(8).choice(n, 60, replace=False)]))
    compare_spgemm(full.to_numpy(), Hq, Hq, Hq, -1.0 if up else 1.0, 2.0 if up else 0.0, 1e-5, fp32=dt == S.SP2_F32,
                   rows=rows)


def test_cascade_levels_of_the_symmetric_step(gpu):
    """A banded X whose product rows span about 1920 columns above the diagonal: more 8-column
    blocks than the tight compact pass holds, fewer than the loose one.  Started at each level
    (sp2_step compact_level 0, 1, 2) the cascade gives the same bits as the full-row product,
    no row reaches the deferred-row bins, and sampled rows match the oracle (tau = 0: every
    structural entry kept)."""
    S = gpu
    n, band = 3000, 960
    X = ell(I.banded(n, band=band, seed=21, delta=10.0))
    dX = dev(S, X)
    rc, info = S.sp2_step(dX, S.Ellpack.empty(n, 32), n / 2, 0.0, raise_on_overflow=False)
    w = ((info.required_width + 31) // 32) * 32
    full = S.Ellpack.empty(n, w)
    info_f = S.sp2_step(dX, full, n / 2, 0.0)
    ref = full.to_numpy()
    for level in (0, 1, 2):
        out = S.Ellpack.empty(n, w)
        info_l = S.sp2_step(dX, out, n / 2, 0.0, symmetric=True, compact_level=level)
        assert info_l.rows_deferred == 0, level
        assert rows_equal(out.to_numpy(), ref), level
        assert (info_l.trXn, info_l.nnz_total) == (info_f.trXn, info_f.nnz_total)
    up = info_f.branch == 2
    rows = np.array([0, 1, 959, 960, 1500, 2040, 2999])
    compare_spgemm(ref, X, X, X, -1.0 if up else 1.0, 2.0 if up else 0.0, 0.0, rows=rows)
