"""Pins of the CPU oracle against what mathematics fixes independently of it.

Each check compares the oracle with something it does not compute itself: dense numpy
products on tiny inputs, closed-form projectors, LAPACK eigendecompositions, exact
special cases.  The mutation tests at the end plant a plausible mistake in a copy of
the oracle source and show that one of these pins fails on it.
"""
import math
import os

import numpy as np
import pytest

from oracle import build as obuild
from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I


def ell(t):
    return O.Ell(*t)


def structural(E):
    """0/1 pattern matrix built from the stored indices (not from the values)."""
    P = np.zeros((E.n, E.n), np.int64)
    for i in range(E.n):
        P[i, E.row(i)[0]] = 1
    return P


def abs_scale(A, B, C, alpha, beta):
    Ad, Bd = np.abs(A.to_dense()), np.abs(B.to_dense())
    s = abs(alpha) * Ad @ Bd
    if C is not None and beta != 0:
        s = s + abs(beta) * np.abs(C.to_dense())
    return s


CASES = [
    # n, seed, min_nnz, max_nnz, full_rows, empty_rows
    (17, 0, 0, 5, (3,), (0, 7)),
    (40, 1, 1, 9, (5, 6), (11,)),
    (64, 2, 0, 12, (), (1, 2, 3)),
]
ALPHA_BETA = [(1.0, 0.0), (-1.0, 2.0), (0.75, -1.25)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("ab", ALPHA_BETA)
def test_spgemm_tau0_matches_dense_bruteforce(case, ab):
    n, seed, lo, hi, full, empty = case
    alpha, beta = ab
    A = ell(I.random_sparse(n, seed=seed, min_nnz=lo, max_nnz=hi, full_rows=full, empty_rows=empty, width=hi))
    B = ell(I.random_sparse(n, seed=seed + 100, min_nnz=lo, max_nnz=hi, empty_rows=empty[:1]))
    C = ell(I.random_sparse(n, seed=seed + 200, min_nnz=0, max_nnz=4))
    out = O.spgemm(A, B, C, alpha, beta, 0.0)
    ref = alpha * A.to_dense() @ B.to_dense() + beta * C.to_dense()
    scale = abs_scale(A, B, C, alpha, beta)
    got = out.to_dense()
    assert np.all(np.abs(got - ref) <= 1e-14 * scale + 1e-300)
    # exact structural pattern (independent of cancellation)
    pat = (structural(A) @ structural(B)) > 0
    if beta != 0:
        pat |= structural(C) > 0
    assert np.array_equal(structural(out) > 0, pat)
    # rows sorted, no duplicates
    for i in range(n):
        c = out.row(i)[0]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("tau", [1e-3, 0.05, 0.3])
def test_spgemm_drop_rule(tau):
    n = 48
    A = ell(I.random_sparse(n, seed=5, min_nnz=1, max_nnz=10))
    B = ell(I.random_sparse(n, seed=6, min_nnz=1, max_nnz=10))
    out = O.spgemm(A, B, None, 1.0, 0.0, tau)
    ref = A.to_dense() @ B.to_dense()
    pat = (structural(A) @ structural(B)) > 0
    keep = pat & (np.abs(ref) > tau)
    near = np.abs(np.abs(ref) - tau) <= 1e-14 * abs_scale(A, B, None, 1.0, 0.0)
    got = structural(out) > 0
    assert np.all((got == keep) | near)
    assert np.allclose(out.to_dense()[got], ref[got], rtol=0, atol=1e-14)


def test_keep_rule_is_strict():
    """An entry equal to tau is dropped, one just above is kept, and tau = 0 keeps
    structural zeros."""
    B = O.from_dense(np.array([[0.25, -0.5, 0.0], [0.0, -0.25, 0.25000000000000006], [0.0, 0.0, 1.0]]))
    out = O.spgemm(O.from_dense(np.eye(3)), B, None, 1.0, 0.0, 0.25)
    assert [set(out.row(i)[0].tolist()) for i in range(3)] == [{1}, {2}, {2}]
    Z = O.Ell(np.array([[0, 1], [0, 0]], np.int32), np.array([[1.0, 0.0], [0.0, 0.0]]), np.array([2, 0], np.int32))
    out = O.spgemm(O.from_dense(np.eye(2)), Z, None, 1.0, 0.0, 0.0)
    assert out.nnz.tolist() == [2, 0] and out.row(0)[1].tolist() == [1.0, 0.0]


def test_spgemm_identity_and_diagonal_are_exact():
    n = 30
    B = ell(I.random_sparse(n, seed=9, min_nnz=0, max_nnz=7))
    Id = O.from_dense(np.eye(n))
    out = O.spgemm(Id, B)
    assert np.array_equal(out.to_dense(), B.to_dense())
    d = np.linspace(-2.0, 3.0, n) + 0.1
    Dm = O.from_dense(np.diag(d))
    out = O.spgemm(Dm, B)
    assert np.array_equal(out.to_dense(), d[:, None] * B.to_dense())  # one product per entry: exact
    out = O.spgemm(B, Dm)
    assert np.array_equal(out.to_dense(), B.to_dense() * d[None, :])


def test_spgemm_order_of_operands():
    """A*B differs from B*A and from A^T*B on non-symmetric inputs: catches a transposed
    operand."""
    n = 25
    A = ell(I.random_sparse(n, seed=11, min_nnz=2, max_nnz=6))
    B = ell(I.random_sparse(n, seed=12, min_nnz=2, max_nnz=6))
    got = O.spgemm(A, B).to_dense()
    Ad, Bd = A.to_dense(), B.to_dense()
    assert np.allclose(got, Ad @ Bd, atol=1e-14)
    assert not np.allclose(got, Bd @ Ad, atol=1e-6)
    assert not np.allclose(got, Ad.T @ Bd, atol=1e-6)


def test_spgemm_rows_subset_matches_full():
    n = 50
    A = ell(I.random_sparse(n, seed=21, min_nnz=0, max_nnz=8))
    full = O.spgemm(A, A, A, -1.0, 2.0, 0.01)
    rows = [49, 0, 17, 17, 3]
    part = O.spgemm(A, A, A, -1.0, 2.0, 0.01, rows=rows)
    for r, i in enumerate(rows):
        assert np.array_equal(part.row(r)[0], full.row(i)[0])
        assert np.array_equal(part.row(r)[1], full.row(i)[1])


@pytest.mark.parametrize("ab", ALPHA_BETA)
def test_add_matches_dense(ab):
    alpha, beta = ab
    n = 40
    A = ell(I.random_sparse(n, seed=31, min_nnz=0, max_nnz=6))
    B = ell(I.random_sparse(n, seed=32, min_nnz=0, max_nnz=6))
    out = O.add(A, B, alpha, beta, 0.0)
    assert np.allclose(out.to_dense(), alpha * A.to_dense() + beta * B.to_dense(), rtol=0, atol=1e-15)
    assert np.array_equal(structural(out) > 0, (structural(A) + structural(B)) > 0)


def test_trace_and_gershgorin_dense():
    H = ell(I.banded(96, band=5, seed=3))
    Hd = H.to_dense()
    assert abs(O.trace(H) - np.trace(Hd)) <= 1e-13 * np.abs(np.diag(Hd)).sum()
    lo, hi = O.gershgorin(H)
    radius = np.abs(Hd).sum(axis=1) - np.abs(np.diag(Hd))
    assert lo == pytest.approx(np.min(np.diag(Hd) - radius), abs=1e-13)
    assert hi == pytest.approx(np.max(np.diag(Hd) + radius), abs=1e-13)
    ev = np.linalg.eigvalsh(Hd)
    assert lo <= ev.min() + 1e-12 and ev.max() <= hi + 1e-12


def test_x0_dense_formula_and_spectrum():
    H = ell(I.banded(80, band=4, seed=4))
    lo, hi = O.gershgorin(H)
    X = O.x0(H, lo, hi, 0.0)
    ref = (hi * np.eye(80) - H.to_dense()) / (hi - lo)
    assert np.allclose(X.to_dense(), ref, rtol=0, atol=1e-15)
    ev = np.linalg.eigvalsh(X.to_dense())
    assert ev.min() >= -1e-12 and ev.max() <= 1 + 1e-12  # Gershgorin maps the spectrum into [0, 1]
    # a Hamiltonian without diagonal entries still gets one per row
    Hz = O.from_dense(H.to_dense() - np.diag(np.diag(H.to_dense())))
    lo, hi = O.gershgorin(Hz)
    Xz = O.x0(Hz, lo, hi, 0.0)
    for i in range(80):
        assert i in set(Xz.row(i)[0].tolist())
    assert np.allclose(np.diag(Xz.to_dense()), hi / (hi - lo))


def test_sp2_diagonal_closed_form():
    """Diagonal H: D is the 0/1 indicator of the nocc lowest diagonal entries."""
    rng = np.random.default_rng(7)
    n, nocc = 64, 23
    h = rng.permutation(np.linspace(-3.0, 2.0, n))
    D, st = O.sp2(O.from_dense(np.diag(h)), nocc, 1e-12, 0.0, max_iter=100)
    want = np.zeros(n)
    want[np.argsort(h)[:nocc]] = 1.0
    assert np.allclose(np.diag(D.to_dense()), want, atol=1e-10)
    assert st["status"] == "converged"


def test_sp2_two_by_two_blocks_closed_form():
    """Block-diagonal H of 2x2 blocks [[a, b], [b, c]]: with every lower eigenvalue below
    every upper one and nocc = number of blocks, D is block-diagonal with v v^T, v the
    lower eigenvector, given in closed form."""
    rng = np.random.default_rng(8)
    m = 20
    a = rng.uniform(-1.0, 1.0, m)
    c = rng.uniform(-1.0, 1.0, m)
    b = rng.uniform(2.0, 3.0, m)
    Hd = np.zeros((2 * m, 2 * m))
    Dref = np.zeros_like(Hd)
    for t in range(m):
        Hd[2 * t:2 * t + 2, 2 * t:2 * t + 2] = [[a[t], b[t]], [b[t], c[t]]]
        lam = 0.5 * (a[t] + c[t]) - math.sqrt(0.25 * (a[t] - c[t]) ** 2 + b[t] ** 2)
        v = np.array([b[t], lam - a[t]])
        v /= np.linalg.norm(v)
        Dref[2 * t:2 * t + 2, 2 * t:2 * t + 2] = np.outer(v, v)
    D, st = O.sp2(O.from_dense(Hd), m, 1e-13, 0.0)
    assert np.allclose(D.to_dense(), Dref, atol=1e-10)


def test_sp2_tridiagonal_toeplitz_closed_form():
    """Tridiagonal Toeplitz H (diagonal a, off-diagonal b < 0): eigenpairs
    a + 2b cos(k pi/(n+1)), sqrt(2/(n+1)) sin(j k pi/(n+1)) (k = 1..n, ascending)."""
    n, nocc, a, b = 40, 20, 0.3, -1.0
    Hd = a * np.eye(n) + b * (np.eye(n, k=1) + np.eye(n, k=-1))
    j = np.arange(1, n + 1)
    V = np.stack([np.sqrt(2.0 / (n + 1)) * np.sin(j * k * np.pi / (n + 1)) for k in range(1, nocc + 1)], axis=1)
    Dref = V @ V.T
    D, st = O.sp2(O.from_dense(Hd), nocc, 1e-13, 0.0)
    assert np.allclose(D.to_dense(), Dref, atol=1e-9)


def test_sp2_matches_eigen_projector_gapped_banded():
    n = 256
    H = ell(I.banded(n, band=16, seed=1, delta=10.0))
    D, st = O.sp2(H, n // 2, 1e-13, 0.0)
    c = O.checks(H.to_dense(), D.to_dense(), n // 2)
    assert c["gap"] > 1.0
    assert c["proj_err"] < 1e-10
    assert c["trace_err"] < 1e-8
    assert c["idem_err"] < 1e-8
    assert c["comm_err"] < 1e-8
    # the recorded trace sequence obeys the branch rule that was taken
    for t, br in enumerate(st["branch"]):
        up = abs(2 * st["trX"][t] - st["trX2"][t] - n // 2) < abs(st["trX2"][t] - n // 2)
        assert br == ("2X-X2" if up else "X2")
        nxt = (2 * st["trX"][t] - st["trX2"][t]) if up else st["trX2"][t]
        assert st["trX"][t + 1] == pytest.approx(nxt, abs=1e-9)


def test_sp2_thresholded_invariants():
    """tau > 0: not the exact projector, but trace and idempotency stay small and the
    stall rule stops the loop."""
    n = 512
    H = ell(I.banded(n, band=16, seed=2, delta=10.0))
    D, st = O.sp2(H, n // 2, 1e-10, 1e-5)
    Dd = D.to_dense()
    c = O.checks(H.to_dense(), Dd, n // 2)
    assert c["trace_err"] < 1e-3
    assert c["idem_err"] < 1e-3
    assert c["proj_err"] < 1e-3
    assert st["status"] in ("converged", "stalled")


def tie_matrix(n, seed, tau, with_zeros=True):
    """Sparse matrix whose stored values include exact ties at +-tau, exact zeros (stored
    structurally) and values one ulp on either side of tau, beside random values."""
    rng = np.random.default_rng(seed)
    idx, val, nnz = I.random_sparse(n, seed=seed, min_nnz=0, max_nnz=9)
    special = [tau, -tau, np.nextafter(tau, 1.0), -np.nextafter(tau, 1.0), np.nextafter(tau, 0.0),
               -np.nextafter(tau, 0.0)] + ([0.0, -0.0] if with_zeros else [])
    for i in range(n):
        for s_ in range(nnz[i]):
            if rng.random() < 0.4:
                val[i, s_] = special[int(rng.integers(len(special)))]
    return O.Ell(idx, val, nnz)


@pytest.mark.parametrize("tau", [0.0, 0.05, 0.25])
def test_drop_matches_dense(tau):
    """The drop of the X^2 branch: keep (j, v) iff |v| > tau (an entry equal to tau is
    removed, one ulp above it stays); tau = 0 keeps every stored entry, zeros included.
    Reference: numpy thresholding of the dense matrix."""
    n = 48
    A = tie_matrix(n, 61, tau if tau > 0 else 0.125)
    out = O.drop(A, tau)
    Ad = A.to_dense()
    if tau == 0.0:
        assert np.array_equal(structural(out), structural(A))
        assert np.array_equal(out.to_dense(), Ad)
        return
    keep = (structural(A) > 0) & (np.abs(Ad) > tau)
    assert np.array_equal(structural(out) > 0, keep)
    assert np.array_equal(out.to_dense(), np.where(keep, Ad, 0.0))
    for i in range(n):  # stored order stays ascending
        assert np.all(np.diff(out.row(i)[0]) > 0)


@pytest.mark.parametrize("ab", ALPHA_BETA)
@pytest.mark.parametrize("tau", [0.05, 0.25])
def test_add_thresholded_matches_dense(ab, tau):
    """drop_tau(alpha A + beta B) at tau > 0 against the dense numpy formula: the pattern
    is the union of the two patterns where |alpha a + beta b| > tau, values exact (both
    sides round alpha*a and beta*b separately and then add them)."""
    alpha, beta = ab
    n = 48
    A = tie_matrix(n, 71, tau)
    B = tie_matrix(n, 72, tau)
    out = O.add(A, B, alpha, beta, tau)
    v = alpha * A.to_dense() + beta * B.to_dense()
    union = (structural(A) + structural(B)) > 0
    keep = union & (np.abs(v) > tau)
    assert np.array_equal(structural(out) > 0, keep)
    assert np.array_equal(out.to_dense(), np.where(keep, v, 0.0))


def test_add_exact_tie_is_dropped():
    """alpha*a + beta*b landing exactly on tau is dropped; one ulp above is kept."""
    tau = 0.25
    up = np.nextafter(0.125, 1.0)  # 0.125 + 2^-55; twice that is 0.25 + 2^-54, one ulp above tau
    A = O.from_dense(np.array([[0.125, up, 0.5], [0.0, 0.25, 0.0], [0.0, 0.0, 0.125]]))
    B = O.from_dense(np.array([[0.125, up, -0.25], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0625]]))
    out = O.add(A, B, 1.0, 1.0, tau)
    # row 0: 0.25 (tie, dropped), 0.25 + ulp (kept), 0.25 (tie, dropped); row 1: 0.25 (tie);
    # row 2: 0.1875 (below)
    assert out.nnz.tolist() == [1, 0, 0]
    assert out.row(0)[0].tolist() == [1]
    out2 = O.add(A, B, 2.0, 0.0, tau)  # 2 * 0.125 = tau: dropped; 2 * up, 2 * 0.5, 2 * 0.25 kept
    assert out2.nnz.tolist() == [2, 1, 0]
    assert out2.row(0)[0].tolist() == [1, 2]


def dense_sp2(Hd, nocc, tol, tau, max_iter=100, stall_arm=0.1, stall_ratio=1.0):
    """SP2 restated on dense numpy arrays with the same readings (Gershgorin X0, branch on
    the trace rule, drop |v| > tau after each update, error |trX - trX2| / N, stall rule).
    Dense matrix products and thresholding; no code shared with the oracle."""
    n = Hd.shape[0]
    d = np.diag(Hd)
    rad = np.abs(Hd).sum(axis=1) - np.abs(d)
    lo, hi = float(np.min(d - rad)), float(np.max(d + rad))
    X = (hi * np.eye(n) - Hd) / (hi - lo)
    X = np.where(np.abs(X) > tau, X, 0.0)
    errs, branch = [], []
    armed = False
    it = 0
    while True:
        P = X @ X
        trX, trX2 = float(np.trace(X)), float(np.trace(P))
        err = abs(trX - trX2) / n
        errs.append(err)
        if err < tol:
            status = "converged"
            break
        if stall_arm > 0:
            if abs(trX - trX2) < stall_arm:
                armed = True
            if armed and it >= 2 and err >= stall_ratio * errs[it - 2]:
                status = "stalled"
                break
        if it >= max_iter:
            status = "max_iter"
            break
        if abs(2 * trX - trX2 - nocc) < abs(trX2 - nocc):
            branch.append("2X-X2")
            X = 2.0 * X - P
        else:
            branch.append("X2")
            X = P
        X = np.where(np.abs(X) > tau, X, 0.0)
        it += 1
    return X, {"iterations": it, "branch": branch, "err": np.array(errs), "status": status}


@pytest.mark.parametrize("tau", [1e-4, 1e-3])
def test_sp2_thresholded_matches_dense_restatement(tau):
    """tau > 0: the oracle's SP2 (sparse products, its own drop and add) against the dense
    restatement above: the same iterations, branches and stop, D's pattern exactly the
    dense nonzeros, values within 1e-12."""
    n = 96
    H = ell(I.banded(n, band=6, seed=4, delta=10.0))
    D, st = O.sp2(H, n // 2, 1e-10, tau)
    Dd, sd = dense_sp2(H.to_dense(), n // 2, 1e-10, tau)
    assert st["iterations"] == sd["iterations"]
    assert st["branch"] == sd["branch"]
    assert st["status"] == sd["status"]
    assert "X2" in st["branch"] and "2X-X2" in st["branch"]
    assert np.array_equal(structural(D) > 0, Dd != 0.0)
    assert np.max(np.abs(D.to_dense() - Dd)) < 1e-12


# ---------------------------------------------------------------- planted mistakes
MUTANTS = {
    "dropped_beta_term": [("double v = alpha * acc[j] + beta * cv[j];", "double v = alpha * acc[j];")],
    "wrong_sign_alpha": [("double v = alpha * acc[j] + beta * cv[j];", "double v = -alpha * acc[j] + beta * cv[j];")],
    "wrong_row_index": [("double b = B->val[(size_t)k * B->w + s];", "double b = B->val[(size_t)j * B->w + s];")],
    "keep_rule_ge": [("if (tau == 0.0 || fabs(v) > tau) list[kept++] = j, acc[j] = v;",
                      "if (tau == 0.0 || fabs(v) >= tau) list[kept++] = j, acc[j] = v;")],
    "x0_sign": [("if (j == i) { x = (emax - h) / (emax - emin); has_diag = 1; }",
                 "if (j == i) { x = (emax + h) / (emax - emin); has_diag = 1; }")],
    "branch_flipped": [("if (fabs(2.0 * trX - trX2 - nocc) < fabs(trX2 - nocc)) {",
                        "if (fabs(2.0 * trX - trX2 - nocc) > fabs(trX2 - nocc)) {")],
    "gershgorin_radius": [("if (j == i) d = v; else r = r + fabs(v);", "if (j == i) d = v; else r = r + v;")],
    "drop_ignores_tau": [("      if (tau == 0.0 || fabs(v) > tau) {\n        out->idx[(size_t)i * out->w + kept]",
                          "      if (1) {\n        out->idx[(size_t)i * out->w + kept]")],
    "add_keep_ge": [("if (tau == 0.0 || fabs(v) > tau) { list[kept++] = j; av[j] = v; }",
                     "if (tau == 0.0 || fabs(v) >= tau) { list[kept++] = j; av[j] = v; }")],
}


def _pins_pass():
    """A compact subset of the pins above; returns False as soon as one fails."""
    try:
        n = 24
        A = ell(I.random_sparse(n, seed=41, min_nnz=1, max_nnz=6))
        B = ell(I.random_sparse(n, seed=42, min_nnz=1, max_nnz=6))
        C = ell(I.random_sparse(n, seed=43, min_nnz=1, max_nnz=4))
        out = O.spgemm(A, B, C, 0.75, -1.25, 0.0)
        ref = 0.75 * A.to_dense() @ B.to_dense() - 1.25 * C.to_dense()
        if not np.allclose(out.to_dense(), ref, atol=1e-13):
            return False
        out = O.spgemm(A, B, None, 1.0, 0.0, 0.05)
        refp = A.to_dense() @ B.to_dense()
        pat = ((structural(A) @ structural(B)) > 0) & (np.abs(refp) > 0.05)
        if not np.array_equal(structural(out) > 0, pat):
            return False
        # an entry exactly at the tolerance is dropped (strict keep rule |v| > tau)
        Bt = O.from_dense(np.array([[0.25, -0.5], [0.0, -0.25]]))
        kept = O.spgemm(O.from_dense(np.eye(2)), Bt, None, 1.0, 0.0, 0.25)
        if kept.nnz.tolist() != [1, 0]:
            return False
        H = ell(I.banded(64, band=3, seed=3))
        lo, hi = O.gershgorin(H)
        Hd = H.to_dense()
        radius = np.abs(Hd).sum(axis=1) - np.abs(np.diag(Hd))
        if abs(lo - np.min(np.diag(Hd) - radius)) > 1e-13 or abs(hi - np.max(np.diag(Hd) + radius)) > 1e-13:
            return False
        ref0 = (hi * np.eye(64) - H.to_dense()) / (hi - lo)
        if not np.allclose(O.x0(H, lo, hi, 0.0).to_dense(), ref0, atol=1e-14):
            return False
        Hg = ell(I.banded(64, band=4, seed=5, delta=10.0))
        D, st = O.sp2(Hg, 32, 1e-12, 0.0, max_iter=60)
        c = O.checks(Hg.to_dense(), D.to_dense(), 32)
        if not c["proj_err"] < 1e-9:
            return False
        # drop and add at tau > 0 with exact ties, against dense thresholding
        T = tie_matrix(24, 81, 0.25)
        Td = T.to_dense()
        if not np.array_equal(O.drop(T, 0.25).to_dense(), np.where(np.abs(Td) > 0.25, Td, 0.0)):
            return False
        T2 = tie_matrix(24, 82, 0.25)
        v = T.to_dense() + T2.to_dense()
        if not np.array_equal(O.add(T, T2, 1.0, 1.0, 0.25).to_dense(), np.where(np.abs(v) > 0.25, v, 0.0)):
            return False
        Ht = ell(I.banded(64, band=5, seed=4, delta=10.0))
        Dt, stt = O.sp2(Ht, 32, 1e-10, 1e-3)
        Dtd, sdt = dense_sp2(Ht.to_dense(), 32, 1e-10, 1e-3)
        return (stt["branch"] == sdt["branch"] and np.array_equal(structural(Dt) > 0, Dtd != 0.0)
                and np.max(np.abs(Dt.to_dense() - Dtd)) < 1e-12)
    except Exception:
        return False


def test_pins_pass_on_the_oracle():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    path = obuild.build_variant(MUTANTS[name], str(tmp_path / ("mut_%s.so" % name)))
    with O.use_variant(path):
        assert not _pins_pass(), "planted mistake %r was not caught by the pins" % name


def test_stall_arm_threshold_variants():
    """The stall rule's arming threshold: never armed (tiny threshold) is the same run as no
    stall rule; armed from the start (huge threshold) stops a gapless system no later than
    the reading's 0.1, and the stop is by the stall rule."""
    H = ell(I.banded(256, band=8, seed=1, delta=0.0))
    D0, s0 = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall=False)
    Dn, sn = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall_arm=1e-300)
    assert sn["iterations"] == s0["iterations"] and sn["status"] == s0["status"] == "max_iter"
    assert np.array_equal(Dn.to_dense(), D0.to_dense())
    Dd, sd = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60)
    Da, sa = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall_arm=1e300)
    assert sa["status"] == "stalled" and sa["iterations"] <= sd["iterations"]
    # armed from the start, the rule fires at the first n >= 2 with err_n >= err_{n-2}
    e = sa["err"]
    first = next(k for k in range(2, len(e)) if e[k] >= e[k - 2])
    assert sa["iterations"] == first


def test_stall_ratio_variants():
    """The stall rule's ratio on the gapless banded Hamiltonian at tau = 1e-5 (its error
    settles at a floor): ratio 1 is the default run; with a smaller ratio the rule fires at
    the first armed n with err_n >= ratio * err_{n-2} of the unstopped run's error sequence,
    never later than with a larger ratio; the iterates before the stop are the unstopped
    run's."""
    H = ell(I.banded(256, band=8, seed=1, delta=0.0))
    D0, s0 = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall=False)
    Dd, sd = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60)
    D1, s1 = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall_ratio=1.0)
    assert s1["iterations"] == sd["iterations"] and np.array_equal(D1.to_dense(), Dd.to_dense())
    e = s0["err"]
    armed_from = next(k for k in range(len(e)) if 256 * e[k] < 0.1)
    last = 10 ** 9
    for ratio in (1.0, 0.99, 0.9, 0.5):
        Dr, sr = O.sp2(H, 128, 1e-14, 1e-5, max_iter=60, stall_ratio=ratio)
        want = next((k for k in range(max(2, armed_from), len(e)) if e[k] >= ratio * e[k - 2]), None)
        if want is None:
            assert sr["status"] == "max_iter"
            continue
        assert sr["status"] == "stalled" and sr["iterations"] == want
        assert np.array_equal(sr["err"], e[:want + 1]) and sr["branch"] == s0["branch"][:want]
        assert want <= last
        last = want
    with pytest.raises(ValueError):
        O.sp2(H, 128, 1e-14, 1e-5, max_iter=5, stall_ratio=0.0)
    with pytest.raises(ValueError):
        O.sp2(H, 128, 1e-14, 1e-5, max_iter=5, stall_ratio=1.5)
