"""Pins of the oracle's standalone ELLPACK operations against dense numpy (CPU):
transpose, norms, drop threshold, scale and dense conversion."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2102_08505_gb300 import inputs as I


def _rand(n, seed, sym=False):
    return O.Ell(*I.random_sparse(n, seed=seed, min_nnz=0, max_nnz=9, symmetric=sym))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_transpose_is_the_dense_transpose(seed):
    A = _rand(40, seed)
    T = O.transpose(A)
    assert np.array_equal(T.to_dense(), A.to_dense().T)
    for j in range(T.n):
        c, _ = T.row(j)
        assert np.all(np.diff(c) > 0)
    TT = O.transpose(T, width=A.w)
    for i in range(A.n):
        assert np.array_equal(TT.row(i)[0], A.row(i)[0]) and np.array_equal(TT.row(i)[1], A.row(i)[1])


def test_transpose_of_a_permutation_is_its_inverse():
    n = 17
    p = np.random.default_rng(3).permutation(n)
    P = O.Ell(p[:, None].astype(np.int32), np.ones((n, 1)), np.ones(n, np.int32))
    Pt = O.transpose(P)
    assert np.array_equal(P.to_dense() @ Pt.to_dense(), np.eye(n))


def test_norms_match_numpy():
    A = _rand(50, 4)
    D = A.to_dense()
    mx, inf, fro = O.norms(A)
    assert mx == np.abs(D).max()
    assert inf == pytest.approx(np.linalg.norm(D, np.inf), rel=1e-15)
    assert fro == pytest.approx(np.linalg.norm(D, "fro"), rel=1e-15)
    assert O.norms(O.Ell(np.zeros((3, 1), np.int32), np.zeros((3, 1)), np.zeros(3, np.int32))) == (0.0, 0.0, 0.0)
    # identity: 1, 1, sqrt(n)
    n = 9
    E = O.Ell(np.arange(n)[:, None].astype(np.int32), np.ones((n, 1)), np.ones(n, np.int32))
    assert O.norms(E) == (1.0, 1.0, pytest.approx(3.0))


def test_threshold_and_scale():
    A = _rand(30, 5)
    D = A.to_dense()
    T = O.threshold(A, 0.3)
    assert np.array_equal(T.to_dense(), np.where(np.abs(D) > 0.3, D, 0.0))
    # strict rule: an entry equal to tau is dropped
    E = O.Ell(np.array([[0, 1]], np.int32), np.array([[0.5, 0.25]]), np.array([2], np.int32))
    assert O.threshold(E, 0.25).nnz[0] == 1
    Z = O.Ell(np.array([[0, 1]], np.int32), np.array([[0.0, -1.0]]), np.array([2], np.int32))
    assert O.threshold(Z, 0.0).nnz[0] == 1  # exact zeros are dropped at tau = 0
    S = O.scale(A, -2.5)
    assert np.array_equal(S.to_dense(), -2.5 * D)


def test_from_dense_round_trip():
    A = _rand(25, 6)
    D = A.to_dense()
    B = O.from_dense_tau(D, 0.0)
    assert np.array_equal(B.to_dense(), D)
    C = O.from_dense_tau(D, 0.4)
    assert np.array_equal(C.to_dense(), np.where(np.abs(D) > 0.4, D, 0.0))
