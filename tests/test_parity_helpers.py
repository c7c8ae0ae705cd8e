"""The parity helpers the GPU tests compare with are themselves right: the sparse copy of an
ELLPACK matrix equals the dense one, padding ignored, and its Frobenius norm is numpy's (CPU)."""
import numpy as np

from paper_2102_08505_gb300 import inputs as I
from parity import dense_of, sparse_fro, sparse_of


def test_sparse_copy_matches_dense():
    for seed in range(4):
        n = 70
        a = I.random_sparse(n, seed=seed, min_nnz=0, max_nnz=12, full_rows=(3,))
        b = I.random_sparse(n, seed=seed + 10, min_nnz=0, max_nnz=12)
        Da, Db = dense_of(*a, n), dense_of(*b, n)
        Sa, Sb = sparse_of(*a, n), sparse_of(*b, n)
        assert np.array_equal(Sa.toarray(), Da)
        assert np.isclose(sparse_fro(Sa - Sb), np.linalg.norm(Da - Db), rtol=1e-14)
        assert Sa.nnz == int(a[2].sum())
