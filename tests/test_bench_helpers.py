"""The product counts the benchmark's roofline is built on (CPU): fma_count is the number of
products of X*X and fma_count_upper the number the upper-triangle product executes, both
against brute force; for a symmetric pattern the upper count is (all products + stored
entries) / 2, since (i, k, j) <-> (j, k, i) pairs the products with j > i and j < i."""
import numpy as np

import bench
from paper_2102_08505_gb300 import inputs as I


def brute(idx, nnz):
    n = len(nnz)
    rows = [idx[i, :nnz[i]] for i in range(n)]
    total = sum(len(rows[k]) for i in range(n) for k in rows[i])
    upper = sum(int((rows[k] >= i).sum()) for i in range(n) for k in rows[i])
    return total, upper


def test_counts_match_brute_force():
    for seed in range(5):
        idx, val, nnz = I.random_sparse(90, seed=seed, min_nnz=0, max_nnz=15, full_rows=(7,), empty_rows=(3,))
        total, upper = brute(idx, nnz)
        assert bench.fma_count(idx, nnz) == total
        assert bench.fma_count_upper(idx, nnz) == upper


def test_upper_count_closed_form_for_symmetric_patterns():
    for make in (lambda: I.banded(150, band=6, seed=2), lambda: I.tight_binding(600, seed=4),
                 lambda: I.random_sparse(120, seed=9, max_nnz=10, symmetric=True)):
        idx, val, nnz = make()
        total = bench.fma_count(idx, nnz)
        assert 2 * bench.fma_count_upper(idx, nnz) == total + int(nnz.sum())
