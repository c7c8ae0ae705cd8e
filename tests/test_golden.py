"""Stored oracle results (tests/golden/*.json, written by tests/golden/make_golden.py from
the oracle alone) recomputed: same iterations, status, branches and nnz; traces and
bounds to 1e-13 relative (CPU).  The GPU side of the same cases is checked against them
in tests/test_gpu_golden.py."""
import glob
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

FILES = sorted(glob.glob(os.path.join(HERE, "golden", "*.json")))


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(p) for p in FILES])
def test_oracle_reproduces_stored_result(path):
    d = json.load(open(path))
    r = make_golden.run(d["case"])
    s = d["result"]
    for k in ("iterations", "status", "branch", "nnz_D"):
        assert r[k] == s[k], k
    for k in ("trX", "trX2"):
        assert np.allclose(r[k], s[k], rtol=1e-13, atol=1e-12), k
    for k in ("emin", "emax", "trace_D"):
        assert r[k] == pytest.approx(s[k], rel=1e-13), k


def test_golden_cases_exist():
    assert len(FILES) == len(make_golden.CASES) >= 2
