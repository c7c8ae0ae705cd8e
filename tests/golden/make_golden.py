"""Writes the stored oracle results under tests/golden/ (run from the repository root:
python tests/golden/make_golden.py).  It calls only the oracle and the seeded input
generators; the paper prints no worked example whose values could be stored instead.

The files pin the oracle against unintended change: tests/test_golden.py recomputes each
case and requires the same branch sequence and iteration count, and traces equal to the
stored ones to 1e-13 relative."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2102_08505_gb300 import inputs as I  # noqa: E402

CASES = {
    # banded, gapped (A/B splitting 10), n = 256, band 8, tau 1e-5, tol 1e-10
    "sp2_banded_gapped_n256": dict(gen="banded", args=dict(n=256, band=8, seed=3, delta=10.0), nocc=128,
                                   tol=1e-10, tau=1e-5),
    # 3D tight-binding, gapped, open cluster, n = 512, tau 1e-5
    "sp2_tb_gapped_n512": dict(gen="tight_binding", args=dict(n=512, seed=5, delta=10.0, periodic=False),
                               nocc=256, tol=1e-10, tau=1e-5),
}


def run(case):
    gen = getattr(I, case["gen"])
    H = O.Ell(*gen(**case["args"]))
    D, st = O.sp2(H, case["nocc"], case["tol"], case["tau"], max_iter=100)
    return {"iterations": int(st["iterations"]), "status": st["status"], "branch": list(st["branch"]),
            "trX": [float(x) for x in st["trX"]], "trX2": [float(x) for x in st["trX2"]],
            "emin": float(st["emin"]), "emax": float(st["emax"]), "nnz_D": int(D.nnz.sum()),
            "trace_D": float(O.trace(D))}


def main():
    for name, case in CASES.items():
        out = {"case": case, "result": run(case)}
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print("wrote", name)


if __name__ == "__main__":
    main()
