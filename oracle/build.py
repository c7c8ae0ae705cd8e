"""Builds the CPU oracle shared library (test infrastructure only).

The oracle is compiled with plain gcc and -ffp-contract=off so that the arithmetic is
exactly the separately rounded multiplies and adds written in sp2_oracle.c.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sp2_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def build_variant(replacements, out_path):
    """Compiles a copy of sp2_oracle.c with textual replacements (old -> new) applied.
    Used only by tests that plant a mistake in the oracle to show that a pin catches it."""
    src = open(SRC).read()
    for old, new in replacements:
        if old not in src:
            raise ValueError("replacement target not found: %r" % old)
        src = src.replace(old, new)
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", out_path, c_path, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


if __name__ == "__main__":
    print(build(force=True))
