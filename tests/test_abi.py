"""The C-ABI library builds for sm_103a, loads, and exports every function declared in
include/sp2ell.h; the Python binding names the same functions.  No compute call (CPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sp2ell.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|double)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which(os.environ.get("NVCC", "nvcc")) is None:
        pytest.skip("nvcc not available")
    from paper_2102_08505_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["ellpack_create", "ellpack_multiply", "ellpack_add", "ellpack_trace", "sp2_purify"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, "declared but not exported: %s" % missing


def test_library_loads_and_binding_matches(libpath):
    L = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(L, n)
    from paper_2102_08505_gb300 import sp2ell
    assert sp2ell.lib.sp2_version() >= 10000
    for n in declared_functions():
        assert hasattr(sp2ell.lib, n)
    # host-side argument checks run without a GPU and report through the error string
    rc = sp2ell.lib.ellpack_wrap(0, 32, 0, None, None, None, ctypes.byref(sp2ell.ellpack_t()))
    assert rc == sp2ell.SP2E_ARG
    assert b"n = 0" in sp2ell.lib.sp2_last_error_string()


def test_options_defaults(libpath):
    from paper_2102_08505_gb300 import sp2ell
    o = sp2ell.sp2_options_default()
    assert (o.precision, o.max_iter, o.stall_rule, o.n_fp64_tail, o.tau) == (0, 100, 1, 2, 1e-5)
    assert (o.stall_arm, o.stall_ratio, o.symmetric) == (0.1, 1.0, 1)
    assert (o.route_rows, o.small_path, o.level_up_frac) == (1, 1, 1.0)


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of its C
    declaration in include/sp2ell.h (a C program built against the header prints them)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2102_08505_gb300 import sp2ell
    structs = [sp2ell.ellpack_t, sp2ell.nnzpred_t, sp2ell.sp2_options, sp2ell.sp2_stats, sp2ell.sp2_step_info,
               sp2ell.sp2_profile]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sp2ell.h"', 'int main(void) {']
    for st in structs:
        c = st.__name__
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (c, c))
        for f in st._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (c, f[0], c, f[0]))
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = dict(l.split() for l in out if l.strip())
    for st in structs:
        c = st.__name__
        assert int(c_layout[c]) == ctypes.sizeof(st), c
        for f in st._fields_:
            assert int(c_layout["%s.%s" % (c, f[0])]) == getattr(st, f[0]).offset, (c, f[0])
