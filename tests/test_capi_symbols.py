"""The C-ABI library builds, loads and exports every function its header
declares.  No compute call is made (these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for h in os.listdir(INCLUDE):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:int|void|const\s+char\s*\*)\s*\*?\s*(gb_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2603_07850_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gb_init", "gb_verify_range", "gb_submit", "gb_poll", "gb_set_option",
                     "gb_verify_range_segments", "gb_stats", "gb_last_error", "gb_shutdown"]:
        assert required in names


def test_header_is_plain_c():
    # the public header must compile as C99 with no CUDA or C++ headers
    subprocess.check_call(["gcc", "-std=c99", "-fsyntax-only", "-Wall", "-Werror", "-x", "c",
                           os.path.join(INCLUDE, "goldbach_gb300.h")])


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_build_exports_the_same_boundary():
    # the GB_DEBUG variant (bounds checks on the shared-memory window) is the
    # same library with the checks compiled in
    from paper_2603_07850_gb300 import build
    dbg = ctypes.CDLL(build.build(debug=True))
    missing = [n for n in declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_2603_07850_gb300 import binding
    for n in declared_functions():
        assert callable(getattr(binding, n)), n


def test_struct_sizes_match_header():
    # sizes of the public structs as compiled by the C compiler vs the binding
    from paper_2603_07850_gb300 import binding
    prog = r'''
#include <stdio.h>
#include "goldbach_gb300.h"
int main(void){printf("%zu %zu %zu\n", sizeof(gb_result), sizeof(gb_seg_record), sizeof(gb_stats_t));return 0;}
'''
    exe = os.path.join(ROOT, "oracle", "_build", "sizes_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    src = exe + ".c"
    open(src, "w").write(prog)
    subprocess.check_call(["gcc", "-std=c99", "-I", INCLUDE, src, "-o", exe])
    out = subprocess.check_output([exe]).decode().split()
    assert [int(x) for x in out] == [ctypes.sizeof(binding.GbResult), ctypes.sizeof(binding.GbSegRecord),
                                     ctypes.sizeof(binding.GbStats)]


def test_last_error_without_init(lib):
    # callable before gb_init and without a GPU: returns a C string
    lib.gb_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.gb_last_error(), bytes)
