"""The host table of tier-A lane skews (paper_2603_07850_gb300/csrc/gb_skew.h).

In a warp-per-prime crossing-off step lane l clears the bit r + l p (plus a
common offset), so it touches window word floor((r + l p) / 32) and shared-
memory bank (that word mod 32).  A lane may start d_l < 4 multiples later,
which moves its bank by d_l p; the table picks the d_l per (p mod 1024, r).
These tests compile the header with the host compiler and check every entry:
the d_l are in range, no entry makes a step's worst bank worse, and on a
seeded sample the worst bank is the smallest any choice of d_l allows, found
here as a maximum flow.  The skews only reorder the marks, so the window's
contents never depend on them (that is covered by the GPU parity tests).
"""
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_07850_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "gb_skew.h"
int main()
{
    std::vector<unsigned long long> t(gbk::ASKEW_ENTRIES);
    gbk::tier_a_skew_table(t.data());
    fwrite(t.data(), 8, t.size(), stdout);
    return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("skew")
    src, exe = d / "skew.cpp", d / "skew"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    raw = subprocess.run([str(exe)], check=True, capture_output=True).stdout
    t = np.frombuffer(raw, dtype="<u8")
    assert t.size == 512 * 32
    return t.reshape(512, 32)


def banks(p: int, r: int, d=None) -> list[int]:
    return [((((r + l * p) >> 5) + (0 if d is None else d[l]) * p) & 31) for l in range(32)]


def skews(entry: int) -> list[int]:
    return [(int(entry) >> (2 * l)) & 3 for l in range(32)]


def worst(bs: list[int]) -> int:
    return max(np.bincount(bs, minlength=32))


def test_no_entry_makes_a_step_worse(table):
    for h in range(512):
        p = 2 * h + 1
        for r in range(32):
            assert worst(banks(p, r, skews(table[h, r]))) <= worst(banks(p, r)), (p, r)


def test_known_cases(table):
    # p = 37: 32 lanes span 37 words, so banks 0..4 take two lanes each
    # unskewed; the table spreads them over all 32 banks
    assert worst(banks(37, 0)) == 2 and worst(banks(37, 0, skews(table[18, 0]))) == 1
    # p = 1025 (p mod 1024 = 1): every lane on bank 0 or 1 unskewed
    assert worst(banks(1025, 0)) >= 16
    assert worst(banks(1025, 0, skews(table[0, 0]))) < worst(banks(1025, 0))


def min_worst_by_flow(p: int, r: int) -> int:
    nx = pytest.importorskip("networkx")
    base = banks(p, r)
    for cap in range(1, 33):
        g = nx.DiGraph()
        for l in range(32):
            g.add_edge("s", ("lane", l), capacity=1)
            for d in range(4):
                g.add_edge(("lane", l), ("bank", (base[l] + d * p) & 31), capacity=1)
        for b in range(32):
            g.add_edge(("bank", b), "t", capacity=cap)
        if nx.maximum_flow_value(g, "s", "t") == 32:
            return cap
    return 32


def test_sampled_entries_are_optimal(table):
    rnd = random.Random(0x5EE)
    cases = [(rnd.randrange(512), rnd.randrange(32)) for _ in range(60)]
    cases += [(0, 0), (511, 31), (18, 0), (256, 7)]
    for h, r in cases:
        p = 2 * h + 1
        assert worst(banks(p, r, skews(table[h, r]))) == min_worst_by_flow(p, r), (p, r)
