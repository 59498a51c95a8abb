"""The per-phase cycle counters (the library variant built with
GB_PHASE_CLOCKS) account for the whole kernel and leave results unchanged.
Runs the phase tool in a child process, since it loads a second library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_phase_split_of_a_range():
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    lo, hi = 4, 2 * 10**10 + 1
    gb.gb_init(1 << 16, 20)
    gb.gb_set_option("search_chunks", 6)
    try:
        ref = gb.gb_verify_range(lo, hi)
    finally:
        gb.gb_shutdown()
    out = subprocess.run([sys.executable, "-m", "paper_2603_07850_gb300.phases", "--lo", str(lo), "--hi", str(hi)],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["n_count"] == ref["n_count"]
    shares = d["cta_share"]
    assert abs(sum(shares.values()) - 1.0) < 1e-9
    # every phase of a tile takes time, and building and searching dominate
    assert all(v > 0 for v in shares.values()), shares
    assert shares["mark"] + shares["search"] > 0.5, shares
    assert 0 < d["search_warp_share"]["bulk"] < 1
