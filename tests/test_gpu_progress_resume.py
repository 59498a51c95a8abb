"""Live progress of a long call, and segment-granular resume.

Records depend only on their own range, so a range verified in pieces that
split at record boundaries gives the same records, and merged aggregate, as
one call: an interrupted run resumes from its first unfinished record.  The
records around the cut, and seeded others, are checked against the oracle.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import recutil
from paper_2603_07850_gb300 import multi
from paper_2603_07850_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture()
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    binding.gb_init(1 << 16, 20)
    yield binding
    binding.gb_shutdown()


def test_progress_is_readable_while_a_call_runs(gb):
    lo, hi = 4, 4 * 10**11
    gb.gb_verify_range(4, 10**6)                         # warm: table, kernels
    out = {}
    th = threading.Thread(target=lambda: out.update(r=gb.gb_verify_range(lo, hi)))
    th.start()
    seen = []
    while th.is_alive():
        seen.append(gb.gb_progress())
        time.sleep(0.01)
    th.join()
    last = gb.gb_progress()
    tile_n = 1 << gb.gb_get_option("tile_bits")
    n_total = W.num_even(lo, hi)
    assert last["tiles_total"] == (n_total + tile_n - 1) // tile_n
    assert last["tiles_done"] == last["tiles_total"]
    assert last["n_done"] == last["n_total"] == n_total and last["eta_s"] == 0.0
    mid = [p for p in seen if 0 < p["tiles_done"] < p["tiles_total"]]
    assert mid, seen[:5]
    for p in mid:
        # a rate and a time left are reported while the call runs
        assert p["n_done"] == p["tiles_done"] * tile_n and p["n_total"] == n_total
        assert p["n_per_s"] > 0 and p["eta_s"] > 0
        assert abs(p["eta_s"] - (n_total - p["n_done"]) / p["n_per_s"]) < 1e-6 * max(1.0, p["eta_s"])
    assert all(a["tiles_done"] <= b["tiles_done"] for a, b in zip(seen, seen[1:]))   # never goes back
    assert out["r"]["status"] == 0


def test_resume_from_a_record_boundary(gb):
    lo, hi, seg = 10**10, 10**10 + 3 * 10**9 + 7, 20
    nrec = W.num_records(lo, hi, seg)
    whole, agg, _ = gb.gb_verify_range_segments(lo, hi, nrec)
    cut = 1234                                           # "interrupted" after 1,234 records
    mid, _ = W.record_bounds(lo, hi, seg, cut)
    a, agg_a, _ = gb.gb_verify_range_segments(lo, mid, nrec)
    b, agg_b, _ = gb.gb_verify_range_segments(mid, hi, nrec)
    assert len(a) == cut and len(a) + len(b) == nrec
    assert np.array_equal(np.concatenate([a, b]), whole)
    merged = multi.merge_results([agg_a, agg_b])
    for k in ("n_first", "n_count", "max_pmin", "argmax_n", "sum_pmin", "wsum_pmin", "hist", "n_slow"):
        assert merged[k] == agg[k], k
    # the records on both sides of the cut, the ragged last one and seeded
    # others equal the oracle's
    cfg = W.RangeConfig("resume", lo, hi, 1 << 16, seg, 0, "")
    rs = np.concatenate([a, b])
    for r in sorted({cut - 1, cut, nrec - 1, *W.sample_records(cfg, 3, 0xF3)}):
        ra, rb = W.record_bounds(lo, hi, seg, r)
        st, orecs, _, _ = oracle.pmin_range(ra, rb, p_max=1 << 16, seg_bits=seg)
        assert st == 0 and recutil.canon(rs[r]) == recutil.canon(orecs[0]), r
