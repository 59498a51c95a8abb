"""Live progress of a long call, and segment-granular resume.

Records depend only on their own range, so a range verified in pieces that
split at record boundaries gives the same records, and merged aggregate, as
one call: an interrupted run resumes from its first unfinished record.
"""
import threading
import time

import numpy as np
import pytest

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
    done, total = gb.gb_progress()
    assert total == (W.num_even(lo, hi) + (1 << 20) - 1) >> 20 and done == total
    assert any(0 < d < t for d, t in seen), seen[:5]
    assert all(a[0] <= b[0] for a, b in zip(seen, seen[1:]))   # never goes back
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
