"""The command-line verifier (the paper's `goldbach [--start=N] LIMIT`
shape) against the oracle on a small range."""
import json
import os
import subprocess
import sys

import pytest

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cli_range_matches_oracle():
    lo, limit = 10**9 + 1, 10**9 + 2 * 10**6
    out = subprocess.run([sys.executable, "-m", "paper_2603_07850_gb300.verify", "--start", str(lo),
                          "--progress", "--warm", "1000", str(limit)],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    r = d["result"]
    st, recs, _, _ = oracle.pmin_range(lo, limit + 1, p_max=1 << 16, seg_bits=40)
    o = recs[0]
    assert (r["n_first"], r["n_count"], r["max_pmin"], r["argmax_n"], r["sum_pmin"], r["wsum_pmin"], r["n_slow"]) == \
        (o.n_first, o.n_count, o.max_pmin, o.argmax_n, o.sum_pmin, o.wsum_pmin, o.n_slow)
    assert {int(b): c for b, c in r["hist"].items()} == {b: c for b, c in enumerate(o.hist) if c}
    assert r["status"] == 0 and r["counterexample_n"] == 0
