"""The library built with GB_DEBUG checks every access to a sieve window in
shared memory against the CTA's allocation.

* With no limit set, its records equal the oracle's on every kernel form
  (single-role, pipelined, per-n, bucketed, plain, serving) and no check
  fails.
* A failed check skips the access and fails the call with GB_EINTERNAL,
  naming the site and byte offset. The test forces one with the option
  debug_smem_limit, which lowers the bound the checks use. Every access
  then still lies inside the allocation, so nothing can fault; the checks
  only report the ones above the lowered bound.

The checked library runs in a child process, since it is a second library.
"""
import json
import os
import subprocess
import sys

import pytest

import oracle
import recutil

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LO, HI = 10**13 + 2, 10**13 + 2 + 4 * 10**6 + 6
SEG_BITS = 12
FORMS = {
    "persistent_bc6": {"search_chunks": 6},
    "persistent_per_n": {"search_chunks": 0},
    "pipelined": {"builder_warps": 8, "search_chunks": 6, "tile_bits": 18},
    "bucketed": {"tile_bits": 14, "bucket_min": 64, "bucket_chunk_tiles": 3},
}
PLAIN = {"plain_per_n": 0, "plain_bit_parallel": 6}
# a range where every n has p_min below 2^16: with the window unreadable
# the forced failure must not send every n into a long slow path
NEG_LO, NEG_HI = 10**6, 10**6 + 2 * 10**4


def child():
    sys.path.insert(0, ROOT)
    from paper_2603_07850_gb300 import binding as gb, build
    gb.load(build.build(debug=True))
    out = {"debug_build": gb.gb_get_option("debug_build")}
    nrec = ((HI - LO + 1) // 2 + (1 << SEG_BITS) - 1) >> SEG_BITS
    for name, opts in FORMS.items():
        gb.gb_init(1 << 16, SEG_BITS)
        for k, v in opts.items():
            gb.gb_set_option(k, v)
        recs, agg, n = gb.gb_verify_range_segments(LO, HI, nrec, check=False)
        out[name] = {"status": agg["status"], "site": gb.gb_get_option("debug_bounds_site"),
                     "recs": [list(recutil.canon(r)) for r in recs]}
        gb.gb_shutdown()
    for name, pbc in PLAIN.items():
        gb.gb_init(1 << 16, SEG_BITS)
        gb.gb_set_option("plain_search_chunks", pbc)
        recs, agg, n = gb.gb_verify_range_plain(LO, HI, nrec)
        out[name] = {"status": agg["status"], "site": gb.gb_get_option("debug_bounds_site"),
                     "recs": [list(recutil.canon(r)) for r in recs]}
        gb.gb_shutdown()
    gb.gb_init(1 << 16, SEG_BITS)
    tickets = [gb.gb_submit(LO, LO + 2 * 10**5), gb.gb_submit(LO + 10**6, LO + 3 * 10**6)]
    out["serving"] = [gb.gb_poll(t, -1, check=False)[0] for t in tickets]
    # the forced failure, then the same context again without it
    gb.gb_set_option("search_chunks", 6)
    gb.gb_set_option("debug_smem_limit", 4096)
    bad = gb.gb_verify_range(NEG_LO, NEG_HI, check=False)
    out["forced"] = {"status": bad["status"], "site": gb.gb_get_option("debug_bounds_site"),
                     "offset": gb.gb_get_option("debug_bounds_offset")}
    gb.gb_set_option("debug_smem_limit", 0)
    good = gb.gb_verify_range(NEG_LO, NEG_HI, check=False)
    out["after"] = {"status": good["status"], "site": gb.gb_get_option("debug_bounds_site"),
                    "sum_pmin": good["sum_pmin"], "n_count": good["n_count"]}
    gb.gb_shutdown()
    print(json.dumps(out), flush=True)


@pytest.fixture(scope="module")
def result():
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "child"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_is_the_checked_build(result):
    assert result["debug_build"] == 1


@pytest.mark.parametrize("name", list(FORMS) + list(PLAIN))
def test_checked_build_matches_oracle(result, name):
    st, orecs, _, _ = oracle.pmin_range(LO, HI, p_max=1 << 16, seg_bits=SEG_BITS)
    got = result[name]
    assert got["status"] == 0 and got["site"] == 0, got["status"]
    want = [list(recutil.canon(r)) for r in orecs]
    assert got["recs"] == want


def test_checked_build_serves(result):
    assert result["serving"] == [0, 0]


def test_failed_check_fails_the_call(result):
    f = result["forced"]
    assert f["status"] == -7                           # GB_EINTERNAL
    assert 1 <= f["site"] <= 7, f                      # a window access of the persistent kernel
    assert f["offset"] >= 4096 - 3, f


def test_context_usable_after_a_failed_check(result):
    a = result["after"]
    assert a["status"] == 0 and a["site"] == 0
    st, _, pm, _ = oracle.pmin_range(NEG_LO, NEG_HI, p_max=1 << 16, seg_bits=SEG_BITS, want_pmin=True)
    assert a["n_count"] == len(pm) and a["sum_pmin"] == int(sum(int(x) for x in pm))


if __name__ == "__main__" and sys.argv[1:] == ["child"]:
    child()
