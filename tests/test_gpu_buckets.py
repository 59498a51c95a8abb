"""GPU parity of the bucketed large-prime pass and the high-offset windows.

Large base primes (p >= the bucket bound) are not crossed off per tile; a
pre-pass scatters each of their hits into per-tile buckets.  These tests
force that pass on with small bounds and tiny chunks, and run the
high-offset windows (base primes up to 2^32) at full size against the
oracle's stored records.  Every comparison is exact.
"""
import json
import os

import pytest

import oracle
import recutil
from paper_2603_07850_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    yield binding
    binding.gb_shutdown()


def run(gb, lo, hi, p_max, seg_bits, **opts):
    gb.gb_init(p_max, seg_bits)
    for k, v in opts.items():
        gb.gb_set_option(k, v)
    nrec = W.num_records(lo, hi, seg_bits)
    recs, agg, n = gb.gb_verify_range_segments(lo, hi, max(nrec, 1))
    assert n == nrec
    return list(recs), agg


@pytest.mark.parametrize("bucket_min,chunk,tile_bits", [
    (1024, 7, 16),        # primes hitting a window many times, several chunks
    (1 << 15, 1, 16),     # one tile per chunk
    (64, 3, 14),          # almost every prime bucketed
    (0, 2048, 16),        # the automatic bound (window span)
])
@pytest.mark.parametrize("builders", [0, 8], ids=["persistent", "pipelined"])
def test_buckets_match_oracle(gb, bucket_min, chunk, tile_bits, builders):
    lo, hi = 10**13 + 2, 10**13 + 2 * 10**7 + 7
    recs, agg = run(gb, lo, hi, 1 << 16, 12, tile_bits=tile_bits, bucket_min=bucket_min,
                    bucket_chunk_tiles=chunk, builder_warps=builders)
    st, orecs, _, _ = oracle.pmin_range(lo, hi, p_max=1 << 16, seg_bits=12)
    d = recutil.diff(recs, orecs)
    assert not d, d
    assert agg["status"] == 0


def test_buckets_largest_chunk(gb):
    """One chunk of 7,935 tiles: the bucket fill's per-tile arrays at nearly
    their largest size (chunks of at most 8,192 tiles), and windows that
    overlap two earlier ones (2^14-n tiles, K = 2^15 bits)."""
    lo, hi = 10**13 + 2, 10**13 + 2 + 260_000_000
    recs, agg = run(gb, lo, hi, 1 << 16, 12, tile_bits=14, bucket_min=1 << 15, bucket_chunk_tiles=8192)
    st, orecs, _, _ = oracle.pmin_range(lo, hi, p_max=1 << 16, seg_bits=12)
    d = recutil.diff(recs, orecs)
    assert not d, d
    assert agg["status"] == 0


def _golden_windows():
    g = json.load(open(os.path.join(GOLDEN, "c3_windows.json")))
    out = []
    for name, block in g.items():
        for w in block["windows"]:
            out.append((name, w["lo"], w["hi"], w["record"]))
    return out


@pytest.mark.parametrize("name,lo,hi,rec", _golden_windows(),
                         ids=lambda v: str(v)[:12] if not isinstance(v, dict) else "rec")
def test_high_offset_subwindows(gb, name, lo, hi, rec):
    recs, agg = run(gb, lo, hi, 1 << 16, 20)
    assert len(recs) == 1
    assert recutil.canon(recs[0]) == recutil.canon(rec)


@pytest.mark.parametrize("cfg", [W.C3A, W.C3B], ids=lambda c: c.name)
@pytest.mark.parametrize("kopts", [{"builder_warps": 0, "tile_bits": 20}, {"builder_warps": 8, "tile_bits": 19}],
                         ids=["persistent", "pipelined"])
def test_high_offset_full_windows(gb, cfg, kopts):
    g = json.load(open(os.path.join(GOLDEN, "c3_windows.json")))[cfg.name]
    recs, agg = run(gb, cfg.lo, cfg.hi, cfg.p_max, 20, **kopts)
    n0 = W.first_even(cfg.lo)
    for w in g["windows"]:
        r = (w["lo"] - n0) // 2 >> 20
        assert recutil.canon(recs[r]) == recutil.canon(w["record"]), r
    assert agg["n_count"] == W.num_even(cfg.lo, cfg.hi)
    assert agg["status"] == 0 and agg["n_slow"] == 0
    # the reported maximum is attained where the oracle says
    assert oracle.pmin_single(agg["argmax_n"]) == agg["max_pmin"]
    assert max(int(r["max_pmin"]) for r in recs) == agg["max_pmin"]


# The largest minimal Goldbach partition found below 4 x 10^18 (Oliveira e
# Silva, Herzog and Pardi, Math. Comp. 83 (2014)): n = 3,325,581,707,333,960,528
# needs p = 9,781, and no smaller even n needs as much.
RECORD_N, RECORD_P = 3325581707333960528, 9781


def test_published_pmin_record(gb):
    # base primes to 1.8e9 (bucketed), the record found in the window with
    # P_max = 2^16 and by the Miller-Rabin slow path with P_max = 4096; the
    # records agree except for n_slow
    lo, hi = RECORD_N - 2 * 2048, RECORD_N + 2 * 2048
    out = {}
    for p_max in (1 << 16, 4096):
        recs, agg = run(gb, lo, hi, p_max, 12)
        assert agg["status"] == 0 and agg["counterexample_n"] == 0
        assert agg["max_pmin"] == RECORD_P and agg["argmax_n"] == RECORD_N
        out[p_max] = (recs, agg)
    (r_win, a_win), (r_slow, a_slow) = out[1 << 16], out[4096]
    assert a_win["n_slow"] == 0 and a_slow["n_slow"] >= 1
    def without_nslow(recs):
        out = []
        for r in recs:
            d = recutil.to_dict(recutil.canon(r))
            del d["n_slow"]
            out.append(d)
        return out
    assert without_nslow(r_win) == without_nslow(r_slow)


@pytest.mark.parametrize("kopts", [{}, {"builder_warps": 16, "tile_bits": 18}], ids=["persistent", "pipelined"])
def test_top_of_u64_range(gb, kopts):
    # hi = 2^64 - 1 includes n = 2^64 - 2; nothing may wrap
    e = W.C3_EDGE
    g = json.load(open(os.path.join(GOLDEN, "c3_windows.json")))[e.name]["windows"][0]
    recs, agg = run(gb, e.lo, e.hi, e.p_max, 20, **kopts)
    assert len(recs) == 1 and int(recs[0]["n_count"]) == 1 << 20
    assert recutil.canon(recs[0]) == recutil.canon(g["record"])
    assert agg["argmax_n"] <= (1 << 64) - 2
