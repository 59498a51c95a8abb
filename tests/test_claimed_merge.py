"""Record merge for callers that claim tiles of one range from a shared
counter (gb_verify_range_claimed), checked on CPU against the oracle: the
tiles of a range are dealt at random to three callers, each caller's records
are folded from the oracle's per-tile results the way the kernel folds them
(record-relative weighted sums), and multi.merge_record_sets must give the
oracle's records of the whole range exactly."""
import random

import numpy as np
import pytest

import oracle
import recutil
from paper_2603_07850_gb300 import multi
from paper_2603_07850_gb300 import workloads as W
from paper_2603_07850_gb300.binding import SEG_DTYPE

MASK = (1 << 64) - 1


def caller_records(lo, hi, seg_bits, tile_bits, tiles):
    """Records of one caller that verified the given tiles (oracle per tile)."""
    n0 = W.first_even(lo)
    nrec = W.num_records(lo, hi, seg_bits)
    out = np.zeros(nrec, dtype=SEG_DTYPE)
    for r in range(nrec):
        out[r]["n_first"] = n0 + (2 * r << seg_bits)
    for t in tiles:
        a = n0 + (2 * t << tile_bits)
        b = min(hi, n0 + (2 * (t + 1) << tile_bits))
        st, recs, _, _ = oracle.pmin_range(a, b, p_max=1 << 16, seg_bits=40)
        x = recs[0]
        r = (t << tile_bits) >> seg_bits
        dk = ((t << tile_bits) - (r << seg_bits))          # tile start - record start, in n
        o = out[r]
        o["n_count"] += x.n_count
        o["sum_pmin"] = (int(o["sum_pmin"]) + x.sum_pmin) & MASK
        o["wsum_pmin"] = (int(o["wsum_pmin"]) + x.wsum_pmin + x.sum_pmin * dk) & MASK
        o["hist"] += np.array(x.hist[:64], dtype=np.uint64)
        o["n_slow"] += x.n_slow
        if x.max_pmin > o["max_pmin"] or (x.max_pmin == o["max_pmin"] and x.max_pmin and x.argmax_n < o["argmax_n"]):
            o["max_pmin"], o["argmax_n"] = x.max_pmin, x.argmax_n
        if x.counterexample_n and (o["counterexample_n"] == 0 or x.counterexample_n < o["counterexample_n"]):
            o["counterexample_n"] = x.counterexample_n
    return out


@pytest.mark.parametrize("lo,hi,seg_bits,tile_bits,seed", [
    (4, 300_001, 14, 11, 1), (10**9 + 1, 10**9 + 200_000, 12, 10, 2), (6, 40_000, 15, 10, 3)])
def test_dealt_tiles_merge_to_the_whole_range(lo, hi, seg_bits, tile_bits, seed):
    n_total = W.num_even(lo, hi)
    ntiles = (n_total + (1 << tile_bits) - 1) >> tile_bits
    rng = random.Random(seed)
    owner = [rng.randrange(3) for _ in range(ntiles)]
    parts = [caller_records(lo, hi, seg_bits, tile_bits, [t for t in range(ntiles) if owner[t] == c])
             for c in range(3)]
    merged = multi.merge_record_sets(parts, n_total=n_total)
    st, want, _, _ = oracle.pmin_range(lo, hi, p_max=1 << 16, seg_bits=seg_bits)
    assert len(merged) == len(want)
    for r in range(len(want)):
        assert recutil.canon(merged[r]) == recutil.canon(want[r]), r


def test_merge_of_nothing():
    assert multi.merge_record_sets([]) == []


def test_a_tile_taken_twice_or_never_fails_the_merge():
    lo, hi, seg_bits, tile_bits = 10**6, 10**6 + 2 * 5000 + 1, 12, 10
    n_total = W.num_even(lo, hi)
    ntiles = (n_total + (1 << tile_bits) - 1) >> tile_bits
    every = list(range(ntiles))
    twice = [caller_records(lo, hi, seg_bits, tile_bits, every),
             caller_records(lo, hi, seg_bits, tile_bits, [0])]
    with pytest.raises(ValueError):
        multi.merge_record_sets(twice, n_total=n_total)
    never = [caller_records(lo, hi, seg_bits, tile_bits, every[1:])]
    with pytest.raises(ValueError):
        multi.merge_record_sets(never, n_total=n_total)
    assert multi.merge_record_sets([caller_records(lo, hi, seg_bits, tile_bits, every)],
                                   n_total=n_total) is not None
