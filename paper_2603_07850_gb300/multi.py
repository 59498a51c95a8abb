"""Several GPUs, one process each: range sharding and the final result merge.

Ranks verify disjoint blocks of the range independently (no collective on
the data path, the device form of the paper's pool needs none across GPUs);
the only exchange is one gather of fixed-size results, merged in range
order.  Alternatively the callers claim tiles of one range from a shared
host counter (gb_verify_range_claimed) and merge their record arrays.  This
module holds the host logic only; each caller's records come from the
library on its own GPU.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def shard_range(lo: int, hi: int, rank: int, world: int, align_bits: int = 20):
    """Rank's half-open block of [lo, hi): the even-n grid from max(lo, 4) is
    cut into `world` contiguous pieces aligned to 2^align_bits even n."""
    n0 = max(lo, 4)
    n0 += n0 & 1
    if n0 >= hi:
        return n0, n0
    total = ((hi - 1) & ~1) - n0
    total = total // 2 + 1 if total >= 0 else 0
    unit = 1 << align_bits
    units = (total + unit - 1) // unit
    per = (units + world - 1) // world
    a = min(total, rank * per * unit)
    b = min(total, (rank + 1) * per * unit)
    lo_r = n0 + 2 * a
    hi_r = min(hi, n0 + 2 * b) if b > a else lo_r
    return lo_r, hi_r


def merge_results(parts: list[dict]) -> dict:
    """Merge gb_result dicts of consecutive disjoint blocks (in range order)
    into the result of their union."""
    parts = [p for p in parts if p["n_count"]]
    if not parts:
        return {"n_first": 0, "n_count": 0, "max_pmin": 0, "argmax_n": 0, "sum_pmin": 0,
                "wsum_pmin": 0, "hist": [0] * 64, "n_slow": 0, "counterexample_n": 0, "status": 0}
    n0 = parts[0]["n_first"]
    out = {"n_first": n0, "n_count": 0, "max_pmin": 0, "argmax_n": 0, "sum_pmin": 0,
           "wsum_pmin": 0, "hist": [0] * 64, "n_slow": 0, "counterexample_n": 0, "status": 0}
    for p in parts:
        k0 = (p["n_first"] - n0) // 2
        out["wsum_pmin"] = (out["wsum_pmin"] + p["wsum_pmin"] + p["sum_pmin"] * k0) & MASK64
        out["sum_pmin"] = (out["sum_pmin"] + p["sum_pmin"]) & MASK64
        out["n_count"] += p["n_count"]
        out["n_slow"] += p["n_slow"]
        out["hist"] = [a + b for a, b in zip(out["hist"], p["hist"])]
        if p["max_pmin"] > out["max_pmin"]:          # blocks ascend: first max wins ties
            out["max_pmin"], out["argmax_n"] = p["max_pmin"], p["argmax_n"]
        if p["counterexample_n"] and not out["counterexample_n"]:
            out["counterexample_n"] = p["counterexample_n"]
        if p["status"] and not out["status"]:
            out["status"] = p["status"]
    return out


def merge_record_sets(sets, n_total: int | None = None):
    """Merge the record arrays (SEG_DTYPE, same range and seg_bits) of callers
    that each verified part of the tiles of one range, as from
    gb_verify_range_claimed: counts, sums (mod 2^64) and histograms add, the
    largest p_min wins with its smallest n, the smallest counterexample wins.
    The result equals the records of one call over the whole range.  With
    n_total (the range's number of even n) the merged counts must add up to
    it: a tile verified twice or never makes the merge fail."""
    import numpy as np
    sets = [s for s in sets if len(s)]
    if not sets:
        if n_total:
            raise ValueError(f"no records, but the range holds {n_total} even n")
        return []
    out = sets[0].copy()
    for s in sets[1:]:
        assert len(s) == len(out) and (s["n_first"] == out["n_first"]).all()
        out["n_count"] += s["n_count"]
        out["sum_pmin"] += s["sum_pmin"]                 # uint64 arithmetic wraps mod 2^64
        out["wsum_pmin"] += s["wsum_pmin"]
        out["hist"] += s["hist"]
        out["n_slow"] += s["n_slow"]
        better = (s["max_pmin"] > out["max_pmin"]) | (
            (s["max_pmin"] == out["max_pmin"]) & (s["max_pmin"] > 0) & (s["argmax_n"] < out["argmax_n"]))
        out["max_pmin"] = np.where(better, s["max_pmin"], out["max_pmin"])
        out["argmax_n"] = np.where(better, s["argmax_n"], out["argmax_n"])
        ce_a, ce_b = out["counterexample_n"], s["counterexample_n"]
        out["counterexample_n"] = np.where((ce_a == 0) | ((ce_b != 0) & (ce_b < ce_a)), ce_b, ce_a)
    if n_total is not None and int(out["n_count"].sum()) != n_total:
        raise ValueError(f"merged records hold {int(out['n_count'].sum())} even n, the range {n_total}")
    return out


def gather_merge(result: dict, group=None) -> dict | None:
    """all-gather every rank's result (torch.distributed) and merge on all
    ranks; returns the merged dict (every rank gets it)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, result, group=group)
    return merge_results(parts)
