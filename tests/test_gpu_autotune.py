"""Autotuner: picks a kernel configuration per range class, caches it, and
never changes a result."""
import os

import pytest

pytestmark = pytest.mark.gpu

KEYS = ("tile_bits", "threads", "search_chunks", "pattern_max", "search_pmax", "tier_b_min", "wheel",
        "builder_warps", "bucket_min", "bucket_chunk_tiles")


def test_autotune_keeps_results_and_caches(tmp_path, monkeypatch):
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("GB_TUNE_CACHE", str(cache))
    lo, hi = 10**11, 10**11 + 4 * 10**9
    gb.gb_init(1 << 16, 20)
    try:
        ref = gb.gb_verify_range_segments(lo, hi, 4096)
        gb.gb_set_option("autotune", 1)
        got = gb.gb_verify_range_segments(lo, hi, 4096)
        tuned = {k: gb.gb_get_option(k) for k in KEYS}
        again = gb.gb_verify_range_segments(lo, hi, 4096)          # cached choice
    finally:
        gb.gb_shutdown()
    assert (got[0] == ref[0]).all() and (again[0] == ref[0]).all()
    assert got[1] == ref[1] == again[1]
    lines = cache.read_text().split("\n")
    assert any(l.split()[1:] == [str(tuned[k]) for k in KEYS] for l in lines if l)
    # a fresh context reads the saved choice
    gb.gb_init(1 << 16, 20)
    try:
        gb.gb_set_option("autotune", 1)
        gb.gb_verify_range(lo, hi)
        assert {k: gb.gb_get_option(k) for k in tuned} == tuned
    finally:
        gb.gb_shutdown()


def test_autotune_a_bucketed_range(tmp_path, monkeypatch):
    # sqrt(n) far above four window spans: the probe runs the bucket
    # pre-pass and kernel per chunk, and the tuner also varies where the
    # pre-pass starts and its chunk size; the records never change
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    monkeypatch.setenv("GB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    lo, hi = 10**16, 10**16 + 2 * 10**9
    gb.gb_init(1 << 16, 20)
    try:
        ref = gb.gb_verify_range_segments(lo, hi, 1024)
        gb.gb_set_option("autotune", 1)
        got = gb.gb_verify_range_segments(lo, hi, 1024)
        tuned = {k: gb.gb_get_option(k) for k in KEYS}
    finally:
        gb.gb_shutdown()
    assert (got[0] == ref[0]).all() and got[1] == ref[1]
    lines = (tmp_path / "tune.txt").read_text().split("\n")
    assert any(l.split()[1:] == [str(tuned[k]) for k in KEYS] for l in lines if l)
