"""Serving (gb_submit / gb_poll): continuous batching over the persistent pool.

Each request's result must be identical whether it runs alone
(gb_verify_range) or mixed with others in the serving loop (tolerance 0: all
outputs are integers); requests that arrive while a large one is on the GPU
must be admitted and finish first; a seeded sample is checked against the
oracle.
"""
import time

import pytest

import oracle
from paper_2603_07850_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIMESTAMPS = ("submit_ns", "done_ns")


@pytest.fixture()
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    binding.gb_init(1 << 16, 20)
    yield binding
    binding.gb_shutdown()


def strip(r):
    return {k: v for k, v in r.items() if k not in TIMESTAMPS}


def mix(count, seed, lo_max=10**13, w_hi_exp=8.0):
    return W.serving_stream(count=count, rate_per_s=1e9, seed=seed, lo_max=lo_max,
                            w_lo_exp=4.0, w_hi_exp=w_hi_exp)


def test_results_same_alone_and_in_the_mix(gb):
    reqs = mix(48, W.SEED_C4)
    alone = [strip(gb.gb_verify_range(r.lo, r.hi)) for r in reqs]
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(gb.gb_submit(r.lo, r.hi))
        if i == 15:
            time.sleep(0.02)          # the rest arrive while the first ones run
    mixed = []
    for t in tickets:
        st, res = gb.gb_poll(t, -1)
        assert st == 0
        mixed.append(res)
    for a, m in zip(alone, mixed):
        assert a == strip(m)
        assert m["done_ns"] >= m["submit_ns"] > 0
    s = gb.gb_stats()
    assert s["requests_completed"] >= len(reqs)


@pytest.mark.parametrize("opts", [{"wheel": 7}, {"threads": 512, "search_chunks": 4}],
                         ids=["wheel7", "threads512"])
def test_settings_without_a_serving_build(gb, opts):
    # these settings have no serving instantiation: the loop runs the
    # wheel-13, 1,024-thread serving kernel with tables and shared memory
    # sized for that kernel, and every result still equals the range call's
    for k, v in opts.items():
        gb.gb_set_option(k, v)
    reqs = mix(12, W.SEED_C4 + 7, lo_max=10**12, w_hi_exp=7.0)
    alone = [strip(gb.gb_verify_range(r.lo, r.hi)) for r in reqs]
    tickets = [gb.gb_submit(r.lo, r.hi) for r in reqs]
    for a, t in zip(alone, tickets):
        st, res = gb.gb_poll(t, -1)
        assert st == 0
        assert a == strip(res)


def test_small_requests_overtake_a_large_one(gb):
    ref_big = strip(gb.gb_verify_range(4, 4 * 10**10))      # also grows the table
    gb.gb_verify_range(10**12, 10**12 + 10)
    big = gb.gb_submit(4, 4 * 10**10)                        # 2e10 even n, many batches
    time.sleep(0.01)
    small = [gb.gb_submit(10**12 + 2 * 10**6 * i, 10**12 + 2 * 10**6 * i + 10**5) for i in range(8)]
    res_small = [gb.gb_poll(t, -1)[1] for t in small]
    st, res_big = gb.gb_poll(big, -1)
    assert st == 0
    assert strip(res_big) == ref_big
    t0 = res_big["submit_ns"]
    timeline = [("big", 0, (res_big["done_ns"] - t0) / 1e6)] + [
        ("small", (r["submit_ns"] - t0) / 1e6, (r["done_ns"] - t0) / 1e6) for r in res_small]
    print("timeline ms (submit, done):", timeline)
    # the small ones arrived while the large one was on the device, were
    # admitted into the running batches and finished before it
    assert max(r["submit_ns"] for r in res_small) < res_big["done_ns"], timeline
    assert max(r["done_ns"] for r in res_small) < res_big["done_ns"], timeline


def test_seeded_sample_against_oracle(gb):
    reqs = [r for r in mix(200, W.SEED_C4 + 1, lo_max=10**15, w_hi_exp=7.0)
            if r.hi - r.lo <= 10**6][:4]
    assert reqs
    tickets = [gb.gb_submit(r.lo, r.hi) for r in reqs]
    for r, t in zip(reqs, tickets):
        st, g = gb.gb_poll(t, -1)
        assert st == 0
        ost, orecs, _, _ = oracle.pmin_range(r.lo, r.hi, p_max=1 << 16, seg_bits=40)
        o = orecs[0]
        assert (g["n_first"], g["n_count"], g["max_pmin"], g["argmax_n"], g["sum_pmin"],
                g["wsum_pmin"], g["n_slow"]) == (o.n_first, o.n_count, o.max_pmin, o.argmax_n,
                                                 o.sum_pmin, o.wsum_pmin, o.n_slow)
        assert g["hist"] == o.hist


def test_admission_budget_and_empty_requests(gb):
    gb.gb_set_option("mem_budget_mb", 16)
    with pytest.raises(gb.GbError) as ei:
        gb.gb_submit(1 << 63, (1 << 63) + 1000)          # needs base primes to 2^32: 2.4 GB
    assert ei.value.code == gb.GB_ENOMEM
    t = gb.gb_submit(0, 4)                               # no even n >= 4
    st, r = gb.gb_poll(t, -1)
    assert st == 0 and r["n_count"] == 0
    t = gb.gb_submit(10**9, 10**9 + 1000)                # small table: admitted
    st, r = gb.gb_poll(t, -1)
    assert st == 0 and r["n_count"] == 500
    assert gb.gb_stats()["requests_rejected"] == 1


@pytest.mark.parametrize("small_first", [True, False], ids=["small_first", "big_first"])
def test_request_status_is_its_own(gb, small_first):
    # P_max = 2 sends every n >= 6 to the slow path; a cap of 2^7 = 64
    # candidates (p <= 129) resolves every n below 1,000 (largest p_min 73)
    # but not n = 5,372 (p_min above 129, found by the oracle).  With 1,024-n
    # tiles [5300, 7400) is two tiles and only the first fails; with two tiles
    # per batch the small request shares a batch with that tile or with the
    # clean one, depending on arrival.
    gb.gb_init(2, 20)
    for k, v in {"slow_cap": 7, "tile_bits": 10, "serve_batch_tiles": 2}.items():
        gb.gb_set_option(k, v)
    small_alone = strip(gb.gb_verify_range(4, 1000))
    assert small_alone["status"] == 0
    order = [(4, 1000), (5300, 7400)] if small_first else [(5300, 7400), (4, 1000)]
    tickets = {r: gb.gb_submit(*r) for r in order}
    st_s, rs = gb.gb_poll(tickets[(4, 1000)], -1, check=False)
    st_b, rb = gb.gb_poll(tickets[(5300, 7400)], -1, check=False)
    # the failing request fails on its own flags, whichever batch held the
    # failing tile, and a capped search is not a counterexample
    assert st_b == gb.GB_ESLOWPATH_LIMIT and rb["status"] == st_b
    assert rb["counterexample_n"] == 0
    # the other request is untouched by it
    assert st_s == 0 and strip(rs) == small_alone


def test_capped_slow_path_is_not_a_counterexample(gb):
    gb.gb_init(2, 5)
    gb.gb_set_option("slow_cap", 7)
    for form in ("range", "segments"):
        if form == "range":
            r = gb.gb_verify_range(5300, 7400, check=False)
            recs = []
        else:
            recs, r, _ = gb.gb_verify_range_segments(5300, 7400, 64, check=False)
        assert r["status"] == gb.GB_ESLOWPATH_LIMIT
        assert r["counterexample_n"] == 0
        assert all(int(x["counterexample_n"]) == 0 for x in recs)
