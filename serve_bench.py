"""Serving benchmark: seeded Poisson stream of range requests on one GB300.

    python serve_bench.py [--requests 10000] [--load 0.7] [--capacity-requests 2000]

Workload (all from paper_2603_07850_gb300.workloads, seed 0xC4): lo an even
integer uniform in [4, 1e15), width log-uniform in [1e4, 1e10], Poisson
arrivals.  First the capacity is measured closed-loop (the first
--capacity-requests requests submitted at once), then the full stream is
replayed with exponential gaps at --load x capacity.  Latency = result on the
host - gb_submit, from the library's own timestamps.  A seeded 1% sample with
width <= 1e7 is checked against the CPU oracle.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(round(q * (len(xs) - 1)))))
    return xs[i]


def run(gb, reqs, rate):
    """Submit reqs on their arrival schedule (rate = None: all at once); return results."""
    results = [None] * len(reqs)
    tickets = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def poller():
        for i in range(len(reqs)):
            ready.acquire()
            st, res = gb.gb_poll(tickets[i], -1)
            results[i] = (st, res)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        if rate:
            delay = t0 + r.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
        tickets[i] = gb.gb_submit(r.lo, r.hi)
        ready.release()
    th.join()
    return results


def measure(gb, requests: int = 10_000, capacity_requests: int = 2000, load: float = 0.7,
            budget_mb: int = 8192, oracle_sample: float = 0.01) -> dict:
    """Capacity closed-loop, then the seeded Poisson stream at load x capacity,
    then the oracle on a seeded sample; returns the summary dict.  Runs on a
    fresh library context (gb_init) and shuts it down."""
    from paper_2603_07850_gb300 import workloads as W
    gb.gb_init(1 << 16, 20)
    gb.gb_set_option("mem_budget_mb", budget_mb)
    gb.gb_set_option("base_limit", 32_000_000)          # base primes kept resident

    # capacity: closed loop on a prefix of the stream
    cap_reqs = W.serving_stream(count=capacity_requests, rate_per_s=1.0, seed=W.SEED_C4)
    t = time.perf_counter()
    res = run(gb, cap_reqs, None)
    cap_s = time.perf_counter() - t
    assert all(st == 0 for st, _ in res)
    capacity = len(cap_reqs) / cap_s
    cap_n = sum(r["n_count"] for _, r in res)

    # the Poisson stream at load x capacity
    rate = load * capacity
    reqs = W.serving_stream(count=requests, rate_per_s=rate, seed=W.SEED_C4)
    t = time.perf_counter()
    res = run(gb, reqs, rate)
    wall = time.perf_counter() - t
    bad = [i for i, (st, _) in enumerate(res) if st != 0]
    lat = [(r["done_ns"] - r["submit_ns"]) * 1e-9 for _, r in res]
    n_total = sum(r["n_count"] for _, r in res)
    first = min(r["submit_ns"] for _, r in res)
    last = max(r["done_ns"] for _, r in res)

    # oracle on a seeded sample with width <= 1e7
    import oracle
    rng = W.SplitMix64(W.SEED_C4 + 1)
    picked = [i for i in range(len(reqs))
              if rng.uniform() < oracle_sample and reqs[i].hi - reqs[i].lo <= 10**7]
    base = oracle.primes_upto(32_000_000)
    mism = 0
    for i in picked:
        r = reqs[i]
        st, orecs, _, _ = oracle.pmin_range(r.lo, r.hi, p_max=1 << 16, seg_bits=40,
                                            base=(base, 32_000_000))
        g = res[i][1]
        o = orecs[0] if orecs else None
        ok = (o is None and g["n_count"] == 0) or (
            o is not None and (g["n_count"], g["max_pmin"], g["argmax_n"], g["sum_pmin"],
                               g["wsum_pmin"], g["hist"]) ==
            (o.n_count, o.max_pmin, o.argmax_n, o.sum_pmin, o.wsum_pmin, o.hist))
        mism += 0 if ok else 1
    stats = gb.gb_stats()
    gb.gb_shutdown()
    return {
        "metric": f"serving latency at {round(100 * load)}% load", "requests": len(reqs), "load": load,
        "capacity_req_per_s": capacity, "capacity_even_n_per_s": cap_n / cap_s,
        "capacity_requests": len(cap_reqs),
        "arrival_rate_req_per_s": rate, "p50_s": percentile(lat, 0.5), "p99_s": percentile(lat, 0.99),
        "mean_s": sum(lat) / len(lat), "max_s": max(lat),
        "throughput_even_n_per_s": n_total / ((last - first) * 1e-9),
        "wall_s": wall, "failed": len(bad), "budget_mb": budget_mb,
        "oracle_checked": len(picked), "oracle_mismatches": mism,
        "kernel_launches": stats["kernel_launches"], "data": "synthetic",
        "workload": "lo uniform even in [4, 1e15), width log-uniform in [1e4, 1e10], seed 0xC4",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=10_000)
    ap.add_argument("--capacity-requests", type=int, default=2000)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--budget-mb", type=int, default=8192)
    ap.add_argument("--oracle-sample", type=float, default=0.01)
    args = ap.parse_args()

    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    out = measure(gb, args.requests, args.capacity_requests, args.load, args.budget_mb, args.oracle_sample)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
