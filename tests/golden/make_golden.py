"""Write the stored expected records used by the GPU parity tests.

Every value written here comes from the CPU oracle (``oracle/``) and nothing
else; the inputs (which segments, which windows) come from the seeded recipes
in ``paper_2603_07850_gb300.workloads``.

    python tests/golden/make_golden.py [c1] [c2] [c3]

Outputs (JSON, next to this script):
  c1_digest.json   : sha256 over all 152,588 records of 2^15 even n covering
                     [4, 10^10], plus their aggregate (oracle run split over
                     processes by record blocks; each block is an ordinary
                     oracle call).
  c2_samples.json  : 64 records of 2^20 even n drawn with seed 0xC2 from the
                     2^20 grid of [4, 10^12], plus p_min of the max candidates.
  c3_windows.json  : 16 sub-windows of 2^20 even n for each high-offset window
                     (seeds 0xC3A, 0xC3B) and the top-of-range window
                     [2^64 - 2^21, 2^64 - 1).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2603_07850_gb300 import workloads as W  # noqa: E402
import recutil  # noqa: E402


def _block(args):
    lo, hi, p_max, seg_bits = args
    st, recs, _, _ = oracle.pmin_range(lo, hi, p_max=p_max, seg_bits=seg_bits)
    assert st == 0
    return [recutil.canon(r) for r in recs]


def aggregate(canon_recs, n0):
    """Whole-range aggregate from records (n_first given by the range)."""
    best_p, best_n = 0, 0
    tot = {"n_count": 0, "sum_pmin": 0, "wsum_pmin": 0, "n_slow": 0, "hist": [0] * 64}
    for t in canon_recs:
        d = recutil.to_dict(t)
        if d["max_pmin"] > best_p:
            best_p, best_n = d["max_pmin"], d["argmax_n"]
        k0 = (d["n_first"] - n0) // 2
        tot["n_count"] += d["n_count"]
        tot["sum_pmin"] = (tot["sum_pmin"] + d["sum_pmin"]) % (1 << 64)
        tot["wsum_pmin"] = (tot["wsum_pmin"] + d["wsum_pmin"] + d["sum_pmin"] * k0) % (1 << 64)
        tot["n_slow"] += d["n_slow"]
        tot["hist"] = [a + b for a, b in zip(tot["hist"], d["hist"])]
    tot["max_pmin"], tot["argmax_n"], tot["n_first"] = best_p, best_n, n0
    return tot


def make_c1(procs: int):
    cfg = W.C1
    nrec = W.num_records(cfg.lo, cfg.hi, cfg.seg_bits)
    per = 4096
    jobs = []
    for r0 in range(0, nrec, per):
        a, _ = W.record_bounds(cfg.lo, cfg.hi, cfg.seg_bits, r0)
        _, b = W.record_bounds(cfg.lo, cfg.hi, cfg.seg_bits, min(r0 + per, nrec) - 1)
        jobs.append((a, b, cfg.p_max, cfg.seg_bits))
    t = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_block, jobs)
    recs = [r for p in parts for r in p]
    assert len(recs) == nrec
    out = {
        "config": cfg.name, "lo": cfg.lo, "hi": cfg.hi, "p_max": cfg.p_max,
        "seg_bits": cfg.seg_bits, "n_records": nrec, "sha256": recutil.digest(recs),
        "aggregate": aggregate(recs, W.first_even(cfg.lo)),
        "oracle_seconds": round(time.time() - t, 1), "oracle_processes": procs,
    }
    json.dump(out, open(os.path.join(HERE, "c1_digest.json"), "w"), indent=1)
    print("c1", out["n_records"], out["sha256"], out["oracle_seconds"], "s")


def make_c2():
    cfg = W.C2
    idx = W.sample_records(cfg, 64, W.SEED_C2)
    base = oracle.primes_upto(1 << 20)
    out = {"config": cfg.name, "lo": cfg.lo, "hi": cfg.hi, "p_max": cfg.p_max,
           "seg_bits": cfg.seg_bits, "seed": W.SEED_C2, "records": []}
    for r in idx:
        a, b = W.record_bounds(cfg.lo, cfg.hi, cfg.seg_bits, r)
        st, recs, _, _ = oracle.pmin_range(a, b, p_max=cfg.p_max, seg_bits=cfg.seg_bits,
                                           base=(base, 1 << 20))
        assert st == 0 and len(recs) == 1
        out["records"].append({"index": r, "record": recutil.to_dict(recutil.canon(recs[0]))})
    json.dump(out, open(os.path.join(HERE, "c2_samples.json"), "w"), indent=1)
    print("c2", len(out["records"]))


def make_c3():
    base32 = oracle.primes_upto((1 << 32) - 1)
    out = {}
    for cfg, seed in ((W.C3A, W.SEED_C3A), (W.C3B, W.SEED_C3B)):
        wins = W.sample_subwindows(cfg, 16, seed)
        lst = []
        for a, b in wins:
            st, recs, _, _ = oracle.pmin_range(a, b, p_max=cfg.p_max, seg_bits=20,
                                               base=(base32, (1 << 32) - 1))
            assert st == 0 and len(recs) == 1
            lst.append({"lo": a, "hi": b, "record": recutil.to_dict(recutil.canon(recs[0]))})
        out[cfg.name] = {"lo": cfg.lo, "hi": cfg.hi, "seed": seed, "windows": lst}
        print(cfg.name, len(lst))
    e = W.C3_EDGE
    st, recs, _, _ = oracle.pmin_range(e.lo, e.hi, p_max=e.p_max, seg_bits=20,
                                       base=(base32, (1 << 32) - 1))
    assert st == 0 and len(recs) == 1
    out[e.name] = {"lo": e.lo, "hi": e.hi,
                   "windows": [{"lo": e.lo, "hi": e.hi,
                                "record": recutil.to_dict(recutil.canon(recs[0]))}]}
    json.dump(out, open(os.path.join(HERE, "c3_windows.json"), "w"), indent=1)


if __name__ == "__main__":
    what = sys.argv[1:] or ["c1", "c2", "c3"]
    if "c2" in what:
        make_c2()
    if "c3" in what:
        make_c3()
    if "c1" in what:
        make_c1(os.cpu_count() or 1)
