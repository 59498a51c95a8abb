"""Command-line verification of a range, in the shape of the paper's tool
(Sec. 3.5: `goldbach [--start=N] LIMIT` with a live `--progress` monitor).

    python -m paper_2603_07850_gb300.verify [--start N] [--progress] [--warm W]
                                            [--p-max P] [--seg-bits B] [--option KEY=VALUE ...] LIMIT

Verifies every even n with max(start, 4) <= n <= LIMIT on the current GPU
through gb_verify_range and prints one JSON line: the aggregate record,
the status, and the wall time of the call.  --warm W first verifies
[start, start + W) untimed (base-prime table, buffers, tuning).  --progress
prints the library's progress (tiles, rate, time left) to stderr every half
second while the call runs.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2603_07850_gb300 import binding, build  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("limit", type=int, help="largest even n to verify (inclusive)")
    ap.add_argument("--start", type=int, default=4)
    ap.add_argument("--progress", action="store_true")
    ap.add_argument("--warm", type=int, default=0, metavar="W")
    ap.add_argument("--p-max", type=int, default=1 << 16)
    ap.add_argument("--seg-bits", type=int, default=20)
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE")
    args = ap.parse_args(argv)
    gb = binding
    gb.load(build.build())
    gb.gb_init(args.p_max, args.seg_bits)
    for kv in args.option:
        k, v = kv.split("=", 1)
        gb.gb_set_option(k, int(v))
    lo, hi = args.start, min(args.limit + 1, (1 << 64) - 1)
    if args.warm:
        gb.gb_verify_range(lo, min(hi, lo + args.warm), check=False)
    stop = threading.Event()

    def monitor():
        while not stop.wait(0.5):
            p = gb.gb_progress()
            sys.stderr.write(f"{p['tiles_done']}/{p['tiles_total']} tiles, {p['n_per_s']:.3e} n/s, "
                             f"eta {p['eta_s']:.1f} s\n")

    th = threading.Thread(target=monitor, daemon=True) if args.progress else None
    if th:
        th.start()
    t = time.perf_counter()
    r = gb.gb_verify_range(lo, hi, check=False)
    wall = time.perf_counter() - t
    stop.set()
    if th:
        th.join()
    gb.gb_shutdown()
    r = {k: v for k, v in r.items() if k not in ("submit_ns", "done_ns")}
    r["hist"] = {b: c for b, c in enumerate(r["hist"]) if c}
    print(json.dumps({"range": [lo, hi], "wall_s": wall, "n_per_s": r["n_count"] / wall if wall else None,
                      "result": r}), flush=True)
    return 0 if r["status"] in (0, 2) else 1


if __name__ == "__main__":
    sys.exit(main())
