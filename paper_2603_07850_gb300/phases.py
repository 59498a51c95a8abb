"""Where the persistent kernel's time goes, from its own cycle counters.

    python -m paper_2603_07850_gb300.phases [--lo 4] [--hi 1000000000001] [--option KEY=VALUE ...]

Builds the library variant with per-phase clock64 counters (GB_PHASE_CLOCKS,
a separate file; the ordinary library has none of this code), verifies the
range once with the single-role persistent kernel and prints one JSON line:
the share of CTA cycles spent claiming tiles, filling the window, crossing
off, searching and reducing (thread 0 of each CTA, between the CTA's
barriers), and the split of the searching warps' cycles between the
bit-parallel bulk loop and the per-n walk of the open n, and of the
crossing-off warps' cycles between tier A (a warp per prime) and tier B (a
lane per prime).  The counters add a
few instructions per tile and per warp, so the kernel time it prints runs a
little above the ordinary build's.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2603_07850_gb300 import binding, build  # noqa: E402

PHASES = ("phase_claim", "phase_fill", "phase_mark", "phase_search", "phase_reduce")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lo", type=int, default=4)
    ap.add_argument("--hi", type=int, default=10**12 + 1)
    ap.add_argument("--p-max", type=int, default=1 << 16)
    ap.add_argument("--seg-bits", type=int, default=20)
    ap.add_argument("--option", action="append", default=["search_chunks=6"], metavar="KEY=VALUE")
    args = ap.parse_args()
    binding.load(build.build(phases=True))
    gb = binding
    gb.gb_init(args.p_max, args.seg_bits)
    gb.gb_set_option("use_graph", 0)
    gb.gb_set_option("time_kernel", 1)
    for kv in args.option:
        k, v = kv.split("=", 1)
        gb.gb_set_option(k, int(v))
    gb.gb_verify_range(args.lo, args.hi)                    # warm: table, buffers
    r = gb.gb_verify_range(args.lo, args.hi)
    kus = gb.gb_get_option("last_kernel_us")
    cyc = {k: gb.gb_get_option(k) for k in PHASES + ("phase_warp_bulk", "phase_warp_tail", "phase_warp_tier_a",
                                                       "phase_warp_tier_b")}
    gb.gb_shutdown()
    cta = sum(cyc[k] for k in PHASES)
    # a range that takes the bucket pre-pass runs several launches and has
    # no single kernel time: its split is in cycles only
    ks = kus * 1e-6 if kus > 0 else None
    warp = cyc["phase_warp_bulk"] + cyc["phase_warp_tail"]
    marks = cyc["phase_warp_tier_a"] + cyc["phase_warp_tier_b"]
    print(json.dumps({
        "range": [args.lo, args.hi], "n_count": r["n_count"], "kernel_s": ks,
        "options": args.option,
        "cta_share": {k[len("phase_"):]: cyc[k] / cta for k in PHASES},
        "cta_seconds": {k[len("phase_"):]: ks * cyc[k] / cta if ks else None for k in PHASES},
        "search_warp_share": {"bulk": cyc["phase_warp_bulk"] / warp if warp else None,
                              "per_n_walk": cyc["phase_warp_tail"] / warp if warp else None},
        "mark_warp_share": {"tier_a": cyc["phase_warp_tier_a"] / marks if marks else None,
                            "tier_b": cyc["phase_warp_tier_b"] / marks if marks else None},
        "cycles": cyc,
    }), flush=True)


if __name__ == "__main__":
    main()
