"""Benchmark: even n verified per second over [4, 10^12] on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole hot path (claim -> window sieve -> p_min
search -> slow path -> records -> merge) over every even n in [4, 10^12].

value : device throughput of gb_verify_range_async on a torch stream, each
        step one replay of the captured CUDA graph (set-params -> clear ->
        persistent kernel -> merge), timed with CUDA events per step, L2
        flushed between steps (a 512 MB write), max over ranks.
e2e   : the same metric through the blocking C-ABI call gb_verify_range with
        host buffers (params H2D and the gb_result D2H inside the timed
        region), wall clock.
plain : the plain per-segment form (one launch sequence per segment plus a
        status round trip), per-n search and bit-parallel search, each at the
        best segment size of a sweep over [4, 10^11]; then both at 10^12, their
        record arrays compared with the persistent kernel's, record by record.
extra : C1 [4, 10^10] and C3a [10^18, 10^18 + 10^10) throughput, and a
        shortened C4 serving run (p50 / p99 at 70% of measured capacity, with
        an oracle sample).

Multi-GPU (torchrun): every rank verifies its own block of 10^12 integers
[r 10^12 + 4, (r + 1) 10^12], no collective on the data path (weak scaling);
rank 0 gathers the tiny results.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_TOP = 10**12
LO, HI = 4, N_TOP + 1
P_MAX, SEG_BITS = 1 << 16, 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-top", type=int, default=N_TOP)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-records", type=int, default=600)
    ap.add_argument("--cpu-all-cores", type=int, default=100, metavar="RECORDS_PER_CORE",
                    help="records per host core for the all-cores oracle run (0 = skip)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default configuration")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="set a library option before the run (repeatable; e.g. search_chunks=6)")
    ap.add_argument("--no-extra", action="store_true", help="skip the C1, C3a, C3b and C4 figures")
    ap.add_argument("--serve-requests", type=int, default=2000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

# Lane-instruction cost of each primitive of the algorithm (the model the
# roofline counts; see the roofline section of the design notes):
#   crossing-off mark           4  (word index, bit mask, shared RMW, stride step)
#   window fill word            4 + in-register pattern primes
#   bit-parallel step (word, p) 3 + popcount(p)  (shift, and-not, or, plane ors)
#   word statistics             100 per 32-n word (popcounts over 8 planes)
#   per-n tail                  20 + 6 per 32-candidate chunk
MODEL = {"mark": 4, "fill": 4, "step": 3, "word_stats": 100, "tail": 20, "tail_chunk": 6}
MODEL_WHEEL = 13          # primes pre-sieved by the fill in the model
MODEL_BOUND = 255         # bit-parallel candidates of the model: the odd primes below 256


def odd_primes_upto(x: int):
    import numpy as np
    sieve = np.ones(x + 1, dtype=bool)
    sieve[:2] = False
    sieve[4::2] = False
    for i in range(3, int(x ** 0.5) + 1, 2):
        if sieve[i]:
            sieve[i * i::2 * i] = False
    return np.nonzero(sieve)[0][1:]


def algorithmic_instructions(n0: int, n_total: int, k_words: int, hist) -> dict:
    """Lane instructions a fixed statement of the algorithm needs for n_total
    even n from n0, independent of the kernel's tuning (tile size, pattern
    primes, search chunks):

    * fill: one word per 32 odd q in [n0 + 1 - 2K, n_last - 1], wheel 3..13;
    * marks: every odd multiple from p^2 of every prime 13 < p <= sqrt(q_max)
      in that q range, counted exactly;
    * search: per word of 32 n, one bit-parallel step per odd prime below 256
      plus the word statistics; per n with p_min above 251 (from the run's own
      histogram), the per-n walk.
    """
    import numpy as np
    K = 32 * k_words
    n_last = n0 + 2 * (n_total - 1)
    q_lo = max(n0 + 1 - 2 * K, 1)
    q_hi = n_last - 1
    primes = odd_primes_upto(int(q_hi ** 0.5) + 1).astype(np.float64)
    primes = primes[(primes > MODEL_WHEEL) & (primes * primes <= q_hi)]
    start = np.maximum(primes * primes, np.ceil(q_lo / primes) * primes)
    start = np.where(start % 2 == 0, start + primes, start)
    marks = float(np.sum(np.maximum(0.0, np.floor((q_hi - start) / (2 * primes)) + 1)))
    words = n_total / 32
    fill_words = (q_hi - q_lo) / 64 + 1
    cands = [int(c) for c in odd_primes_upto(MODEL_BOUND)]
    step_cost = sum(MODEL["step"] + bin(c).count("1") for c in cands)
    tail_n = sum(hist[b] for b in range(len(hist)) if (1 << b) > MODEL_BOUND)
    instr = (marks * MODEL["mark"] + fill_words * MODEL["fill"] + words * step_cost
             + words * MODEL["word_stats"] + tail_n * (MODEL["tail"] + 1.5 * MODEL["tail_chunk"]))
    # shared-memory accesses: a read-modify-write per mark, a store per fill
    # word, two window loads per 32-candidate chunk of a word (4 chunks), two
    # per chunk of the per-n walk
    smem = marks + fill_words + words * 8 + tail_n * 1.5 * 2
    return {"instr": instr, "per_n": instr / n_total, "marks_per_n": marks / n_total,
            "smem": smem, "tail_fraction": tail_n / n_total}


# the sources the persistent kernel is compiled from (its profile is void
# once any of them changes)
KERNEL_SOURCES = ("gb_device.cuh", "gb_search.cuh", "gb_persist.cuh", "gb_types.h", "gb_persist_1024.cu")


def csrc_digest() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_2603_07850_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def measured_profile(n_count: int):
    """The last ncu capture of the persistent kernel
    (profiles/persistent_traffic.json): DRAM bytes (read + write) and executed
    warp instructions of one launch, for a launch over n_count even n --
    scaled by n when the capture covered another range, which the result
    says; None when the kernel sources changed since the capture."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "persistent_traffic.json")))
    except (OSError, ValueError):
        return None
    if t.get("csrc_sha256") != csrc_digest():
        return None
    f = n_count / t["n_even"]
    return {"traffic": t["dram_bytes"] * f, "inst_executed": t.get("inst_executed", 0) * f or None,
            "scaled": t["n_even"] != n_count, "captured_n": t["n_even"]}


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------

def cpu_sample(n_top: int, count: int, seed: int = 0xB0):
    import oracle
    from paper_2603_07850_gb300 import workloads as W
    cfg = W.RangeConfig("bench", 4, n_top + 1, P_MAX, SEG_BITS, 0, "")
    idx = W.sample_records(cfg, count, seed)
    base = oracle.primes_upto(int(n_top ** 0.5) + 2)
    lim = int(n_top ** 0.5) + 2
    t = time.perf_counter()
    n = 0
    for r in idx:
        a, b = W.record_bounds(cfg.lo, cfg.hi, SEG_BITS, r)
        st, recs, _, _ = oracle.pmin_range(a, b, p_max=P_MAX, seg_bits=SEG_BITS, base=(base, lim))
        n += recs[0].n_count
    dt = time.perf_counter() - t
    return n / dt, n, dt, len(idx)


def _oracle_records(job):
    """Worker of the all-cores oracle run: fold the given records."""
    n_top, recs = job
    import oracle
    from paper_2603_07850_gb300 import workloads as W
    cfg = W.RangeConfig("bench", 4, n_top + 1, P_MAX, SEG_BITS, 0, "")
    base = oracle.primes_upto(int(n_top ** 0.5) + 2)
    lim = int(n_top ** 0.5) + 2
    n = 0
    for r in recs:
        a, b = W.record_bounds(cfg.lo, cfg.hi, SEG_BITS, r)
        st, out, _, _ = oracle.pmin_range(a, b, p_max=P_MAX, seg_bits=SEG_BITS, base=(base, lim))
        n += out[0].n_count
    return n


def cpu_sample_all_cores(n_top: int, per_core: int, seed: int = 0xB1):
    """The same oracle, one process per host core (spawned: this process
    already holds a CUDA context), each folding its share of seeded records."""
    import multiprocessing as mp
    import platform
    from paper_2603_07850_gb300 import workloads as W
    cores = os.cpu_count() or 1
    cfg = W.RangeConfig("bench", 4, n_top + 1, P_MAX, SEG_BITS, 0, "")
    idx = list(W.sample_records(cfg, per_core * cores, seed))
    jobs = [(n_top, idx[c::cores]) for c in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_records, [(n_top, idx[:1])] * cores)      # start-up outside the clock
        t = time.perf_counter()
        n = sum(pool.map(_oracle_records, jobs))
        dt = time.perf_counter() - t
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return n / dt, n, dt, len(idx), cores, model


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    per_step = 2
    for i in range(args.warmup + args.steps):
        v, n, dt, k = cpu_sample(args.n_top, per_step, seed=0xB0 + i)
        if i >= args.warmup:
            steps.append((n, dt))
    n = sum(s[0] for s in steps)
    dt = sum(s[1] for s in steps)
    value = n / dt
    line = {
        "impl": "reference", "metric": "even n verified/s at N=1e12", "value": value,
        "unit": "even_n/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "every even n in [4, 1e12]", "p_max": P_MAX, "seg_bits": SEG_BITS,
                   "sample": f"{per_step} seeded records of 2^20 even n per step"},
        "cpu_baseline": {"value": value, "unit": "even_n/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} seeded records of 2^20 even n per step, "
                                   "single-threaded C oracle"},
        "e2e": {"value": value, "unit": "even_n/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def kernel_seconds(gb, lo, hi, res, stream):
    """One timed gb_verify_range_async on `stream`: the persistent kernel's
    CUDA-event duration (time_kernel must be on) and the result."""
    gb.gb_verify_range_async(lo, hi, res.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    out = gb.result_from_bytes(bytes(res.cpu().numpy()))
    return gb.gb_get_option("last_kernel_us") * 1e-6, out


def measure_plain(gb, lo, hi, ref, flush, torch, stream, res):
    """The plain per-segment form with the per-n search (the paper's shape)
    and with the bit-parallel search.  Each sweeps plain_seg_bits over
    [lo, lo + 10^11] and runs the whole range at its best size; every record
    of both runs must equal the persistent kernel's.  Then the persistent
    kernel with the per-n search over the whole range, for the ratio at equal
    search."""
    sweep_hi = min(hi, lo + 10**11)
    bc = gb.gb_get_option("search_chunks") or 6
    nrec = (ref["n_count"] + (1 << SEG_BITS) - 1) >> SEG_BITS
    prec, pagg, _ = gb.gb_verify_range_segments(lo, hi, nrec)
    out = {}
    for name, pbc in (("per_n", 0), ("bit_parallel", bc)):
        gb.gb_set_option("plain_search_chunks", pbc)
        sweep = []
        for sb in (22, 24, 26, 28, 30):
            gb.gb_set_option("plain_seg_bits", sb)
            gb.gb_verify_range_plain(lo, lo + 10**8)                 # buffers for this size
            flush.fill_(7)
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, r, _ = gb.gb_verify_range_plain(lo, sweep_hi, 0)
            sweep.append({"plain_seg_bits": sb, "value": r["n_count"] / (time.perf_counter() - t)})
        best = max(sweep, key=lambda x: x["value"])
        gb.gb_set_option("plain_seg_bits", best["plain_seg_bits"])
        flush.fill_(5)
        torch.cuda.synchronize()
        t = time.perf_counter()
        recs, r, n = gb.gb_verify_range_plain(lo, hi, nrec)
        dt = time.perf_counter() - t
        # the two forms agree on every field of every record, not just the totals
        assert n == nrec and len(recs) == nrec and (recs == prec).all(), name
        assert {k: r[k] for k in pagg if k != "status"} == {k: pagg[k] for k in pagg if k != "status"}
        out[name] = {"value": r["n_count"] / dt, "unit": "even_n/s", "seconds": dt,
                     "plain_seg_bits": best["plain_seg_bits"], "search_chunks": pbc, "sweep": sweep,
                     "records_compared": nrec, "records_equal": True}
    gb.gb_set_option("plain_search_chunks", 0)
    gb.gb_set_option("plain_seg_bits", 26)
    # the persistent kernel with the per-n search (the tuned shape, or the
    # single-role kernel where the tuned pipelined shape has no per-n build)
    keep = {k: gb.gb_get_option(k) for k in ("search_chunks", "autotune", "builder_warps", "tile_bits")}
    gb.gb_set_option("autotune", 0)
    gb.gb_set_option("search_chunks", 0)
    try:
        kernel_seconds(gb, lo, lo + 10**8, res, stream)
    except gb.GbError:
        gb.gb_set_option("builder_warps", 0)
        gb.gb_set_option("tile_bits", 20)
    with torch.cuda.stream(stream):
        flush.fill_(9)
    ks, r = kernel_seconds(gb, lo, hi, res, stream)
    assert r["sum_pmin"] == ref["sum_pmin"] and r["argmax_n"] == ref["argmax_n"]
    out["persistent_per_n"] = {"value": r["n_count"] / ks, "unit": "even_n/s", "kernel_s": ks,
                               "builder_warps": gb.gb_get_option("builder_warps"),
                               "tile_bits": gb.gb_get_option("tile_bits")}
    for k, v in keep.items():
        gb.gb_set_option(k, v)
    return out


def measure_extra(gb, torch, args):
    """C1, C3a and C3b throughput, and a shortened C4 serving run, each on a
    fresh context (rank 0 only)."""
    from paper_2603_07850_gb300 import workloads as W
    import serve_bench
    extra = {}
    stream = torch.cuda.Stream()
    res = torch.zeros(gb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    # C1: every even n in [4, 1e10], records of 2^15, autotuned, graph replays
    c = W.C1
    gb.gb_init(c.p_max, c.seg_bits)
    gb.gb_set_option("time_kernel", 1)
    gb.gb_set_option("autotune", 1)
    kernel_seconds(gb, c.lo, c.hi, res, stream)                    # tunes
    ts = [kernel_seconds(gb, c.lo, c.hi, res, stream) for _ in range(5)]
    ks = min(t for t, _ in ts)
    extra["C1"] = {"workload": "every even n in [4, 1e10], records of 2^15", "value": ts[0][1]["n_count"] / ks,
                   "unit": "even_n/s", "kernel_s": ks, "tile_bits": gb.gb_get_option("tile_bits"),
                   "builder_warps": gb.gb_get_option("builder_warps"),
                   "search_chunks": gb.gb_get_option("search_chunks")}
    # C3a: [1e18, 1e18 + 1e10), base primes to 2^30 - 1, bucket pre-pass; the
    # whole blocking call after a warm-up call that builds the table and tunes
    c = W.C3A
    gb.gb_init(c.p_max, c.seg_bits)
    gb.gb_set_option("autotune", 1)
    gb.gb_verify_range(c.lo, c.hi)
    walls = []
    for _ in range(3):
        t = time.perf_counter()
        r = gb.gb_verify_range(c.lo, c.hi)
        walls.append(time.perf_counter() - t)
    extra["C3a"] = {"workload": "[1e18, 1e18 + 1e10)", "value": r["n_count"] / min(walls), "unit": "even_n/s",
                    "call_s": min(walls), "max_pmin": r["max_pmin"], "status": r["status"],
                    "tuned": {k: gb.gb_get_option(k) for k in ("tile_bits", "threads", "search_chunks", "builder_warps",
                                                               "bucket_min", "bucket_chunk_tiles", "tier_b_min")}}
    gb.gb_shutdown()
    # C3b: [2^64 - 2^33, 2^64 - 2), base primes to 2^32 - 1, the same way
    c = W.C3B
    gb.gb_init(c.p_max, c.seg_bits)
    gb.gb_set_option("autotune", 1)
    gb.gb_verify_range(c.lo, c.hi)
    walls = []
    for _ in range(3):
        t = time.perf_counter()
        r = gb.gb_verify_range(c.lo, c.hi)
        walls.append(time.perf_counter() - t)
    extra["C3b"] = {"workload": "[2^64 - 2^33, 2^64 - 2)", "value": r["n_count"] / min(walls), "unit": "even_n/s",
                    "call_s": min(walls), "max_pmin": r["max_pmin"], "status": r["status"],
                    "tuned": {k: gb.gb_get_option(k) for k in ("tile_bits", "threads", "search_chunks", "builder_warps",
                                                               "bucket_min", "bucket_chunk_tiles", "tier_b_min")}}
    gb.gb_shutdown()
    # C4: the seeded serving stream, shortened
    extra["C4"] = serve_bench.measure(gb, requests=args.serve_requests, capacity_requests=args.serve_requests,
                                      load=0.7, oracle_sample=0.05)
    return extra


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2603_07850_gb300 import binding as gb, build
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    gb.load()
    unit_peaks = gb.gb_measure_peaks()          # microbenchmarks, before anything is timed
    gb.gb_init(P_MAX, SEG_BITS)
    gb.gb_set_option("time_kernel", 1)
    gb.gb_set_option("autotune", 0 if args.no_autotune else 1)   # the first warm-up step tunes
    for kv in args.option:
        k, v = kv.split("=", 1)
        gb.gb_set_option(k, int(v))
    lo = rank * args.n_top + 4
    hi = (rank + 1) * args.n_top + 1
    n_total = (hi - 1 - lo) // 2 + 1 if lo % 2 == 0 else None

    stream = torch.cuda.Stream()
    res = torch.zeros(gb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step():
        gb.gb_verify_range_async(lo, hi, res.data_ptr(), stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            step()
    stream.synchronize()

    replays0 = gb.gb_stats()["graph_replays"]
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_us = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xFF)              # L2 flush between steps (not timed)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stream.synchronize()
            kernel_us.append(gb.gb_get_option("last_kernel_us"))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    replays = gb.gb_stats()["graph_replays"] - replays0
    assert replays == args.steps, (replays, args.steps)     # every timed step was one graph replay
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    out = gb.result_from_bytes(bytes(res.cpu().numpy()))
    if out["status"] not in (0,):
        raise SystemExit(f"device status {out['status']}: {gb.gb_last_error()}")

    # end to end through the blocking C-ABI call with host buffers
    e2e_t = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(3)
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = gb.gb_verify_range(lo, hi)
        e2e_t.append(time.perf_counter() - t)
        assert r["n_count"] == out["n_count"] and r["sum_pmin"] == out["sum_pmin"]
    e2e_s = sum(e2e_t) / len(e2e_t)

    plain = None
    if not args.no_plain and rank == 0:
        plain = measure_plain(gb, lo, hi, out, flush, torch, stream, res)

    # max over ranks of the step time and of the e2e time; the results of the
    # ranks' blocks merge into one (the only exchange)
    tot_n = out["n_count"]
    merged = out
    if dist:
        from paper_2603_07850_gb300 import multi
        merged = multi.gather_merge(out)
        t = torch.tensor([ms, e2e_s, float(out["n_count"])], dtype=torch.float64, device="cuda")
        g = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(g, t)
        ms = max(float(x[0]) for x in g)
        e2e_s = max(float(x[1]) for x in g)
        tot_n = sum(int(x[2]) for x in g)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    opt = {k: gb.gb_get_option(k) for k in ("k_words", "tile_bits", "wheel", "pattern_max",
                                            "search_chunks", "threads", "sms")}
    alg = algorithmic_instructions(out["n_first"], out["n_count"], opt["k_words"], out["hist"])
    kus = statistics.mean(kernel_us) if kernel_us else None
    sm_clock = (peaks or {}).get("sm_max_mhz", 2070.0)
    peak = opt["sms"] * 128 * sm_clock * 1e6          # 4 schedulers x 32 lanes per SM per clock
    achieved = alg["instr"] / (kus * 1e-6) if kus else None
    prof = measured_profile(out["n_count"])
    traffic = prof["traffic"] if prof else None
    executed = prof["inst_executed"] if prof else None
    line = {
        "metric": "even n verified/s at N=1e12", "value": tot_n / (ms * 1e-3),
        "unit": "even_n/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "every even n in [4, 1e12] (per rank: its own 1e12 block)",
                   "p_max": P_MAX, "seg_bits": SEG_BITS,
                   "tile_bits": gb.gb_get_option("tile_bits"),
                   "threads": gb.gb_get_option("threads"), "wheel": gb.gb_get_option("wheel"),
                   "search_chunks": gb.gb_get_option("search_chunks"),
                   "pattern_max": gb.gb_get_option("pattern_max"),
                   "search_pmax": gb.gb_get_option("search_pmax"),
                   "tier_b_min": gb.gb_get_option("tier_b_min"),
                   "builder_warps": gb.gb_get_option("builder_warps"),
                   "l2": "flushed between steps (512 MB write)", "form": "persistent",
                   "launch": "one captured CUDA graph replay per step"},
        "e2e": {"value": tot_n / e2e_s, "unit": "even_n/s", "h2d_bytes_per_step": 64,
                "d2h_bytes_per_step": gb.RESULT_BYTES},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9 if achieved else None,
                     "peak": peak / 1e9, "unit": "Ginstr/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_note": (None if not prof else
                                      f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch over "
                                      f"{prof['captured_n']} even n" + (", scaled to this launch by n"
                                                                        if prof["scaled"] else "")),
                     "frac_executed": (executed * 32 / (kus * 1e-6) / peak) if (executed and kus) else None,
                     "executed_note": "ncu smsp__inst_executed.sum x 32 lanes / (kernel time x issue-slot "
                                      "peak): the issue slots the kernel filled, useful or not",
                     "kernel": "persistent_kernel", "kernel_us": kus,
                     "algorithmic_instr_per_n": alg["per_n"], "marks_per_n": alg["marks_per_n"],
                     "tail_fraction": alg["tail_fraction"],
                     "peak_note": "issue slots: SMs x 4 schedulers x 32 lanes x max SM clock "
                                  "(derived, of measured clock)",
                     "measured_units": {k: v / 1e9 for k, v in unit_peaks.items() if k != "sms"},
                     "frac_vs_measured_int": (achieved / (unit_peaks["int_logic_ops"] + unit_peaks["int_mad_ops"])
                                              if achieved else None),
                     "frac_vs_measured_smem": (alg["smem"] / (kus * 1e-6) / unit_peaks["smem_atomic_ops"]
                                               if kus else None),
                     "measured_note": "G lane-ops/s of our microbenchmarks (gb_measure_peaks): INT32 "
                                      "logic/shift, integer mad, popc, conflict-free shared atomicAnd; the "
                                      "integer fraction divides by logic + mad (two pipes)"},
        "plain": plain,
        "speedup_vs_plain": (tot_n / (ms * 1e-3)) / plain["per_n"]["value"] if plain else None,
        "speedup_same_search_per_n": (plain["persistent_per_n"]["value"] / plain["per_n"]["value"]
                                      if plain else None),
        "speedup_same_search_bit_parallel": ((out["n_count"] / (ms * 1e-3)) / plain["bit_parallel"]["value"]
                                             if plain else None),
        "result": {k: merged[k] for k in ("n_count", "max_pmin", "argmax_n", "sum_pmin", "n_slow")},
    }
    try:
        v, n, dt, k = cpu_sample(args.n_top, args.cpu_records)
        line["cpu_baseline"] = {"value": v, "unit": "even_n/s", "cores": 1, "kind": "oracle",
                                "sample": f"{k} seeded records of 2^20 even n in [4, 1e12], "
                                          f"{dt:.1f} s single-threaded"}
    except Exception as e:  # noqa: BLE001
        line["cpu_baseline"] = {"value": None, "unit": "even_n/s", "cores": 1, "kind": "oracle",
                                "sample": f"failed: {e}"}
    if args.cpu_all_cores > 0:
        try:
            v, n, dt, k, cores, model = cpu_sample_all_cores(args.n_top, args.cpu_all_cores)
            line["cpu_baseline_all_cores"] = {
                "value": v, "unit": "even_n/s", "cores": cores, "kind": "oracle", "cpu": model,
                "sample": f"{k} seeded records of 2^20 even n in [4, 1e12], one oracle process per "
                          f"core, {dt:.1f} s wall"}
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline_all_cores"] = {"value": None, "sample": f"failed: {e}"}
    if not args.no_extra:
        line["configs_extra"] = measure_extra(gb, torch, args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
