"""gb_verify_range_claimed: callers verify one range together by claiming its
tiles from a counter in shared host memory (the kernels bump it with
system-scope atomics), and their merged records equal one ordinary call and,
on seeded records, the oracle.

Two processes on the one GPU share the counter; their kernels never wait on
each other, they only take the next tile.  Records of 2^22 n hold four
2^20-n tiles, so a record can be split between the callers and the merge
has to add.
"""
import ctypes
import mmap
import multiprocessing as mp
from multiprocessing import shared_memory

import numpy as np
import pytest

import oracle
import recutil
from paper_2603_07850_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LO, HI = 10**10, 10**10 + 8 * 10**10 + 17       # 4e10 even n, 38,147 tiles of 2^20
SEG_BITS = 22


def _caller(shm_name, barrier, q, lo, hi):
    from paper_2603_07850_gb300 import binding as gb
    gb.load()
    gb.gb_init(1 << 16, SEG_BITS)
    gb.gb_verify_range(4, 10**6)                    # warm: context, table, kernels
    shm = shared_memory.SharedMemory(name=shm_name)
    ptr = ctypes.addressof(ctypes.c_uint64.from_buffer(shm.buf))
    barrier.wait(timeout=300)
    recs, agg, n = gb.gb_verify_range_claimed(lo, hi, ptr, 1 << 16)
    q.put((recs.tobytes(), agg["n_count"], agg["status"]))
    gb.gb_shutdown()
    del ptr
    shm.close()


def oracle_check(recs, lo, hi, seed, count=3):
    """Seeded records of a merged set against the oracle, record-exact."""
    cfg = W.RangeConfig("claimed", lo, hi, 1 << 16, SEG_BITS, 0, "")
    for r in W.sample_records(cfg, count, seed):
        a, b = W.record_bounds(lo, hi, SEG_BITS, r)
        st, orecs, _, _ = oracle.pmin_range(a, b, p_max=1 << 16, seg_bits=SEG_BITS)
        assert st == 0 and len(orecs) == 1
        assert recutil.canon(recs[r]) == recutil.canon(orecs[0]), r


@pytest.fixture(scope="module")
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    yield binding
    binding.gb_shutdown()


def test_single_caller_equals_the_plain_call(gb):
    gb.gb_init(1 << 16, SEG_BITS)
    ref, ref_agg, n = gb.gb_verify_range_segments(LO, HI, 1 << 16)
    mm = mmap.mmap(-1, mmap.PAGESIZE)               # page-aligned host memory, zeroed
    counter = ctypes.c_uint64.from_buffer(mm)
    recs, agg, n2 = gb.gb_verify_range_claimed(LO, HI, ctypes.addressof(counter), 1 << 16)
    assert n2 == n and (recs == ref).all()
    assert agg == ref_agg
    ntiles = -(-ref_agg["n_count"] // (1 << 20))
    assert counter.value >= ntiles                  # every tile claimed, then a final claim per CTA
    oracle_check(recs, LO, HI, seed=0xF1)
    del counter
    mm.close()


def test_a_caller_with_other_settings_is_refused(gb):
    mm = mmap.mmap(-1, mmap.PAGESIZE)
    block = ctypes.addressof(ctypes.c_uint64.from_buffer(mm))
    gb.gb_init(1 << 16, SEG_BITS)
    lo, hi = 10**9, 10**9 + 4 * 10**7
    recs, agg, n = gb.gb_verify_range_claimed(lo, hi, block, 1 << 10)
    assert agg["n_count"] == W.num_even(lo, hi)
    used = ctypes.c_uint64.from_buffer(mm, 0).value
    # another tile size, another range or another P_max would index other n
    for change in ({"tile_bits": 18}, {"range": (lo, hi + 2)}, {"p_max": 1 << 12}):
        gb.gb_init(change.get("p_max", 1 << 16), SEG_BITS)
        if "tile_bits" in change:
            gb.gb_set_option("tile_bits", change["tile_bits"])
        a, b = change.get("range", (lo, hi))
        with pytest.raises(gb.GbError) as ei:
            gb.gb_verify_range_claimed(a, b, block, 1 << 10)
        assert ei.value.code == gb.GB_EINVAL
        assert ctypes.c_uint64.from_buffer(mm, 0).value == used    # nothing was claimed
    gb.gb_shutdown()
    mm.close()


def test_two_processes_share_the_tiles(gb):
    from paper_2603_07850_gb300 import multi
    from paper_2603_07850_gb300.binding import SEG_DTYPE
    gb.gb_init(1 << 16, SEG_BITS)
    ref, ref_agg, n = gb.gb_verify_range_segments(LO, HI, 1 << 16)
    gb.gb_shutdown()
    shm = shared_memory.SharedMemory(create=True, size=64)
    shm.buf[:gb.CLAIM_BYTES] = bytes(gb.CLAIM_BYTES)
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(2), ctx.Queue()
    procs = [ctx.Process(target=_caller, args=(shm.name, barrier, q, LO, HI)) for _ in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
    shm.close()
    shm.unlink()
    sets = [np.frombuffer(b, dtype=SEG_DTYPE) for b, _, _ in out]
    counts = [c for _, c, _ in out]
    assert all(st == 0 for _, _, st in out)
    assert sum(counts) == ref_agg["n_count"]        # every tile verified exactly once
    assert min(counts) > 0                          # both callers took tiles
    # the record-add path ran: some records hold n of both callers
    assert ((sets[0]["n_count"] > 0) & (sets[1]["n_count"] > 0)).any()
    merged = multi.merge_record_sets(sets, n_total=W.num_even(LO, HI))
    assert (merged == ref).all()
    oracle_check(merged, LO, HI, seed=0xF2)
    print("tiles' n per caller:", counts)
