"""gb_verify_range_claimed: callers verify one range together by claiming its
tiles from a counter in shared host memory (the kernels bump it with
system-scope atomics), and their merged records equal one ordinary call.

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

pytestmark = pytest.mark.gpu

LO, HI = 10**10, 10**10 + 8 * 10**10 + 17       # 4e10 even n, 38,147 tiles of 2^20


def _caller(shm_name, barrier, q, lo, hi):
    from paper_2603_07850_gb300 import binding as gb
    gb.load()
    gb.gb_init(1 << 16, 22)
    gb.gb_verify_range(4, 10**6)                    # warm: context, table, kernels
    shm = shared_memory.SharedMemory(name=shm_name)
    ptr = ctypes.addressof(ctypes.c_uint64.from_buffer(shm.buf))
    barrier.wait(timeout=300)
    recs, agg, n = gb.gb_verify_range_claimed(lo, hi, ptr, 1 << 16)
    q.put((recs.tobytes(), agg["n_count"], agg["status"]))
    gb.gb_shutdown()
    del ptr
    shm.close()


@pytest.fixture(scope="module")
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    yield binding
    binding.gb_shutdown()


def test_single_caller_equals_the_plain_call(gb):
    gb.gb_init(1 << 16, 22)
    ref, ref_agg, n = gb.gb_verify_range_segments(LO, HI, 1 << 16)
    mm = mmap.mmap(-1, mmap.PAGESIZE)               # page-aligned host memory, zeroed
    counter = ctypes.c_uint64.from_buffer(mm)
    recs, agg, n2 = gb.gb_verify_range_claimed(LO, HI, ctypes.addressof(counter), 1 << 16)
    assert n2 == n and (recs == ref).all()
    assert agg == ref_agg
    ntiles = -(-ref_agg["n_count"] // (1 << 20))
    assert counter.value >= ntiles                  # every tile claimed, then a final claim per CTA
    del counter
    mm.close()


def test_two_processes_share_the_tiles(gb):
    from paper_2603_07850_gb300 import multi
    from paper_2603_07850_gb300.binding import SEG_DTYPE
    gb.gb_init(1 << 16, 22)
    ref, ref_agg, n = gb.gb_verify_range_segments(LO, HI, 1 << 16)
    gb.gb_shutdown()
    shm = shared_memory.SharedMemory(create=True, size=64)
    shm.buf[:8] = bytes(8)
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
    merged = multi.merge_record_sets(sets)
    assert (merged == ref).all()
    print("tiles' n per caller:", counts)
