"""Multi-rank host logic on CPU ranks (gloo, world size 2): sharding, the
final gather-and-merge, and a rank that leaves before the exchange.

Each rank's block is computed by the CPU oracle as a stand-in for its GPU;
the merged result must equal the oracle's result for the whole range.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import oracle
from paper_2603_07850_gb300 import multi

FIELDS = ("n_first", "n_count", "max_pmin", "argmax_n", "sum_pmin", "wsum_pmin", "n_slow",
          "counterexample_n", "hist")


def whole(lo, hi):
    st, recs, _, _ = oracle.pmin_range(lo, hi, p_max=1 << 16, seg_bits=40)
    r = recs[0].as_dict()
    r["status"] = st
    return r


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, lo, hi, out_q, leave_early):
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    a, b = multi.shard_range(lo, hi, rank, world, align_bits=10)
    part = whole(a, b) if b > a else multi.merge_results([])
    if leave_early and rank == 1:
        os._exit(0)                          # leaves between steps, nothing in flight
    try:
        merged = multi.gather_merge(part)
        out_q.put((rank, "ok", {k: merged[k] for k in FIELDS}))
    except Exception as e:                   # noqa: BLE001
        out_q.put((rank, "error", type(e).__name__))
    dist.destroy_process_group()


def run_world(lo, hi, leave_early=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, lo, hi, q, leave_early)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    out = []
    while not q.empty():
        out.append(q.get())
    return sorted(out)


@pytest.mark.parametrize("lo,hi", [(4, 3_000_001), (10**9 + 1, 10**9 + 777_777), (4, 5)])
def test_two_ranks_merge_to_the_whole_range(lo, hi):
    out = run_world(lo, hi)
    assert [o[1] for o in out] == ["ok", "ok"]
    ref = whole(lo, hi) if hi > 4 else multi.merge_results([])
    for _, _, merged in out:
        assert {k: merged[k] for k in FIELDS} == {k: ref[k] for k in FIELDS}


def test_shards_cover_the_range_exactly():
    for lo, hi, world in [(4, 10**6, 3), (5, 1234567, 4), (10**12, 10**12 + 10, 8), (4, 4, 2)]:
        blocks = [multi.shard_range(lo, hi, r, world, align_bits=6) for r in range(world)]
        ns = [n for a, b in blocks for n in range(a, b, 2)]
        n0 = max(lo, 4) + (max(lo, 4) & 1)
        assert ns == list(range(n0, hi, 2))


def test_a_rank_that_leaves_is_detected():
    out = run_world(4, 1_000_001, leave_early=True)
    # the surviving rank's exchange ends with an error instead of hanging
    assert out and out[0][0] == 0 and out[0][1] == "error"
