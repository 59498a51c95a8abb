"""Failure paths, all provoked on the host or by bounded waits (no GPU fault,
trap or hang is ever caused):

* GB_FAULT makes the k-th cudaMalloc / kernel launch / cudaMemcpy of the
  library fail before it reaches CUDA: calls return clean status codes,
  nothing leaks, and the context keeps working;
* the slow-path candidate cap turns into GB_ESLOWPATH_LIMIT;
* a serving batch that outlives timeout_ms turns into GB_ETIMEOUT and the
  loop recovers; gb_poll with a zero timeout reports GB_PENDING.
"""
import os

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture()
def gb():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    yield binding
    binding.gb_shutdown()
    os.environ.pop("GB_FAULT", None)


def free_mem():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_malloc_failures_leak_nothing(gb):
    torch = pytest.importorskip("torch")
    torch.cuda.init()
    gb.gb_init(1 << 16, 20)
    ref = gb.gb_verify_range(10**12, 10**12 + 10**7)
    gb.gb_shutdown()
    base = free_mem()
    outcomes = []
    for k in range(1, 25):                 # past the allocations of init and the first call
        os.environ["GB_FAULT"] = f"malloc:{k}"
        try:
            gb.gb_init(1 << 16, 20)
        except gb.GbError as e:
            assert e.code == gb.GB_ENOMEM and "injected" in gb.gb_last_error()
            outcomes.append("init")
            with pytest.raises(gb.GbError):
                gb.gb_verify_range(4, 100)                  # no context was left behind
            continue
        try:
            r = gb.gb_verify_range(10**12, 10**12 + 10**7)
            assert r == ref
            outcomes.append("ok")
        except gb.GbError as e:
            assert e.code == gb.GB_ENOMEM
            outcomes.append("call")
            assert gb.gb_verify_range(10**12, 10**12 + 10**7) == ref   # still usable
        gb.gb_shutdown()
    os.environ.pop("GB_FAULT")
    assert "init" in outcomes and "call" in outcomes and "ok" in outcomes
    assert abs(free_mem() - base) < 64 << 20


def test_injected_failure_in_a_large_table_build_frees_it(gb):
    pytest.importorskip("torch")
    base = free_mem()
    # base primes up to 2^32 need the bitset, block counts and offsets, then
    # the 0.8 GB prime array and the 1.6 GB reciprocal array: fail the last
    os.environ["GB_FAULT"] = "malloc:12"
    gb.gb_init(1 << 16, 20)
    with pytest.raises(gb.GbError) as ei:
        gb.gb_verify_range((1 << 64) - 10**6, (1 << 64) - 2)
    assert ei.value.code == gb.GB_ENOMEM
    gb.gb_shutdown()
    os.environ.pop("GB_FAULT")
    assert abs(free_mem() - base) < 64 << 20


@pytest.mark.parametrize("kind", ["launch", "memcpy"])
def test_injected_launch_and_copy_failures(gb, kind):
    gb.gb_init(1 << 16, 15)
    gb.gb_set_option("use_graph", 0)
    recs, ref, n = gb.gb_verify_range_segments(10**9, 10**9 + 10**7, 1024)
    gb.gb_shutdown()
    failed = 0
    for k in range(1, 6):
        os.environ["GB_FAULT"] = f"{kind}:{k}"
        try:
            gb.gb_init(1 << 16, 15)
            gb.gb_set_option("use_graph", 0)
        except gb.GbError as e:
            assert e.code == gb.GB_ECUDA
            failed += 1
            continue
        try:
            r2, g2, _ = gb.gb_verify_range_segments(10**9, 10**9 + 10**7, 1024)
            assert g2 == ref and (r2 == recs).all()
        except gb.GbError as e:
            assert e.code == gb.GB_ECUDA and "injected" in gb.gb_last_error()
            failed += 1
            r2, g2, _ = gb.gb_verify_range_segments(10**9, 10**9 + 10**7, 1024)
            assert g2 == ref and (r2 == recs).all()
        gb.gb_shutdown()
    os.environ.pop("GB_FAULT")
    assert failed >= 1


def test_slow_path_cap_reports_a_status(gb):
    # P_max = 2 sends every n >= 6 to the slow path; a cap of 64 candidates
    # cannot reach p_min of the hardest n below 10^6
    gb.gb_init(2, 12)
    gb.gb_set_option("slow_cap", 6)
    with pytest.raises(gb.GbError) as ei:
        gb.gb_verify_range(4, 10**6)
    assert ei.value.code == gb.GB_ESLOWPATH_LIMIT
    gb.gb_set_option("slow_cap", 24)
    r = gb.gb_verify_range(4, 10**6)                         # the context still works
    assert r["status"] == 0 and r["n_slow"] == r["n_count"] - 1


def test_serving_timeout_and_recovery(gb):
    gb.gb_init(1 << 16, 20)
    t = gb.gb_submit(4, 4 * 10**11)                          # ~100 batches
    st, r = gb.gb_poll(t, 0)
    assert st == gb.GB_PENDING and r is None
    gb.gb_poll(t, -1)
    gb.gb_set_option("timeout_ms", 1)                        # shorter than one batch
    t = gb.gb_submit(4, 4 * 10**11)
    with pytest.raises(gb.GbError) as ei:
        gb.gb_poll(t, -1)
    assert ei.value.code == gb.GB_ETIMEOUT
    gb.gb_set_option("timeout_ms", 600000)
    t = gb.gb_submit(10**9, 10**9 + 10**6)
    st, r = gb.gb_poll(t, -1)
    assert st == 0 and r == {**gb.gb_verify_range(10**9, 10**9 + 10**6),
                             "submit_ns": r["submit_ns"], "done_ns": r["done_ns"]}
