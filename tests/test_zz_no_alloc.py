"""The allocation-free entry point against the ordinary one.

gb_verify_range_noalloc serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or an allocation would stall a
latency-critical loop): it works out of a fixed static device scratch.  Its
results must equal gb_verify_range's exactly (all outputs are integers), on
consecutive calls that reuse the same scratch.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_verify_range_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    out = torch.zeros(gb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    calls = [
        (4, 10**9 + 1, 1 << 16, 22),                  # near the origin, records inside tiles' reach
        (10**11, 10**11 + 6 * 10**8 + 7, 64, 16),     # far out, P_max = 64: slow path busy
        (4, 10**9 + 1, 1 << 16, 22),                  # the first call again on the reused scratch
    ]
    for lo, hi, p_max, seg_bits in calls:
        out.fill_(0xAB)                               # stale bytes must not leak into the result
        gb.gb_verify_range_noalloc(lo, hi, p_max, seg_bits, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = gb.result_from_bytes(bytes(out.cpu().numpy()))
        gb.gb_init(p_max, seg_bits)
        try:
            ref = gb.gb_verify_range(lo, hi)
        finally:
            gb.gb_shutdown()
        assert got == ref, (lo, hi, p_max, seg_bits)
        assert got["status"] == 0 and got["n_count"] > 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    out = torch.zeros(gb.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for lo, hi, p_max, seg_bits in [
        (4, 10**10, 1 << 16, 15),         # 152,588 records > 8192
        (1 << 40, (1 << 40) + 100, 1 << 16, 20),   # n beyond 2^40
        (4, 1000, 1 << 17, 20),           # P_max beyond 2^16
    ]:
        with pytest.raises(gb.GbError) as ei:
            gb.gb_verify_range_noalloc(lo, hi, p_max, seg_bits, out.data_ptr(), stream)
        assert ei.value.code == gb.GB_EINVAL
