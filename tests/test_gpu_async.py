"""gb_verify_range_async: the pipeline enqueued on a caller stream and
replayed from a captured CUDA graph, against the blocking call.

Each call rewrites only the parameter kernel's arguments in the instantiated
graph, so consecutive calls over different ranges must give exactly the
blocking call's results (all outputs are integers), and every call is one
graph replay.
"""
import pytest

pytestmark = pytest.mark.gpu

RANGES = [(4, 10**8 + 1), (10**11, 10**11 + 2 * 10**8 + 7), (10**9 + 1, 10**9 + 3 * 10**7), (4, 10**8 + 1)]


@pytest.fixture()
def env():
    torch = pytest.importorskip("torch")
    from paper_2603_07850_gb300 import binding as gb, build
    build.build()
    gb.load()
    yield torch, gb
    gb.gb_shutdown()


def run_async(torch, gb, lo, hi, out, stream):
    gb.gb_verify_range_async(lo, hi, out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return gb.result_from_bytes(bytes(out.cpu().numpy()))


@pytest.mark.parametrize("opts", [{}, {"use_graph": 0}, {"builder_warps": 16, "tile_bits": 19},
                                  {"time_kernel": 1}],
                         ids=["graph", "direct", "graph_pipelined", "graph_timed"])
def test_async_matches_blocking_call(env, opts):
    torch, gb = env
    gb.gb_init(1 << 16, 20)
    for k, v in opts.items():
        gb.gb_set_option(k, v)
    ref = [gb.gb_verify_range(lo, hi) for lo, hi in RANGES]
    stream = torch.cuda.Stream()
    outs = [torch.zeros(gb.RESULT_BYTES, dtype=torch.uint8, device="cuda") for _ in range(2)]
    before = gb.gb_stats()["graph_replays"]
    for i, ((lo, hi), want) in enumerate(zip(RANGES, ref)):
        outs[i % 2].fill_(0xCD)                    # stale bytes must not survive
        got = run_async(torch, gb, lo, hi, outs[i % 2], stream)
        assert got == want, (lo, hi)
        if opts.get("time_kernel"):
            assert gb.gb_get_option("last_kernel_us") > 0
    replays = gb.gb_stats()["graph_replays"] - before
    assert replays == (0 if opts.get("use_graph") == 0 else len(RANGES))
