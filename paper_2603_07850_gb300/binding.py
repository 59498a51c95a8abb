"""Thin ctypes binding over libgoldbach_gb300.so (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all of the sieve, search and reduction work runs in
the library's CUDA kernels.  If the shared library is missing or fails to
load, importing this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgoldbach_gb300.so")

GB_OK = 0
GB_PENDING = 1
GB_COUNTEREXAMPLE = 2
GB_EINVAL = -1
GB_ENOMEM = -2
GB_ECUDA = -3
GB_ETIMEOUT = -4
GB_ESLOWPATH_LIMIT = -5
GB_EOVERFLOW = -6
GB_EINTERNAL = -7

U64 = ctypes.c_uint64


class GbResult(ctypes.Structure):
    _fields_ = [
        ("n_first", U64), ("n_count", U64), ("max_pmin", U64), ("argmax_n", U64),
        ("sum_pmin", U64), ("wsum_pmin", U64), ("hist", U64 * 64), ("n_slow", U64),
        ("counterexample_n", U64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("submit_ns", U64), ("done_ns", U64),
    ]

    def as_dict(self) -> dict:
        return {f: (list(getattr(self, f)) if f == "hist" else int(getattr(self, f)))
                for f, _ in self._fields_ if f != "reserved"}


class GbSegRecord(ctypes.Structure):
    _fields_ = [
        ("n_first", U64), ("n_count", U64), ("max_pmin", U64), ("argmax_n", U64),
        ("sum_pmin", U64), ("wsum_pmin", U64), ("hist", U64 * 64), ("n_slow", U64),
        ("counterexample_n", U64),
    ]


SEG_DTYPE = np.dtype([
    ("n_first", "<u8"), ("n_count", "<u8"), ("max_pmin", "<u8"), ("argmax_n", "<u8"),
    ("sum_pmin", "<u8"), ("wsum_pmin", "<u8"), ("hist", "<u8", (64,)), ("n_slow", "<u8"),
    ("counterexample_n", "<u8"),
])
assert SEG_DTYPE.itemsize == ctypes.sizeof(GbSegRecord)


class GbStats(ctypes.Structure):
    _fields_ = [(n, U64) for n in (
        "calls", "tiles", "n_verified", "n_slow", "kernel_launches", "graph_replays",
        "requests_submitted", "requests_completed", "requests_rejected", "base_prime_count",
        "base_prime_limit", "device_bytes")]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class GbProgress(ctypes.Structure):
    _fields_ = [("tiles_done", U64), ("tiles_total", U64), ("n_done", U64), ("n_total", U64),
                ("elapsed_s", ctypes.c_double), ("n_per_s", ctypes.c_double), ("eta_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class GbPeaks(ctypes.Structure):
    _fields_ = [("int_logic_ops", ctypes.c_double), ("int_mad_ops", ctypes.c_double),
                ("popc_ops", ctypes.c_double), ("smem_atomic_ops", ctypes.c_double),
                ("sms", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class GbError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2603_07850_gb300.build.build()")
    lib = ctypes.CDLL(path)
    u32, i32, i64, sz = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "gb_init": ([u32, u32], ctypes.c_int),
        "gb_set_option": ([ctypes.c_char_p, i64], ctypes.c_int),
        "gb_get_option": ([ctypes.c_char_p, P(i64)], ctypes.c_int),
        "gb_shutdown": ([], None),
        "gb_verify_range": ([U64, U64, P(GbResult)], ctypes.c_int),
        "gb_verify_range_segments": ([U64, U64, ctypes.c_void_p, sz, P(sz), P(GbResult)], ctypes.c_int),
        "gb_verify_range_plain": ([U64, U64, ctypes.c_void_p, sz, P(sz), P(GbResult)], ctypes.c_int),
        "gb_verify_range_claimed": ([U64, U64, ctypes.c_void_p, ctypes.c_void_p, sz, P(sz), P(GbResult)],
                                    ctypes.c_int),
        "gb_verify_range_async": ([U64, U64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
        "gb_verify_range_noalloc": ([U64, U64, u32, u32, ctypes.c_void_p, ctypes.c_void_p],
                                    ctypes.c_int),
        "gb_submit": ([U64, U64, P(U64)], ctypes.c_int),
        "gb_poll": ([U64, P(GbResult), i32], ctypes.c_int),
        "gb_stats": ([P(GbStats)], ctypes.c_int),
        "gb_progress": ([P(GbProgress)], ctypes.c_int),
        "gb_measure_peaks": ([P(GbPeaks)], ctypes.c_int),
        "gb_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(fn: str, rc: int, ok=(GB_OK,)) -> int:
    if rc not in ok:
        raise GbError(fn, rc, gb_last_error())
    return rc


def gb_last_error() -> str:
    v = load().gb_last_error()
    return v.decode() if v else ""


def gb_init(p_max: int = 1 << 16, seg_bits: int = 20) -> None:
    _check("gb_init", load().gb_init(p_max, seg_bits))


def gb_set_option(key: str, value: int) -> None:
    _check("gb_set_option", load().gb_set_option(key.encode(), int(value)))


def gb_get_option(key: str) -> int:
    v = ctypes.c_int64(0)
    _check("gb_get_option", load().gb_get_option(key.encode(), ctypes.byref(v)))
    return v.value


def gb_shutdown() -> None:
    load().gb_shutdown()


def gb_verify_range(lo: int, hi: int, check: bool = True) -> dict:
    """check=False returns the result (its "status" field set) instead of
    raising on an error status."""
    r = GbResult()
    rc = load().gb_verify_range(lo, hi, ctypes.byref(r))
    if check:
        _check("gb_verify_range", rc, ok=(GB_OK, GB_COUNTEREXAMPLE))
    return r.as_dict()


def _segments(fn_name: str, lo: int, hi: int, cap: int, check: bool = True):
    lib = load()
    buf = np.zeros(max(cap, 1), dtype=SEG_DTYPE)
    n = ctypes.c_size_t(0)
    r = GbResult()
    rc = getattr(lib, fn_name)(lo, hi, buf.ctypes.data, cap, ctypes.byref(n), ctypes.byref(r))
    if check:
        _check(fn_name, rc, ok=(GB_OK, GB_COUNTEREXAMPLE))
    return buf[:min(cap, n.value)], r.as_dict(), n.value


def gb_verify_range_segments(lo: int, hi: int, cap: int, check: bool = True):
    """Returns (records ndarray[SEG_DTYPE], aggregate dict, number of records);
    check=False returns them with the aggregate's "status" set instead of
    raising on an error status."""
    return _segments("gb_verify_range_segments", lo, hi, cap, check)


def gb_verify_range_plain(lo: int, hi: int, cap: int = 0):
    return _segments("gb_verify_range_plain", lo, hi, cap)


CLAIM_BYTES = 16              # sizeof(gb_claim_t): tile counter and fingerprint


def gb_verify_range_claimed(lo: int, hi: int, claim_ptr: int, cap: int):
    """Cooperative form: claim_ptr is the host address of a gb_claim_t
    (CLAIM_BYTES, zeroed before the first call) shared by every caller.
    Returns (records of this caller's tiles, its aggregate, number of
    records)."""
    lib = load()
    buf = np.zeros(max(cap, 1), dtype=SEG_DTYPE)
    n = ctypes.c_size_t(0)
    r = GbResult()
    rc = lib.gb_verify_range_claimed(lo, hi, ctypes.c_void_p(claim_ptr), buf.ctypes.data, cap,
                                     ctypes.byref(n), ctypes.byref(r))
    _check("gb_verify_range_claimed", rc, ok=(GB_OK, GB_COUNTEREXAMPLE))
    return buf[:min(cap, n.value)], r.as_dict(), n.value


def gb_verify_range_async(lo: int, hi: int, dev_out_ptr: int, stream_ptr: int = 0) -> None:
    """dev_out_ptr: device address of a gb_result-sized buffer; stream_ptr: cudaStream_t."""
    _check("gb_verify_range_async",
           load().gb_verify_range_async(lo, hi, ctypes.c_void_p(dev_out_ptr),
                                        ctypes.c_void_p(stream_ptr or None)))


def gb_verify_range_noalloc(lo: int, hi: int, p_max: int, seg_bits: int, dev_out_ptr: int,
                            stream_ptr: int = 0) -> None:
    """Allocation-free verification into a caller-owned device gb_result
    (for callers that cannot call cudaMalloc; see the C header)."""
    _check("gb_verify_range_noalloc",
           load().gb_verify_range_noalloc(lo, hi, p_max, seg_bits, ctypes.c_void_p(dev_out_ptr),
                                          ctypes.c_void_p(stream_ptr or None)))


def gb_submit(lo: int, hi: int) -> int:
    t = U64(0)
    _check("gb_submit", load().gb_submit(lo, hi, ctypes.byref(t)))
    return t.value


def gb_poll(ticket: int, timeout_ms: int = -1, check: bool = True):
    """Returns (status, result dict or None while pending); check=False also
    returns (status, result) for an error status instead of raising."""
    r = GbResult()
    rc = load().gb_poll(ticket, ctypes.byref(r), timeout_ms)
    if rc == GB_PENDING:
        return rc, None
    if check:
        _check("gb_poll", rc, ok=(GB_OK, GB_COUNTEREXAMPLE))
    return rc, r.as_dict()


def gb_progress() -> dict:
    """Progress of the running or last verification call: tiles_done,
    tiles_total, n_done, n_total, elapsed_s, n_per_s, eta_s."""
    p = GbProgress()
    _check("gb_progress", load().gb_progress(ctypes.byref(p)))
    return p.as_dict()


def gb_stats() -> dict:
    s = GbStats()
    _check("gb_stats", load().gb_stats(ctypes.byref(s)))
    return s.as_dict()


def gb_measure_peaks() -> dict:
    """Measured lane operations/s of INT32 logic, integer mad, popc and
    conflict-free shared atomicAnd on the current GPU."""
    p = GbPeaks()
    _check("gb_measure_peaks", load().gb_measure_peaks(ctypes.byref(p)))
    return p.as_dict()


def result_from_bytes(raw: bytes) -> dict:
    """Decode a gb_result read back from device memory."""
    return GbResult.from_buffer_copy(raw).as_dict()


RESULT_BYTES = ctypes.sizeof(GbResult)
