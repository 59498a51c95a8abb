"""ctypes wrapper around the plain-C oracle (``goldbach_oracle.c``).

Test infrastructure only: the product path never imports this module.
The shared object is compiled with gcc into ``oracle/_build/`` on first use
(or by ``build()``), on whatever host runs the tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "goldbach_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _CRecord(ctypes.Structure):
    _fields_ = [
        ("n_first", ctypes.c_uint64),
        ("n_count", ctypes.c_uint64),
        ("max_pmin", ctypes.c_uint64),
        ("argmax_n", ctypes.c_uint64),
        ("sum_pmin", ctypes.c_uint64),
        ("wsum_pmin", ctypes.c_uint64),
        ("hist", ctypes.c_uint64 * 64),
        ("n_slow", ctypes.c_uint64),
        ("counterexample_n", ctypes.c_uint64),
    ]


@dataclass
class OracleRecord:
    n_first: int
    n_count: int
    max_pmin: int
    argmax_n: int
    sum_pmin: int
    wsum_pmin: int
    hist: list = field(default_factory=lambda: [0] * 64)
    n_slow: int = 0
    counterexample_n: int = 0

    def as_dict(self) -> dict:
        return {
            "n_first": self.n_first, "n_count": self.n_count, "max_pmin": self.max_pmin,
            "argmax_n": self.argmax_n, "sum_pmin": self.sum_pmin, "wsum_pmin": self.wsum_pmin,
            "hist": list(self.hist), "n_slow": self.n_slow,
            "counterexample_n": self.counterexample_n,
        }


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u64, u32, i64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64
    lib.oracle_isqrt.argtypes = [u64]
    lib.oracle_isqrt.restype = u64
    lib.oracle_is_prime_td.argtypes = [u64]
    lib.oracle_is_prime_td.restype = ctypes.c_int
    lib.oracle_pi.argtypes = [u64]
    lib.oracle_pi.restype = u64
    lib.oracle_primes_upto.argtypes = [u64, ctypes.c_void_p, u64]
    lib.oracle_primes_upto.restype = i64
    lib.oracle_pmin_range.argtypes = [u64, u64, u32, u32, u32, ctypes.c_void_p, u64,
                                      ctypes.POINTER(u64), ctypes.c_void_p, u64,
                                      ctypes.POINTER(u64)]
    lib.oracle_pmin_range.restype = ctypes.c_int
    lib.oracle_pmin_range_base.argtypes = lib.oracle_pmin_range.argtypes + [
        ctypes.c_void_p, u64, u64]
    lib.oracle_pmin_range_base.restype = ctypes.c_int
    lib.oracle_pmin_single.argtypes = [u64, u32]
    lib.oracle_pmin_single.restype = u64
    lib.oracle_record_size.restype = u64
    assert lib.oracle_record_size() == ctypes.sizeof(_CRecord)
    _lib = lib
    return lib


def isqrt(x: int) -> int:
    return int(_load().oracle_isqrt(x))


def is_prime_td(x: int) -> bool:
    return bool(_load().oracle_is_prime_td(x))


def pi(x: int) -> int:
    return int(_load().oracle_pi(x))


def primes_upto(limit: int) -> np.ndarray:
    lib = _load()
    n = lib.oracle_primes_upto(limit, None, 0)
    if n < 0:
        raise MemoryError("oracle_primes_upto")
    out = np.empty(max(n, 1), dtype=np.uint32)
    lib.oracle_primes_upto(limit, out.ctypes.data, n)
    return out[:n]


def _num_records(lo: int, hi: int, seg_bits: int) -> int:
    n0 = max(lo, 4)
    n0 += n0 & 1
    if n0 >= hi:
        return 0
    n_last = (hi - 1) & ~1
    if n_last < n0:
        return 0
    total = (n_last - n0) // 2 + 1
    return (total + (1 << seg_bits) - 1) >> seg_bits


def pmin_range(lo: int, hi: int, p_max: int = 1 << 16, seg_bits: int = 18,
               x_ext: int = 1 << 17, want_pmin: bool = False, base=None):
    """Records (and optionally every p_min) for even n with max(lo,4) <= n < hi.

    ``base`` may be ``(primes_array, limit)`` from ``primes_upto(limit)`` with
    ``limit >= isqrt(hi)``, shared across calls far from the origin.

    Returns ``(status, records, pmin_array_or_None, counterexample_n)``;
    status 0 = ok, 2 = counterexample found.
    """
    lib = _load()
    nrec = _num_records(lo, hi, seg_bits)
    recs = (_CRecord * max(nrec, 1))()
    got = ctypes.c_uint64(0)
    ce = ctypes.c_uint64(0)
    pm = None
    pm_ptr, pm_cap = None, 0
    if want_pmin:
        n0 = max(lo, 4)
        n0 += n0 & 1
        total = 0 if n0 >= hi else max(0, ((hi - 1) & ~1) - n0) // 2 + 1
        pm = np.zeros(max(total, 1), dtype=np.uint32)
        pm_ptr, pm_cap = pm.ctypes.data, total
        pm = pm[:total]
    if base is None:
        st = lib.oracle_pmin_range(lo, hi, p_max, seg_bits, x_ext, ctypes.addressof(recs),
                                   nrec, ctypes.byref(got), pm_ptr, pm_cap, ctypes.byref(ce))
    else:
        arr, limit = base
        arr = np.ascontiguousarray(arr, dtype=np.uint32)
        st = lib.oracle_pmin_range_base(lo, hi, p_max, seg_bits, x_ext, ctypes.addressof(recs),
                                        nrec, ctypes.byref(got), pm_ptr, pm_cap,
                                        ctypes.byref(ce), arr.ctypes.data, len(arr), limit)
    if st < 0:
        raise RuntimeError(f"oracle_pmin_range failed: {st}")
    assert got.value == nrec, (got.value, nrec)
    out = []
    for i in range(nrec):
        r = recs[i]
        out.append(OracleRecord(r.n_first, r.n_count, r.max_pmin, r.argmax_n, r.sum_pmin,
                                r.wsum_pmin, list(r.hist), r.n_slow, r.counterexample_n))
    return st, out, pm, ce.value


def pmin_single(n: int, x_ext: int = 1 << 17) -> int:
    return int(_load().oracle_pmin_single(n, x_ext))
