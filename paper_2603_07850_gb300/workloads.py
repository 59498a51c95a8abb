"""Seeded synthetic workloads: ranges, sampled segments and request streams.

This module holds only the input recipes (which ranges of even n are
verified, which segments are sampled, which requests arrive when).  It holds
none of the method's arithmetic, so both the CUDA path's tests and the CPU
oracle can draw from it.

All randomness comes from splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

MASK64 = (1 << 64) - 1
U64_MAX = MASK64


class SplitMix64:
    """splitmix64 as published: a Weyl sequence with a 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) by a 64x64 -> high-64 multiply (m < 2^64)."""
        return (self.next() * m) >> 64

    def uniform(self) -> float:
        """Uniform float in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


@dataclass(frozen=True)
class RangeConfig:
    """One verification workload: every even n with max(lo, 4) <= n < hi."""
    name: str
    lo: int
    hi: int
    p_max: int
    seg_bits: int          # report granularity: 2^seg_bits even n per record
    base_limit: int        # base primes resident on the device go up to here
    description: str


# The five workloads (plain 10^8; batched 10^10; 10^12; two high-offset
# windows).  Ranges are half-open; "[4, N]" inclusive maps to hi = N + 1.
C0 = RangeConfig("C0_plain_1e8", 4, 10**8 + 1, 1 << 16, 18, 10**4,
                 "every even n in [4, 1e8], segments of 2^18, P_max = 2^16")
C0_PMAX64 = RangeConfig("C0_plain_1e8_pmax64", 4, 10**8 + 1, 64, 18, 10**4,
                        "as C0 with P_max = 64: exercises the GPU over-bound path")
C1 = RangeConfig("C1_batched_1e10", 4, 10**10 + 1, 1 << 16, 15, 10**5,
                 "every even n in [4, 1e10], persistent kernel, records of 2^15")
C2 = RangeConfig("C2_full_1e12", 4, 10**12 + 1, 1 << 16, 20, 10**6,
                 "every even n in [4, 1e12], base primes <= 1e6, records of 2^20")
C3A = RangeConfig("C3a_1e18", 10**18, 10**18 + 10**10, 1 << 16, 20, (1 << 32) - 1,
                  "[1e18, 1e18 + 1e10), base primes <= 2^32")
C3B = RangeConfig("C3b_2p64", (1 << 64) - (1 << 33), (1 << 64) - 2, 1 << 16, 20,
                  (1 << 32) - 1, "[2^64 - 2^33, 2^64 - 2), base primes <= 2^32")
C3_EDGE = RangeConfig("C3_edge", (1 << 64) - (1 << 21), U64_MAX, 1 << 16, 20,
                      (1 << 32) - 1, "[2^64 - 2^21, 2^64 - 1): includes n = 2^64 - 2")

SEED_C2 = 0xC2
SEED_C3A = 0xC3A
SEED_C3B = 0xC3B
SEED_C4 = 0xC4


def first_even(lo: int) -> int:
    n0 = max(lo, 4)
    return n0 + (n0 & 1)


def num_even(lo: int, hi: int) -> int:
    n0 = first_even(lo)
    if n0 >= hi:
        return 0
    return (((hi - 1) & ~1) - n0) // 2 + 1


def num_records(lo: int, hi: int, seg_bits: int) -> int:
    t = num_even(lo, hi)
    return (t + (1 << seg_bits) - 1) >> seg_bits


def record_bounds(lo: int, hi: int, seg_bits: int, r: int) -> tuple[int, int]:
    """Half-open n-range [a, b) of record r of the range [lo, hi)."""
    n0 = first_even(lo)
    a = n0 + (r << (seg_bits + 1))
    b = min(a + (1 << (seg_bits + 1)), hi)
    return a, b


def sample_records(cfg: RangeConfig, count: int, seed: int) -> list[int]:
    """`count` distinct record indices drawn uniformly over the range's grid."""
    nrec = num_records(cfg.lo, cfg.hi, cfg.seg_bits)
    rng = SplitMix64(seed)
    out: list[int] = []
    seen = set()
    while len(out) < min(count, nrec):
        r = rng.below(nrec)
        if r not in seen:
            seen.add(r)
            out.append(r)
    return out


def sample_subwindows(cfg: RangeConfig, count: int, seed: int, width_bits: int = 20):
    """`count` seeded sub-windows [a, b) of 2^width_bits even n inside cfg's range,
    aligned to the 2^width_bits grid that starts at the range's first even n."""
    idx = sample_records(RangeConfig(cfg.name, cfg.lo, cfg.hi, cfg.p_max, width_bits,
                                     cfg.base_limit, ""), count, seed)
    return [record_bounds(cfg.lo, cfg.hi, width_bits, r) for r in idx]


@dataclass(frozen=True)
class Request:
    rid: int
    lo: int
    hi: int
    arrival_s: float


def serving_stream(count: int = 10_000, rate_per_s: float = 100.0, seed: int = SEED_C4,
                   lo_max: int = 10**15, w_lo_exp: float = 4.0, w_hi_exp: float = 10.0):
    """Request mix: lo an even integer uniform in [4, lo_max), width w log-uniform
    in [10^w_lo_exp, 10^w_hi_exp], Poisson arrivals at `rate_per_s`."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        lo = 2 * rng.below((lo_max - 4) // 2) + 4
        w = int(10 ** (w_lo_exp + (w_hi_exp - w_lo_exp) * rng.uniform()))
        u = rng.uniform()
        t += -math.log(1.0 - u) / rate_per_s
        out.append(Request(i, lo, min(lo + w, U64_MAX), t))
    return out
