"""Pins for the CPU oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself:
published prime counts, brute-force trial division written independently
here, a record fold written from the record definition, the sympy primality
routine, or the paper's stated bounds.  A dropped term, an off-by-one in a
sieve bound, a wrong histogram bin or a wrong argmax tie rule fails at least
one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_07850_gb300 import workloads as W

MASK64 = (1 << 64) - 1


# --------------------------------------------------------------------------
# independent helpers (plain trial division, written for these pins only)
# --------------------------------------------------------------------------

def td_is_prime(x: int) -> bool:
    if x < 2:
        return False
    if x % 2 == 0:
        return x == 2
    d = 3
    while d * d <= x:
        if x % d == 0:
            return False
        d += 2
    return True


def brute_pmin_table(limit: int) -> dict[int, int]:
    """p_min(n) for every even 4 <= n < limit by trial-division primality."""
    isp = [td_is_prime(i) for i in range(limit)]
    out = {}
    for n in range(4, limit, 2):
        for p in range(2, n // 2 + 1):
            if isp[p] and isp[n - p]:
                out[n] = p
                break
    return out


def python_fold(pmins: dict[int, int], lo: int, hi: int, seg_bits: int, p_max: int):
    """Records straight from their definition: one per 2^seg_bits even n from
    n0 = first even >= max(lo, 4); argmax is the smallest n with the max."""
    n0 = max(lo, 4)
    n0 += n0 & 1
    recs = []
    n = n0
    while n < hi:
        a = n
        b = min(a + (2 << seg_bits), hi)
        ns = list(range(a, b, 2))
        ps = [pmins[m] for m in ns]
        mx = max(ps)
        rec = {
            "n_first": a,
            "n_count": len(ns),
            "max_pmin": mx,
            "argmax_n": min(m for m, p in zip(ns, ps) if p == mx),
            "sum_pmin": sum(ps) & MASK64,
            "wsum_pmin": sum(p * (k + 1) for k, p in enumerate(ps)) & MASK64,
            "hist": [0] * 64,
            "n_slow": sum(1 for p in ps if p > p_max),
            "counterexample_n": 0,
        }
        for p in ps:
            rec["hist"][p.bit_length() - 1] += 1
        recs.append(rec)
        n = b if b % 2 == 0 else b + 1
    return recs


@pytest.fixture(scope="module")
def brute_1e5():
    return brute_pmin_table(10**5)


# --------------------------------------------------------------------------
# prime counts
# --------------------------------------------------------------------------

def test_prime_counts_small():
    # pi(10^6) = 78,498 is the candidate-prime count the paper states for
    # P_SMALL = 10^6 (Sec. 3.1, Sec. 4); the others are the standard values.
    assert oracle.pi(10**6) == 78498
    assert len(oracle.primes_upto(10**6)) == 78498
    assert oracle.pi(10**4) == 1229
    assert oracle.pi(10**5) == 9592
    assert oracle.pi(10**8) == 5761455
    # boundary behaviour of the odd-only sieve
    assert [oracle.pi(x) for x in range(0, 12)] == [0, 0, 1, 2, 2, 3, 3, 4, 4, 4, 4, 5]
    assert list(oracle.primes_upto(30)) == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]


def test_prime_count_1e9():
    assert oracle.pi(10**9) == 50847534


@pytest.fixture(scope="module")
def base32():
    return oracle.primes_upto((1 << 32) - 1)


def test_prime_count_2p32(base32):
    # pi(2^32) = 203,280,221: the size of the base-prime table near 2^64.
    assert len(base32) == 203280221
    assert int(base32[-1]) == 4294967291          # largest prime below 2^32
    assert int(base32[0]) == 2


def test_isqrt_edges():
    for x in [0, 1, 2, 3, 4, 15, 16, 17, 10**12, (1 << 64) - 1, (1 << 62), 2**63 + 12345]:
        assert oracle.isqrt(x) == math.isqrt(x)


def test_trial_division_prime():
    for x in range(0, 2000):
        assert oracle.is_prime_td(x) == td_is_prime(x)
    assert oracle.is_prime_td(4294967291)
    assert not oracle.is_prime_td(4294967297)      # 641 * 6700417


# --------------------------------------------------------------------------
# p_min against brute force
# --------------------------------------------------------------------------

def test_pmin_matches_brute_force_below_1e5(brute_1e5):
    st, recs, pm, ce = oracle.pmin_range(4, 10**5, seg_bits=10, want_pmin=True)
    assert st == 0 and ce == 0
    ns = range(4, 10**5, 2)
    assert len(pm) == len(ns)
    expect = np.array([brute_1e5[n] for n in ns], dtype=np.uint32)
    assert np.array_equal(pm, expect)


@pytest.mark.parametrize("x_ext", [3, 5, 11, 64])
def test_pmin_trial_division_fallback(brute_1e5, x_ext):
    # A tiny small-candidate table forces the oracle's trial-division branch.
    st, recs, pm, ce = oracle.pmin_range(4, 30001, seg_bits=8, x_ext=x_ext, want_pmin=True)
    assert st == 0
    expect = np.array([brute_1e5[n] for n in range(4, 30001, 2)], dtype=np.uint32)
    assert np.array_equal(pm, expect)


def test_pmin_first_values():
    # p_min(4..20) by hand: 4=2+2, 6=3+3, 8=3+5, 10=3+7, 12=5+7, 14=3+11,
    # 16=3+13, 18=5+13, 20=3+17.
    st, recs, pm, ce = oracle.pmin_range(4, 21, seg_bits=4, want_pmin=True)
    assert list(pm) == [2, 3, 3, 3, 5, 3, 3, 5, 3]


# --------------------------------------------------------------------------
# records against a fold written from the definition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lo,hi,seg_bits,p_max", [
    (4, 10**5, 10, 1 << 16),
    (0, 77777, 7, 64),
    (1001, 77778, 5, 32),
    (5, 6, 3, 64),
    (4, 5, 0, 64),
    (98, 99999, 12, 8),
])
def test_records_match_definition(brute_1e5, lo, hi, seg_bits, p_max):
    st, recs, _, _ = oracle.pmin_range(lo, hi, p_max=p_max, seg_bits=seg_bits)
    expect = python_fold(brute_1e5, lo, hi, seg_bits, p_max)
    assert [r.as_dict() for r in recs] == expect


def test_empty_ranges():
    for lo, hi in [(0, 4), (4, 4), (5, 6), (10, 3), (7, 8)]:
        st, recs, _, _ = oracle.pmin_range(lo, hi, seg_bits=4)
        assert st == 0 and recs == []


def test_single_n4_record():
    st, recs, _, _ = oracle.pmin_range(0, 5, seg_bits=0)
    r = recs[0]
    assert (r.n_first, r.n_count, r.max_pmin, r.argmax_n, r.sum_pmin, r.wsum_pmin) == \
        (4, 1, 2, 4, 2, 2)
    assert r.hist[1] == 1 and sum(r.hist) == 1


def test_argmax_tie_takes_smallest_n(brute_1e5):
    # In [4, 40) the max p_min is 7 (n = 30); below it the value 5 recurs, so a
    # record that stops before 30 must report the first n with p_min = 5.
    st, recs, _, _ = oracle.pmin_range(4, 30, seg_bits=6)
    ties = [n for n in range(4, 30, 2) if brute_1e5[n] == recs[0].max_pmin]
    assert len(ties) > 1
    assert recs[0].argmax_n == min(ties)


# --------------------------------------------------------------------------
# invariants far from the origin, checked with sympy's primality routine
# --------------------------------------------------------------------------

def _check_invariants(n: int, p: int):
    sympy = pytest.importorskip("sympy")
    assert p >= 2 and sympy.isprime(p) and sympy.isprime(n - p), (n, p)
    for c in range(3, p, 2):
        assert not (sympy.isprime(c) and sympy.isprime(n - c)), (n, p, c)


@pytest.mark.parametrize("center", [10**12, 10**15])
def test_invariants_sampled(center):
    rng = W.SplitMix64(0x0A11 ^ center)
    lo = center - 2 * 2000
    st, recs, pm, _ = oracle.pmin_range(lo, center + 2 * 2000, seg_bits=12, want_pmin=True)
    n0 = W.first_even(lo)
    for _ in range(40):
        k = rng.below(len(pm))
        _check_invariants(n0 + 2 * k, int(pm[k]))


def test_invariants_1e18():
    base = oracle.primes_upto(10**9 + 1000)
    lo = 10**18
    st, recs, pm, _ = oracle.pmin_range(lo, lo + 2 * 4096, seg_bits=12, want_pmin=True,
                                        base=(base, 10**9 + 1000))
    rng = W.SplitMix64(0x1E18)
    for _ in range(30):
        k = rng.below(len(pm))
        _check_invariants(lo + 2 * k, int(pm[k]))
    assert recs[0].max_pmin == max(pm)


# The largest minimal Goldbach partition found below 4 x 10^18 (Oliveira e
# Silva, Herzog and Pardi, Math. Comp. 83 (2014), the verification the paper
# builds on): n = 3,325,581,707,333,960,528 needs p = 9,781, and no smaller
# even n needs as much.
RECORD_N, RECORD_P = 3325581707333960528, 9781


def test_published_pmin_record(base32):
    # the window sieve and candidate walk reach the record's p, and in a
    # window around it that p is the max with the record n as smallest argmax
    lo, hi = RECORD_N - 2 * 2048, RECORD_N + 2 * 2048
    st, recs, pm, _ = oracle.pmin_range(lo, hi, seg_bits=12, want_pmin=True,
                                        base=(base32, (1 << 32) - 1))
    assert st == 0 and len(recs) == 1
    assert int(pm[2048]) == RECORD_P
    assert recs[0].max_pmin == RECORD_P and recs[0].argmax_n == RECORD_N
    assert all(int(x) < RECORD_P for x in pm[:2048])
    _check_invariants(RECORD_N, RECORD_P)


def test_top_of_u64_range(base32):
    # The last even n below 2^64 is 2^64 - 2; hi = 2^64 - 1 must include it
    # without any wrap.
    lo, hi = (1 << 64) - 2 * 512, (1 << 64) - 1
    st, recs, pm, _ = oracle.pmin_range(lo, hi, seg_bits=9, want_pmin=True,
                                        base=(base32, (1 << 32) - 1))
    assert st == 0 and len(recs) == 1 and recs[0].n_count == 512 == len(pm)
    assert recs[0].n_first == lo
    rng = W.SplitMix64(0x2064)
    for k in [511, 510, 0] + [rng.below(512) for _ in range(20)]:
        _check_invariants(lo + 2 * k, int(pm[k]))
    # hi = 2^64 - 2 (exclusive) stops one n earlier
    st, recs2, pm2, _ = oracle.pmin_range(lo, (1 << 64) - 2, seg_bits=9, want_pmin=True,
                                          base=(base32, (1 << 32) - 1))
    assert recs2[0].n_count == 511 and np.array_equal(pm2, pm[:511])


# --------------------------------------------------------------------------
# the paper's own bounds
# --------------------------------------------------------------------------

def test_paper_bounds_to_1e8():
    # Sec. 4: no n in the tested ranges needed a candidate beyond the small
    # bound, and the comet envelope H(10^13) is about 4,305; so with
    # P_max = 2^16 no n <= 10^8 is over-bound and max p_min stays far below.
    st, recs, _, ce = oracle.pmin_range(4, 10**8 + 1, p_max=1 << 16, seg_bits=18)
    assert st == 0 and ce == 0
    assert sum(r.n_slow for r in recs) == 0
    assert max(r.max_pmin for r in recs) <= 4305
    assert sum(r.n_count for r in recs) == 49999999
    assert sum(sum(r.hist) for r in recs) == 49999999
