"""The algorithmic-work model behind bench.py's roofline figures.

The model counts crossing-off marks exactly: every odd multiple m of every
prime 13 < p <= sqrt(q_max) with max(p^2, q_lo) <= m <= q_max.  Here that
count is pinned to a brute-force enumeration on small ranges.  The other
terms are pinned to their definitions: one fill word per 32 odd q, the 53 odd
primes below 256 as bit-parallel candidates, and the tail as the n with
p_min above 251 from the histogram.
"""
import pytest

import bench


def brute_marks(q_lo, q_hi):
    root = int(q_hi ** 0.5)
    primes = [p for p in range(17, root + 1, 2) if all(p % d for d in range(3, int(p ** 0.5) + 1, 2))]
    marks = 0
    for p in primes:
        if p * p > q_hi:
            continue
        m0 = max(p * p, -(-q_lo // p) * p)            # first multiple >= max(p^2, q_lo)
        if m0 % 2 == 0:
            m0 += p                                    # odd multiples only
        for m in range(m0, q_hi + 1, 2 * p):
            marks += 1
    return marks


@pytest.mark.parametrize("n0,n_total,k_words", [
    (4, 50_000, 4), (1_000_000, 20_000, 32), (123_456_788, 30_000, 2), (10_000_000_000, 5_000, 64)])
def test_marks_match_brute_force(n0, n_total, k_words):
    hist = [0] * 64
    got = bench.algorithmic_instructions(n0, n_total, k_words, hist)
    K = 32 * k_words
    q_lo = max(n0 + 1 - 2 * K, 1)
    q_hi = n0 + 2 * (n_total - 1) - 1
    assert round(got["marks_per_n"] * n_total) == brute_marks(q_lo, q_hi)


def test_fill_search_and_tail_terms():
    n0, n_total, k_words = 1_000_000, 64_000, 32
    hist = [0] * 64
    hist[3], hist[7], hist[8], hist[9] = 1000, 50, 7, 2        # bins 8 and 9: p_min >= 256
    a = bench.algorithmic_instructions(n0, n_total, k_words, hist)
    base = bench.algorithmic_instructions(n0, n_total, k_words, [0] * 64)
    M = bench.MODEL
    assert a["tail_fraction"] == 9 / n_total
    assert a["instr"] - base["instr"] == pytest.approx(9 * (M["tail"] + 1.5 * M["tail_chunk"]))
    cands = [p for p in range(3, 256, 2) if all(p % d for d in range(3, int(p ** 0.5) + 1, 2))]
    assert len(cands) == 53
    words = n_total / 32
    step = sum(M["step"] + bin(p).count("1") for p in cands)
    K = 32 * k_words
    q_lo, q_hi = n0 + 1 - 2 * K, n0 + 2 * (n_total - 1) - 1
    fill = (q_hi - q_lo) / 64 + 1
    marks = base["marks_per_n"] * n_total
    expect = marks * M["mark"] + fill * M["fill"] + words * (step + M["word_stats"])
    assert base["instr"] == pytest.approx(expect)
