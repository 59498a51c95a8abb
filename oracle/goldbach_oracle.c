/*
 * goldbach_oracle.c -- plain, slow, single-threaded CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes (paper, Sec. 1 and Sec. 3.3): for every even n with
 * max(lo, 4) <= n < hi, the smallest prime p such that n - p is also prime,
 *
 *     p_min(n) = min { p prime : n - p prime },
 *
 * written out directly: a textbook odd-only byte sieve of Eratosthenes for
 * the primes q near n, a second byte sieve for the small candidates p, and
 * an ascending walk over the candidates p.  Candidates beyond the small
 * table (never needed in practice) fall back to trial division, on purpose
 * not Miller-Rabin, so that the oracle stays independent of the GPU slow
 * path.  The walk stops at p > n/2; reaching that bound without a hit means
 * n is a counterexample to the binary conjecture (paper, Fig. 2 abort path).
 *
 * The values are folded into per-segment records (one per 2^seg_bits even
 * n, counted from n0 = the first even n >= max(lo, 4)):
 *   n_count, max p_min, the smallest n attaining it, hist[floor(log2 p_min)],
 *   sum of p_min mod 2^64, wsum = sum of p_min * (k + 1) mod 2^64 with k the
 *   index of n inside its record, n_slow = #n with p_min > p_max.
 *
 * Sieve arithmetic follows the paper's overflow guards (Sec. 3.4): a prime p
 * sieves only while p <= q_hi / p, and the first multiple inside a window is
 * found by division, never by forming p * p unguarded or stepping past
 * 2^64 - 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    uint64_t n_first;
    uint64_t n_count;
    uint64_t max_pmin;
    uint64_t argmax_n;
    uint64_t sum_pmin;
    uint64_t wsum_pmin;
    uint64_t hist[64];
    uint64_t n_slow;
    uint64_t counterexample_n;
} oracle_record;

enum { ORACLE_OK = 0, ORACLE_COUNTEREXAMPLE = 2, ORACLE_EINVAL = -1, ORACLE_ENOMEM = -2 };

/* ------------------------------------------------------------------ */
/* integer helpers                                                     */
/* ------------------------------------------------------------------ */

/* floor(sqrt(x)) for any 64-bit x, corrected with division so that no
 * product can overflow. */
uint64_t oracle_isqrt(uint64_t x)
{
    uint64_t r = (uint64_t)sqrt((double)x);
    if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
    while (r > 0 && r > x / r) r--;
    while (r + 1 <= 0xFFFFFFFFull && (r + 1) <= x / (r + 1)) r++;
    return r;
}

/* Primality by trial division with every odd d <= sqrt(x). */
int oracle_is_prime_td(uint64_t x)
{
    if (x < 2) return 0;
    if (x < 4) return 1;
    if ((x & 1) == 0) return 0;
    for (uint64_t d = 3; d <= x / d; d += 2)
        if (x % d == 0) return 0;
    return 1;
}

/* Odd-only byte sieve of [0, limit]: entry i stands for 2i+1, 1 = prime.
 * Caller frees.  Textbook Eratosthenes: every odd p with p*p <= limit clears
 * p*p, p*p + 2p, ... */
static uint8_t *odd_sieve_upto(uint64_t limit, uint64_t *n_entries)
{
    uint64_t n = limit / 2 + 1;           /* odd numbers 1, 3, ..., <= limit (+1 slack) */
    uint8_t *s = (uint8_t *)malloc(n ? n : 1);
    if (!s) return NULL;
    memset(s, 1, n);
    s[0] = 0;                              /* 1 is not prime */
    for (uint64_t p = 3; p <= limit / p; p += 2) {
        if (!s[p / 2]) continue;
        for (uint64_t m = p * p; m <= limit; m += 2 * p) {
            s[m / 2] = 0;
            if (m > limit - 2 * p) break;  /* no wrap past 2^64 - 1 */
        }
    }
    *n_entries = n;
    return s;
}

/* pi(x): number of primes <= x. */
uint64_t oracle_pi(uint64_t x)
{
    if (x < 2) return 0;
    uint64_t n = 0;
    uint8_t *s = odd_sieve_upto(x, &n);
    if (!s) return 0;
    uint64_t c = 1;                        /* the prime 2 */
    for (uint64_t i = 1; i < n; i++)
        if (s[i] && 2 * i + 1 <= x) c++;
    free(s);
    return c;
}

/* All primes <= limit (2 included), ascending, in a malloc'd array. */
static uint32_t *primes_array(uint64_t limit, uint64_t *count)
{
    *count = 0;
    if (limit > 0xFFFFFFFFull) return NULL;
    uint64_t n = 0;
    uint8_t *s = odd_sieve_upto(limit < 2 ? 2 : limit, &n);
    if (!s) return NULL;
    uint64_t c = limit >= 2 ? 1 : 0;
    for (uint64_t i = 1; i < n; i++)
        if (s[i] && 2 * i + 1 <= limit) c++;
    uint32_t *out = (uint32_t *)malloc((size_t)(c ? c : 1) * sizeof(uint32_t));
    if (!out) { free(s); return NULL; }
    uint64_t k = 0;
    if (limit >= 2) out[k++] = 2;
    for (uint64_t i = 1; i < n; i++)
        if (s[i] && 2 * i + 1 <= limit) out[k++] = (uint32_t)(2 * i + 1);
    free(s);
    *count = c;
    return out;
}

/* All primes <= limit (2 included), ascending.  Returns the count, writes at
 * most cap of them.  Returns -1 on allocation failure or limit >= 2^32. */
int64_t oracle_primes_upto(uint64_t limit, uint32_t *out, uint64_t cap)
{
    if (limit < 2) return 0;
    uint64_t c = 0;
    uint32_t *a = primes_array(limit, &c);
    if (!a) return -1;
    if (out) memcpy(out, a, (size_t)(c < cap ? c : cap) * sizeof(uint32_t));
    free(a);
    return (int64_t)c;
}

/* ------------------------------------------------------------------ */
/* p_min over a range                                                  */
/* ------------------------------------------------------------------ */

static unsigned floor_log2_u64(uint64_t v)
{
    unsigned b = 0;
    while (v > 1) { v >>= 1; b++; }
    return b;
}

/* Odd-only byte sieve of the window [qlo, qhi] (qlo, qhi odd, qlo >= 3):
 * entry j stands for qlo + 2j.  base[] holds every odd prime <= sqrt(qhi). */
static void sieve_window(uint64_t qlo, uint64_t qhi, const uint32_t *base, uint64_t nbase,
                         uint8_t *win)
{
    uint64_t len = (qhi - qlo) / 2 + 1;
    memset(win, 1, len);
    for (uint64_t b = 0; b < nbase; b++) {
        uint64_t p = base[b];
        if (p == 2) continue;
        if (p > qhi / p) break;            /* guard: p*p > qhi, nothing left to clear */
        uint64_t pp = p * p;               /* < 2^64 because p <= qhi / p */
        uint64_t d;                        /* first odd multiple of p >= max(p*p, qlo) is qlo + d */
        if (pp >= qlo) {
            d = pp - qlo;
        } else {
            /* distance from qlo to the next multiple of p, by division; it is
             * kept as a distance so that nothing is formed above qhi */
            uint64_t rem = qlo % p;
            d = rem ? p - rem : 0;
            if (d & 1) d += p;             /* qlo is odd: qlo + d odd <=> d even */
        }
        if (d > qhi - qlo) continue;
        for (uint64_t j = d / 2; j < len; j += p) win[j] = 0;
    }
}

static void fold(oracle_record *r, uint64_t n, uint64_t p, uint32_t p_max)
{
    uint64_t k = (n - r->n_first) / 2;
    r->n_count++;
    r->sum_pmin += p;
    r->wsum_pmin += p * (k + 1);
    if (p > r->max_pmin) { r->max_pmin = p; r->argmax_n = n; }
    r->hist[floor_log2_u64(p)]++;
    if (p > p_max) r->n_slow++;
}

/*
 * Compute p_min(n) for every even n, max(lo,4) <= n < hi, and fold into
 * records of 2^seg_bits even n each.
 *
 *   p_max     : only used for the n_slow count (p_min > p_max).
 *   seg_bits  : record granularity (log2 of even n per record), 0..40.
 *   x_ext     : the small-candidate bound X: candidates p <= X are tested with
 *               a byte sieve, larger ones by trial division (and the q-window
 *               is extended X below each chunk).  Must be >= 3.
 *   recs      : caller array of cap records (zeroed here).  *n_rec receives
 *               the number of records the range needs; records past cap are
 *               computed but dropped.
 *   pmin_out  : optional; receives p_min for the first pmin_cap even n, in
 *               order from n0 (0 for a counterexample).
 *
 * Returns ORACLE_OK, ORACLE_COUNTEREXAMPLE (the first counterexample goes to
 * *counterexample), ORACLE_EINVAL or ORACLE_ENOMEM.
 *
 * base_in / base_limit: optional.  When base_in is given it must hold every
 * prime <= base_limit in ascending order, with base_limit >= sqrt(hi); it is
 * then used instead of sieving the base primes again (many sub-windows far
 * from the origin can share one table).
 */
int oracle_pmin_range_base(uint64_t lo, uint64_t hi, uint32_t p_max, uint32_t seg_bits,
                           uint32_t x_ext, oracle_record *recs, uint64_t cap, uint64_t *n_rec,
                           uint32_t *pmin_out, uint64_t pmin_cap, uint64_t *counterexample,
                           const uint32_t *base_in, uint64_t nbase_in, uint64_t base_limit)
{
    if (seg_bits > 40 || x_ext < 3 || !n_rec) return ORACLE_EINVAL;
    if (counterexample) *counterexample = 0;
    *n_rec = 0;
    uint64_t n0 = lo < 4 ? 4 : lo;
    if (n0 & 1) {
        if (n0 == UINT64_MAX) return ORACLE_OK;
        n0++;
    }
    if (n0 >= hi) return ORACLE_OK;
    uint64_t n_last = ((hi - 1) & ~1ull);  /* largest even n < hi */
    if (n_last < n0) return ORACLE_OK;
    uint64_t total = (n_last - n0) / 2 + 1;
    uint64_t per_rec = 1ull << seg_bits;
    uint64_t nrec = (total + per_rec - 1) / per_rec;
    *n_rec = nrec;
    for (uint64_t r = 0; r < nrec && r < cap; r++) {
        memset(&recs[r], 0, sizeof(oracle_record));
        recs[r].n_first = n0 + 2 * per_rec * r;
    }

    /* small candidates: odd-only byte sieve up to X */
    uint64_t nsmall = 0;
    uint8_t *small = odd_sieve_upto(x_ext, &nsmall);
    if (!small) return ORACLE_ENOMEM;

    /* base primes up to sqrt(largest q) = sqrt(n_last - 3) */
    uint64_t qmax = n_last >= 7 ? n_last - 3 : 3;
    uint64_t root = oracle_isqrt(qmax);
    uint64_t nb = 0;
    uint32_t *owned = NULL;
    const uint32_t *base;
    if (base_in) {
        if (base_limit < root) { free(small); return ORACLE_EINVAL; }
        base = base_in;
        nb = nbase_in;
    } else {
        owned = primes_array(root < 2 ? 2 : root, &nb);
        if (!owned) { free(small); return ORACLE_ENOMEM; }
        base = owned;
    }

    const uint64_t CHUNK = 1ull << 22;      /* even n per chunk */
    uint64_t win_cap = CHUNK + x_ext + 4;
    uint8_t *win = (uint8_t *)malloc(win_cap);
    if (!win) { free(small); free(owned); return ORACLE_ENOMEM; }

    int status = ORACLE_OK;
    for (uint64_t c0 = 0; c0 < total; c0 += CHUNK) {
        uint64_t cn = total - c0 < CHUNK ? total - c0 : CHUNK;
        uint64_t a = n0 + 2 * c0;           /* first n of the chunk */
        uint64_t b = a + 2 * (cn - 1);      /* last n of the chunk (no wrap: <= n_last) */
        /* q window: odd q with max(3, a - X) <= q <= b - 3 */
        uint64_t qlo = (a > x_ext + 3) ? a - x_ext : 3;
        if ((qlo & 1) == 0) qlo--;
        if (qlo < 3) qlo = 3;
        uint64_t qhi = b >= 6 ? b - 3 : 3;
        if (qhi < qlo) qhi = qlo;
        sieve_window(qlo, qhi, base, nb, win);

        for (uint64_t t = 0; t < cn; t++) {
            uint64_t n = a + 2 * t;
            uint64_t idx = c0 + t;
            uint64_t r = idx >> seg_bits;
            uint64_t found = 0;
            if (n == 4) {
                found = 2;
            } else {
                /* ascending odd candidates p <= X from the small table */
                for (uint64_t p = 3; p <= x_ext && p <= n / 2; p += 2) {
                    if (!small[p / 2]) continue;
                    uint64_t q = n - p;   /* >= n/2 >= 3 and >= a - X >= qlo */
                    if (win[(q - qlo) / 2]) { found = p; break; }
                }
                if (!found) {
                    /* trial-division fallback beyond X */
                    uint64_t p = (x_ext + 1) | 1;
                    for (; p <= n / 2; p += 2) {
                        if (oracle_is_prime_td(p) && oracle_is_prime_td(n - p)) { found = p; break; }
                    }
                }
            }
            if (!found) {
                status = ORACLE_COUNTEREXAMPLE;
                if (counterexample && *counterexample == 0) *counterexample = n;
                if (r < cap && recs[r].counterexample_n == 0) recs[r].counterexample_n = n;
                if (r < cap) recs[r].n_count++;
            } else if (r < cap) {
                fold(&recs[r], n, found, p_max);
            }
            if (pmin_out && idx < pmin_cap) pmin_out[idx] = (uint32_t)found;
        }
    }
    free(win);
    free(owned);
    free(small);
    return status;
}

int oracle_pmin_range(uint64_t lo, uint64_t hi, uint32_t p_max, uint32_t seg_bits,
                      uint32_t x_ext, oracle_record *recs, uint64_t cap, uint64_t *n_rec,
                      uint32_t *pmin_out, uint64_t pmin_cap, uint64_t *counterexample)
{
    return oracle_pmin_range_base(lo, hi, p_max, seg_bits, x_ext, recs, cap, n_rec,
                                  pmin_out, pmin_cap, counterexample, NULL, 0, 0);
}

/* p_min of a single even n >= 4 (0 for a counterexample), same method. */
uint64_t oracle_pmin_single(uint64_t n, uint32_t x_ext)
{
    oracle_record r;
    uint64_t nrec = 0, ce = 0;
    uint32_t p = 0;
    if (n < 4 || (n & 1)) return 0;
    uint64_t hi = n + 1;                   /* n <= 2^64 - 2 so no wrap */
    oracle_pmin_range(n, hi, 0xFFFFFFFFu, 0, x_ext, &r, 1, &nrec, &p, 1, &ce);
    return p;
}

uint64_t oracle_record_size(void) { return sizeof(oracle_record); }
