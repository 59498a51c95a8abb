// gb_device.cuh -- device-side building blocks of the Goldbach range verifier.
//
// Sieve window (paper Sec. 3.1, rebuilt for sm_103a): the odd integers of a
// window are one bit each, bit j <-> q = wbase + 2j, in shared memory.  A
// window is built in three passes:
//   1. fill    : every word is written once as the AND of pre-sieved
//                patterns (3*5*7*11*13, 17*19*23, 29*31; 3*5*7 with wheel 7)
//                and, when configured, in-register masks of primes above 31
//                (no shared-memory read-modify-write at all);
//   2. marking : the remaining base primes p <= sqrt(q_hi) clear their odd
//                multiples from p^2 on with shared-memory atomicAnd, one warp
//                per prime for the dense small primes (tier A, in an order
//                balanced over the warps) and one lane per prime for the
//                sparse large ones (tier B); primes above the bucket bound
//                come from the pre-pass's buckets;
//   3. fix-ups : q <= 1 cleared, the pattern primes themselves set again.
// Overflow guards follow paper Sec. 3.4: a prime sieves only while
// p*p <= q_hi (p < 2^32 so p*p cannot wrap), and the first multiple is found
// from wbase mod p as a distance, never by forming a value above q_hi.
//
// Per-n p_min search (paper Sec. 3.1 phase 1; gb_search.cuh), the
// search_chunks = 0 form and the tail of the bit-parallel one: for one n,
// candidate p = 2i+1 maps to the window bit c - i with c the bit of q = n - 1.
// Chunk t is the 32 window bits [c - 32t - 31, c - 32t], one funnel shift of
// two words, ANDed with the bit-reversed candidate word t; the smallest
// candidate is 32t + clz(mask).
//
// Slow path (paper Sec. 3.3, moved onto the GPU): an n with no candidate
// p <= P_max is finished by its warp, 32 odd candidates p > P_max per step,
// each p and n - p tested by deterministic Miller-Rabin with the first 12
// primes as bases (paper Sec. 3.4), Montgomery multiplication in 64 bits.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "gb_types.h"

namespace gbk {

#define GB_FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// bounds-checked window accesses (GB_DEBUG builds)
// ---------------------------------------------------------------------------
//
// Every read, store and atomic on a sieve window goes through wld / wst /
// wand / wor.  In an ordinary build they are the plain access.  In a build
// with GB_DEBUG an access to shared memory is first checked against the
// CTA's dynamic shared memory (or its first RangeParams::dbg_lim bytes): one
// outside is skipped (a load reads 0), and the first failing site and its
// byte offset are kept in shared memory.  The kernel's epilogue (dbg_end, or
// dbg_report per serving tile) moves them to the control block with
// F_BOUNDS | F_INTERNAL, so the call fails with GB_EINTERNAL instead of the
// access faulting.  dbg_check does the same for a logical index bound.
// Accesses to global memory are not checked.
enum DbgSite : uint32_t {
    DS_FILL = 1, DS_MARK_A = 2, DS_MARK_BIT = 3, DS_FIXUP = 4, DS_BULK = 5, DS_TAIL = 6, DS_PERN = 7,
    DS_STAGE = 8
};

#ifdef GB_DEBUG
extern __shared__ __align__(16) uint32_t gb_dyn_smem[];
static __shared__ uint32_t gb_dbg_site, gb_dbg_off, gb_dbg_lim;

__device__ __forceinline__ void dbg_fail(uint32_t site, uint32_t off)
{
    if (atomicCAS(&gb_dbg_site, 0u, site) == 0u) gb_dbg_off = off;
}

__device__ __forceinline__ bool dbg_ok(const void *p, uint32_t site)
{
    if (!__isShared(p)) return true;
    uint32_t size;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(gb_dyn_smem);
    const uint32_t off = (uint32_t)__cvta_generic_to_shared(p);
    const uint32_t lim = gb_dbg_lim && gb_dbg_lim < size ? gb_dbg_lim : size;
    if (off >= base && off - base + 4u <= lim) return true;
    dbg_fail(site, off - base);
    return false;
}

__device__ __forceinline__ bool dbg_check(bool in, uint32_t site, uint32_t value)
{
    if (!in) dbg_fail(site, value);
    return in;
}

// Before the kernel's first barrier, by every thread (thread 0 writes).
__device__ __forceinline__ void dbg_begin(uint32_t lim)
{
    if (threadIdx.x == 0) {
        gb_dbg_site = 0u;
        gb_dbg_off = 0u;
        gb_dbg_lim = lim;
    }
}

// Thread 0, with every other thread of the CTA past its last window access:
// move a failure into ctrl and clear it.
__device__ __forceinline__ void dbg_report(Ctrl *ctrl)
{
    const uint32_t site = atomicExch(&gb_dbg_site, 0u);
    if (site && ctrl) {
        if (atomicCAS(&ctrl->dbg_site, 0u, site) == 0u) ctrl->dbg_off = gb_dbg_off;
        atomicOr(&ctrl->flags, F_BOUNDS | F_INTERNAL);
    }
}

// At the end of the kernel, by every thread of the CTA.
__device__ __forceinline__ void dbg_end(Ctrl *ctrl)
{
    __syncthreads();
    if (threadIdx.x == 0) dbg_report(ctrl);
}
#else
__device__ __forceinline__ bool dbg_ok(const void *, uint32_t) { return true; }
__device__ __forceinline__ bool dbg_check(bool, uint32_t, uint32_t) { return true; }
__device__ __forceinline__ void dbg_begin(uint32_t) {}
__device__ __forceinline__ void dbg_report(Ctrl *) {}
__device__ __forceinline__ void dbg_end(Ctrl *) {}
#endif

__device__ __forceinline__ uint32_t wld(const uint32_t *p, uint32_t site) { return dbg_ok(p, site) ? *p : 0u; }
__device__ __forceinline__ void wst(uint32_t *p, uint32_t v, uint32_t site)
{
    if (dbg_ok(p, site)) *p = v;
}
__device__ __forceinline__ void wand(uint32_t *p, uint32_t m, uint32_t site)
{
    if (dbg_ok(p, site)) atomicAnd(p, m);
}
__device__ __forceinline__ void wor(uint32_t *p, uint32_t m, uint32_t site)
{
    if (dbg_ok(p, site)) atomicOr(p, m);
}

// Primes cleared by in-register masks during the fill (those above the wheel).
// A constexpr function so that, in unrolled loops, every p is a compile-time
// constant and every "mod p" becomes a multiply-high.
constexpr int NPAT = 14;
__host__ __device__ constexpr uint32_t pat_prime(int i)
{
    return i == 0 ? 11u : i == 1 ? 13u : i == 2 ? 17u : i == 3 ? 19u : i == 4 ? 23u :
           i == 5 ? 29u : i == 6 ? 31u : i == 7 ? 37u : i == 8 ? 41u : i == 9 ? 43u :
           i == 10 ? 47u : i == 11 ? 53u : i == 12 ? 59u : 61u;
}

// ---------------------------------------------------------------------------
// small integer helpers
// ---------------------------------------------------------------------------

// x mod p for 64-bit x and 32-bit p, with m = floor((2^64-1)/p): the quotient
// estimate umulhi(x, m) is at most one below floor(x / p).
__device__ __forceinline__ uint32_t mod_recip(unsigned long long x, uint32_t p,
                                              unsigned long long m)
{
    unsigned long long q = __umul64hi(x, m);
    unsigned long long r = x - q * (unsigned long long)p;
    if (r >= p) r -= p;
    return (uint32_t)r;
}

// floor(sqrt(x)) for any 64-bit x, exact: a double-precision estimate (off by
// at most one) corrected with 64-bit products, never above 2^32 - 1.
__device__ __forceinline__ unsigned long long isqrt_u64(unsigned long long x)
{
    unsigned long long r = (unsigned long long)sqrt((double)x);
    if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
    while (r > 0 && r * r > x) r--;
    while (r < 0xFFFFFFFFull && (r + 1) * (r + 1) <= x) r++;
    return r;
}

// Number of table primes <= v (table is ascending, odd primes from 3).
__device__ __forceinline__ uint32_t count_le(const uint32_t *primes, uint32_t n,
                                             unsigned long long v)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if ((unsigned long long)primes[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The same count by a whole warp (every lane calls it, all get the answer):
// each round the 32 lanes test 32 evenly spaced entries and a ballot narrows
// the range 32-fold, so a 2^20-prime table takes four dependent loads.
__device__ __forceinline__ uint32_t count_le_warp(const uint32_t *primes, uint32_t n, unsigned long long v)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = n;                             // the count lies in [lo, hi]
    while (lo < hi) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + (lane + 1) * step - 1;
        const bool le = idx < hi && (unsigned long long)primes[idx] <= v;
        const uint32_t cnt = __popc(__ballot_sync(GB_FULL_MASK, le));
        const uint32_t nhi = lo + (cnt + 1) * step - 1;
        lo += cnt * step;
        hi = nhi < hi ? nhi : hi;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GB_FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(GB_FULL_MASK, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// ---------------------------------------------------------------------------
// deterministic Miller-Rabin, bases = the first 12 primes (paper Sec. 3.4;
// correct for every x < 2^64 -- Sorenson and Webster 2015 prove the 12-prime
// set for x < 3.18e23).  Montgomery arithmetic modulo odd x (Montgomery 1985).
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long mont_mul(unsigned long long a, unsigned long long b,
                                                       unsigned long long x,
                                                       unsigned long long ninv)
{
    unsigned long long lo = a * b, hi = __umul64hi(a, b);
    unsigned long long m = lo * ninv;                // lo + m*x == 0 mod 2^64
    unsigned long long mxhi = __umul64hi(m, x);
    unsigned long long t = hi + mxhi;
    bool ov = t < hi;
    unsigned long long c = (lo != 0ull) ? 1ull : 0ull;
    unsigned long long t2 = t + c;
    ov |= (t2 < t);
    if (ov || t2 >= x) t2 -= x;                      // result < 2x, one subtraction
    return t2;
}

static __device__ bool is_prime_u64(unsigned long long x)
{
    if (x < 2) return false;
    const uint32_t sp[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
#pragma unroll
    for (int i = 0; i < 12; i++) {
        if (x == sp[i]) return true;
        if (x % sp[i] == 0) return false;
    }
    if (x < 41ull * 41ull) return true;             // no factor <= 37 and x < 41^2
    // -x^{-1} mod 2^64 by Newton's iteration (x odd: x*x == 1 mod 8)
    unsigned long long inv = x;
#pragma unroll
    for (int i = 0; i < 5; i++) inv *= 2ull - x * inv;
    unsigned long long ninv = 0ull - inv;
    unsigned long long r1 = (0ull - x) % x;          // 2^64 mod x  (Montgomery 1)
    unsigned long long r2 = r1;                      // 2^128 mod x by 64 doublings
    for (int i = 0; i < 64; i++) {
        unsigned long long d = r2 << 1;
        if ((r2 >> 63) || d >= x) d -= x;
        r2 = d;
    }
    unsigned long long xm1 = x - 1;
    int s = __ffsll((long long)xm1) - 1;
    unsigned long long d = xm1 >> s;
    unsigned long long mone = x - r1;                // Montgomery -1
    int top = 63 - __clzll((long long)d);
    for (int i = 0; i < 12; i++) {
        unsigned long long a = mont_mul(sp[i], r2, x, ninv);   // sp[i] * 2^64 mod x
        unsigned long long y = a;                    // leading bit of d
        for (int b = top - 1; b >= 0; b--) {
            y = mont_mul(y, y, x, ninv);
            if ((d >> b) & 1ull) y = mont_mul(y, a, x, ninv);
        }
        if (y == r1 || y == mone) continue;
        bool comp = true;
        for (int k = 1; k < s; k++) {
            y = mont_mul(y, y, x, ninv);
            if (y == mone) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// slow_pmin's result when it stopped without an answer: its candidate cap ran
// out, or another warp's had already run out (the call has failed).  Distinct
// from 0, which means no p <= n/2 works (a counterexample).
constexpr unsigned long long SLOW_GAVE_UP = ~0ull;

// Warp-cooperative exact search for p_min(n) over odd p >= p_start (all lanes
// call with the same n).  Returns p_min; 0 with F_COUNTEREX set if no
// p <= n/2 works (the counterexample is recorded in *ce_inv); SLOW_GAVE_UP
// with F_SLOWCAP set if the candidate cap ran out first.  flags and ce_inv
// belong to the call (or, when serving, to the request) the n is part of.
// Kept out of line: it runs for a tiny share of n, and inlined its 64-bit
// Montgomery state would weigh on the register allocation of the hot loops.
static __device__ __noinline__ unsigned long long slow_pmin(unsigned long long n, unsigned long long p_start,
                                        uint32_t cap_log2, unsigned int *flags,
                                        unsigned long long *ce_inv)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long half = n >> 1;
    const unsigned long long steps = cap_log2 >= 6 ? (1ull << (cap_log2 - 6)) : 1ull;
    // once any warp has exhausted its cap the call has failed: stop early
    // (lane 0 reads the flag and broadcasts it so the warp stays converged)
    unsigned int fl = lane == 0 ? *(volatile unsigned int *)flags : 0u;
    fl = __shfl_sync(GB_FULL_MASK, fl, 0);
    if (fl & (F_SLOWCAP | F_INTERNAL)) return SLOW_GAVE_UP;
    for (unsigned long long it = 0; it < steps; ++it) {
        unsigned long long base = p_start + 64ull * it;
        if (base > half) break;
        unsigned long long p = base + 2ull * lane;
        bool ok = (p <= half) && is_prime_u64(p) && is_prime_u64(n - p);
        uint32_t m = __ballot_sync(GB_FULL_MASK, ok);
        if (m) return base + 2ull * (unsigned long long)(__ffs(m) - 1);
        if (it + 1 == steps) {
            if (lane == 0) atomicOr(flags, F_SLOWCAP);
            return SLOW_GAVE_UP;
        }
    }
    if (lane == 0) {
        atomicOr(flags, F_COUNTEREX);
        atomicMax(ce_inv, ~n);
    }
    return 0;
}

// Per-phase cycle counters (builds with GB_PHASE_CLOCKS only; elsewhere no
// code): the leader thread, just after a barrier, adds the cycles since its
// previous mark to slot `slot` (slot < 0 only starts the clock).  The last
// mark lives in one shared word per CTA, so only whole-CTA phases use it.
__device__ __forceinline__ void phase_mark(const Tables &t, int slot, bool leader)
{
#ifdef GB_PHASE_CLOCKS
    __shared__ unsigned long long s_last;
    if (leader && t.phase) {
        const unsigned long long c = clock64();
        if (slot >= 0) atomicAdd(&t.phase[slot], c - s_last);
        s_last = c;
    }
#else
    (void)t; (void)slot; (void)leader;
#endif
}

// The same for one warp's own phase: cycles since `since` (a clock64 value
// taken by the warp), added by lane 0; returns the current clock.
__device__ __forceinline__ unsigned long long phase_warp(const Tables &t, int slot, unsigned long long since)
{
#ifdef GB_PHASE_CLOCKS
    __syncwarp();                                    // the warp's slowest lane ends the phase
    const unsigned long long c = clock64();
    if ((threadIdx.x & 31) == 0 && t.phase && slot >= 0) atomicAdd(&t.phase[slot], c - since);
    return c;
#else
    (void)t; (void)slot; (void)since;
    return 0ull;
#endif
}

// Barrier of a group of NTH threads: the whole CTA (BAR = 0, __syncthreads)
// or a named barrier shared by a subset of its warps (BAR = 1..15).
template <int BAR, int NTH>
__device__ __forceinline__ void group_sync()
{
    if (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NTH) : "memory");
}

// ---------------------------------------------------------------------------
// window geometry
// ---------------------------------------------------------------------------

// Bit j of a window stands for q = wbase + 2j.  The true value of wbase may be
// below 1 near the origin; it is kept modulo 2^64 in `wbase` and described
// exactly by (half_abs, neg): (wbase - 1) / 2 == neg ? -half_abs : +half_abs.
struct WinGeom {
    unsigned long long wbase;
    unsigned long long half_abs;
    unsigned long long q_hi;           // q of bit j_end - 1
    uint32_t neg;
    uint32_t j_end;                    // bits [0, j_end) are sieved, the rest zero
    uint32_t clear_upto;               // bits [0, clear_upto) stand for q <= 1
    uint32_t nfill;                    // words written by the fill pass
};

__device__ __forceinline__ WinGeom make_geom(unsigned long long half_abs, bool neg, uint32_t j_end)
{
    WinGeom g;
    g.half_abs = half_abs;
    g.neg = neg ? 1u : 0u;
    g.wbase = neg ? (1ull - 2ull * half_abs) : (2ull * half_abs + 1ull);
    g.j_end = j_end;
    g.q_hi = g.wbase + 2ull * (unsigned long long)(j_end - 1);   // exact when j_end > 0
    g.clear_upto = (neg || half_abs == 0) ? (uint32_t)(neg ? half_abs + 1 : 1) : 0u;
    g.nfill = (j_end + 31) / 32 + 1;
    return g;
}

// Window of a verification tile whose first even n is n_lo, holding cnt n:
// it starts K_bits odd numbers below n_lo + 1 so every q = n - p with
// p < 2 K_bits is inside, and ends at q = n_last - 1.
__device__ __forceinline__ WinGeom tile_geom(unsigned long long n_lo, uint32_t cnt, uint32_t k_bits)
{
    unsigned long long h = n_lo >> 1;
    bool neg = h < k_bits;
    unsigned long long half_abs = neg ? (k_bits - h) : (h - k_bits);
    return make_geom(half_abs, neg, cnt + k_bits - 1);
}

// ---------------------------------------------------------------------------
// sieve passes
// ---------------------------------------------------------------------------

template <int WHEEL> struct WheelM;
template <> struct WheelM<13> { static constexpr uint32_t M = 3u * 5u * 7u * 11u * 13u; };
template <> struct WheelM<7> { static constexpr uint32_t M = 3u * 5u * 7u; };

// Pre-sieved patterns in shared memory.  Bit u of a pattern of period M is 1
// iff 2u+1 is coprime to M; M + 64 bits are stored so any 32-bit run starting
// below M is one funnel shift of two words.  The block holds the wheel
// (3*5*7*11*13 or 3*5*7) and, with wheel 13, two group patterns that the fill
// may also apply: 17*19*23 and 29*31.
constexpr uint32_t G1_M = 17u * 19u * 23u;        // 7,429
constexpr uint32_t G2_M = 29u * 31u;              // 899
__host__ __device__ constexpr uint32_t pattern_span(uint32_t M) { return ((M + 64 + 31) / 32 + 3) & ~3u; }
template <int WHEEL>
__host__ __device__ constexpr uint32_t pattern_block_words()
{
    return pattern_span(WheelM<WHEEL>::M) + (WHEEL == 13 ? pattern_span(G1_M) + pattern_span(G2_M) : 0u);
}

template <int NT>
__device__ void build_pattern(uint32_t *pat, uint32_t M, uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3,
                              uint32_t p4)
{
    const uint32_t nw = (M + 64 + 31) / 32;
    for (uint32_t w = threadIdx.x; w < nw; w += NT) {
        uint32_t word = 0;
        for (uint32_t b = 0; b < 32; b++) {
            const uint32_t o = 2u * ((32u * w + b) % M) + 1u;
            const bool cop = (o % p0) && (o % p1) && (o % p2) && (o % p3) && (o % p4);
            word |= (cop ? 1u : 0u) << b;
        }
        pat[w] = word;
    }
}

template <int WHEEL, int NT>
__device__ void build_wheel_pattern(uint32_t *pat)
{
    if (WHEEL == 13) {
        build_pattern<NT>(pat, WheelM<13>::M, 3, 5, 7, 11, 13);
        uint32_t *g1 = pat + pattern_span(WheelM<13>::M);
        build_pattern<NT>(g1, G1_M, 17, 19, 23, 17, 17);
        build_pattern<NT>(g1 + pattern_span(G1_M), G2_M, 29, 31, 29, 29, 29);
    } else {
        build_pattern<NT>(pat, WheelM<7>::M, 3, 5, 7, 3, 3);
    }
}

// Phase of window word 0 in a pattern of period M: ((wbase - 1) / 2) mod M,
// exact for negative values; then this thread's first word.
__device__ __forceinline__ uint32_t pattern_phase(const WinGeom &g, uint32_t M)
{
    uint32_t u0 = (uint32_t)(g.half_abs % M);
    if (g.neg && u0) u0 = M - u0;
    return (uint32_t)((u0 + 32ull * threadIdx.x) % M);
}

// The fill loop; REG = some primes are cleared by in-register masks, GROUPS =
// group patterns applied.  Only the words at the window's two edges take
// the masks of [clear_upto, j_end).
template <int WHEEL, int NT, bool REG, int GROUPS>
__device__ __forceinline__ void fill_words(uint32_t *win, const uint32_t *wpat, const WinGeom &g,
                                           uint32_t pat_lo, uint32_t pat_hi)
{
    constexpr bool use1 = GROUPS >= 1, use2 = GROUPS >= 2;
    // words fully inside [clear_upto, j_end) need no edge mask
    const uint32_t w_lo = (g.clear_upto + 31u) >> 5, w_hi = g.j_end >> 5;
    const uint32_t nint = w_hi > w_lo ? w_hi - w_lo : 0u;
    constexpr uint32_t M = WheelM<WHEEL>::M;
    constexpr uint32_t STEP_M = (32u * NT) % M;
    constexpr uint32_t STEP_1 = (32u * NT) % G1_M, STEP_2 = (32u * NT) % G2_M;
    const uint32_t *gp1 = wpat + pattern_span(M);
    const uint32_t *gp2 = gp1 + pattern_span(G1_M);
    uint32_t u = pattern_phase(g, M);
    uint32_t u1 = use1 ? pattern_phase(g, G1_M) : 0u;
    uint32_t u2 = use2 ? pattern_phase(g, G2_M) : 0u;
    uint32_t r[NPAT];
#pragma unroll
    for (int i = 0; i < NPAT; i++) {
        const uint32_t p = pat_prime(i);
        uint32_t v = REG ? (uint32_t)(g.half_abs % p) : 0u;
        if (g.neg && v) v = p - v;
        r[i] = REG ? (v + 32u * threadIdx.x) % p : 0u;
    }
    for (uint32_t w = threadIdx.x; w < g.nfill; w += NT) {
        uint32_t word = __funnelshift_r(wpat[u >> 5], wpat[(u >> 5) + 1], u);
        if (use1) word &= __funnelshift_r(gp1[u1 >> 5], gp1[(u1 >> 5) + 1], u1);
        if (use2) word &= __funnelshift_r(gp2[u2 >> 5], gp2[(u2 >> 5) + 1], u2);
        if (REG) {
#pragma unroll
            for (int i = 0; i < NPAT; i++) {
                if (i >= (int)pat_lo && i < (int)pat_hi) {
                    const uint32_t p = pat_prime(i);
                    const uint32_t h = (p - 1) / 2;  // 2u+1 == 0 mod p  <=>  u == h mod p
                    uint32_t b0 = h >= r[i] ? h - r[i] : h + p - r[i];
                    uint32_t clr = (b0 < 32 ? (1u << b0) : 0u);
                    if (p < 32) clr |= (b0 + p < 32 ? (1u << (b0 + p)) : 0u);
                    if (2 * p < 32) clr |= (b0 + 2 * p < 32 ? (1u << (b0 + 2 * p)) : 0u);
                    word &= ~clr;
                    r[i] += (32u * NT) % p;
                    if (r[i] >= p) r[i] -= p;
                }
            }
        }
        if (w - w_lo >= nint) {
            const uint32_t jw = 32u * w;
            if (jw + 32 > g.j_end) word &= (g.j_end > jw) ? (0xffffffffu >> (32 - (g.j_end - jw))) : 0u;
            if (g.clear_upto > jw) word &= (g.clear_upto >= jw + 32) ? 0u : (0xffffffffu << (g.clear_upto - jw));
        }
        wst(&win[w], word, DS_FILL);
        u += STEP_M;
        if (u >= M) u -= M;
        if (use1) { u1 += STEP_1; if (u1 >= G1_M) u1 -= G1_M; }
        if (use2) { u2 += STEP_2; if (u2 >= G2_M) u2 -= G2_M; }
    }
}

// Pass 1: write every window word from the wheel pattern, the group patterns
// (groups = 0, 1 or 2 of them) and the in-register masks of the pattern
// primes PAT[pat_lo .. pat_hi), zeroing bits outside [clear_upto, j_end).
template <int WHEEL, int NT>
__device__ __forceinline__ void fill_pass(uint32_t *win, const uint32_t *wpat, const WinGeom &g,
                                          uint32_t pat_lo, uint32_t pat_hi, uint32_t groups)
{
    const uint32_t gr = WHEEL == 13 ? groups : 0u;
    if (pat_lo < pat_hi) {
        if (gr >= 2) fill_words<WHEEL, NT, true, 2>(win, wpat, g, pat_lo, pat_hi);
        else if (gr == 1) fill_words<WHEEL, NT, true, 1>(win, wpat, g, pat_lo, pat_hi);
        else fill_words<WHEEL, NT, true, 0>(win, wpat, g, pat_lo, pat_hi);
    } else {
        if (gr >= 2) fill_words<WHEEL, NT, false, 2>(win, wpat, g, pat_lo, pat_hi);
        else if (gr == 1) fill_words<WHEEL, NT, false, 1>(win, wpat, g, pat_lo, pat_hi);
        else fill_words<WHEEL, NT, false, 0>(win, wpat, g, pat_lo, pat_hi);
    }
}

// First window bit of the odd multiples of p that are >= max(p^2, wbase).
// Returns 0xffffffff when p has nothing to clear in [0, j_end).
__device__ __forceinline__ uint32_t first_bit(const WinGeom &g, uint32_t p, unsigned long long m)
{
    unsigned long long pp = (unsigned long long)p * p;      // p < 2^32: no wrap
    if (pp > g.q_hi) return 0xffffffffu;
    unsigned long long j;
    if (g.neg || pp >= g.wbase) {
        j = (pp - g.wbase) >> 1;                            // true distance, wrap-safe
    } else {
        uint32_t r = mod_recip(g.wbase, p, m);
        unsigned long long d = r ? (unsigned long long)(p - r) : 0ull;
        if (d & 1ull) d += p;                                // wbase odd: need d even
        j = d >> 1;
    }
    return j < g.j_end ? (uint32_t)j : 0xffffffffu;
}

// Clear mask m in words w, w + p, ... below w_end (unrolled by eight, then
// four: marks in flight per lane keep the shared-memory atomics busy).
__device__ __forceinline__ void mark_words(uint32_t *win, uint32_t w, uint32_t w_end, uint32_t p, uint32_t m)
{
    for (; w + 7u * p < w_end; w += 8u * p) {
        wand(&win[w], m, DS_MARK_A);
        wand(&win[w + p], m, DS_MARK_A);
        wand(&win[w + 2u * p], m, DS_MARK_A);
        wand(&win[w + 3u * p], m, DS_MARK_A);
        wand(&win[w + 4u * p], m, DS_MARK_A);
        wand(&win[w + 5u * p], m, DS_MARK_A);
        wand(&win[w + 6u * p], m, DS_MARK_A);
        wand(&win[w + 7u * p], m, DS_MARK_A);
    }
    if (w + 3u * p < w_end) {
        wand(&win[w], m, DS_MARK_A);
        wand(&win[w + p], m, DS_MARK_A);
        wand(&win[w + 2u * p], m, DS_MARK_A);
        wand(&win[w + 3u * p], m, DS_MARK_A);
        w += 4u * p;
    }
    for (; w < w_end; w += p) wand(&win[w], m, DS_MARK_A);
}

// Tier-A primes below this bound get the lane skews (measured: 512 and 1024
// alike, 2048 and all primes slower).
constexpr uint32_t SKEW_PMAX = 1024;

// The same for a lane that starts at its d-th multiple w + d p and takes the
// first d (w, w + p, ...) last: the same marks in another order.
__device__ __forceinline__ void mark_words_skew(uint32_t *win, uint32_t w, uint32_t w_end, uint32_t p, uint32_t m,
                                                uint32_t d)
{
    mark_words(win, w + d * p, w_end, p, m);
    for (uint32_t k = 0; k < d && w < w_end; k++, w += p) wand(&win[w], m, DS_MARK_A);
}

__device__ __forceinline__ void clear_bit(uint32_t *win, uint32_t j)
{
    // ~(1 << (j mod 32)) as one rotate: a funnel shift of 0xfffffffe with itself
    wand(&win[j >> 5], __funnelshift_l(0xfffffffeu, 0xfffffffeu, j), DS_MARK_BIT);
}

// Pass 2: cross off the odd multiples of primes[iA0 .. np) in the window.
template <int NT>
__device__ __forceinline__ void mark_pass(uint32_t *win, const WinGeom &g, const Tables &t, uint32_t np)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    constexpr int NWARP = NT / 32;
    const uint32_t j_end = g.j_end;
    // tier A: one warp per prime, lane l clears multiples l, l+32, ... of it.
    // A lane's step, 32 p bits, is exactly p words, so its bit position and
    // clear mask stay fixed and each mark is one atomicAnd plus an add.  Warp
    // w takes every NWARP-th entry of the prime order (balanced by the host,
    // else the ascending primes), 32 at a time: lane q finds the first
    // multiple of the q-th, then the warp marks the 32 primes in turn.
    // The 32 words of one warp step, floor((r + l p) / 32) + const (r = the
    // first bit mod 32), often share shared-memory banks; for p < SKEW_PMAX
    // lane l then starts at its d_l-th multiple (d_l < 4, from the host's
    // table for p mod 1024 and r), which moves its bank by d_l p, and marks
    // its first d_l last.  A larger p has too few marks per lane: the
    // reordered tails cost more than the conflicts they save.
    const uint32_t a_end = t.iB0 < np ? t.iB0 : np;
    unsigned long long tw = phase_warp(t, -1, 0ull);
    // batch entry e of this warp (lane q holds entry e0 + q NWARP): a prime
    // index, from the balanced order when the host provides one
    const uint32_t e_beg = t.aperm ? 0u : t.iA0, e_end = t.aperm ? t.aperm_len : a_end;
    for (uint32_t e0 = e_beg + warp; e0 < e_end; e0 += 32u * NWARP) {
        const uint32_t e = e0 + lane * NWARP;
        const uint32_t iq = e < e_end ? (t.aperm ? t.aperm[e] : e) : 0xffffffffu;
        const bool in = iq < a_end;
        const uint32_t pq = in ? t.primes[iq] : 0u;
        const uint32_t jq = in ? first_bit(g, pq, t.recip[iq]) : 0xffffffffu;
        const unsigned long long sq = t.askew && jq != 0xffffffffu && pq < SKEW_PMAX
                                          ? t.askew[(((pq & 1023u) >> 1) << 5) | (jq & 31u)] : 0ull;
        const bool bskew = __any_sync(GB_FULL_MASK, sq != 0ull);  // some prime of the batch is skewed
        const uint32_t nq = (e_end - e0 + NWARP - 1) / NWARP;   // entries of this batch
        for (uint32_t q = 0; q < nq && q < 32u; q++) {
            const uint32_t j0 = __shfl_sync(GB_FULL_MASK, jq, q);
            if (j0 == 0xffffffffu) continue;
            const uint32_t p = __shfl_sync(GB_FULL_MASK, pq, q);
            uint32_t d = 0;
            if (bskew) {
                const uint32_t s_lo = __shfl_sync(GB_FULL_MASK, (uint32_t)sq, q);
                const uint32_t s_hi = __shfl_sync(GB_FULL_MASK, (uint32_t)(sq >> 32), q);
                d = ((lane < 16 ? s_lo : s_hi) >> (2u * (lane & 15u))) & 3u;
            }
            const uint32_t jl = j0 + lane * p;              // j0 < 2^21, p < 2^16: no wrap
            if (jl >= j_end) continue;
            const uint32_t b = jl & 31u;
            const uint32_t w_end = (j_end - b + 31u) >> 5;  // words w with 32 w + b < j_end
            const uint32_t m = __funnelshift_l(0xfffffffeu, 0xfffffffeu, b);
            if (bskew) mark_words_skew(win, jl >> 5, w_end, p, m, d);
            else mark_words(win, jl >> 5, w_end, p, m);
        }
    }
    tw = phase_warp(t, PH_WARP_TIER_A, tw);
    // tier B: one lane per prime; the next prime's table entries are loaded
    // while the current one is marked
    const uint32_t iB = (t.iB0 > t.iA0 ? t.iB0 : t.iA0) + threadIdx.x;
    uint32_t p_nx = iB < np ? t.primes[iB] : 0u;
    unsigned long long m_nx = iB < np ? t.recip[iB] : 0ull;
    for (uint32_t i = iB; i < np; i += NT) {
        const uint32_t p = p_nx;
        const unsigned long long m = m_nx;
        if (i + NT < np) {
            p_nx = t.primes[i + NT];
            m_nx = t.recip[i + NT];
        }
        uint32_t j = first_bit(g, p, m);
        if (j == 0xffffffffu) continue;
        if (p >= j_end) {                                   // one multiple at most
            clear_bit(win, j);
            continue;
        }
        // p < j_end < 2^21: no index below wraps
        for (; j + 3u * p < j_end; j += 4u * p) {
            clear_bit(win, j);
            clear_bit(win, j + p);
            clear_bit(win, j + 2u * p);
            clear_bit(win, j + 3u * p);
        }
        for (; j < j_end; j += p) clear_bit(win, j);
    }
    phase_warp(t, PH_WARP_TIER_B, tw);
}

// Pass 3: give back the pattern and wheel primes that lie in the window
// (the patterns cleared every multiple of them, themselves included).
template <int WHEEL>
__device__ __forceinline__ void fixup_pass(uint32_t *win, const WinGeom &g, uint32_t pat_hi)
{
    if (threadIdx.x != 0) return;
    if (!g.neg && g.wbase > 61) return;
    uint32_t lim = pat_hi ? pat_prime((int)pat_hi - 1) : (uint32_t)WHEEL;
    if (lim < (uint32_t)WHEEL) lim = WHEEL;
#pragma unroll
    for (int i = -3; i < NPAT; i++) {                         // 3, 5, 7, then 11 .. 61
        const uint32_t sp = i == -3 ? 3u : i == -2 ? 5u : i == -1 ? 7u : pat_prime(i);
        if (sp > lim) continue;
        const unsigned long long q = sp;
        const unsigned long long d = q - g.wbase;             // true distance if q >= wbase
        const bool inside = g.neg ? true : (q >= g.wbase);
        if (!inside || q > g.q_hi) continue;
        const unsigned long long j = d >> 1;
        if (j < g.j_end) wor(&win[j >> 5], 1u << (j & 31), DS_FIXUP);
    }
}

// Pass 2b: clear the hits of the large primes that the bucket pre-pass
// scattered to this window (one bit per entry, coalesced entry loads).
template <int NT>
__device__ __forceinline__ void bucket_pass(uint32_t *win, const WinGeom &g, const uint32_t *ent,
                                            unsigned long long b0, unsigned long long b1, Ctrl *ctrl)
{
    for (unsigned long long e = b0 + threadIdx.x; e < b1; e += NT) {
        const uint32_t j = ent[e];
        if (j < g.j_end) clear_bit(win, j);
        else atomicOr(&ctrl->flags, F_INTERNAL);          // a bucket entry outside its window
    }
}

// Build the whole window (passes 1-3).  Primes from index np_cap on are left
// to the bucket entries [b0, b1) of ent (none when ent is null).  Run by
// threads [0, NT) of the CTA, which meet at barrier BAR (0 = the whole CTA);
// ends with that barrier.
template <int WHEEL, int NT, int BAR = 0>
__device__ __forceinline__ void build_window(uint32_t *win, const uint32_t *wpat, const WinGeom &g,
                                             const Tables &t, uint32_t np_cap = 0xffffffffu,
                                             const uint32_t *ent = nullptr,
                                             unsigned long long b0 = 0, unsigned long long b1 = 0,
                                             Ctrl *ctrl = nullptr)
{
    fill_pass<WHEEL, NT>(win, wpat, g, t.pat_lo, t.pat_hi, t.groups);
    group_sync<BAR, NT>();
    phase_mark(t, PH_FILL, BAR == 0 && threadIdx.x == 0);
    uint32_t np = count_le_warp(t.primes, t.nprimes, isqrt_u64(g.q_hi));
    if (np > np_cap) np = np_cap;
    mark_pass<NT>(win, g, t, np);
    if (ent) bucket_pass<NT>(win, g, ent, b0, b1, ctrl);
    fixup_pass<WHEEL>(win, g, t.pat_hi);
    group_sync<BAR, NT>();
    phase_mark(t, PH_MARK, BAR == 0 && threadIdx.x == 0);
}

// First odd multiple of p that is >= max(p^2, w), as a distance from w;
// w is a window base described by (w mod 2^64, neg).  Returns ~0 when
// p^2 > q_hi.  Used by the bucket pre-pass (64-bit distances).
__device__ __forceinline__ unsigned long long first_dist(unsigned long long w, bool neg,
                                                         unsigned long long q_hi, uint32_t p,
                                                         unsigned long long m)
{
    unsigned long long pp = (unsigned long long)p * p;
    if (pp > q_hi) return ~0ull;
    if (neg || pp >= w) return pp - w;
    uint32_t r = mod_recip(w, p, m);
    unsigned long long d = r ? (unsigned long long)(p - r) : 0ull;
    if (d & 1ull) d += p;
    return d;
}

}  // namespace gbk
