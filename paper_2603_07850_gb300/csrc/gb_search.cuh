// gb_search.cuh -- bit-parallel p_min search over one tile window.
//
// For the 32 consecutive even n of one word w (n index k = 32w + b), the
// candidate p = 2i + 1 maps to window bit k + K - 1 - i, so the 32 lookups of
// one candidate for the whole word are one funnel shift of two window words
// by the constant 31 - (i mod 32) (paper Sec. 5.3: bitwise bulk marking,
// 32 n per instruction).  A lane owns one word and walks the odd primes
// p < 64 BC (BC <= 8, so p < 512) in ascending order (compile-time unrolled);
// each candidate resolves the bits that are still open:
//     x = funnelshift(window words);  V |= x;
// and p is recorded in bit-sliced form: plane j holds the n whose p_min has
// bit j set.  V only gains bits, so the n a run of consecutive candidates
// resolved are V(after the run) - V(before it); plane j adds that difference
// once per run of candidates with bit j set (bits 1..4 of p), and planes 5..
// once per 32-wide range of candidates.  The record statistics come from the
// planes: the sums through bit-sliced per-position accumulators, the log2
// histogram from popcounts of V at the candidate boundaries 2^b, and the max
// with its smallest n.  The few n left open (p_min >= 64 BC) are compacted
// through a per-warp shared ring into full rounds of 32 and finish with the
// per-n search from chunk BC on, then the exact slow path.
#pragma once
#include "gb_device.cuh"

namespace gbk {

constexpr int CAND_COUNT = 96;             // odd primes below 512

__host__ __device__ constexpr uint32_t cand_prime(int i)
{
    switch (i) {
        case 0: return 3u;
        case 1: return 5u;
        case 2: return 7u;
        case 3: return 11u;
        case 4: return 13u;
        case 5: return 17u;
        case 6: return 19u;
        case 7: return 23u;
        case 8: return 29u;
        case 9: return 31u;
        case 10: return 37u;
        case 11: return 41u;
        case 12: return 43u;
        case 13: return 47u;
        case 14: return 53u;
        case 15: return 59u;
        case 16: return 61u;
        case 17: return 67u;
        case 18: return 71u;
        case 19: return 73u;
        case 20: return 79u;
        case 21: return 83u;
        case 22: return 89u;
        case 23: return 97u;
        case 24: return 101u;
        case 25: return 103u;
        case 26: return 107u;
        case 27: return 109u;
        case 28: return 113u;
        case 29: return 127u;
        case 30: return 131u;
        case 31: return 137u;
        case 32: return 139u;
        case 33: return 149u;
        case 34: return 151u;
        case 35: return 157u;
        case 36: return 163u;
        case 37: return 167u;
        case 38: return 173u;
        case 39: return 179u;
        case 40: return 181u;
        case 41: return 191u;
        case 42: return 193u;
        case 43: return 197u;
        case 44: return 199u;
        case 45: return 211u;
        case 46: return 223u;
        case 47: return 227u;
        case 48: return 229u;
        case 49: return 233u;
        case 50: return 239u;
        case 51: return 241u;
        case 52: return 251u;
        case 53: return 257u;
        case 54: return 263u;
        case 55: return 269u;
        case 56: return 271u;
        case 57: return 277u;
        case 58: return 281u;
        case 59: return 283u;
        case 60: return 293u;
        case 61: return 307u;
        case 62: return 311u;
        case 63: return 313u;
        case 64: return 317u;
        case 65: return 331u;
        case 66: return 337u;
        case 67: return 347u;
        case 68: return 349u;
        case 69: return 353u;
        case 70: return 359u;
        case 71: return 367u;
        case 72: return 373u;
        case 73: return 379u;
        case 74: return 383u;
        case 75: return 389u;
        case 76: return 397u;
        case 77: return 401u;
        case 78: return 409u;
        case 79: return 419u;
        case 80: return 421u;
        case 81: return 431u;
        case 82: return 433u;
        case 83: return 439u;
        case 84: return 443u;
        case 85: return 449u;
        case 86: return 457u;
        case 87: return 461u;
        case 88: return 463u;
        case 89: return 467u;
        case 90: return 479u;
        case 91: return 487u;
        case 92: return 491u;
        case 93: return 499u;
        case 94: return 503u;
        case 95: return 509u;
        default: return 0u;
    }
}

// Number of candidates below 64 * bc (bc = 1..8).
__host__ __device__ constexpr int cand_count(int bc)
{
    return bc == 1 ? 17 : bc == 2 ? 30 : bc == 3 ? 42 : bc == 4 ? 53 : bc == 5 ? 65 : bc == 6 ? 75 : bc == 7 ? 85 : 96;
}

// Largest candidate below 64 * bc (bc = 1..8).
__host__ __device__ constexpr uint32_t cand_last(int bc)
{
    return cand_prime(cand_count(bc) - 1);
}

// sum over the set bits b of x of b
__device__ __forceinline__ uint32_t bitpos_sum(uint32_t x)
{
    return __popc(x & 0xAAAAAAAAu) + 2u * __popc(x & 0xCCCCCCCCu) + 4u * __popc(x & 0xF0F0F0F0u) +
           8u * __popc(x & 0xFF00FF00u) + 16u * __popc(x & 0xFFFF0000u);
}

// Per-lane running state of one sub-record: sums relative to the sub-record
// start (k_rel = k - ks), converted to record-relative values at the end.
// The histogram bins 1..8 are 16-bit counts, two to a word (a lane folds at
// most 2^20 / 256 n of one sub-record).  The rare n_slow and counterexample
// updates go to the CTA's shared counters instead of registers.
struct SubAcc {
    uint32_t mx, arg;                       // max p_min, its k_rel
    unsigned long long sum, wsum;           // sum p, sum p * (k_rel + 1)
    uint32_t h[4];                          // bin b (1..8) in h[(b-1)/2] bits 16((b-1)%2) ..
    __device__ __forceinline__ void reset()
    {
        mx = 0; arg = 0xffffffffu; sum = 0; wsum = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) h[b] = 0;
    }
    __device__ __forceinline__ void take_max(uint32_t p, uint32_t k)
    {
        if (p > mx || (p == mx && k < arg)) { mx = p; arg = k; }
    }
    __device__ __forceinline__ uint32_t bin(int b) const
    {
        return (h[(b - 1) >> 1] >> (16 * ((b - 1) & 1))) & 0xffffu;
    }
};

// CTA-wide counters of one sub-record that lanes touch only rarely.
struct SubShared {
    uint32_t *hist;                         // bins >= 9
    uint32_t *slow;                         // #(p_min > P_max)
    unsigned long long *ce;                 // max ~n over counterexamples
};

// Bit-sliced sums of p_min per bit position over the words a lane has folded
// since the last flush: plane j of T holds bit j of sum_w p_w(b) for every bit
// position b (p_w(b) = p_min of n 32 w + b, 0 when open).  A word adds its
// nine bit planes with a ripple of three-input logic ops, so the position
// weights of wsum cost popcounts once per flush instead of once per word
// (sum_b b p(b) is what wsum needs beyond the per-word sum).  Every p_min of
// the bulk phase is below 512, so CAP = 2^(TW - 9) words never overflow the
// TW planes.
constexpr int POS_TW = 12;
struct PosAcc {
    uint32_t T[POS_TW];
    uint32_t G;                             // sum over the pass's words of gi * (sum of p over word gi)
    static constexpr uint32_t CAP = 1u << (POS_TW - 9);
};

// Fold sum_b b T(b) of the nw words in pa into acc.wsum.  Plane j can be set
// only when nw * 511 >= 2^j.
__device__ __forceinline__ void pos_flush(const PosAcc &pa, uint32_t nw, SubAcc &acc)
{
    uint32_t sb = 0;                        // <= 496 * 2^POS_TW: no wrap
#pragma unroll
    for (int j = 0; j < POS_TW; j++)
        if (j < 9 || nw > (1u << (j - 9))) sb += bitpos_sum(pa.T[j]) << j;
    acc.wsum += sb;
}

// One word of the bulk phase: resolves candidates p < 64 BC with p <= bb,
// folds the resolved bits into acc and pa (word gi of the lane's pass, wl =
// its index in the sub-record) and returns the still-open bits.  bb never
// exceeds P_max, so nothing resolved here counts towards n_slow.  ALL = every
// candidate below 64 BC is <= bb (the usual case), so no candidate is tested
// against bb at run time.
// `one` is 1 and `mone` -1, passed at run time: a run's plane update
// B += V_end - V_start is then two integer multiply-adds, issued on the FMA
// pipe beside the ALU pipe that runs the funnel shifts and the ORs (the loop
// is bound by the ALU pipe; plane 3 takes a three-input add on it, which
// measured best).  The difference holds no bit of any plane, so the add is
// an OR.
// The word statistics bulk_word folds: the sums and the histogram (BW_SUMS),
// the largest p_min and its smallest n (BW_MAX).
enum : int { BW_SUMS = 1, BW_MAX = 2 };

// Histogram bin b (1..8) of acc gains v.
__device__ __forceinline__ void hist_add(SubAcc &acc, int b, uint32_t v)
{
    acc.h[(b - 1) >> 1] += v << (16 * ((b - 1) & 1));
}

template <int BC, bool ALL, int PART = BW_SUMS | BW_MAX>
__device__ __forceinline__ uint32_t bulk_word(const uint32_t *win, uint32_t w, uint32_t wl, uint32_t gi,
                                              uint32_t KW, uint32_t valid, uint32_t bb, uint32_t one,
                                              SubAcc &acc, PosAcc &pa)
{
    // Every candidate is odd, so plane 0 collects exactly the resolved bits:
    // it doubles as the "already resolved" mask V (invalid bits start set).
    // The candidates of one 32-wide range of p share the bits of p from bit 5
    // up, so planes 5.. take the bits the range resolved once, after it;
    // planes 1..4 take theirs once per run of candidates (Rj = B0 where the
    // run of plane j began).
    // Candidates run in ascending order, so the n of histogram bin b (p_min in
    // [2^b, 2^(b+1))) are those resolved between the candidate boundaries 2^b
    // and 2^(b+1): with BW_SUMS each bin is the difference of two popcounts of
    // B0 taken at those boundaries.
    constexpr bool SUMS = (PART & BW_SUMS) != 0;
    uint32_t B0 = ~valid, B1 = 0, B2 = 0, B3 = 0, B4 = 0, B5 = 0, B6 = 0, B7 = 0, B8 = 0;
    const uint32_t c0 = SUMS ? (uint32_t)__popc(B0) : 0u;
    uint32_t cp = c0;                                 // popcount of B0 at the last bin boundary
    uint32_t R1 = 0, R2 = 0, R3 = 0, R4 = 0;          // B0 where the open run of plane j began
    const uint32_t mone = 0u - one;
#pragma unroll
    for (int c = 0; c < BC; c++) {
        // a chunk past the window's K bits holds no candidate <= bb (only
        // possible when !ALL, with a search bound below 64 BC): it loads
        // nothing, so no index runs below the window
        const bool cin = ALL || (uint32_t)c < KW;
        const uint32_t lo = cin ? wld(&win[w + KW - 1 - c], DS_BULK) : 0u,
                       hi = cin ? wld(&win[w + KW - c], DS_BULK) : 0u;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t g = 2u * c + h;                // p in [32 g, 32 g + 32)
            const uint32_t B_start = B0;
#pragma unroll
            for (int ci = 0; ci < cand_count(BC); ci++) {
                const uint32_t p = cand_prime(ci);
                const uint32_t i = (p - 1) >> 1;
                if ((p >> 5) == g) {
                    // the candidates of this range just before and after p
                    const uint32_t pv = ci > 0 && (cand_prime(ci - 1) >> 5) == g ? cand_prime(ci - 1) : 0u;
                    const uint32_t pn = (cand_prime(ci + 1) >> 5) == g ? cand_prime(ci + 1) : 0u;
                    if ((p & 2u) && !(pv & 2u)) R1 = B0;
                    if ((p & 4u) && !(pv & 4u)) R2 = B0;
                    if ((p & 8u) && !(pv & 8u)) R3 = B0;
                    if ((p & 16u) && !(pv & 16u)) R4 = B0;
                    if (ALL || p <= bb) B0 |= __funnelshift_r(lo, hi, 31u - (i & 31u));
                    if ((p & 2u) && !(pn & 2u)) B1 = R1 * mone + (B0 * one + B1);
                    if ((p & 4u) && !(pn & 4u)) B2 = R2 * mone + (B0 * one + B2);
                    if ((p & 8u) && !(pn & 8u)) B3 = B3 + B0 - R3;
                    if ((p & 16u) && !(pn & 16u)) B4 = R4 * mone + (B0 * one + B4);
                }
                // bins 1, 2, 3 end after the candidates 3, 7 and 13 (range 0)
                if (SUMS && g == 0u && (p == 3u || p == 7u || p == 13u)) {
                    const uint32_t cn = __popc(B0);
                    hist_add(acc, p == 3u ? 1 : p == 7u ? 2 : 3, cn - cp);
                    cp = cn;
                }
            }
            if (g != 0u) {
                const uint32_t D = B0 & ~B_start;       // resolved by this range
                if ((32u * g) & 32u) B5 = D * one + B5;
                if ((32u * g) & 64u) B6 = D * one + B6;
                if ((32u * g) & 128u) B7 = D * one + B7;
                if ((32u * g) & 256u) B8 = D * one + B8;
            }
            // bins 4.. end with the ranges g = 2^(b-4) - 1; the last bin
            // with candidates ends with the loop
            if (SUMS && (g == 0u || g == 1u || g == 3u || g == 7u || g == 15u || g + 1u == 2u * BC)) {
                const uint32_t cn = __popc(B0);
                hist_add(acc, g == 0u ? 4 : 5 + (31 - __clz(g)), cn - cp);
                cp = cn;
            }
        }
    }
    const uint32_t V = B0;
    B0 &= valid;
    if (SUMS) {
        // sum over the word, plane by plane (plane 0 has cp - c0 bits)
        constexpr int NPL = BC > 4 ? 9 : 8;
        const uint32_t Bs[9] = {B0, B1, B2, B3, B4, B5, B6, B7, B8};
        uint32_t s = cp - c0;
#pragma unroll
        for (int j = 1; j < NPL; j++) s += __popc(Bs[j]) << j;
        acc.sum += s;
        pa.G += gi * s;
        // the position-weighted part: add the planes to pa (the first word
        // after a flush starts it)
        if ((gi & (PosAcc::CAP - 1u)) == 0u) {
#pragma unroll
            for (int j = 0; j < POS_TW; j++) pa.T[j] = j < NPL ? Bs[j] : 0u;
        } else {
            uint32_t cy = pa.T[0] & B0;
            pa.T[0] ^= B0;
#pragma unroll
            for (int j = 1; j < POS_TW; j++) {
                const uint32_t t = pa.T[j];
                if (j < NPL) {
                    const uint32_t x = Bs[j];
                    pa.T[j] = t ^ x ^ cy;
                    cy = (t & x) | (cy & (t ^ x));
                } else {
                    pa.T[j] = t ^ cy;
                    cy = t & cy;
                }
            }
        }
    }
    if (PART & BW_MAX) {
        const uint32_t R = V & valid;                 // resolved n of this word
        if (R) {
            // max over the word and its smallest n
            const uint32_t Bs[9] = {B0, B1, B2, B3, B4, B5, B6, B7, B8};
            uint32_t cand = R, mx = 0;
#pragma unroll
            for (int j = (BC > 4 ? 8 : 7); j >= 0; j--) {
                const uint32_t t = cand & Bs[j];
                if (t) { cand = t; mx |= 1u << j; }
            }
            acc.take_max(mx, 32u * wl + (uint32_t)(__ffs(cand) - 1));
        }
    }
    return valid & ~V;
}

// p_min of one n per lane (tile index k) from candidate index i_start on,
// then the exact slow path.  Warp-collective (all 32 lanes call it; `act`
// marks the lanes that hold an n).  Returns p_min, or 0: a counterexample
// (gave_up false; F_COUNTEREX is set) or a slow path that gave up (gave_up
// true; the call fails with GB_ESLOWPATH_LIMIT).
__device__ __forceinline__ uint32_t tail_pmin(const uint32_t *win, const uint32_t *PR, uint32_t KW, uint32_t k,
                                              bool act, unsigned long long n_lo, uint32_t i_start,
                                              const RangeParams &prm, Ctrl *ctrl, bool &gave_up)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t KB = 32u * KW;
    const uint32_t t0 = i_start >> 5;
    const uint32_t mask0 = 0xffffffffu >> (i_start & 31u);
    const unsigned long long n = n_lo + 2ull * k;
    uint32_t pm = 0;
    gave_up = false;
    if (act) {
        if (n == 4ull) {
            pm = 2u;
        } else if (t0 < KW) {
            // chunk t covers the 32 window bits from s_t = k + K - 32 - 32 t:
            // the shift is the same for every t and chunk t+1's high word is
            // chunk t's low word, so each step loads one window word
            const uint32_t s0 = k + KB - 32u - 32u * t0;
            const uint32_t sh = s0 & 31u;
            uint32_t w = s0 >> 5, hi = wld(&win[w + 1], DS_TAIL);
            uint32_t lo = wld(&win[w], DS_TAIL);
            uint32_t m = __funnelshift_r(lo, hi, sh) & PR[t0] & mask0;
            uint32_t t = t0;
            while (!m && ++t < KW) {
                hi = lo;
                lo = wld(&win[--w], DS_TAIL);
                m = __funnelshift_r(lo, hi, sh) & PR[t];
            }
            if (m) pm = 2u * (32u * t + __clz(m)) + 1u;
        }
    }
    uint32_t pend = __ballot_sync(GB_FULL_MASK, act && pm == 0u);
    while (pend) {
        const int src = __ffs(pend) - 1;
        pend &= pend - 1;
        const unsigned long long ns = __shfl_sync(GB_FULL_MASK, n, src);
        unsigned long long ps = slow_pmin(ns, prm.p_slow_start, prm.slow_cap_log2, &ctrl->flags, &ctrl->ce_inv);
        const bool gu = ps == SLOW_GAVE_UP;
        if (!gu && ps >= PMIN_LIMIT) {
            if (lane == 0) atomicOr(&ctrl->flags, F_OVERFLOW);
            ps = PMIN_LIMIT - 1;
        }
        if ((int)lane == src) {
            pm = gu ? 0u : (uint32_t)ps;
            gave_up = gu;
        }
    }
    return pm;
}

// Fold one p_min (kr = its index in the sub-record) into the lane's record state.
__device__ __forceinline__ void fold_pmin(uint32_t pm, uint32_t kr, const RangeParams &prm, SubAcc &acc,
                                          const SubShared &ss)
{
    acc.take_max(pm, kr);
    acc.sum += pm;
    acc.wsum += (unsigned long long)pm * (kr + 1ull);
    if (pm > prm.p_max) atomicAdd(ss.slow, 1u);
    const uint32_t bin = 31u - __clz(pm);
    if (bin <= 8) {
        const uint32_t hb = bin - 1u, inc = 1u << (16u * (hb & 1u));
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) acc.h[q] += (hb >> 1) == q ? inc : 0u;
    } else {
        atomicAdd(&ss.hist[bin], 1u);
    }
}

// Per-n search of one open n (tile index k) per lane, from candidate index
// i_start on, then the exact slow path; folds p_min into acc (a
// counterexample into the sub-record's shared counter, a slow path that gave
// up nowhere: the call fails).  Warp-collective (all 32 lanes call it; `act`
// marks the lanes that hold an n).
__device__ __forceinline__ void tail_one(const uint32_t *win, const uint32_t *PR, uint32_t KW, uint32_t k,
                                         bool act, unsigned long long n_lo, uint32_t ks, uint32_t i_start,
                                         const RangeParams &prm, SubAcc &acc, const SubShared &ss, Ctrl *ctrl)
{
    bool gave_up;
    const uint32_t pm = tail_pmin(win, PR, KW, k, act, n_lo, i_start, prm, ctrl, gave_up);
    if (act && pm) fold_pmin(pm, k - ks, prm, acc, ss);
    else if (act && !gave_up) atomicMax(ss.ce, ~(n_lo + 2ull * k));
}

// The per-n phase of one sub-record for one warp.  During the bulk phase the
// warp stored the open mask of each of its words (p_min above the
// bit-parallel bound); here each step every lane hands over the lowest open
// bit of its word, its slot in the warp's 64-entry
// shared ring given by a ballot and a popcount (about three steps per group at
// 10^12), and a full round of 32 is searched as soon as the ring holds one.
struct OpenRing {
    uint32_t *q;
    uint32_t head, tail;                               // warp-uniform positions
};

// Groups [g0, g1) of the warp's open masks mb (lane l of group gi at
// mb[32 gi + l], word wg0 + 32 NWARP gi + l).
template <int NWARP>
__device__ __forceinline__ void ring_groups(OpenRing &rg, const uint32_t *mb, uint32_t g0, uint32_t g1, uint32_t wg0,
                                            const uint32_t *win, const uint32_t *PR, uint32_t KW,
                                            unsigned long long n_lo, uint32_t ks, uint32_t i_start,
                                            const RangeParams &prm, SubAcc &acc, const SubShared &ss, Ctrl *ctrl)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    uint32_t U_nx = g0 < g1 ? mb[32u * g0 + lane] : 0u; // the next group's masks load ahead
    for (uint32_t gi = g0; gi < g1; gi++) {
        uint32_t U = U_nx;
        if (gi + 1 < g1) U_nx = mb[32u * (gi + 1) + lane];
        const uint32_t kw = 32u * (wg0 + 32u * NWARP * gi + lane);
        for (;;) {
            const uint32_t has = __ballot_sync(GB_FULL_MASK, U != 0u);
            if (!has) break;
            if (U) {
                rg.q[(rg.tail + __popc(has & below)) & 63u] = kw + (uint32_t)(__ffs(U) - 1);
                U &= U - 1u;
            }
            rg.tail += __popc(has);                    // at most 63 entries are pending
            if (rg.tail - rg.head >= 32u) {
                __syncwarp();
                const uint32_t k = rg.q[(rg.head + lane) & 63u];
                __syncwarp();
                tail_one(win, PR, KW, k, true, n_lo, ks, i_start, prm, acc, ss, ctrl);
                rg.head += 32u;
            }
        }
    }
}

// Search the entries still in the ring (fewer than 32).
__device__ __forceinline__ void ring_flush(OpenRing &rg, const uint32_t *win, const uint32_t *PR, uint32_t KW,
                                           unsigned long long n_lo, uint32_t ks, uint32_t i_start,
                                           const RangeParams &prm, SubAcc &acc, const SubShared &ss, Ctrl *ctrl)
{
    const uint32_t lane = threadIdx.x & 31;
    __syncwarp();
    if (rg.tail != rg.head) {
        const uint32_t k = rg.q[(rg.head + lane) & 63u];
        tail_one(win, PR, KW, k, lane < rg.tail - rg.head, n_lo, ks, i_start, prm, acc, ss, ctrl);
    }
    __syncwarp();
    rg.head = rg.tail = 0;
}

// First pass of the per-n search for one warp of NWARP: the warp takes the
// same words as the bit-parallel bulk loop (word wg0 + 32 NWARP gi + j, j =
// 0..31), one word (32 n, one per lane) per step.  Each lane looks its n up
// in the first chunk of 32 candidates (two window words the whole warp
// shares), folds the resolved ones, and lane j keeps word j's open mask,
// stored at mb[32 gi + j] like the bulk loop's; ring_groups then finishes the
// open n from candidate 32.  Returns the number of word groups.
template <int NWARP>
__device__ __forceinline__ uint32_t pern_first(const uint32_t *win, const uint32_t *PR, uint32_t KW,
                                               unsigned long long n_lo, uint32_t ks, uint32_t ke, int warp,
                                               uint32_t *mb, uint32_t gmax, const RangeParams &prm, SubAcc &acc,
                                               const SubShared &ss)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t PR0 = PR[0];
    const uint32_t wbeg = ks >> 5, wend = (ke + 31) >> 5;
    uint32_t gi = 0;
    for (uint32_t wb = wbeg + 32u * (uint32_t)warp; wb < wend; wb += 32u * NWARP, gi++) {
        uint32_t keep = 0;
        const uint32_t jn = wend - wb < 32u ? wend - wb : 32u;
        for (uint32_t j = 0; j < jn; j++) {
            const uint32_t w = wb + j;
            const uint32_t k = 32u * w + lane;
            const bool valid = k < ke;
            uint32_t pm = 0;
            if (valid && n_lo + 2ull * k != 4ull) {
                const uint32_t m = __funnelshift_r(wld(&win[w + KW - 1u], DS_PERN), wld(&win[w + KW], DS_PERN), lane) & PR0;
                if (m) pm = 2u * __clz(m) + 1u;
            }
            if (pm) fold_pmin(pm, k - ks, prm, acc, ss);
            const uint32_t open = __ballot_sync(GB_FULL_MASK, valid && pm == 0u);
            if (lane == j) keep = open;
        }
        if (gi < gmax) mb[32u * gi + lane] = keep;
    }
    return gi;
}

// Per-n search (one lane per n) of the n [ks, ke) of a tile for one warp of
// NWARP in one loop, for a launch without open-mask slots, with warp
// compaction: each lane looks its n up in the first chunk of
// 32 candidates (p < 64; one funnel shift of two window words that the whole
// warp shares); the n left open (and n = 4) go to the warp's ring and finish
// in full rounds of 32 from candidate 32 on, so no lane idles while another
// walks far.
template <int NWARP>
__device__ __forceinline__ void pern_groups(OpenRing &rg, int warp, const uint32_t *win, const uint32_t *PR,
                                            uint32_t KW, unsigned long long n_lo, uint32_t ks, uint32_t ke,
                                            const RangeParams &prm, SubAcc &acc, const SubShared &ss, Ctrl *ctrl)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t PR0 = PR[0];
    for (uint32_t g32 = (ks >> 5) + (uint32_t)warp; (g32 << 5) < ke; g32 += NWARP) {
        const uint32_t k = (g32 << 5) + lane;
        const bool valid = k < ke;
        const unsigned long long n = n_lo + 2ull * k;
        uint32_t pm = 0;
        if (valid && n != 4ull) {
            const uint32_t m =
                __funnelshift_r(wld(&win[g32 + KW - 1u], DS_PERN), wld(&win[g32 + KW], DS_PERN), lane) & PR0;
            if (m) pm = 2u * __clz(m) + 1u;
        }
        if (pm) fold_pmin(pm, k - ks, prm, acc, ss);
        const bool open = valid && pm == 0u;
        const uint32_t has = __ballot_sync(GB_FULL_MASK, open);
        if (open) rg.q[(rg.tail + __popc(has & below)) & 63u] = k;
        rg.tail += __popc(has);                        // at most 63 entries are pending
        if (rg.tail - rg.head >= 32u) {
            __syncwarp();
            const uint32_t kk = rg.q[(rg.head + lane) & 63u];
            __syncwarp();
            tail_one(win, PR, KW, kk, true, n_lo, ks, 32u, prm, acc, ss, ctrl);
            rg.head += 32u;
        }
    }
}

}  // namespace gbk
