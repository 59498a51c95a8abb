// gb_types.h -- layouts shared by the kernels and the host side of the library.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/goldbach_gb300.h"

namespace gbk {

// Ctrl::flags bits
// (F_BOUNDS: a bounds check of a GB_DEBUG build failed; F_INTERNAL is raised
// with it, so the call fails)
enum : uint32_t { F_COUNTEREX = 1u, F_SLOWCAP = 2u, F_OVERFLOW = 4u, F_INTERNAL = 8u, F_BOUNDS = 16u };

// Record key: (max_pmin << 40) | (2^40 - 1 - k_argmax), so one 64-bit
// atomicMax keeps the largest p_min and, on ties, the smallest n.
constexpr int KEY_SHIFT = 40;
constexpr uint64_t KEY_KMASK = (1ull << KEY_SHIFT) - 1;
constexpr uint32_t PMIN_LIMIT = 1u << 24;   // p_min must stay below this for the key
constexpr int HIST_BINS = 32;

struct __align__(16) DevRec {         // 304 bytes
    unsigned long long key;            // 0 = no n folded yet
    unsigned long long sum;
    unsigned long long wsum;
    unsigned long long n_count;
    unsigned long long n_slow;
    unsigned long long ce_inv;         // ~n of the smallest counterexample, 0 = none
    unsigned long long hist[HIST_BINS];
};

struct __align__(16) Ctrl {
    unsigned long long tile_ctr;       // next tile to claim (device atomic pool)
    unsigned long long ce_inv;         // ~n of the smallest counterexample
    unsigned long long slow_total;
    unsigned int flags;
    unsigned int merge_done;
    unsigned long long work_ctr;       // serving: next work item
    unsigned int dbg_site;             // GB_DEBUG builds: site of the first failed bounds check
    unsigned int dbg_off;              //   and its byte offset in the dynamic shared memory
    unsigned long long pad[2];
};

// Everything a launch needs to know about one call, kept in device memory so a
// captured graph can be replayed with new ranges.
struct __align__(16) RangeParams {
    unsigned long long n0;             // first even n of the range
    unsigned long long n_total;        // number of even n
    unsigned long long ntiles;
    unsigned long long nrec;
    unsigned long long p_slow_start;   // smallest odd p > P_max
    unsigned int tile_bits;            // log2 even n per tile
    unsigned int rec_bits;             // log2 even n per record
    unsigned int k_words;              // candidate words (K_bits = 32 k_words)
    unsigned int p_max;
    unsigned int slow_cap_log2;
    unsigned int bk_prime0;            // primes with index >= this come from buckets
    unsigned int dbg_lim;              // GB_DEBUG builds: window accesses allowed in the first
                                       // dbg_lim bytes of dynamic shared memory (0 = all of it)
    unsigned int dbg_pad;
    unsigned long long tile0;          // this launch processes tiles [tile0, tile_end)
    unsigned long long tile_end;
    const unsigned long long *bk_off;  // bucket of tile t: entries [bk_off[t-tile0], bk_off[t-tile0+1])
    const uint32_t *bk_ent;            // window bit indices; nullptr = no buckets
    unsigned long long *progress;      // finished-tile counter in mapped host memory, or nullptr
    unsigned long long *claim;         // tile counter shared by several callers (mapped host
                                       // memory, system-scope atomics), or nullptr = Ctrl::tile_ctr
};

// Serving: one admitted request.  Its params have rec_bits = 40 so the whole
// request folds into the single record acc (requests have fewer than 2^40 n).
// ctl holds the request's own status flags and counterexample, accumulated
// over every batch that runs one of its tiles (its tile counter is unused).
struct __align__(16) SlotDev {
    RangeParams prm;
    DevRec acc;
    Ctrl ctl;
};
constexpr int SERVE_SLOT_SHIFT = 40;       // work item = (slot << 40) | tile

// Words of one tile window in shared memory: 2^tile_bits + 32 k_words bits,
// two spare words for the funnel shifts, rounded up to 16 bytes.
__host__ __device__ constexpr uint32_t pipe_window_words(uint32_t tile_bits, uint32_t k_words)
{
    return (((1u << tile_bits) + 32u * k_words) / 32u + 2u + 3u) & ~3u;
}

// Read-only device tables shared by every kernel.
struct Tables {
    // both arrays are padded with zeros to a multiple of four entries
    const uint32_t *primes;            // odd primes ascending, primes[0] = 3
    const unsigned long long *recip;   // floor((2^64 - 1) / p)
    const uint32_t *PR;                // bit-reversed candidate words
    uint32_t nprimes;
    uint32_t iA0;                      // first prime index that is marked (above the patterns)
    uint32_t iB0;                      // first prime index marked lane-per-prime
    uint32_t pat_lo, pat_hi;           // in-register pattern primes PAT[pat_lo .. pat_hi)
    uint32_t groups;                   // group patterns in the fill: 1 = 17*19*23, 2 = also 29*31
    uint32_t k_words;
    // scratch of the bit-parallel search: warp w of CTA c stores the open
    // mask of each of its words in olist[(c * warps_per_cta + w) * olist_wcap
    // ..], olist_wcap >= its words per tile; a launch of the bit-parallel
    // kernels must provide it for CTAs c < olist_ctas = the grid
    uint32_t *olist;
    uint32_t olist_wcap, olist_ctas;
    // order of the tier-A primes over the warps: warp w takes the prime
    // indices aperm[w], aperm[w + warps_per_cta], ... (0xffffffff = none),
    // balanced by work; null = round-robin over the ascending primes
    const uint32_t *aperm;
    uint32_t aperm_len;
    // lane skews of the tier-A marks (2 bits a lane) by ((p mod 1024) >> 1,
    // first bit mod 32): 512 x 32 entries; null = no skew
    const unsigned long long *askew;
    // per-phase clock64 sums of builds with GB_PHASE_CLOCKS defined (slots
    // PH_*), null otherwise
    unsigned long long *phase;
};

// phase slots: CTA cycles (thread 0, between barriers) of the window fill,
// the crossing-off (marks, buckets, fix-ups), the search and the record
// reduction; warp cycles (lane 0, summed over warps) of the bit-parallel
// bulk loop and of the per-n walk of the open n; CTA cycles of the tile
// claims; warp cycles of the tier-A (warp per prime) and tier-B (lane per
// prime) crossing-off
enum : int {
    PH_FILL = 0, PH_MARK, PH_SEARCH, PH_REDUCE, PH_WARP_BULK, PH_WARP_TAIL, PH_CLAIM, PH_WARP_TIER_A,
    PH_WARP_TIER_B, PH_COUNT
};

}  // namespace gbk
