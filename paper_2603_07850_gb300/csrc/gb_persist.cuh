// gb_persist.cuh -- the persistent fused kernel and the record reduction it
// shares with the plain form.  Instantiated per thread count in
// gb_persist_<NT>.cu so the variants compile in parallel.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "gb_device.cuh"
#include "gb_search.cuh"

namespace gbk {

// ---------------------------------------------------------------------------
// persistent fused kernel
// ---------------------------------------------------------------------------

struct RedScratch {
    uint32_t ring[32][64];                   // per-warp rings of open n (bit-parallel search)
    unsigned long long arg[32], sum[32], wsum[32], ce[32];
    uint32_t mx[32], slow[32];
    uint32_t hist[HIST_BINS];
    uint32_t xslow;                          // n_slow and counterexample of the sub-record,
    unsigned long long xce;                  //   folded by lanes of the bit-parallel search
    unsigned long long tile;
    RangeParams prm;                         // the current tile's call
    uint32_t one;                            // holds 1 (multiplier of the plane updates)
};

// Fold one p_min into a lane's running record state.
struct LaneAcc {
    uint32_t mx, slow;
    unsigned long long arg, sum, wsum, ce, hA, hB;
    __device__ __forceinline__ void reset()
    {
        mx = 0; slow = 0; arg = ~0ull; sum = 0; wsum = 0; ce = 0; hA = 0; hB = 0;
    }
    __device__ __forceinline__ void add(uint32_t pm, unsigned long long kr, uint32_t p_max,
                                        uint32_t *s_hist)
    {
        if (pm > mx) { mx = pm; arg = kr; }           // k ascends per lane: first max wins
        sum += pm;
        wsum += (unsigned long long)pm * (kr + 1ull);
        slow += pm > p_max ? 1u : 0u;
        uint32_t b = 31u - __clz(pm);                 // floor(log2 p_min) >= 1
        if (b <= 4) hA += 1ull << (16u * (b - 1u));
        else if (b <= 8) hB += 1ull << (16u * (b - 5u));
        else atomicAdd(&s_hist[b], 1u);
    }
};

// Reduction of the lanes' state over a group of NWARP warps into record r;
// `warp` is the warp's index in the group (0 combines) and `gt` the thread's,
// BAR the group's barrier (0 = the whole CTA).  `whole` = the tile owns the
// record (plain stores) instead of sharing it (atomics).
template <int NWARP, int BAR>
__device__ __forceinline__ void reduce_group(LaneAcc &a, RedScratch &s, DevRec *rec, uint32_t n_cnt, bool whole,
                                             Ctrl *ctrl, int warp, const Tables *tp = nullptr)
{
    const int lane = threadIdx.x & 31;
    uint32_t wmax = __reduce_max_sync(GB_FULL_MASK, a.mx);
    unsigned long long warg = warp_min_u64(a.mx == wmax ? a.arg : ~0ull);
    unsigned long long wsum = warp_sum_u64(a.sum), wws = warp_sum_u64(a.wsum);
    unsigned long long wce = a.ce;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(GB_FULL_MASK, wce, o);
        wce = v > wce ? v : wce;
    }
    uint32_t wslow = __reduce_add_sync(GB_FULL_MASK, a.slow);
#pragma unroll
    for (int f = 0; f < 4; f++) {
        uint32_t ca = __reduce_add_sync(GB_FULL_MASK, (uint32_t)(a.hA >> (16 * f)) & 0xffffu);
        uint32_t cb = __reduce_add_sync(GB_FULL_MASK, (uint32_t)(a.hB >> (16 * f)) & 0xffffu);
        if (lane == 0) {
            if (ca) atomicAdd(&s.hist[1 + f], ca);
            if (cb) atomicAdd(&s.hist[5 + f], cb);
        }
    }
    if (lane == 0) {
        s.mx[warp] = wmax; s.arg[warp] = warg; s.sum[warp] = wsum; s.wsum[warp] = wws;
        s.slow[warp] = wslow; s.ce[warp] = wce;
    }
    group_sync<BAR, 32 * NWARP>();
    if (tp) phase_mark(*tp, PH_SEARCH, BAR == 0 && threadIdx.x == 0);
    if (warp == 0) {
        uint32_t m = lane < NWARP ? s.mx[lane] : 0u;
        unsigned long long ar = lane < NWARP ? s.arg[lane] : ~0ull;
        uint32_t cm = __reduce_max_sync(GB_FULL_MASK, m);
        unsigned long long ca = warp_min_u64(m == cm ? ar : ~0ull);
        unsigned long long su = warp_sum_u64(lane < NWARP ? s.sum[lane] : 0ull);
        unsigned long long ws = warp_sum_u64(lane < NWARP ? s.wsum[lane] : 0ull);
        uint32_t sl = __reduce_add_sync(GB_FULL_MASK, lane < NWARP ? s.slow[lane] : 0u) + s.xslow;
        unsigned long long ce = lane < NWARP ? s.ce[lane] : 0ull;
        if (lane == 0 && s.xce > ce) ce = s.xce;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long v = __shfl_xor_sync(GB_FULL_MASK, ce, o);
            ce = v > ce ? v : ce;
        }
        unsigned long long key = cm ? (((unsigned long long)cm << KEY_SHIFT) | (KEY_KMASK - ca)) : 0ull;
        if (whole) {
            if (lane == 0) {
                rec->key = key; rec->sum = su; rec->wsum = ws; rec->n_count = n_cnt;
                rec->n_slow = sl; rec->ce_inv = ce;
            }
            rec->hist[lane] = s.hist[lane];
        } else {
            if (lane == 0) {
                if (key) atomicMax(&rec->key, key);
                atomicAdd(&rec->sum, su);
                atomicAdd(&rec->wsum, ws);
                atomicAdd(&rec->n_count, (unsigned long long)n_cnt);
                if (sl) atomicAdd(&rec->n_slow, (unsigned long long)sl);
                if (ce) atomicMax(&rec->ce_inv, ce);
            }
            if (s.hist[lane]) atomicAdd(&rec->hist[lane], (unsigned long long)s.hist[lane]);
        }
        if (lane == 0 && sl) atomicAdd(&ctrl->slow_total, (unsigned long long)sl);
    }
    if (tp) phase_mark(*tp, PH_REDUCE, BAR == 0 && threadIdx.x == 0);
}

// CTA-wide reduction (every thread of an NT-thread CTA).
template <int NT>
__device__ __forceinline__ void reduce_to_record(LaneAcc &a, RedScratch &s, DevRec *rec,
                                                 uint32_t n_cnt, bool whole, Ctrl *ctrl)
{
    reduce_group<NT / 32, 0>(a, s, rec, n_cnt, whole, ctrl, (int)(threadIdx.x >> 5));
}

// Bit-parallel phase bound of a call: candidates p <= bb (never above P_max
// or the search bound) resolve in the bulk phase; the per-n phase starts at
// candidate index (bb + 1) / 2.
template <int SEARCH_BC>
__device__ __forceinline__ uint32_t bulk_bound(const RangeParams &prm)
{
    const uint32_t ps_odd = (uint32_t)(prm.p_slow_start - 2ull);
    uint32_t bb = SEARCH_BC ? 64u * SEARCH_BC - 1u : 0u;
    if (bb > ps_odd) bb = ps_odd;
    if (bb > prm.p_max) bb = prm.p_max;
    return bb;
}

// The bit-parallel pass over one warp's words of the sub-record [ks, ke):
// word (ks >> 5) + 32 NWARP gi + lane for gi = 0, 1, ...; PART selects the
// statistics folded into acc.  With BW_SUMS it also stores each word's open
// mask at mb[32 gi + lane] while gi < gmax.  Returns the number of groups.
template <int NWARP, int SEARCH_BC, int PART>
__device__ __forceinline__ uint32_t bulk_pass(const uint32_t *win, uint32_t KW, uint32_t ks, uint32_t ke, int warp,
                                              bool ball, uint32_t bb, uint32_t one, uint32_t *mb, uint32_t gmax,
                                              SubAcc &acc)
{
    const int lane = threadIdx.x & 31;
    const uint32_t wbeg = ks >> 5, wend = (ke + 31) >> 5;
    uint32_t gi = 0;
    // with BW_SUMS the pass starts with acc's sums at zero: it adds the sum
    // of p over its words to acc.sum, sum_b b T(b) to acc.wsum, and the word
    // weights at the end
    PosAcc pa;
    pa.G = 0u;
    for (uint32_t wb = wbeg + 32u * warp; wb < wend; wb += 32u * NWARP, gi++) {
        const uint32_t w = wb + lane;
        const bool inw = w < wend;
        uint32_t valid = 0u;
        if (inw) {
            const uint32_t kw0 = 32u * w;
            valid = (kw0 + 32u <= ke) ? 0xffffffffu : (0xffffffffu >> (32u - (ke - kw0)));
        }
        const uint32_t wl = w - wbeg;
        const uint32_t wr = inw ? w : wend - 1u;
        const uint32_t U = ball ? bulk_word<SEARCH_BC, true, PART>(win, wr, wl, gi, KW, valid, bb, one, acc, pa)
                                : bulk_word<SEARCH_BC, false, PART>(win, wr, wl, gi, KW, valid, bb, one, acc, pa);
        if (PART & BW_SUMS) {
            if (gi < gmax) mb[32u * gi + lane] = U;
            if ((gi & (PosAcc::CAP - 1u)) == PosAcc::CAP - 1u) pos_flush(pa, PosAcc::CAP, acc);
        }
    }
    if (PART & BW_SUMS) {
        // words since the last flush
        if (gi & (PosAcc::CAP - 1u)) pos_flush(pa, gi & (PosAcc::CAP - 1u), acc);
        // word gi of this lane is wl = wl0 + 32 NWARP gi: its n weigh
        // 32 wl + b + 1 = (32 wl0 + 1) + 1024 NWARP gi + b
        const uint32_t wl0 = 32u * (uint32_t)warp + (uint32_t)lane;
        acc.wsum += acc.sum * (32ull * wl0 + 1ull) + (unsigned long long)pa.G * (1024ull * NWARP);
    }
    return gi;
}

// Search every n of a tile whose window is built, and reduce it into its
// record(s).  Run by a group of NWARP warps (the whole CTA, BAR = 0, or the
// searching warps of the pipelined kernel); `warp` and `gt` are the warp's
// and the thread's index in the group.  ONE_LOOP: the per-n search in one
// loop, for a launch without open-mask slots (the allocation-free entry
// point); otherwise both search forms store open masks and finish the open n
// in a second pass.
template <int NWARP, int SEARCH_BC, int BAR, bool ONE_LOOP = false>
__device__ __forceinline__ void search_tile(const RangeParams &prm, unsigned long long tile, const Tables &t,
                                            const uint32_t *PR, const uint32_t *win, RedScratch &s,
                                            DevRec *recs, Ctrl *ctrl, int warp, uint32_t gt)
{
    const int lane = threadIdx.x & 31;
    const uint32_t KW = prm.k_words;
    const uint32_t rbits = prm.rec_bits < prm.tile_bits ? prm.rec_bits : prm.tile_bits;
    const bool whole = prm.tile_bits >= prm.rec_bits;
    const unsigned long long rmask = (1ull << prm.rec_bits) - 1ull;
    const uint32_t bb = bulk_bound<SEARCH_BC>(prm);
    const uint32_t i_start = (bb + 1u) >> 1;
    const bool ball = SEARCH_BC && bb >= cand_last(SEARCH_BC ? SEARCH_BC : 1);
    const unsigned long long k0 = tile << prm.tile_bits;
    const unsigned long long left = prm.n_total - k0;
    const uint32_t cnt = left < (1ull << prm.tile_bits) ? (uint32_t)left : (1u << prm.tile_bits);
    const unsigned long long n_lo = prm.n0 + 2ull * k0;

    for (uint32_t ks = 0; ks < cnt; ks += (1u << rbits)) {
        const uint32_t ke = (cnt - ks) < (1u << rbits) ? cnt : ks + (1u << rbits);
        const unsigned long long kg = k0 + ks;
        DevRec *rec = &recs[kg >> prm.rec_bits];
        const unsigned long long kr0 = kg & rmask;
        LaneAcc a;
        a.reset();
        if (gt < HIST_BINS) s.hist[gt] = 0u;
        if (gt == 0) { s.xslow = 0u; s.xce = 0ull; }
        group_sync<BAR, 32 * NWARP>();
        SubAcc acc;
        acc.reset();
        const SubShared ss{s.hist, &s.xslow, &s.xce};
        OpenRing rg{&s.ring[warp][0], 0u, 0u};
        unsigned long long tw = phase_warp(t, -1, 0ull);
        // this warp's open-mask slots (sized by the host for a whole tile)
        const bool has_list = t.olist && blockIdx.x < t.olist_ctas;
        uint32_t *mb = has_list ? t.olist + ((size_t)blockIdx.x * NWARP + warp) * t.olist_wcap : nullptr;
        const uint32_t gmax = has_list ? t.olist_wcap / 32u : 0u;
        if (SEARCH_BC == 0 && !ONE_LOOP) {
            // per-n search: first chunk per lane, then the open n through the
            // ring from candidate 32, as in the bit-parallel search
            uint32_t gi = pern_first<NWARP>(win, PR, KW, n_lo, ks, ke, warp, mb, gmax, prm, acc, ss);
            if (gi > gmax) {                                 // the host sized the slots too small
                if (lane == 0) atomicOr(&ctrl->flags, F_INTERNAL);
                gi = gmax;
            }
            __syncwarp();
            tw = phase_warp(t, PH_WARP_BULK, tw);
            ring_groups<NWARP>(rg, mb, 0u, gi, (ks >> 5) + 32u * warp, win, PR, KW, n_lo, ks, 32u, prm, acc, ss, ctrl);
            ring_flush(rg, win, PR, KW, n_lo, ks, 32u, prm, acc, ss, ctrl);
            tw = phase_warp(t, PH_WARP_TAIL, tw);
        } else if (SEARCH_BC == 0) {
            // no open-mask slots: the per-n search in one loop
            pern_groups<NWARP>(rg, warp, win, PR, KW, n_lo, ks, ke, prm, acc, ss, ctrl);
            ring_flush(rg, win, PR, KW, n_lo, ks, 32u, prm, acc, ss, ctrl);
            tw = phase_warp(t, PH_WARP_TAIL, tw);
        } else {
            const uint32_t one = s.one;                       // 1, a value the compiler cannot see
            uint32_t gi = bulk_pass<NWARP, SEARCH_BC, BW_SUMS>(win, KW, ks, ke, warp, ball, bb, one, mb, gmax, acc);
            if (gi > gmax) {                                 // the host sized the slots too small
                if (lane == 0) atomicOr(&ctrl->flags, F_INTERNAL);
                gi = gmax;
            }
            __syncwarp();
            tw = phase_warp(t, PH_WARP_BULK, tw);
            ring_groups<NWARP>(rg, mb, 0u, gi, (ks >> 5) + 32u * warp, win, PR, KW, n_lo, ks, i_start, prm, acc, ss,
                               ctrl);
            ring_flush(rg, win, PR, KW, n_lo, ks, i_start, prm, acc, ss, ctrl);
            // Every p_min the per-n walk found exceeds every bit-parallel one
            // (it is above bb), so the warp's largest p_min comes from the
            // bit-parallel pass only when the walk found none; then that pass
            // runs again for the max alone.  At scale nearly every warp has
            // open n, and the per-word max stays out of the main loop.
            if (!__any_sync(GB_FULL_MASK, acc.mx > bb))
                bulk_pass<NWARP, SEARCH_BC, BW_MAX>(win, KW, ks, ke, warp, ball, bb, one, mb, 0u, acc);
            tw = phase_warp(t, PH_WARP_TAIL, tw);
        }
        a.mx = acc.mx;
        a.arg = acc.mx ? kr0 + acc.arg : ~0ull;
        a.sum = acc.sum;
        a.wsum = acc.wsum + kr0 * acc.sum;
        a.hA = (unsigned long long)acc.h[0] | ((unsigned long long)acc.h[1] << 32);
        a.hB = (unsigned long long)acc.h[2] | ((unsigned long long)acc.h[3] << 32);
        reduce_group<NWARP, BAR>(a, s, rec, ke - ks, whole, ctrl, warp, &t);
    }
}

// Build the window of one tile.  Run by threads [0, NT) of the CTA, which
// meet at barrier BAR; ends with that barrier.
template <int WHEEL, int NT, int BAR>
__device__ __forceinline__ void build_tile(const RangeParams &prm, unsigned long long tile, const Tables &t,
                                           const uint32_t *wpat, uint32_t *win, Ctrl *ctrl)
{
    const uint32_t KW = prm.k_words;
    const unsigned long long k0 = tile << prm.tile_bits;
    const unsigned long long left = prm.n_total - k0;
    const uint32_t cnt = left < (1ull << prm.tile_bits) ? (uint32_t)left : (1u << prm.tile_bits);
    const unsigned long long n_lo = prm.n0 + 2ull * k0;
    const WinGeom g = tile_geom(n_lo, cnt, 32u * KW);
    unsigned long long b0 = 0, b1 = 0;
    if (prm.bk_ent) {
        b0 = prm.bk_off[tile - prm.tile0];
        b1 = prm.bk_off[tile - prm.tile0 + 1];
    }
    build_window<WHEEL, NT, BAR>(win, wpat, g, t, prm.bk_prime0, prm.bk_ent, b0, b1, ctrl);
}

// One tile: build its window, search every n, reduce into its record(s).
// Called by every thread of the CTA (it contains barriers).
template <int WHEEL, int NT, int SEARCH_BC, bool ONE_LOOP = false>
__device__ __forceinline__ void run_tile(const RangeParams &prm, unsigned long long tile, const Tables &t,
                                         const uint32_t *wpat, const uint32_t *PR, uint32_t *win,
                                         RedScratch &s, DevRec *recs, Ctrl *ctrl)
{
    build_tile<WHEEL, NT, 0>(prm, tile, t, wpat, win, ctrl);
    search_tile<NT / 32, SEARCH_BC, 0, ONE_LOOP>(prm, tile, t, PR, win, s, recs, ctrl, (int)(threadIdx.x >> 5),
                                                 threadIdx.x);
}

// SEARCH_BC = 0: per-n search (one lane per n, 32 candidates per step).
// SEARCH_BC = 4, 6, 8: bit-parallel search of the candidates p < 64 SEARCH_BC
// (one lane per 32 n), the rest per n after warp compaction.
// 512-thread CTAs are built for two per SM (64 registers a thread), so that with
// tiles of at most 2^19 n one CTA can build its window while the other searches.
template <int NT> constexpr int min_ctas() { return NT == 512 ? 2 : 1; }

template <int WHEEL, int NT, int SEARCH_BC, bool ONE_LOOP = false>
__global__ void __launch_bounds__(NT, min_ctas<NT>())
persistent_kernel(const RangeParams *__restrict__ prm_g, Tables t, DevRec *__restrict__ recs,
                  Ctrl *ctrl)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ RedScratch s;
    constexpr uint32_t WP = pattern_block_words<WHEEL>();
    dbg_begin(prm_g->dbg_lim);
    // the call's parameters live in shared memory, not in registers
    if (threadIdx.x == 0) { s.prm = *prm_g; s.one = 1u; }
    const RangeParams &prm = s.prm;
    const uint32_t KW = prm_g->k_words;
    uint32_t *wpat = smem;
    uint32_t *PR = wpat + WP;
    uint32_t *win = PR + ((KW + 3) & ~3u);
    build_wheel_pattern<WHEEL, NT>(wpat);
    for (uint32_t i = threadIdx.x; i < KW; i += NT) PR[i] = t.PR[i];
    phase_mark(t, -1, threadIdx.x == 0);
    for (;;) {
        if (threadIdx.x == 0)
            s.tile = prm.tile0 + (prm.claim ? atomicAdd_system(prm.claim, 1ull) : atomicAdd(&ctrl->tile_ctr, 1ull));
        __syncthreads();
        phase_mark(t, PH_CLAIM, threadIdx.x == 0);
        const unsigned long long tile = s.tile;
        if (tile >= prm.tile_end) break;
        run_tile<WHEEL, NT, SEARCH_BC, ONE_LOOP>(prm, tile, t, wpat, PR, win, s, recs, ctrl);
        if (threadIdx.x == 0 && prm.progress) atomicAdd_system(prm.progress, 1ull);
    }
    dbg_end(ctrl);
}

// ---------------------------------------------------------------------------
// pipelined persistent kernel: warp-specialised, two window buffers
// ---------------------------------------------------------------------------
//
// The window build is bound by shared-memory atomics and the search by
// instruction issue, so the two overlap: warps [0, NP) (builders) sieve the
// window of the CTA's next tile into one buffer while warps [NP, NP + NC)
// (searchers) search the current tile in the other; the whole CTA meets once
// per tile and the buffers swap.  The builders meet at named barrier 1, the
// searchers at named barrier 2.  Tiles are claimed from the same device atomic
// counter as the persistent kernel (one tile ahead), so records, order of
// folding and results are identical.  Two windows must fit in shared memory:
// tiles of at most 2^19 n at P_max = 2^16.
template <int NP, int NC> constexpr int pipe_threads() { return 32 * (NP + NC); }

template <int WHEEL, int NP, int NC, int SEARCH_BC>
__global__ void __launch_bounds__(pipe_threads<NP, NC>(), 1)
pipe_kernel(const RangeParams *__restrict__ prm_g, Tables t, DevRec *__restrict__ recs, Ctrl *ctrl)
{
    constexpr int NT = pipe_threads<NP, NC>();
    constexpr int NPT = 32 * NP, NCT = 32 * NC;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ RedScratch s;
    __shared__ unsigned long long s_tile[2];
    constexpr uint32_t WP = pattern_block_words<WHEEL>();
    dbg_begin(prm_g->dbg_lim);
    if (threadIdx.x == 0) { s.prm = *prm_g; s.one = 1u; }
    const RangeParams &prm = s.prm;
    const uint32_t KW = prm_g->k_words;
    const uint32_t WW = pipe_window_words(prm_g->tile_bits, KW);
    uint32_t *wpat = smem;
    uint32_t *PR = wpat + WP;
    // buffer b is win0 + b WW: computed from the shared-memory base (an array
    // of the two pointers would hide that they point to shared memory, and
    // every access would become a generic one)
    uint32_t *win0 = PR + ((KW + 3) & ~3u);
    build_wheel_pattern<WHEEL, NT>(wpat);
    for (uint32_t i = threadIdx.x; i < KW; i += NT) PR[i] = t.PR[i];
    const int warp = (int)(threadIdx.x >> 5);
    const bool builder = warp < NP;
    if (threadIdx.x == 0)
        s_tile[0] = prm_g->tile0 + (prm_g->claim ? atomicAdd_system(prm_g->claim, 1ull) : atomicAdd(&ctrl->tile_ctr, 1ull));
    __syncthreads();
    if (builder && s_tile[0] < prm.tile_end) build_tile<WHEEL, NPT, 1>(prm, s_tile[0], t, wpat, win0, ctrl);
    __syncthreads();
    for (uint32_t k = 0;; k++) {
        const unsigned long long tile = s_tile[k & 1u];
        if (tile >= prm.tile_end) break;
        if (builder) {
            if (threadIdx.x == 0)
                s_tile[(k + 1u) & 1u] =
                    prm.tile0 + (prm.claim ? atomicAdd_system(prm.claim, 1ull) : atomicAdd(&ctrl->tile_ctr, 1ull));
            group_sync<1, NPT>();
            const unsigned long long next = s_tile[(k + 1u) & 1u];
            if (next < prm.tile_end)
                build_tile<WHEEL, NPT, 1>(prm, next, t, wpat, win0 + ((k & 1u) ? 0u : WW), ctrl);
        } else {
            const uint32_t gt = threadIdx.x - NPT;
            search_tile<NC, SEARCH_BC, 2>(prm, tile, t, PR, win0 + ((k & 1u) ? WW : 0u), s, recs, ctrl, warp - NP, gt);
            if (gt == 0 && prm.progress) atomicAdd_system(prm.progress, 1ull);
        }
        __syncthreads();
    }
    dbg_end(ctrl);
    (void)NCT;
}

// Serving: CTAs claim work items (slot, tile) of the admitted requests from a
// device counter, so the tiles of many requests share one persistent launch;
// each tile folds into its request's record with atomics, and raises its
// status flags and counterexample in the request's own control block.
template <int WHEEL, int NT, int SEARCH_BC>
__global__ void __launch_bounds__(NT, min_ctas<NT>())
serve_kernel(const unsigned long long *__restrict__ items, unsigned long long n_items, SlotDev *slots,
             Tables t, Ctrl *ctrl)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ RedScratch s;
    constexpr uint32_t WP = pattern_block_words<WHEEL>();
    const uint32_t KW = t.k_words;
    uint32_t *wpat = smem;
    uint32_t *PR = wpat + WP;
    uint32_t *win = PR + ((KW + 3) & ~3u);
    dbg_begin(0u);
    build_wheel_pattern<WHEEL, NT>(wpat);
    for (uint32_t i = threadIdx.x; i < KW; i += NT) PR[i] = t.PR[i];
    if (threadIdx.x == 0) s.one = 1u;
    Ctrl *last_ctl = nullptr;                    // thread 0: the request of the CTA's last tile
    for (;;) {
        __syncthreads();                         // every thread is done with the last tile's params
        if (threadIdx.x == 0) {
            dbg_report(last_ctl);                // a failed bounds check of that tile fails its request
            const unsigned long long i = atomicAdd(&ctrl->work_ctr, 1ull);
            s.tile = i;
            if (i < n_items) s.prm = slots[items[i] >> SERVE_SLOT_SHIFT].prm;
        }
        __syncthreads();
        const unsigned long long idx = s.tile;
        if (idx >= n_items) break;
        const unsigned long long item = items[idx];
        const unsigned long long slot = item >> SERVE_SLOT_SHIFT;
        const unsigned long long tile = item & ((1ull << SERVE_SLOT_SHIFT) - 1ull);
        if (threadIdx.x == 0) last_ctl = &slots[slot].ctl;
        run_tile<WHEEL, NT, SEARCH_BC>(s.prm, tile, t, wpat, PR, win, s, &slots[slot].acc, &slots[slot].ctl);
    }
}

}  // namespace gbk
