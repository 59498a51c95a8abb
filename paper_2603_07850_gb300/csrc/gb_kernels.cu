// gb_kernels.cu -- CUDA kernels of the Goldbach range verifier (sm_103a).
//
// persistent_kernel : the fused hot path.  A grid of (SMs x CTAs/SM) CTAs
//                     claims tiles from one device atomic counter -- the
//                     on-device form of the paper's lock-free work pool
//                     (Sec. 3.2, Alg. 1) -- and for each tile builds the sieve
//                     window in shared memory, finds p_min for every even n,
//                     finishes over-bound n on the spot, and reduces the tile
//                     to its records.  No host round trip per tile.
// merge_kernel      : folds the records of a call into one gb_result.
// plain_*           : the per-segment baseline (sieve -> global bitset,
//                     search -> p_min array, reduce -> records), launched by a
//                     host loop that synchronises on a status word per segment
//                     (paper Alg. 1).
// table_*           : base-prime table builder (segmented sieve + compaction).
#include <stdint.h>
#include <cuda_runtime.h>

#include "gb_device.cuh"
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

// Zero the control block and (when tiles share records) the records.
__global__ void clear_kernel(const RangeParams *__restrict__ prm_g, DevRec *recs, Ctrl *ctrl,
                             int clear_records)
{
    const RangeParams prm = *prm_g;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (tid == 0) {
        ctrl->tile_ctr = 0; ctrl->ce_inv = 0; ctrl->slow_total = 0; ctrl->flags = 0;
        ctrl->merge_done = 0; ctrl->work_ctr = 0;
        ctrl->dbg_site = 0; ctrl->dbg_off = 0;
    }
    if (!clear_records) return;
    const unsigned long long words = prm.nrec * (sizeof(DevRec) / 16);
    uint4 *p = reinterpret_cast<uint4 *>(recs);
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (unsigned long long i = tid; i < words; i += (unsigned long long)gridDim.x * blockDim.x) p[i] = z;
}

// ---------------------------------------------------------------------------
// merge: records -> gb_result
// ---------------------------------------------------------------------------

struct MergePart {
    unsigned long long best_p, best_n, sum, wsum, n_count, n_slow, ce;
    unsigned long long hist[HIST_BINS];
};

__device__ __forceinline__ bool better(unsigned long long p, unsigned long long n,
                                       unsigned long long bp, unsigned long long bn)
{
    return p > bp || (p == bp && p != 0 && n < bn);
}

__global__ void __launch_bounds__(256)
merge_kernel(const RangeParams *__restrict__ prm_g, const DevRec *__restrict__ recs, Ctrl *ctrl,
             MergePart *parts, gb_result *out)
{
    __shared__ unsigned long long s_hist[HIST_BINS];
    __shared__ unsigned long long s_bp[8], s_bn[8], s_sum[8], s_wsum[8], s_cnt[8], s_slow[8], s_ce[8];
    __shared__ int s_last;
    const RangeParams prm = *prm_g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < HIST_BINS) s_hist[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long bp = 0, bn = ~0ull, sum = 0, wsum = 0, cnt = 0, slow = 0, ce = 0;
    for (unsigned long long r = blockIdx.x * 256ull + threadIdx.x; r < prm.nrec;
         r += (unsigned long long)gridDim.x * 256ull) {
        const DevRec &R = recs[r];
        const unsigned long long kfirst = r << prm.rec_bits;
        const unsigned long long key = R.key;
        if (key) {
            unsigned long long p = key >> KEY_SHIFT;
            unsigned long long n = prm.n0 + 2ull * (kfirst + (KEY_KMASK - (key & KEY_KMASK)));
            if (better(p, n, bp, bn)) { bp = p; bn = n; }
        }
        sum += R.sum;
        wsum += R.wsum + R.sum * kfirst;
        cnt += R.n_count;
        slow += R.n_slow;
        ce = R.ce_inv > ce ? R.ce_inv : ce;
        for (int b = 0; b < HIST_BINS; b++)
            if (R.hist[b]) atomicAdd(&s_hist[b], R.hist[b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long op = __shfl_xor_sync(GB_FULL_MASK, bp, o);
        unsigned long long on = __shfl_xor_sync(GB_FULL_MASK, bn, o);
        if (better(op, on, bp, bn)) { bp = op; bn = on; }
        sum += __shfl_xor_sync(GB_FULL_MASK, sum, o);
        wsum += __shfl_xor_sync(GB_FULL_MASK, wsum, o);
        cnt += __shfl_xor_sync(GB_FULL_MASK, cnt, o);
        slow += __shfl_xor_sync(GB_FULL_MASK, slow, o);
        unsigned long long oc = __shfl_xor_sync(GB_FULL_MASK, ce, o);
        ce = oc > ce ? oc : ce;
    }
    if (lane == 0) {
        s_bp[warp] = bp; s_bn[warp] = bn; s_sum[warp] = sum; s_wsum[warp] = wsum;
        s_cnt[warp] = cnt; s_slow[warp] = slow; s_ce[warp] = ce;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) {
            if (better(s_bp[w], s_bn[w], bp, bn)) { bp = s_bp[w]; bn = s_bn[w]; }
            sum += s_sum[w]; wsum += s_wsum[w]; cnt += s_cnt[w]; slow += s_slow[w];
            ce = s_ce[w] > ce ? s_ce[w] : ce;
        }
        MergePart &P = parts[blockIdx.x];
        P.best_p = bp; P.best_n = bn; P.sum = sum; P.wsum = wsum; P.n_count = cnt;
        P.n_slow = slow; P.ce = ce;
    }
    if (threadIdx.x < HIST_BINS) parts[blockIdx.x].hist[threadIdx.x] = s_hist[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&ctrl->merge_done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned long long fp = 0, fn = ~0ull, fs = 0, fw = 0, fc = 0, fsl = 0, fce = 0;
        for (unsigned int b = 0; b < gridDim.x; b++) {
            const volatile MergePart &P = parts[b];
            if (better(P.best_p, P.best_n, fp, fn)) { fp = P.best_p; fn = P.best_n; }
            fs += P.sum; fw += P.wsum; fc += P.n_count; fsl += P.n_slow;
            fce = P.ce > fce ? P.ce : fce;
        }
        out->n_first = prm.n_total ? prm.n0 : 0;
        out->n_count = fc;
        out->max_pmin = fp;
        out->argmax_n = fp ? fn : 0;
        out->sum_pmin = fs;
        out->wsum_pmin = fw;
        out->n_slow = fsl;
        const unsigned long long ci = fce > ctrl->ce_inv ? fce : ctrl->ce_inv;
        const unsigned long long cen = ci ? ~ci : 0ull;
        out->counterexample_n = cen;
        const unsigned int f = ctrl->flags;
        int st = GB_OK;
        if (f & F_INTERNAL) st = GB_EINTERNAL;
        else if (f & F_SLOWCAP) st = GB_ESLOWPATH_LIMIT;
        else if (f & F_OVERFLOW) st = GB_EOVERFLOW;
        else if ((f & F_COUNTEREX) || cen) st = GB_COUNTEREXAMPLE;
        out->status = st;
        out->reserved = 0;
        out->submit_ns = 0;
        out->done_ns = 0;
    }
    if (threadIdx.x < 64) {
        unsigned long long h = 0;
        if (threadIdx.x < HIST_BINS)
            for (unsigned int b = 0; b < gridDim.x; b++)
                h += ((const volatile MergePart &)parts[b]).hist[threadIdx.x];
        out->hist[threadIdx.x] = h;
    }
}

// ---------------------------------------------------------------------------
// plain per-segment form
// ---------------------------------------------------------------------------

// Window slice [z0, z0 + Z) of a window described by (half_abs, neg, j_end).
__device__ __forceinline__ WinGeom slice_geom(unsigned long long half_abs, bool neg, uint32_t j_end,
                                              uint32_t z0, uint32_t Z)
{
    unsigned long long h2;
    bool n2;
    if (neg) {
        n2 = half_abs > z0;
        h2 = n2 ? half_abs - z0 : z0 - half_abs;
    } else {
        n2 = false;
        h2 = half_abs + z0;
    }
    uint32_t je = j_end - z0 < Z ? j_end - z0 : Z;
    return make_geom(h2, n2, je);
}

// One CTA builds slice blockIdx.x of the window in shared memory and flushes
// it to the global bitset with 16-byte stores.
template <int WHEEL, int NT>
__global__ void __launch_bounds__(NT, 1)
slice_sieve_kernel(unsigned long long half_abs, int neg, uint32_t j_end, uint32_t Z, Tables t,
                   uint32_t *__restrict__ gwin, uint32_t gwords, Ctrl *ctrl)
{
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr uint32_t WP = pattern_block_words<WHEEL>();
    uint32_t *wpat = smem;
    uint32_t *win = smem + WP;
    dbg_begin(0u);
    build_wheel_pattern<WHEEL, NT>(wpat);
    __syncthreads();
    const uint32_t z0 = blockIdx.x * Z;
    const WinGeom g = slice_geom(half_abs, neg != 0, j_end, z0, Z);
    build_window<WHEEL, NT>(win, wpat, g, t);
    // words of this slice: Z/32, except the last slice which also writes its
    // trailing zero word(s); never write a word owned by the next slice.
    const uint32_t w0 = z0 >> 5;
    uint32_t nw = (z0 + Z >= j_end) ? g.nfill : (Z >> 5);
    if (w0 + nw > gwords) nw = gwords - w0;
    const uint32_t n4 = nw >> 2;
    uint4 *dst = reinterpret_cast<uint4 *>(gwin + w0);
    const uint4 *src = reinterpret_cast<const uint4 *>(win);
    for (uint32_t i = threadIdx.x; i < n4; i += NT) dst[i] = src[i];
    for (uint32_t i = 4 * n4 + threadIdx.x; i < nw; i += NT) gwin[w0 + i] = win[i];
    dbg_end(ctrl);
}

// Entry of the plain form's p_min array for an n whose slow path gave up.
constexpr uint32_t PM_GAVE_UP = 0xffffffffu;

// p_min for every n of a plain segment, read from the global window bitset:
// the per-n search with warp compaction (first chunk of 32 candidates per
// lane; the n left open finish in full rounds of 32 from candidate 32 on).
__global__ void __launch_bounds__(256)
plain_search_kernel(const RangeParams *__restrict__ prm_g, const uint32_t *__restrict__ gwin,
                    const uint32_t *__restrict__ PR, unsigned long long n_lo, uint32_t cnt,
                    uint32_t *__restrict__ pm_out, Ctrl *ctrl)
{
    __shared__ uint32_t ring[8][64];
    const RangeParams prm = *prm_g;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t KW = prm.k_words, PR0 = PR[0];
    const uint32_t nchunks = (cnt + 31) >> 5;
    uint32_t *q = ring[warp];
    uint32_t head = 0, tail = 0;
    auto finish = [&](uint32_t kk, bool act) {
        bool gave_up;
        const uint32_t pm = tail_pmin(gwin, PR, KW, kk, act, n_lo, 32u, prm, ctrl, gave_up);
        if (act) pm_out[kk] = gave_up ? PM_GAVE_UP : pm;
    };
    for (uint32_t g32 = blockIdx.x * 8u + warp; g32 < nchunks; g32 += gridDim.x * 8u) {
        const uint32_t k = (g32 << 5) + lane;
        const bool valid = k < cnt;
        const unsigned long long n = n_lo + 2ull * k;
        uint32_t pm = 0;
        if (valid && n != 4ull) {
            const uint32_t m = __funnelshift_r(gwin[g32 + KW - 1u], gwin[g32 + KW], lane) & PR0;
            if (m) pm = 2u * __clz(m) + 1u;
        }
        if (pm) pm_out[k] = pm;
        const bool open = valid && pm == 0u;
        const uint32_t has = __ballot_sync(GB_FULL_MASK, open);
        if (open) q[(tail + __popc(has & below)) & 63u] = k;
        tail += __popc(has);
        if (tail - head >= 32u) {
            __syncwarp();
            const uint32_t kk = q[(head + lane) & 63u];
            __syncwarp();
            finish(kk, true);
            head += 32u;
        }
    }
    __syncwarp();
    if (tail != head) finish(q[(head + lane) & 63u], lane < tail - head);
}

// Plain form with the bit-parallel search: the CTAs take sub-tiles of 2^(
// prm.tile_bits) n of the segment and search each in the segment's global
// window bitset (sub-tile u starts at word u 2^(tile_bits - 5)) with the
// persistent kernel's search and reduction, folding into the (zeroed)
// records.  One launch replaces the per-n search and the reduce kernel.
template <int NT, int BC>
__global__ void __launch_bounds__(NT, 1)
plain_bulk_kernel(RangeParams prm, unsigned long long tile_first, uint32_t nsub, Tables t,
                  const uint32_t *__restrict__ gwin, DevRec *recs, Ctrl *ctrl)
{
    extern __shared__ __align__(16) uint32_t PRs[];
    __shared__ RedScratch s;
    dbg_begin(prm.dbg_lim);
    for (uint32_t i = threadIdx.x; i < prm.k_words; i += NT) PRs[i] = t.PR[i];
    if (threadIdx.x == 0) s.one = 1u;
    __syncthreads();
    for (uint32_t u = blockIdx.x; u < nsub; u += gridDim.x) {
        search_tile<NT / 32, BC, 0>(prm, tile_first + u, t, PRs, gwin + ((size_t)u << (prm.tile_bits - 5)), s, recs,
                                    ctrl, (int)(threadIdx.x >> 5), threadIdx.x);
        __syncthreads();
    }
    dbg_end(ctrl);
}

// Reduce chunks of the p_min array into (zeroed) records with atomics.
template <int NT>
__global__ void __launch_bounds__(NT)
plain_reduce_kernel(const RangeParams *__restrict__ prm_g, const uint32_t *__restrict__ pm,
                    unsigned long long k_seg0, unsigned long long n_lo, uint32_t cnt,
                    uint32_t chunk, DevRec *recs, Ctrl *ctrl)
{
    __shared__ RedScratch s;
    const RangeParams prm = *prm_g;
    const uint32_t rbits = prm.rec_bits;
    const unsigned long long rmask = (1ull << rbits) - 1ull;
    // chunk boundaries never straddle a record: chunk divides 2^rec_bits or vice versa
    const uint32_t ks = blockIdx.x * chunk;
    if (ks >= cnt) return;
    const uint32_t ke = cnt - ks < chunk ? cnt : ks + chunk;
    const unsigned long long kg = k_seg0 + ks;
    DevRec *rec = &recs[kg >> rbits];
    const unsigned long long kr0 = kg & rmask;
    LaneAcc a;
    a.reset();
    if (threadIdx.x < HIST_BINS) s.hist[threadIdx.x] = 0u;
    if (threadIdx.x == 0) { s.xslow = 0u; s.xce = 0ull; }
    __syncthreads();
    for (uint32_t k = ks + threadIdx.x; k < ke; k += NT) {
        const uint32_t p = pm[k];
        if (p == PM_GAVE_UP) continue;                     // slow path gave up: the call fails
        if (p) a.add(p, kr0 + (k - ks), prm.p_max, s.hist);
        else a.ce = a.ce > ~(n_lo + 2ull * k) ? a.ce : ~(n_lo + 2ull * k);
    }
    reduce_to_record<NT>(a, s, rec, ke - ks, false, ctrl);
}

// ---------------------------------------------------------------------------
// base-prime table: compaction of a sieved bitset of odd numbers
// ---------------------------------------------------------------------------

constexpr uint32_t TBL_WORDS_PER_BLOCK = 8192;

__global__ void table_count_kernel(const uint32_t *__restrict__ bits, uint32_t nwords,
                                   uint32_t *__restrict__ block_counts)
{
    __shared__ uint32_t s_c;
    if (threadIdx.x == 0) s_c = 0;
    __syncthreads();
    const uint32_t w0 = blockIdx.x * TBL_WORDS_PER_BLOCK;
    uint32_t c = 0;
    for (uint32_t i = threadIdx.x; i < TBL_WORDS_PER_BLOCK && w0 + i < nwords; i += blockDim.x)
        c += __popc(bits[w0 + i]);
    c = __reduce_add_sync(GB_FULL_MASK, c);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_c, c);
    __syncthreads();
    if (threadIdx.x == 0) block_counts[blockIdx.x] = s_c;
}

// Each block re-reads its words; thread i owns 8 consecutive words, a block
// scan of the per-thread counts gives every prime its output slot.
__global__ void __launch_bounds__(1024)
table_scatter_kernel(const uint32_t *__restrict__ bits, uint32_t nwords,
                     const unsigned long long *__restrict__ block_offsets, unsigned long long limit,
                     uint32_t *__restrict__ primes, unsigned long long *__restrict__ recip)
{
    __shared__ uint32_t s_warp[32];
    const uint32_t w0 = blockIdx.x * TBL_WORDS_PER_BLOCK + threadIdx.x * 8u;
    uint32_t wd[8];
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        wd[i] = (w0 + i < nwords) ? bits[w0 + i] : 0u;
        c += __popc(wd[i]);
    }
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(GB_FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(GB_FULL_MASK, v, o);
            if (lane >= o) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    unsigned long long pos = block_offsets[blockIdx.x] + (x - c) + (warp ? s_warp[warp - 1] : 0u);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        uint32_t w = wd[i];
        while (w) {
            const int b = __ffs(w) - 1;
            w &= w - 1;
            const unsigned long long q = 2ull * (32ull * (w0 + i) + b) + 1ull;
            if (q <= limit) {
                primes[pos] = (uint32_t)q;
                recip[pos] = 0xFFFFFFFFFFFFFFFFull / q;
            }
            pos++;
        }
    }
}

// Exclusive scan of n u32 counts into u64 offsets (out[n] = the total), and
// optionally into u32 cursors, by one 1,024-thread block: each thread sums a
// run of ceil(n / 1024) counts, the block scans the run sums (warp shuffles,
// then one warp over the warp totals), and each thread writes its run.  n is
// at most a few tens of thousands (table blocks, bucket tiles).
__global__ void __launch_bounds__(1024) block_scan_kernel(const uint32_t *__restrict__ in, uint32_t n,
                                                          unsigned long long *__restrict__ out,
                                                          unsigned int *__restrict__ cursor)
{
    __shared__ unsigned long long s_w[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (n + 1023u) / 1024u;
    const uint32_t b = threadIdx.x * per;
    const uint32_t e = b + per < n ? b + per : n;
    unsigned long long sum = 0;
    for (uint32_t i = b; i < e; i++) sum += in[i];
    unsigned long long x = sum;                       // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(GB_FULL_MASK, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(GB_FULL_MASK, v, o);
            if ((int)lane >= o) v += y;
        }
        s_w[lane] = v;
    }
    __syncthreads();
    unsigned long long acc = x - sum + (warp ? s_w[warp - 1] : 0ull);
    for (uint32_t i = b; i < e; i++) {
        out[i] = acc;
        if (cursor) cursor[i] = (unsigned int)acc;
        acc += in[i];
    }
    if (threadIdx.x == 1023) out[n] = acc;            // an empty run ends at the total too
}

// ---------------------------------------------------------------------------
// bucket pre-pass for the large base primes (p >= bucket bound): every hit
// of such a prime in the windows of tiles [t0, t0 + nt) becomes one entry
// (window bit index) in that tile's bucket.  Windows overlap by K bits, so a
// hit in the first K - 1 bits of tile t's window is also a hit in the
// extension of tile t - 1.
// ---------------------------------------------------------------------------

struct ChunkGeom {
    unsigned long long w0;     // window base of tile t0 (mod 2^64)
    unsigned long long span;   // q_hi of the last tile - w0 (true distance)
    unsigned long long q_hi;
    uint32_t S, KB, shift, nt;
    bool neg;
};

__device__ __forceinline__ ChunkGeom chunk_geom(const RangeParams &prm, unsigned long long t0, uint32_t nt)
{
    ChunkGeom c;
    c.S = 1u << prm.tile_bits;
    c.KB = 32u * prm.k_words;
    c.shift = prm.tile_bits + 1;
    c.nt = nt;
    const unsigned long long n_lo0 = prm.n0 + 2ull * (t0 << prm.tile_bits);
    const unsigned long long h = n_lo0 >> 1;
    c.neg = h < c.KB;
    const unsigned long long half_abs = c.neg ? (c.KB - h) : (h - c.KB);
    c.w0 = c.neg ? (1ull - 2ull * half_abs) : (2ull * half_abs + 1ull);
    const unsigned long long tl = t0 + nt - 1;
    const unsigned long long kl = tl << prm.tile_bits;
    const unsigned long long left = prm.n_total - kl;
    const unsigned long long cl = left < c.S ? left : c.S;
    const unsigned long long n_last = prm.n0 + 2ull * (kl + cl - 1ull);
    c.q_hi = n_last - 1ull;
    c.span = c.q_hi - c.w0;
    return c;
}

template <class F>
__device__ __forceinline__ void for_each_hit(const ChunkGeom &c, uint32_t p, unsigned long long m, F &&emit)
{
    unsigned long long d = first_dist(c.w0, c.neg, c.q_hi, p, m);
    if (d == ~0ull || d > c.span) return;
    const unsigned long long step = 2ull * p;
    for (;;) {
        // the hit is bit j of tile tt's window and, since consecutive windows
        // overlap by K - 1 bits, bit j + u S of tile tt - u while that stays
        // inside a window (j + u S <= S + K - 2); with K > S that is more
        // than one earlier tile
        unsigned long long tt = d >> c.shift;
        uint32_t j = (uint32_t)((d - (tt << c.shift)) >> 1);
        for (;;) {
            if (tt < c.nt) emit((uint32_t)tt, j);
            if (tt == 0ull || j + 1u >= c.KB) break;
            j += c.S;
            tt--;
        }
        if (c.span - d < step) break;
        d += step;
    }
}

// Count the hits of every bucket prime in the windows of tiles [t0, t0 + nt):
// per block in shared memory, then into counts[k] (all blocks, atomics) and
// into blk[b nt + k] (block b's own count of tile k, all of them written).
template <int NT>
__global__ void __launch_bounds__(NT)
bucket_count_kernel(const RangeParams *__restrict__ prm_g, Tables t, uint32_t i0, unsigned long long t0,
                    uint32_t nt, unsigned int *__restrict__ counts, unsigned int *__restrict__ blk)
{
    extern __shared__ unsigned int h[];
    const RangeParams prm = *prm_g;
    const ChunkGeom c = chunk_geom(prm, t0, nt);
    const uint32_t i1 = count_le(t.primes, t.nprimes, isqrt_u64(c.q_hi));
    for (uint32_t k = threadIdx.x; k < nt; k += NT) h[k] = 0u;
    __syncthreads();
    for (uint32_t i = i0 + blockIdx.x * NT + threadIdx.x; i < i1; i += gridDim.x * NT)
        for_each_hit(c, t.primes[i], t.recip[i], [&](uint32_t tt, uint32_t) { atomicAdd(&h[tt], 1u); });
    __syncthreads();
    unsigned int *mine = blk + (size_t)blockIdx.x * nt;
    for (uint32_t k = threadIdx.x; k < nt; k += NT) {
        mine[k] = h[k];
        if (h[k]) atomicAdd(&counts[k], h[k]);
    }
}

// Turn the blocks' counts into their first entry in each bucket: tile k's
// entries start at off[k], block b's at off[k] + the counts of blocks < b.
__global__ void bucket_block_offsets_kernel(uint32_t nt, uint32_t nblocks, const unsigned long long *__restrict__ off,
                                            unsigned int *__restrict__ blk)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    unsigned int acc = (unsigned int)off[k];         // entries of a chunk stay below 2^32 (host bound)
    for (uint32_t b = 0; b < nblocks; b++) {
        const unsigned int c = blk[(size_t)b * nt + k];
        blk[(size_t)b * nt + k] = acc;
        acc += c;
    }
}

// Block-wide exclusive scan of in[0, n) into out[0, n]; out[n] is the total.
// Each of the NT threads takes a run of consecutive entries; s_w holds 32
// words.  Ends with the block's barrier.
template <int NT>
__device__ __forceinline__ void block_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *s_w)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (n + NT - 1) / NT;
    const uint32_t b = threadIdx.x * per;
    const uint32_t e = b + per < n ? b + per : n;
    uint32_t sum = 0;
    for (uint32_t i = b; i < e; i++) sum += in[i];
    uint32_t x = sum;                                   // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(GB_FULL_MASK, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < NT / 32 ? s_w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(GB_FULL_MASK, v, o);
            if ((int)lane >= o) v += y;
        }
        s_w[lane] = v;
    }
    __syncthreads();
    uint32_t acc = x - sum + (warp ? s_w[warp - 1] : 0u);
    for (uint32_t i = b; i < e; i++) {
        const uint32_t v = in[i];
        out[i] = acc;
        acc += v;
    }
    if (threadIdx.x == NT - 1) out[n] = acc;            // a thread past n holds the total
    __syncthreads();
}

// A thread's position in the enumeration of its primes' entries, in the
// order of for_each_hit: prime index i is the next prime to take; (tt, j)
// is the current entry of the hit at distance d of prime p (p = 0: none).
struct HitCursor {
    unsigned long long d;
    uint32_t i, p, tt, j;
};

__device__ __forceinline__ void cursor_entry(HitCursor &h, const ChunkGeom &c)
{
    h.tt = (uint32_t)(h.d >> c.shift);
    h.j = (uint32_t)((h.d - ((unsigned long long)h.tt << c.shift)) >> 1);
}

// Move to the first entry of the next prime that hits the chunk; false when
// the thread's primes are used up.
__device__ __forceinline__ bool cursor_prime(HitCursor &h, const ChunkGeom &c, const Tables &t, uint32_t i1,
                                             uint32_t stride)
{
    while (h.i < i1) {
        const uint32_t p = t.primes[h.i];
        const unsigned long long m = t.recip[h.i];
        h.i += stride;                                  // i1 < 2^28, stride < 2^20: no wrap
        const unsigned long long d = first_dist(c.w0, c.neg, c.q_hi, p, m);
        if (d == ~0ull || d > c.span) continue;
        h.p = p;
        h.d = d;
        cursor_entry(h, c);
        return true;
    }
    h.p = 0;
    return false;
}

// Step past the current entry: the same hit in the earlier overlapping
// window, else the prime's next hit, else the next prime.
__device__ __forceinline__ bool cursor_next(HitCursor &h, const ChunkGeom &c, const Tables &t, uint32_t i1,
                                            uint32_t stride)
{
    if (h.tt != 0u && h.j + 1u < c.KB) {
        h.j += c.S;
        h.tt--;
        return true;
    }
    if (c.span - h.d < 2ull * h.p) return cursor_prime(h, c, t, i1, stride);
    h.d += 2ull * h.p;
    cursor_entry(h, c);
    return true;
}

// Write the entries, staged in rounds.  Block b takes the primes of the
// count kernel's blocks FOLD b .. FOLD b + FOLD - 1 (its NT threads are
// theirs, the grid is theirs / FOLD), so its share of tile k's bucket
// starts at blk[FOLD b][k].  In each round every thread enumerates its next
// H entries for this chunk's tiles; the block counts them per tile, ranks
// them with a scan, enumerates them again into a tile-sorted staging area in
// shared memory and copies that out, so the entries of one tile leave the
// block as a run of consecutive slots and the stores coalesce.  The order of
// the entries inside a bucket is free: each one clears one bit.
template <int NT, int H, int FOLD>
__global__ void __launch_bounds__(NT, 1)
bucket_fill_staged_kernel(const RangeParams *__restrict__ prm_g, Tables t, uint32_t i0, unsigned long long t0,
                          uint32_t nt, const unsigned int *__restrict__ blk, uint32_t *__restrict__ ent,
                          unsigned long long cap, Ctrl *ctrl)
{
    extern __shared__ uint32_t sm[];
    uint32_t *pos = sm;                                 // [nt] next slot of this block in tile k's bucket
    uint32_t *cnt = pos + nt;                           // [nt] entries of tile k in this round
    uint32_t *base = cnt + nt;                          // [nt + 1] first staging slot of tile k
    uint32_t *s_w = base + nt + 1;                      // [32] scan scratch
    uint32_t *sj = s_w + 32;                            // [NT H] staged window bits, by tile
    uint16_t *stt = (uint16_t *)(sj + NT * H);          // [NT H] their tiles (nt <= 2^16)
    const RangeParams prm = *prm_g;
    const ChunkGeom c = chunk_geom(prm, t0, nt);
    const uint32_t i1 = count_le(t.primes, t.nprimes, isqrt_u64(c.q_hi));
    const unsigned int *mine = blk + (size_t)blockIdx.x * FOLD * nt;
    dbg_begin(0u);
    for (uint32_t k = threadIdx.x; k < nt; k += NT) {
        pos[k] = mine[k];
        cnt[k] = 0u;
    }
    const uint32_t stride = gridDim.x * NT;
    HitCursor h;
    h.i = i0 + blockIdx.x * NT + threadIdx.x;
    h.p = h.tt = h.j = 0u;
    h.d = 0ull;
    bool live = cursor_prime(h, c, t, i1, stride);
    bool over = false;
    __syncthreads();
    for (;;) {
        const HitCursor h0 = h;
        const bool live0 = live;
        for (int e = 0; live && e < H;) {               // count
            if (h.tt < nt) {
                atomicAdd(&cnt[h.tt], 1u);
                e++;
            }
            live = cursor_next(h, c, t, i1, stride);
        }
        if (!__syncthreads_or(live0)) break;            // uniform: every thread sees the same
        block_exclusive_scan<NT>(cnt, base, nt, s_w);
        for (uint32_t k = threadIdx.x; k < nt; k += NT) cnt[k] = 0u;
        __syncthreads();
        HitCursor g = h0;                               // the same entries again, now placed
        bool l = live0;
        for (int e = 0; l && e < H;) {
            if (g.tt < nt) {
                const uint32_t r = base[g.tt] + atomicAdd(&cnt[g.tt], 1u);
                if (dbg_check(r < NT * H, DS_STAGE, r)) {
                    sj[r] = g.j;
                    stt[r] = (uint16_t)g.tt;
                }
                e++;
            }
            l = cursor_next(g, c, t, i1, stride);
        }
        __syncthreads();
        const uint32_t total = base[nt];
        for (uint32_t k = threadIdx.x; k < total; k += NT) {
            const uint32_t tt = stt[k];
            const unsigned long long e = (unsigned long long)pos[tt] + (k - base[tt]);
            if (e < cap) __stcs(&ent[e], sj[k]);
            else over = true;
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < nt; k += NT) {
            pos[k] += base[k + 1] - base[k];
            cnt[k] = 0u;
        }
        __syncthreads();
    }
    if (over) atomicOr(&ctrl->flags, F_INTERNAL);       // the host's capacity bound failed
    dbg_end(ctrl);
}

constexpr int FILL_NT = 1024, FILL_H = 16, FILL_FOLD = FILL_NT / 256;
constexpr uint32_t FILL_MAX_TILES = 8192;     // the largest bucket chunk (192 KB of shared memory)

size_t fill_staged_smem(uint32_t nt) { return 4ull * (3ull * nt + 33ull) + 6ull * FILL_NT * FILL_H; }

__global__ void set_params_kernel(RangeParams *dst, RangeParams p)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = p;
}

// ---------------------------------------------------------------------------
// host-side launch wrappers
// ---------------------------------------------------------------------------

cudaError_t launch_bucket_prepass(cudaStream_t st, int grid, const RangeParams *prm, const Tables &t,
                                  uint32_t i0, unsigned long long t0, uint32_t nt, unsigned int *counts,
                                  unsigned long long *off, unsigned int *blk, uint32_t *ent, int phase,
                                  unsigned long long cap, Ctrl *ctrl)
{
    const size_t smem = 4ull * nt;
    if (phase == 0) {
        bucket_count_kernel<256><<<grid, 256, smem, st>>>(prm, t, i0, t0, nt, counts, blk);
        if (cudaPeekAtLastError() == cudaSuccess) block_scan_kernel<<<1, 1024, 0, st>>>(counts, nt, off, nullptr);
        if (cudaPeekAtLastError() == cudaSuccess)
            bucket_block_offsets_kernel<<<(nt + 255) / 256, 256, 0, st>>>(nt, (uint32_t)grid, off, blk);
    } else {
        // the staged fill: FILL_FOLD count blocks to one fill block
        if (grid % FILL_FOLD != 0 || nt > FILL_MAX_TILES) return cudaErrorInvalidValue;
        const size_t fs = fill_staged_smem(nt);
        const cudaError_t e = cudaFuncSetAttribute(bucket_fill_staged_kernel<FILL_NT, FILL_H, FILL_FOLD>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
        if (e != cudaSuccess) return e;
        bucket_fill_staged_kernel<FILL_NT, FILL_H, FILL_FOLD><<<grid / FILL_FOLD, FILL_NT, fs, st>>>(
            prm, t, i0, t0, nt, blk, ent, cap, ctrl);
    }
    return cudaGetLastError();
}

cudaError_t launch_set_params(cudaStream_t st, RangeParams *dst, const RangeParams &p)
{
    set_params_kernel<<<1, 32, 0, st>>>(dst, p);
    return cudaGetLastError();
}

const void *set_params_kernel_ptr() { return (const void *)set_params_kernel; }

template <int WHEEL, int NT>
static const void *slice_ptr() { return (const void *)slice_sieve_kernel<WHEEL, NT>; }

const void *persistent_kernel_ptr(int wheel, int nt, int bc)
{
    if (nt == 256) return persistent_ptr_256(wheel, bc);
    if (nt == 512) return persistent_ptr_512(wheel, bc);
    if (nt == 768) return persistent_ptr_768(wheel, bc);
    if (nt == 1024) return persistent_ptr_1024(wheel, bc);
    return nullptr;
}

const void *pipe_kernel_ptr(int wheel, int np, int nt, int bc)
{
    if (wheel != 13) return nullptr;
    if (np == 8) return pipe_ptr_8(nt, bc);
    if (np == 12 || np == 16) return pipe_ptr_16(np, nt, bc);
    return nullptr;
}

cudaError_t launch_range_kernel(const void *fn, int nt, int grid, size_t smem, cudaStream_t st,
                                const RangeParams *prm, const Tables &t, DevRec *recs, Ctrl *ctrl)
{
    if (!fn) return cudaErrorInvalidValue;
    Tables tt = t;
    void *args[] = {(void *)&prm, (void *)&tt, (void *)&recs, (void *)&ctrl};
    return cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, st);
}

const void *serve_kernel_ptr(int wheel, int nt, int bc)
{
    if (nt == 512) return serve_ptr_512(wheel, bc);
    if (nt == 1024) return serve_ptr_1024(wheel, bc);
    return nullptr;
}

cudaError_t launch_serve(const void *fn, int nt, int grid, size_t smem, cudaStream_t st,
                         const unsigned long long *items, unsigned long long n_items, SlotDev *slots,
                         const Tables &t, Ctrl *ctrl)
{
    if (!fn) return cudaErrorInvalidValue;
    Tables tt = t;
    void *args[] = {(void *)&items, (void *)&n_items, (void *)&slots, (void *)&tt, (void *)&ctrl};
    return cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, st);
}

const void *slice_kernel_ptr(int wheel, int nt)
{
    if (wheel == 13) {
        if (nt == 256) return slice_ptr<13, 256>();
        if (nt == 512) return slice_ptr<13, 512>();
        if (nt == 1024) return slice_ptr<13, 1024>();
    } else if (wheel == 7) {
        if (nt == 256) return slice_ptr<7, 256>();
        if (nt == 512) return slice_ptr<7, 512>();
        if (nt == 1024) return slice_ptr<7, 1024>();
    }
    return nullptr;
}

uint32_t wheel_pattern_words(int wheel)
{
    return wheel == 13 ? pattern_block_words<13>() : pattern_block_words<7>();
}

cudaError_t launch_clear(cudaStream_t st, const RangeParams *prm, DevRec *recs, Ctrl *ctrl,
                         int clear_records, int grid)
{
    clear_kernel<<<grid, 256, 0, st>>>(prm, recs, ctrl, clear_records);
    return cudaGetLastError();
}

cudaError_t launch_merge(cudaStream_t st, int grid, const RangeParams *prm, const DevRec *recs,
                         Ctrl *ctrl, void *parts, gb_result *out)
{
    merge_kernel<<<grid, 256, 0, st>>>(prm, recs, ctrl, (MergePart *)parts, out);
    return cudaGetLastError();
}

size_t merge_part_bytes() { return sizeof(MergePart); }

const void *plain_bulk_ptr(int bc)
{
    switch (bc) {
        case 4: return (const void *)plain_bulk_kernel<1024, 4>;
        case 6: return (const void *)plain_bulk_kernel<1024, 6>;
        case 8: return (const void *)plain_bulk_kernel<1024, 8>;
    }
    return nullptr;
}

cudaError_t launch_plain_bulk(int bc, int grid, size_t smem, cudaStream_t st, const RangeParams &prm,
                              unsigned long long tile_first, uint32_t nsub, const Tables &t, const uint32_t *gwin,
                              DevRec *recs, Ctrl *ctrl)
{
    const void *fn = plain_bulk_ptr(bc);
    if (!fn) return cudaErrorInvalidValue;
    RangeParams p = prm;
    Tables tt = t;
    void *args[] = {(void *)&p, (void *)&tile_first, (void *)&nsub, (void *)&tt, (void *)&gwin, (void *)&recs,
                    (void *)&ctrl};
    return cudaLaunchKernel(fn, dim3(grid), dim3(1024), args, smem, st);
}

cudaError_t launch_slice_sieve(int wheel, int nt, int grid, size_t smem, cudaStream_t st,
                               unsigned long long half_abs, int neg, uint32_t j_end, uint32_t Z,
                               const Tables &t, uint32_t *gwin, uint32_t gwords, Ctrl *ctrl)
{
    const void *fn = slice_kernel_ptr(wheel, nt);
    if (!fn) return cudaErrorInvalidValue;
    Tables tt = t;
    void *args[] = {(void *)&half_abs, (void *)&neg, (void *)&j_end, (void *)&Z, (void *)&tt,
                    (void *)&gwin, (void *)&gwords, (void *)&ctrl};
    return cudaLaunchKernel(fn, dim3(grid), dim3(nt), args, smem, st);
}

cudaError_t launch_plain_search(cudaStream_t st, int grid, const RangeParams *prm,
                                const uint32_t *gwin, const uint32_t *PR, unsigned long long n_lo,
                                uint32_t cnt, uint32_t *pm, Ctrl *ctrl)
{
    plain_search_kernel<<<grid, 256, 0, st>>>(prm, gwin, PR, n_lo, cnt, pm, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_plain_reduce(cudaStream_t st, const RangeParams *prm, const uint32_t *pm,
                                unsigned long long k_seg0, unsigned long long n_lo, uint32_t cnt,
                                uint32_t chunk, DevRec *recs, Ctrl *ctrl)
{
    const uint32_t grid = (cnt + chunk - 1) / chunk;
    plain_reduce_kernel<256><<<grid, 256, 0, st>>>(prm, pm, k_seg0, n_lo, cnt, chunk, recs, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_table_compact(cudaStream_t st, const uint32_t *bits, uint32_t nwords,
                                 uint32_t *block_counts, unsigned long long *block_offsets,
                                 unsigned long long limit, uint32_t *primes,
                                 unsigned long long *recip, int count_only)
{
    const uint32_t nb = (nwords + TBL_WORDS_PER_BLOCK - 1) / TBL_WORDS_PER_BLOCK;
    if (count_only) {
        table_count_kernel<<<nb, 256, 0, st>>>(bits, nwords, block_counts);
        block_scan_kernel<<<1, 1024, 0, st>>>(block_counts, nb, block_offsets, nullptr);
    } else {
        table_scatter_kernel<<<nb, 1024, 0, st>>>(bits, nwords, block_offsets, limit, primes, recip);
    }
    return cudaGetLastError();
}

uint32_t table_blocks(uint32_t nwords) { return (nwords + TBL_WORDS_PER_BLOCK - 1) / TBL_WORDS_PER_BLOCK; }

}  // namespace gbk
