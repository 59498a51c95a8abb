// gb_capi.cu -- host side of libgoldbach_gb300.so: the library context, the
// base-prime tables, the launch pipelines and the C ABI declared in
// include/goldbach_gb300.h.
//
// Pipelines per call:
//   persistent : params H2D -> clear -> persistent_kernel -> merge -> result D2H,
//                captured once into a CUDA graph and replayed (paper Sec. 5.3
//                proposes graphs to amortise launch cost; here the whole
//                range is one replay and there is no per-segment host step).
//   plain      : the paper's Alg. 1 shape, per segment: sieve kernel (global
//                bitset) -> search kernel -> reduce kernel -> 4-byte status
//                D2H + synchronise.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <queue>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "gb_kernels.h"
#include "gb_types.h"
#include "gb_serve.h"
#include "gb_skew.h"

using namespace gbk;

namespace {

struct Options {
    int64_t tile_bits = 20;
    int64_t threads = 1024;
    int64_t ctas_per_sm = 0;       // 0 = as many as fit
    int64_t wheel = 13;
    int64_t pattern_max = 31;
    int64_t tier_b_min = 8192;     // measured best at 10^10, 10^12 and 10^18 against 2^11 .. 2^16
    int64_t base_limit = 0;
    int64_t mem_budget_mb = 8192;
    int64_t plain_seg_bits = 26;
    int64_t plain_slice_bits = 18;
    int64_t plain_search_chunks = 0;   // plain form: 0 = per-n search kernel, 4/6/8 = bit-parallel
    int64_t use_graph = 1;
    int64_t slow_cap = 24;
    int64_t timeout_ms = 600000;
    int64_t serve_batch_tiles = 1024;
    int64_t time_kernel = 0;       // record CUDA events around the persistent kernel
    int64_t bucket_min = 0;        // smallest bucketed prime; 0 = four window spans 4 (S + K)
    int64_t bucket_chunk_tiles = 2048;
    int64_t search_pmax = 0;       // window search bound; 0 = P_max
    int64_t search_chunks = 4;     // bit-parallel search over p < 64 * this (0 = per-n search)
    int64_t autotune = 0;          // 1: tune the kernel configuration per range class
    int64_t builder_warps = 0;     // > 0: pipelined kernel, this many warps build windows
    int64_t debug_smem_limit = 0;  // builds with GB_DEBUG: bytes of dynamic shared memory the
                                   // window accesses may touch (0 = the whole allocation)
};

struct GraphKey {
    const void *fn = nullptr;
    int grid = 0, nt = 0, wheel = 0, merge_grid = 0, clear_records = 0;
    size_t smem = 0;
    const void *recs = nullptr;
    const void *olist = nullptr;
    uint32_t olist_wcap = 0, olist_ctas = 0;
    const void *aperm = nullptr;
    uint32_t aperm_len = 0;
    const void *askew = nullptr;
    bool operator==(const GraphKey &o) const
    {
        return fn == o.fn && grid == o.grid && nt == o.nt && wheel == o.wheel &&
               merge_grid == o.merge_grid && clear_records == o.clear_records && smem == o.smem &&
               recs == o.recs && olist == o.olist && olist_wcap == o.olist_wcap && olist_ctas == o.olist_ctas &&
               aperm == o.aperm && aperm_len == o.aperm_len && askew == o.askew;
    }
};

struct Ctx {
    bool inited = false;
    int device = 0, sms = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    uint32_t p_max = 0, seg_bits = 0, k_words = 0;
    Options opt;
    // base-prime table (odd primes from 3, ascending) and reciprocals
    uint32_t *d_primes = nullptr;
    unsigned long long *d_recip = nullptr;
    uint64_t nprimes = 0, table_limit = 0;
    std::vector<uint32_t> h_small;           // odd primes <= 2^16
    uint32_t *d_PR = nullptr;
    // per-call scratch
    RangeParams *d_params = nullptr, *h_params = nullptr;
    Ctrl *d_ctrl = nullptr;
    DevRec *d_recs = nullptr;
    size_t rec_cap = 0;
    void *d_parts = nullptr;
    gb_result *d_result = nullptr, *h_result = nullptr;
    unsigned int *h_flags = nullptr;
    // graph
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    // graph of gb_verify_range_async: set-params -> clear -> kernel -> merge
    // into the caller's result; each call rewrites the set-params node's
    // arguments in the instantiated graph and replays it on the caller's stream
    cudaGraphExec_t aexec = nullptr;
    cudaGraph_t agraph = nullptr;          // kept while aexec lives: anode belongs to it
    cudaGraphNode_t anode = nullptr;
    GraphKey akey;
    const void *aout = nullptr;
    // plain-form buffers
    uint32_t *d_gwin = nullptr;
    size_t gwin_words = 0;
    uint32_t *d_pm = nullptr;
    size_t pm_cap = 0;
    gb_stats_t stats{};
    size_t device_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // persistent-kernel timing (time_kernel)
    unsigned long long *h_progress = nullptr, *d_progress = nullptr;   // mapped tile counter
    // bucket pre-pass buffers
    unsigned int *d_bk_counts = nullptr;
    unsigned int *d_bk_blk = nullptr;      // per (pre-pass block, tile): count, then first entry
    unsigned long long *d_bk_off = nullptr;
    size_t bk_tiles_cap = 0;
    uint32_t *d_bk_ent = nullptr;
    size_t bk_ent_cap = 0;
    // open-mask slots of the bit-parallel search (see Tables::olist)
    uint32_t *d_olist = nullptr;
    size_t olist_cap = 0;
    uint32_t olist_wcap = 0, olist_ctas = 0;
    // per-phase cycle sums (builds with GB_PHASE_CLOCKS; see Tables::phase)
    unsigned long long *d_phase = nullptr;
    // balanced order of the tier-A primes (see Tables::aperm) and what it was built for
    uint32_t *d_aperm = nullptr;
    uint32_t aperm_len = 0;
    unsigned long long *d_askew = nullptr;    // tier-A lane skews (ASKEW_ENTRIES)
    uint64_t aperm_key[5] = {0, 0, 0, 0, 0};
    std::map<uint64_t, uint32_t> odd_primes_below;  // cache: bound -> #odd primes below it
    char dev_name[256] = {0};
    struct TuneCfg {
        int64_t tile_bits, threads, search_chunks, pattern_max, search_pmax, tier_b_min, wheel, builder_warps,
            bucket_min, bucket_chunk_tiles;
    };
    std::map<std::string, TuneCfg> tuned;       // autotuner results by range class
    bool ev_pending = false;
};

Ctx g;

// NVTX range over a host-side phase (table build, tuning, bucket pre-pass,
// launch or replay, plain segment, serving batch) for a profiler timeline;
// costs nothing when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// The captured graphs bake in table, record and scratch pointers and launch
// shapes: any change of those makes the next call capture again.
void invalidate_graphs()
{
    g.gkey = GraphKey{};
    g.akey = GraphKey{};
}

std::atomic<bool> g_ready{false};        // gb_init done: readable without the context lock
std::atomic<unsigned long long> g_progress_total{0};   // tiles of the running call
std::atomic<unsigned long long> g_progress_ntotal{0};  // its even n
std::atomic<unsigned long long> g_progress_tile_n{0};  // even n per tile
std::atomic<long long> g_progress_t0{0};               // its start, steady-clock ns
std::atomic<unsigned long long *> g_progress_ptr{nullptr};
uint32_t search_pmax();
int build_candidates();
std::recursive_mutex g_mu;
std::mutex g_err_mu;
std::string g_err = "";
constexpr int MERGE_GRID_CAP = 512;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = buf;
}

int cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GB_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA;
}

// Host-side fault injection for the failure-path tests: GB_FAULT="kind:k"
// (kind = malloc, launch or memcpy) makes the k-th such call, counted from
// gb_init, fail before it reaches CUDA.  No GPU fault is ever provoked.
struct FaultShim {
    int kind = -1;                    // 0 malloc, 1 launch, 2 memcpy
    long long at = 0, seen[3] = {0, 0, 0};
};
FaultShim g_fault;

void fault_configure()
{
    g_fault = FaultShim{};
    const char *f = getenv("GB_FAULT");
    if (!f) return;
    static const char *names[3] = {"malloc:", "launch:", "memcpy:"};
    for (int k = 0; k < 3; k++) {
        size_t n = strlen(names[k]);
        if (!strncmp(f, names[k], n)) { g_fault.kind = k; g_fault.at = atoll(f + n); }
    }
}

// 0, or the status of an injected failure of this call
int fault_pre(int kind, const char *what)
{
    if (g_fault.kind != kind) return GB_OK;
    if (++g_fault.seen[kind] != g_fault.at) return GB_OK;
    set_error("injected failure (GB_FAULT) at %s", what);
    return kind == 0 ? GB_ENOMEM : GB_ECUDA;
}

int fault_kind_of(const char *what)
{
    if (strstr(what, "launch_")) return 1;
    if (strstr(what, "cudaMemcpy")) return 2;
    return -2;
}

#define CK(x)                                                   \
    do {                                                        \
        int rc_ = fault_pre(fault_kind_of(#x), #x);             \
        if (rc_ == GB_OK) rc_ = cuda_status((x), #x);           \
        if (rc_ != GB_OK) return rc_;                           \
    } while (0)

template <class T>
int dev_alloc(T **p, size_t bytes)
{
    if (int frc = fault_pre(0, "cudaMalloc")) return frc;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return GB_ENOMEM;
    }
    *p = (T *)q;
    g.device_bytes += bytes;
    return GB_OK;
}

template <class T>
void dev_free(T **p, size_t bytes)
{
    if (*p) {
        cudaFree((void *)*p);
        g.device_bytes -= std::min(g.device_bytes, bytes);
    }
    *p = nullptr;
}

uint64_t isqrt_host(uint64_t x)
{
    uint64_t r = (uint64_t)std::sqrt((double)x);
    if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
    while (r > 0 && r > x / r) r--;
    while (r < 0xFFFFFFFFull && (r + 1) <= x / (r + 1)) r++;
    return r;
}

// Odd primes <= limit by a plain host sieve (limit <= 2^21): bootstrap table.
std::vector<uint32_t> host_odd_primes(uint32_t limit)
{
    std::vector<uint8_t> c(limit + 1, 1);
    std::vector<uint32_t> out;
    for (uint64_t i = 3; i <= limit; i += 2) {
        if (!c[i]) continue;
        out.push_back((uint32_t)i);
        for (uint64_t m = i * i; m <= limit; m += 2 * i) c[m] = 0;
    }
    return out;
}

uint32_t bitrev32(uint32_t x)
{
    uint32_t r = 0;
    for (int b = 0; b < 32; b++) r |= ((x >> b) & 1u) << (31 - b);
    return r;
}

// Tables of one launch; `wheel` is the WHEEL of the kernel that gets them.
Tables make_tables(int wheel)
{
    Tables t{};
    t.primes = g.d_primes;
    t.recip = g.d_recip;
    t.PR = g.d_PR;
    t.nprimes = (uint32_t)g.nprimes;
    t.k_words = g.k_words;
    // the fill clears every prime above the wheel up to pattern_max: with
    // wheel 13 by the group patterns 17*19*23 (from 23 on) and 29*31 (from 31
    // on), the rest by in-register masks
    static const uint32_t pat[14] = {11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61};
    t.groups = 0;
    if (wheel == 13 && g.opt.pattern_max >= 23) t.groups = 1;
    if (wheel == 13 && g.opt.pattern_max >= 31) t.groups = 2;
    t.pat_lo = wheel == 13 ? 2u + (t.groups >= 1 ? 3u : 0u) + (t.groups >= 2 ? 2u : 0u) : 0u;
    uint32_t hi = wheel == 13 ? 2u : 0u;
    while (hi < 14 && pat[hi] <= (uint32_t)g.opt.pattern_max) hi++;
    t.pat_hi = std::max(hi, t.pat_lo);
    uint32_t lim = (uint32_t)wheel;
    if (hi > (wheel == 13 ? 2u : 0u)) lim = std::max(lim, pat[hi - 1]);
    t.iA0 = (uint32_t)(std::upper_bound(g.h_small.begin(), g.h_small.end(), lim) - g.h_small.begin());
    t.iB0 = (uint32_t)(std::lower_bound(g.h_small.begin(), g.h_small.end(),
                                        (uint32_t)g.opt.tier_b_min) - g.h_small.begin());
    if (t.iB0 < t.iA0) t.iB0 = t.iA0;
    t.olist = g.d_olist;
    t.olist_wcap = g.olist_wcap;
    t.olist_ctas = g.olist_ctas;
    const bool aperm_fits = g.d_aperm && g.aperm_key[0] == t.iA0 && g.aperm_key[1] == t.iB0;
    t.aperm = aperm_fits ? g.d_aperm : nullptr;
    t.aperm_len = aperm_fits ? g.aperm_len : 0u;
    t.askew = g.d_askew;
    t.phase = g.d_phase;
    return t;
}

Tables make_tables() { return make_tables((int)g.opt.wheel); }

size_t window_words(uint32_t tile_bits)
{
    return ((((size_t)1 << tile_bits) + 32ull * g.k_words) / 32 + 2 + 3) & ~(size_t)3;
}

size_t persistent_smem(uint32_t tile_bits, int wheel)
{
    return 4ull * (wheel_pattern_words(wheel) + ((g.k_words + 3) & ~3u) + window_words(tile_bits));
}

size_t persistent_smem(uint32_t tile_bits) { return persistent_smem(tile_bits, (int)g.opt.wheel); }

// The range kernel of the current options: the pipelined kernel when
// builder_warps > 0 (its CTA holds two windows), else the persistent one.
const void *range_kernel()
{
    if (g.opt.builder_warps > 0)
        return pipe_kernel_ptr((int)g.opt.wheel, (int)g.opt.builder_warps, (int)g.opt.threads,
                               (int)g.opt.search_chunks);
    return persistent_kernel_ptr((int)g.opt.wheel, (int)g.opt.threads, (int)g.opt.search_chunks);
}

size_t range_smem(uint32_t tile_bits)
{
    if (g.opt.builder_warps <= 0) return persistent_smem(tile_bits);
    return 4ull * (wheel_pattern_words((int)g.opt.wheel) + ((g.k_words + 3) & ~3u) +
                   2ull * pipe_window_words(tile_bits, g.k_words));
}

// Threads that build windows and threads that search them, per CTA.
int builder_threads() { return g.opt.builder_warps > 0 ? 32 * (int)g.opt.builder_warps : (int)g.opt.threads; }
int searcher_threads()
{
    return g.opt.builder_warps > 0 ? (int)g.opt.threads - 32 * (int)g.opt.builder_warps : (int)g.opt.threads;
}

// Grow the device base-prime table to every prime <= need (or base_limit).
// Builds with GB_DEBUG: true, with the error message set, when a kernel's
// bounds check failed since the control block's debug fields were last
// cleared; the work must have completed.  Ordinary builds: always false.
bool debug_bounds_failed(const char *where)
{
#ifdef GB_DEBUG
    Ctrl hc;
    if (cudaMemcpy(&hc, g.d_ctrl, sizeof hc, cudaMemcpyDeviceToHost) != cudaSuccess || !hc.dbg_site) return false;
    set_error("bounds check failed while %s: site %u, byte %u of dynamic shared memory", where, hc.dbg_site,
              hc.dbg_off);
    return true;
#else
    (void)where;
    return false;
#endif
}

int ensure_table(uint64_t need)
{
    if (need <= g.table_limit) return GB_OK;
    NvtxRange nv("gb: base-prime table");
    uint64_t L = std::max<uint64_t>(need, (uint64_t)g.opt.base_limit);
    // round up to 2^k - 1 so repeated growth stays rare
    uint64_t r = 1;
    while (r - 1 < L && r < (1ull << 32)) r <<= 1;
    L = std::min<uint64_t>(r - 1, 0xFFFFFFFFull);
    if (L <= g.table_limit) return GB_OK;
    // sieve the odd numbers q = 2j + 1, j < j_end, with the bootstrap primes
    const uint32_t j_end = (uint32_t)((L + 1) / 2);
    const uint32_t Z = 1u << 18;
    const uint32_t gwords = (j_end + 31) / 32 + 2;
    uint32_t *bits = nullptr;
    int rc = dev_alloc(&bits, 4ull * gwords);
    if (rc) return rc;
    const int nt = 512;
    const size_t smem = 4ull * (wheel_pattern_words((int)g.opt.wheel) + Z / 32 + 4);
    const void *fn = slice_kernel_ptr((int)g.opt.wheel, nt);
    Tables t = make_tables();                     // still the bootstrap table
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, 4ull * gwords, g.stream);
#ifdef GB_DEBUG
    if (e == cudaSuccess) e = cudaMemsetAsync(&g.d_ctrl->dbg_site, 0, 8, g.stream);   // dbg_site, dbg_off
#endif
    if (e == cudaSuccess)
        e = launch_slice_sieve((int)g.opt.wheel, nt, (int)((j_end + Z - 1) / Z), smem, g.stream, 0ull, 0,
                               j_end, Z, t, bits, gwords, g.d_ctrl);
    const uint32_t nb = table_blocks(gwords);
    uint32_t *bc = nullptr;
    unsigned long long *bo = nullptr;
    if (e == cudaSuccess && (rc = dev_alloc(&bc, 4ull * nb)) == GB_OK &&
        (rc = dev_alloc(&bo, 8ull * (nb + 1))) == GB_OK) {
        e = launch_table_compact(g.stream, bits, gwords, bc, bo, L, nullptr, nullptr, 1);
        unsigned long long total = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, bo + nb, 8, cudaMemcpyDeviceToHost, g.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g.stream);
        if (e == cudaSuccess && debug_bounds_failed("building the base-prime table")) rc = GB_EINTERNAL;
        uint32_t *np = nullptr;
        unsigned long long *nr = nullptr;
        const uint64_t padded = (total + 3) & ~3ull;       // four-wide loads read up to here
        if (e == cudaSuccess && rc == GB_OK && (rc = dev_alloc(&np, 4ull * padded)) == GB_OK &&
            (rc = dev_alloc(&nr, 8ull * padded)) == GB_OK) {
            e = cudaMemsetAsync(np + total, 0, 4ull * (padded - total), g.stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(nr + total, 0, 8ull * (padded - total), g.stream);
            if (e == cudaSuccess) e = launch_table_compact(g.stream, bits, gwords, bc, bo, L, np, nr, 0);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g.stream);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();   // no launch may still read the old table
            if (e == cudaSuccess) {
                dev_free(&g.d_primes, 4ull * ((g.nprimes + 3) & ~3ull));
                dev_free(&g.d_recip, 8ull * ((g.nprimes + 3) & ~3ull));
                g.d_primes = np;
                g.d_recip = nr;
                g.nprimes = total;
                g.table_limit = L;
                np = nullptr;
                nr = nullptr;
                invalidate_graphs();                 // tables changed: recapture
            }
        }
        dev_free(&np, 4ull * padded);
        dev_free(&nr, 8ull * padded);
    }
    dev_free(&bc, 4ull * nb);
    dev_free(&bo, 8ull * (nb + 1));
    dev_free(&bits, 4ull * gwords);
    if (rc) return rc;
    return cuda_status(e, "base-prime table build");
}

int ensure_records(uint64_t nrec)
{
    if (nrec <= g.rec_cap) return GB_OK;
    size_t cap = std::max<uint64_t>(nrec, 1024);
    dev_free(&g.d_recs, sizeof(DevRec) * g.rec_cap);
    g.rec_cap = 0;
    int rc = dev_alloc(&g.d_recs, sizeof(DevRec) * cap);
    if (rc) return rc;
    g.rec_cap = cap;
    invalidate_graphs();
    return GB_OK;
}

struct CallPlan {
    uint64_t n0 = 0, n_total = 0, nrec = 0, ntiles = 0;
};

// Validate a range and compute its even-n grid.  n_total == 0 means empty.
int plan_range(uint64_t lo, uint64_t hi, CallPlan &cp)
{
    cp = CallPlan{};
    uint64_t n0 = lo < 4 ? 4 : lo;
    if (n0 & 1) {
        if (n0 == UINT64_MAX) return GB_OK;
        n0++;
    }
    if (n0 >= hi) return GB_OK;
    uint64_t n_last = (hi - 1) & ~1ull;
    if (n_last < n0) return GB_OK;
    cp.n0 = n0;
    cp.n_total = (n_last - n0) / 2 + 1;
    cp.nrec = ((cp.n_total - 1) >> g.seg_bits) + 1;
    cp.ntiles = ((cp.n_total - 1) >> g.opt.tile_bits) + 1;
    return GB_OK;
}

void fill_params(const CallPlan &cp, uint32_t tile_bits, RangeParams &p)
{
    memset(&p, 0, sizeof p);
    p.n0 = cp.n0;
    p.n_total = cp.n_total;
    p.ntiles = cp.ntiles;
    p.nrec = cp.nrec;
    p.p_slow_start = (search_pmax() + 1ull) | 1ull;
    p.tile_bits = tile_bits;
    p.rec_bits = g.seg_bits;
    p.k_words = g.k_words;
    p.p_max = g.p_max;
    p.slow_cap_log2 = (uint32_t)g.opt.slow_cap;
    p.bk_prime0 = 0xffffffffu;
    p.tile0 = 0;
    p.tile_end = cp.ntiles;
    p.bk_off = nullptr;
    p.bk_ent = nullptr;
    p.progress = g.d_progress;
    p.dbg_lim = (uint32_t)g.opt.debug_smem_limit;
}

void empty_result(gb_result *out)
{
    if (!out) return;
    memset(out, 0, sizeof *out);
    out->status = GB_OK;
}

long long steady_ns()
{
    return (long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A call of `tiles` tiles of tile_n even n each (n_total in all) starts.
void begin_progress(uint64_t tiles, uint64_t n_total, uint64_t tile_n)
{
    if (g.h_progress) *(volatile unsigned long long *)g.h_progress = 0;
    g_progress_total = tiles;
    g_progress_ntotal = n_total;
    g_progress_tile_n = tile_n;
    g_progress_t0 = steady_ns();
}

int prepare_common(const CallPlan &cp)
{
    uint64_t n_last = cp.n0 + 2 * (cp.n_total - 1);
    int rc = ensure_table(isqrt_host(n_last));
    if (rc) return rc;
    return ensure_records(cp.nrec);
}

int occupancy_grid(const void *fn, int nt, size_t smem, int *grid)
{
    if (!fn) {
        set_error("no kernel for this combination of wheel, threads and search_chunks "
                  "(wheel 7 supports search_chunks 0, 4, 8)");
        return GB_EINVAL;
    }
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
    if (per_sm < 1) {
        set_error("tile does not fit in shared memory (%zu bytes)", smem);
        return GB_ENOMEM;
    }
    if (g.opt.ctas_per_sm > 0) per_sm = std::min<int>(per_sm, (int)g.opt.ctas_per_sm);
    *grid = per_sm * g.sms;
    return GB_OK;
}

// Open-mask slots per warp for the bit-parallel search: one u32 per word of
// the warp's share of a tile, i.e. 32 x (its groups of 32 words).
uint32_t olist_slice(int nt, uint32_t tile_bits)
{
    const uint64_t nwarp = (uint64_t)nt / 32;
    const uint64_t groups = ((1ull << tile_bits) + 1024 * nwarp - 1) / (1024 * nwarp);
    return (uint32_t)(32 * groups);
}

uint32_t olist_slice(int nt) { return olist_slice(nt, (uint32_t)g.opt.tile_bits); }

// The context's open-mask slots for a persistent launch of `grid` CTAs.
int ensure_olist(int grid, int nt, uint32_t tile_bits, bool bulk)
{
    if (!bulk) { g.olist_wcap = 0; g.olist_ctas = 0; return GB_OK; }
    const uint32_t wcap = olist_slice(nt, tile_bits);
    const size_t need = (size_t)grid * (size_t)(nt / 32) * wcap;
    if (need > g.olist_cap) {
        dev_free(&g.d_olist, 4 * g.olist_cap);
        g.olist_cap = 0;
        int rc;
        if ((rc = dev_alloc(&g.d_olist, 4 * need))) return rc;
        g.olist_cap = need;
    }
    g.olist_wcap = wcap;
    g.olist_ctas = (uint32_t)grid;
    return GB_OK;
}

// The tier-A lane skews (gb_skew.h), built once per process.
const std::vector<unsigned long long> &tier_a_skews()
{
    static std::vector<unsigned long long> tab;
    if (tab.empty()) {
        tab.assign(ASKEW_ENTRIES, 0ull);
        tier_a_skew_table(tab.data());
    }
    return tab;
}

// The tier-A primes of the current tables spread over the warps of an
// nt-thread CTA by longest processing time first: each prime, heaviest first,
// goes to the least-loaded warp.  A prime's load is its crossing-off steps per
// lane, (S + K) / 32 / p, plus 16 for its first-multiple setup.  The marks
// are exact with any order; this only evens out the warps' work.
int ensure_aperm(int nt)
{
    if (!g.d_askew) {
        const std::vector<unsigned long long> &sk = tier_a_skews();
        int rc;
        if ((rc = dev_alloc(&g.d_askew, 8ull * ASKEW_ENTRIES))) return rc;
        auto upload = [&]() -> int {
            CK(cudaMemcpy(g.d_askew, sk.data(), 8ull * ASKEW_ENTRIES, cudaMemcpyHostToDevice));
            return GB_OK;
        };
        if ((rc = upload())) {                  // no half-written table: the next call uploads again
            dev_free(&g.d_askew, 8ull * ASKEW_ENTRIES);
            return rc;
        }
    }
    const Tables t = make_tables();
    const uint64_t nwarp = (uint64_t)nt / 32;
    const uint64_t key[5] = {t.iA0, t.iB0, nwarp, (uint64_t)g.opt.tile_bits, g.k_words};
    if (g.d_aperm && std::equal(key, key + 5, g.aperm_key)) return GB_OK;
    dev_free(&g.d_aperm, 4ull * g.aperm_len);
    g.aperm_len = 0;
    std::fill(g.aperm_key, g.aperm_key + 5, 0ull);
    const uint32_t n = t.iB0 > t.iA0 ? t.iB0 - t.iA0 : 0u;
    if (n == 0 || t.iB0 > g.h_small.size()) return GB_OK;
    const double span_words = ((double)(1ull << g.opt.tile_bits) + 32.0 * g.k_words) / 32.0;
    std::vector<std::pair<double, uint32_t>> items(n);
    for (uint32_t i = 0; i < n; i++) items[i] = {span_words / g.h_small[t.iA0 + i] + 16.0, t.iA0 + i};
    std::sort(items.begin(), items.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<std::vector<uint32_t>> lists(nwarp);
    std::priority_queue<std::pair<double, uint64_t>, std::vector<std::pair<double, uint64_t>>,
                        std::greater<std::pair<double, uint64_t>>> load;
    for (uint64_t w = 0; w < nwarp; w++) load.push({0.0, w});
    for (const auto &it : items) {
        auto top = load.top();
        load.pop();
        lists[top.second].push_back(it.second);
        load.push({top.first + it.first, top.second});
    }
    size_t len = 0;
    for (const auto &l : lists) len = std::max(len, l.size());
    std::vector<uint32_t> perm(nwarp * len, 0xffffffffu);
    for (uint64_t w = 0; w < nwarp; w++)
        for (size_t k = 0; k < lists[w].size(); k++) perm[w + nwarp * k] = lists[w][k];
    int rc;
    if ((rc = dev_alloc(&g.d_aperm, 4ull * perm.size()))) return rc;
    CK(cudaMemcpy(g.d_aperm, perm.data(), 4ull * perm.size(), cudaMemcpyHostToDevice));
    g.aperm_len = (uint32_t)perm.size();
    std::copy(key, key + 5, g.aperm_key);
    return GB_OK;
}

// Grid of a persistent launch on the context's stream, with its list and the
// tier-A order for its thread count.
int ctx_grid(const void *fn, int nt, size_t smem, int *grid)
{
    int rc = occupancy_grid(fn, nt, smem, grid);
    if (!rc) rc = ensure_aperm(builder_threads());
    return rc ? rc : ensure_olist(*grid, searcher_threads(), (uint32_t)g.opt.tile_bits, true);
}

int merge_grid_for(uint64_t nrec)
{
    uint64_t b = (nrec + 255) / 256;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, MERGE_GRID_CAP));
}

// Enqueue the persistent pipeline (without the params copy) on stream st.
int enqueue_persistent(cudaStream_t st, const CallPlan &cp, gb_result *dev_out, int grid,
                       size_t smem, int merge_grid, bool timed = false)
{
    const int clear_records = g.opt.tile_bits < g.seg_bits ? 1 : 0;
    Tables t = make_tables();
    CK(launch_clear(st, g.d_params, g.d_recs, g.d_ctrl, clear_records, clear_records ? 4 * g.sms : 1));
    if (g.d_phase) CK(cudaMemsetAsync(g.d_phase, 0, 8ull * PH_COUNT, st));
    if (timed) {
        if (!g.ev0) CK(cudaEventCreate(&g.ev0));
        if (!g.ev1) CK(cudaEventCreate(&g.ev1));
        CK(cudaEventRecord(g.ev0, st));
    }
    CK(launch_range_kernel(range_kernel(), (int)g.opt.threads, grid, smem, st, g.d_params, t, g.d_recs, g.d_ctrl));
    if (timed) {
        CK(cudaEventRecord(g.ev1, st));
        g.ev_pending = true;
    }
    CK(launch_merge(st, merge_grid, g.d_params, g.d_recs, g.d_ctrl, g.d_parts, dev_out));
    (void)cp;
    return GB_OK;
}

// Blocks of the bucket pre-pass kernels (four per SM).
size_t bucket_grid() { return 4ull * (size_t)g.sms; }

// Smallest prime handled by the bucket pre-pass for this configuration.
uint64_t bucket_bound()
{
    if (g.opt.bucket_min > 0) return (uint64_t)g.opt.bucket_min;
    // four window spans: measured on GB300 at 1e13, 1e15 and 1e18 against
    // one, two, 16 and 64 spans; below it the lane-per-prime crossing-off
    // costs less than a bucket entry (two enumerations and a scattered store)
    return 4ull * ((1ull << g.opt.tile_bits) + 32ull * g.k_words);
}

uint32_t count_odd_primes_below(uint64_t x)
{
    auto it = g.odd_primes_below.find(x);
    if (it != g.odd_primes_below.end()) return it->second;
    uint32_t c;
    if (x <= (1u << 16)) {
        c = (uint32_t)(std::lower_bound(g.h_small.begin(), g.h_small.end(), (uint32_t)x) - g.h_small.begin());
    } else {
        std::vector<uint32_t> v = host_odd_primes((uint32_t)std::min<uint64_t>(x, 0xFFFFFFFFull));
        c = (uint32_t)(std::lower_bound(v.begin(), v.end(), (uint32_t)std::min<uint64_t>(x, 0xFFFFFFFFull)) -
                       v.begin());
    }
    g.odd_primes_below[x] = c;
    return c;
}

bool needs_buckets(const CallPlan &cp)
{
    const uint64_t n_last = cp.n0 + 2 * (cp.n_total - 1);
    return isqrt_host(n_last) >= bucket_bound();
}

// Upper bound on the bucket entries of one chunk, found without the device:
// a bucket prime p (B <= p <= P) has at most span/p + 1 hits in the chunk's
// `span` window bits (its odd multiples are p bits apart), and each hit is
// entered in at most `dup` overlapping windows.  The sum of 1/p is exact over
// the host's primes up to 2^16; above, Rosser and Schoenfeld's bounds on
// sum_{p <= x} 1/p (within 1/(2 ln^2 x) of ln ln x + M for x >= 286) give
// sum_{lo < p <= P} 1/p < ln ln P - ln ln lo + 1/ln^2 lo.
uint64_t bucket_entries_bound(uint64_t B, uint64_t P, uint64_t nprimes, uint64_t span, uint64_t dup)
{
    double rs = 0.0;
    for (uint32_t q : g.h_small)
        if (q >= B && q <= P) rs += 1.0 / q;
    const double lo = std::max<double>((double)B, 65536.0);
    if ((double)P > lo) {
        const double l = std::log(lo);
        rs += std::log(std::log((double)P)) - std::log(l) + 1.0 / (l * l);
    }
    const double e = (double)dup * ((double)span * rs + (double)nprimes) + 1024.0;
    return (uint64_t)std::ceil(e * 1.01);
}

// Persistent pipeline with the large primes bucketed: tiles are processed in
// chunks; per chunk the pre-pass counts, scans and fills the buckets, then
// the persistent kernel sieves the chunk's tiles.  The entry buffer is sized
// once from bucket_entries_bound, so the chunks are enqueued back to back
// with no host round trip (a fill that would pass the bound sets F_INTERNAL
// instead of writing).
int run_persistent_buckets(const CallPlan &cp, int grid, size_t smem, int mg, gb_result *dev_out,
                           cudaStream_t st, bool sync_result)
{
    int rc;
    const uint64_t B = bucket_bound();
    if (B > (1ull << 28)) { set_error("bucket_min above 2^28 is not supported"); return GB_EINVAL; }
    const uint32_t i0 = count_odd_primes_below(B);
    const uint64_t CT = (uint64_t)g.opt.bucket_chunk_tiles;
    if (g.bk_tiles_cap < CT + 1) {
        dev_free(&g.d_bk_counts, 4 * g.bk_tiles_cap);
        dev_free(&g.d_bk_blk, 4 * g.bk_tiles_cap * bucket_grid());
        dev_free(&g.d_bk_off, 8 * g.bk_tiles_cap);
        g.bk_tiles_cap = 0;
        if ((rc = dev_alloc(&g.d_bk_counts, 4 * (CT + 1)))) return rc;
        if ((rc = dev_alloc(&g.d_bk_blk, 4 * (CT + 1) * bucket_grid()))) return rc;
        if ((rc = dev_alloc(&g.d_bk_off, 8 * (CT + 1)))) return rc;
        g.bk_tiles_cap = CT + 1;
    }
    RangeParams p;
    fill_params(cp, (uint32_t)g.opt.tile_bits, p);
    p.bk_prime0 = i0;
    Tables t = make_tables();
    const int clear_records = g.opt.tile_bits < g.seg_bits ? 1 : 0;
    CK(launch_set_params(st, g.d_params, p));
    CK(launch_clear(st, g.d_params, g.d_recs, g.d_ctrl, clear_records, clear_records ? 4 * g.sms : 1));
    if (g.d_phase) CK(cudaMemsetAsync(g.d_phase, 0, 8ull * PH_COUNT, st));
    const uint64_t S = 1ull << g.opt.tile_bits, K = 32ull * g.k_words;
    const uint64_t P = isqrt_host(cp.n0 + 2 * (cp.n_total - 1));
    const uint64_t cap = bucket_entries_bound(B, P, g.nprimes - i0, CT * S + K, 1 + (K - 1 + S - 1) / S);
    if (cap >= (1ull << 32)) { set_error("bucket chunk too large: lower bucket_chunk_tiles"); return GB_ENOMEM; }
    if (cap > g.bk_ent_cap) {
        dev_free(&g.d_bk_ent, 4 * g.bk_ent_cap);
        g.bk_ent_cap = 0;
        if ((rc = dev_alloc(&g.d_bk_ent, 4 * cap))) return rc;
        g.bk_ent_cap = cap;
    }
    uint64_t launches = 2;
    for (uint64_t t0 = 0; t0 < cp.ntiles; t0 += CT) {
        NvtxRange nv("gb: bucket chunk (pre-pass + kernel)");
        const uint32_t nt = (uint32_t)std::min<uint64_t>(CT, cp.ntiles - t0);
        CK(cudaMemsetAsync(g.d_bk_counts, 0, 4ull * nt, st));
        CK(launch_bucket_prepass(st, (int)bucket_grid(), g.d_params, t, i0, t0, nt, g.d_bk_counts, g.d_bk_off,
                                 g.d_bk_blk, nullptr, 0, 0, nullptr));
        CK(launch_bucket_prepass(st, (int)bucket_grid(), g.d_params, t, i0, t0, nt, g.d_bk_counts, g.d_bk_off,
                                 g.d_bk_blk, g.d_bk_ent, 1, g.bk_ent_cap, g.d_ctrl));
        p.tile0 = t0;
        p.tile_end = t0 + nt;
        p.bk_off = g.d_bk_off;
        p.bk_ent = g.d_bk_ent;
        CK(launch_set_params(st, g.d_params, p));
        CK(cudaMemsetAsync(&g.d_ctrl->tile_ctr, 0, 8, st));
        CK(launch_range_kernel(range_kernel(), (int)g.opt.threads, grid, smem, st, g.d_params, t, g.d_recs, g.d_ctrl));
        launches += 6;
    }
    p.tile0 = 0;
    p.tile_end = cp.ntiles;
    CK(launch_set_params(st, g.d_params, p));
    CK(launch_merge(st, mg, g.d_params, g.d_recs, g.d_ctrl, g.d_parts, dev_out));
    launches += 2;
    if (sync_result) {
        CK(cudaMemcpyAsync(g.h_result, dev_out, sizeof(gb_result), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    g.stats.kernel_launches += launches;
    g.stats.tiles += cp.ntiles;
    return GB_OK;
}

// ---------------------------------------------------------------------------
// autotuner: coordinate descent over the kernel configuration, timed with
// CUDA events on a probe at the top of the caller's range; results cached per
// (GPU, SMs, P_max, log2 of the largest n rounded to even) in memory and, when
// GB_TUNE_CACHE names a file, on disk.
// ---------------------------------------------------------------------------

using TuneCfg = Ctx::TuneCfg;

TuneCfg current_cfg()
{
    return TuneCfg{g.opt.tile_bits, g.opt.threads, g.opt.search_chunks, g.opt.pattern_max,
                   g.opt.search_pmax, g.opt.tier_b_min, g.opt.wheel, g.opt.builder_warps,
                   g.opt.bucket_min, g.opt.bucket_chunk_tiles};
}

int apply_cfg(const TuneCfg &c)
{
    const bool pr = c.search_pmax != g.opt.search_pmax;
    g.opt.tile_bits = c.tile_bits;
    g.opt.threads = c.threads;
    g.opt.search_chunks = c.search_chunks;
    g.opt.pattern_max = c.pattern_max;
    g.opt.search_pmax = c.search_pmax;
    g.opt.tier_b_min = c.tier_b_min;
    g.opt.wheel = c.wheel;
    g.opt.builder_warps = c.builder_warps;
    g.opt.bucket_min = c.bucket_min;
    g.opt.bucket_chunk_tiles = c.bucket_chunk_tiles;
    invalidate_graphs();
    return pr ? build_candidates() : GB_OK;
}

std::string tune_key(const CallPlan &cp)
{
    const uint64_t n_last = cp.n0 + 2 * (cp.n_total - 1);
    const int mag = 63 - __builtin_clzll(n_last);
    char buf[400];
    snprintf(buf, sizeof buf, "%s|sm%d|pmax%u|log2n%d", g.dev_name, g.sms, g.p_max, mag & ~1);
    for (char *c = buf; *c; c++)
        if (*c == ' ') *c = '_';
    return buf;
}

// Kernel time of one persistent launch over the probe range; < 0 if the
// configuration cannot run.
float time_probe(const CallPlan &probe_in)
{
    CallPlan probe = probe_in;
    probe.ntiles = ((probe.n_total - 1) >> g.opt.tile_bits) + 1;
    const int nt = (int)g.opt.threads;
    const size_t smem = range_smem((uint32_t)g.opt.tile_bits);
    const void *fn = range_kernel();
    if (!fn || smem > g.smem_optin) return -1.f;
    int grid = 0;
    if (ctx_grid(fn, nt, smem, &grid)) { cudaGetLastError(); return -1.f; }
    float best = -1.f;
    if (needs_buckets(probe)) {
        // the bucket pipeline (pre-pass and kernel per chunk), timed whole
        if (!g.ev0 && cudaEventCreate(&g.ev0) != cudaSuccess) return -1.f;
        if (!g.ev1 && cudaEventCreate(&g.ev1) != cudaSuccess) return -1.f;
        for (int rep = 0; rep < 2; rep++) {
            if (cudaEventRecord(g.ev0, g.stream) != cudaSuccess) return -1.f;
            if (run_persistent_buckets(probe, grid, smem, merge_grid_for(probe.nrec), g.d_result, g.stream, false))
                { cudaGetLastError(); return -1.f; }
            if (cudaEventRecord(g.ev1, g.stream) != cudaSuccess) return -1.f;
            if (cudaStreamSynchronize(g.stream) != cudaSuccess) return -1.f;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, g.ev0, g.ev1) != cudaSuccess) return -1.f;
            if (best < 0 || ms < best) best = ms;
        }
        return best;
    }
    RangeParams p;
    fill_params(probe, (uint32_t)g.opt.tile_bits, p);
    for (int rep = 0; rep < 2; rep++) {
        if (launch_set_params(g.stream, g.d_params, p) != cudaSuccess) return -1.f;
        if (enqueue_persistent(g.stream, probe, g.d_result, grid, smem, merge_grid_for(probe.nrec), true))
            return -1.f;
        if (cudaStreamSynchronize(g.stream) != cudaSuccess) return -1.f;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g.ev0, g.ev1) != cudaSuccess) return -1.f;
        if (best < 0 || ms < best) best = ms;
    }
    return best;
}

void load_tune_file()
{
    const char *path = getenv("GB_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[400];
    long long a, b, c, d, e, h, w, bw, bm, bt;
    while (fscanf(f, "%399s %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld", key, &a, &b, &c, &d, &e, &h, &w, &bw,
                  &bm, &bt) == 11)
        g.tuned[key] = TuneCfg{a, b, c, d, e, h, w, bw, bm, bt};
    fclose(f);
}

void save_tune_file()
{
    const char *path = getenv("GB_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (const auto &kv : g.tuned)
        fprintf(f, "%s %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld\n", kv.first.c_str(),
                (long long)kv.second.tile_bits, (long long)kv.second.threads, (long long)kv.second.search_chunks,
                (long long)kv.second.pattern_max, (long long)kv.second.search_pmax,
                (long long)kv.second.tier_b_min, (long long)kv.second.wheel, (long long)kv.second.builder_warps,
                (long long)kv.second.bucket_min, (long long)kv.second.bucket_chunk_tiles);
    fclose(f);
}

// Pick (and cache) the configuration for cp's range class; cp.ntiles follows
// the chosen tile size.
int maybe_autotune(CallPlan &cp)
{
    if (!g.opt.autotune) return GB_OK;
    NvtxRange nv("gb: autotune");
    if (g.tuned.empty()) load_tune_file();
    const std::string key = tune_key(cp);
    auto it = g.tuned.find(key);
    int rc;
    if (it == g.tuned.end()) {
        CallPlan probe;
        probe.n_total = std::min<uint64_t>(cp.n_total, 1ull << 30);
        probe.n0 = cp.n0 + 2 * (cp.n_total - probe.n_total);
        probe.nrec = ((probe.n_total - 1) >> g.seg_bits) + 1;
        if ((rc = ensure_records(probe.nrec))) return rc;
        TuneCfg best = current_cfg();
        float best_ms = time_probe(probe);
        std::vector<std::pair<int64_t TuneCfg::*, std::vector<int64_t>>> axes = {
            {&TuneCfg::builder_warps, {0, 8, 12, 16}},       // single-role or pipelined kernel
            {&TuneCfg::search_chunks, {4, 6, 8}},
            {&TuneCfg::tier_b_min, {4096, 8192, 16384, 65536}},
            {&TuneCfg::threads, {256, 512, 768, 1024}},         // 4, 2, 1 or 1 CTAs per SM
            {&TuneCfg::tile_bits, {15, 16, 17, 18, 19, 20, 21}}, // 2^21 never fits shared memory
            {&TuneCfg::wheel, {7, 13}},
            {&TuneCfg::pattern_max, {13, 31, 61}},
            {&TuneCfg::search_pmax, {0, 4096, 8192, 16384}},
        };
        if (needs_buckets(cp)) {
            // where the bucket pre-pass starts (0 = four window spans) and its chunk size
            axes.push_back({&TuneCfg::bucket_min, {0, 1 << 21, 1 << 24}});
            axes.push_back({&TuneCfg::bucket_chunk_tiles, {512, 2048, 8192}});
        }
        for (int pass = 0; pass < 2; pass++) {
            for (const auto &ax : axes) {
                for (int64_t v : ax.second) {
                    TuneCfg c = best;
                    c.*(ax.first) = v;
                    if (c.*(ax.first) == best.*(ax.first)) continue;
                    if (c.search_pmax && c.search_pmax >= (int64_t)g.p_max) continue;
                    if ((rc = apply_cfg(c))) return rc;
                    // the pipelined kernel holds two windows: take the largest
                    // tile that fits next to the other values
                    while (g.opt.tile_bits > 15 && range_smem((uint32_t)g.opt.tile_bits) > g.smem_optin)
                        g.opt.tile_bits--;
                    c.tile_bits = g.opt.tile_bits;
                    const float ms = time_probe(probe);
                    // a change must gain 0.5 % (the probe's repeat spread is below 0.1 %)
                    if (ms > 0.f && (best_ms < 0.f || ms < 0.995f * best_ms)) { best = c; best_ms = ms; }
                }
            }
        }
        if ((rc = apply_cfg(best))) return rc;
        g.tuned[key] = best;
        save_tune_file();
    } else if ((rc = apply_cfg(it->second))) {
        return rc;
    }
    cp.ntiles = ((cp.n_total - 1) >> g.opt.tile_bits) + 1;
    return GB_OK;
}

// The async pipeline's graph for this configuration and result pointer,
// captured on first use, with its set-params node given this call's params.
int async_graph(const CallPlan &cp, const RangeParams &p, gb_result *dev_out, int grid, size_t smem, int mg)
{
    GraphKey key;
    key.fn = range_kernel(); key.grid = grid; key.nt = (int)g.opt.threads; key.wheel = (int)g.opt.wheel;
    key.merge_grid = mg; key.clear_records = g.opt.tile_bits < g.seg_bits ? 1 : 0; key.smem = smem;
    key.recs = g.d_recs; key.olist = g.d_olist; key.olist_wcap = g.olist_wcap; key.olist_ctas = g.olist_ctas;
    const Tables tk = make_tables();
    key.aperm = tk.aperm; key.aperm_len = tk.aperm_len; key.askew = tk.askew;
    if (!g.aexec || !(key == g.akey) || g.aout != dev_out) {
        if (g.aexec) { cudaGraphExecDestroy(g.aexec); g.aexec = nullptr; }
        if (g.agraph) { cudaGraphDestroy(g.agraph); g.agraph = nullptr; }
        g.anode = nullptr;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_set_params(g.stream, g.d_params, p);
        int rc = e == cudaSuccess ? enqueue_persistent(g.stream, cp, dev_out, grid, smem, mg)
                                  : cuda_status(e, "params kernel");
        cudaError_t e2 = cudaStreamEndCapture(g.stream, &graph);
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e2 != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_status(e2, "graph capture"); }
        // the set-params node: the graph's kernel node that runs that kernel
        size_t nn = 0;
        e = cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
        g.anode = nullptr;
        for (size_t i = 0; e == cudaSuccess && i < nn && !g.anode; i++) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess && kp.func == set_params_kernel_ptr())
                g.anode = nodes[i];
        }
        if (e == cudaSuccess && !g.anode) e = cudaErrorInvalidValue;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.aexec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            g.aexec = nullptr;
            g.anode = nullptr;
            return cuda_status(e, "async graph");
        }
        // the node handle stays valid only while its graph exists: keep the
        // graph for later parameter updates of the instantiated copy
        g.agraph = graph;
        g.akey = key;
        g.aout = dev_out;
        return GB_OK;                                  // captured with this call's params
    }
    RangeParams *dst = g.d_params;
    RangeParams pv = p;
    void *args[] = {(void *)&dst, (void *)&pv};
    cudaKernelNodeParams kp{};
    kp.func = (void *)set_params_kernel_ptr();
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CK(cudaGraphExecKernelNodeSetParams(g.aexec, g.anode, &kp));
    return GB_OK;
}

int run_persistent(uint64_t lo, uint64_t hi, CallPlan &cp)
{
    int rc = plan_range(lo, hi, cp);
    if (rc) return rc;
    if (!cp.n_total) return GB_OK;
    if ((rc = prepare_common(cp))) return rc;
    if ((rc = maybe_autotune(cp))) return rc;
    begin_progress(cp.ntiles, cp.n_total, 1ull << g.opt.tile_bits);
    const uint32_t tile_bits = (uint32_t)g.opt.tile_bits;
    const int nt = (int)g.opt.threads;
    const size_t smem = range_smem(tile_bits);
    const void *fn = range_kernel();
    int grid = 0;
    if ((rc = ctx_grid(fn, nt, smem, &grid))) return rc;
    const int mg = merge_grid_for(cp.nrec);
    if (needs_buckets(cp)) return run_persistent_buckets(cp, grid, smem, mg, g.d_result, g.stream, true);
    fill_params(cp, tile_bits, *g.h_params);
    const int clear_records = g.opt.tile_bits < g.seg_bits ? 1 : 0;
    if (g.opt.use_graph) {
        GraphKey key;
        key.fn = fn; key.grid = grid; key.nt = nt; key.wheel = (int)g.opt.wheel; key.merge_grid = mg;
        key.clear_records = clear_records; key.smem = smem; key.recs = g.d_recs;
        key.olist = g.d_olist; key.olist_wcap = g.olist_wcap; key.olist_ctas = g.olist_ctas;
        const Tables tk = make_tables();
        key.aperm = tk.aperm; key.aperm_len = tk.aperm_len; key.askew = tk.askew; key.askew = tk.askew;
        if (!(key == g.gkey) || !g.gexec) {
            if (g.gexec) { cudaGraphExecDestroy(g.gexec); g.gexec = nullptr; }
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemcpyAsync(g.d_params, g.h_params, sizeof(RangeParams),
                                            cudaMemcpyHostToDevice, g.stream);
            int rc2 = e == cudaSuccess ? enqueue_persistent(g.stream, cp, g.d_result, grid, smem, mg)
                                       : cuda_status(e, "params copy");
            if (rc2 == GB_OK) {
                e = cudaMemcpyAsync(g.h_result, g.d_result, sizeof(gb_result), cudaMemcpyDeviceToHost,
                                    g.stream);
                rc2 = cuda_status(e, "result copy");
            }
            cudaError_t e2 = cudaStreamEndCapture(g.stream, &graph);
            if (rc2) { if (graph) cudaGraphDestroy(graph); return rc2; }
            CK(e2);
            e = cudaGraphInstantiate(&g.gexec, graph, 0);
            cudaGraphDestroy(graph);
            CK(e);
            g.gkey = key;
        }
        {
            NvtxRange nv("gb: graph replay");
            CK(cudaGraphLaunch(g.gexec, g.stream));
        }
        g.stats.graph_replays++;
    } else {
        CK(cudaMemcpyAsync(g.d_params, g.h_params, sizeof(RangeParams), cudaMemcpyHostToDevice, g.stream));
        if ((rc = enqueue_persistent(g.stream, cp, g.d_result, grid, smem, mg, g.opt.time_kernel != 0)))
            return rc;
        CK(cudaMemcpyAsync(g.h_result, g.d_result, sizeof(gb_result), cudaMemcpyDeviceToHost, g.stream));
    }
    CK(cudaStreamSynchronize(g.stream));
    CK(cudaGetLastError());
    g.stats.kernel_launches += 3;
    g.stats.tiles += cp.ntiles;
    return GB_OK;
}

void finish_stats(const CallPlan &cp, const gb_result &r)
{
    g.stats.calls++;
    g.stats.n_verified += cp.n_total;
    g.stats.n_slow += r.n_slow;
}

int copy_records(const CallPlan &cp, gb_seg_record *buf, size_t cap, size_t *n_written)
{
    if (n_written) *n_written = (size_t)cp.nrec;
    if (!buf || !cap || !cp.nrec) return GB_OK;
    size_t n = (size_t)std::min<uint64_t>(cap, cp.nrec);
    std::vector<DevRec> h(n);
    CK(cudaMemcpy(h.data(), g.d_recs, n * sizeof(DevRec), cudaMemcpyDeviceToHost));
    for (size_t r = 0; r < n; r++) {
        const DevRec &d = h[r];
        gb_seg_record &o = buf[r];
        memset(&o, 0, sizeof o);
        uint64_t kfirst = (uint64_t)r << g.seg_bits;
        o.n_first = cp.n0 + 2 * kfirst;
        o.n_count = d.n_count;
        o.max_pmin = d.key >> KEY_SHIFT;
        o.argmax_n = d.key ? o.n_first + 2 * (KEY_KMASK - (d.key & KEY_KMASK)) : 0;
        o.sum_pmin = d.sum;
        o.wsum_pmin = d.wsum;
        for (int b = 0; b < HIST_BINS; b++) o.hist[b] = d.hist[b];
        o.n_slow = d.n_slow;
        o.counterexample_n = d.ce_inv ? ~d.ce_inv : 0;
    }
    return GB_OK;
}

int run_plain(uint64_t lo, uint64_t hi, CallPlan &cp)
{
    int rc = plan_range(lo, hi, cp);
    if (rc) return rc;
    if (!cp.n_total) return GB_OK;
    if (needs_buckets(cp)) {
        set_error("the plain form has no bucket pass: its ranges must keep sqrt(n) below the "
                  "bucket bound (%llu)", (unsigned long long)bucket_bound());
        return GB_EINVAL;
    }
    if ((rc = prepare_common(cp))) return rc;
    const uint32_t sbits = (uint32_t)g.opt.plain_seg_bits;
    const uint64_t S = 1ull << sbits;
    const uint32_t Z = 1u << g.opt.plain_slice_bits;
    const uint32_t kb = 32u * g.k_words;
    const size_t need_words = (S + kb) / 32 + 8;
    if (g.gwin_words < need_words) {
        dev_free(&g.d_gwin, 4 * g.gwin_words);
        g.gwin_words = 0;
        if ((rc = dev_alloc(&g.d_gwin, 4 * need_words))) return rc;
        g.gwin_words = need_words;
    }
    // bit-parallel search: 1,024-thread CTAs over sub-tiles of 2^sub_bits n
    const int pbc = (int)g.opt.plain_search_chunks;
    const uint32_t sub_bits = std::min<uint32_t>(sbits, std::max<uint32_t>(12, std::min<uint32_t>(17, sbits - 9)));
    int bgrid = 0;
    size_t bsmem = 0;
    if (pbc) {
        bsmem = 4ull * ((g.k_words + 3) & ~3u);
        const void *bfn = plain_bulk_ptr(pbc);
        if (!bfn) { set_error("plain_search_chunks must be 0, 4, 6 or 8"); return GB_EINVAL; }
        if ((rc = occupancy_grid(bfn, 1024, bsmem, &bgrid))) return rc;
        if ((rc = ensure_olist(bgrid, 1024, sub_bits, true))) return rc;
        invalidate_graphs();                         // the persistent graph's slots changed
    } else if (g.pm_cap < S) {
        dev_free(&g.d_pm, 4 * g.pm_cap);
        g.pm_cap = 0;
        if ((rc = dev_alloc(&g.d_pm, 4 * S))) return rc;
        g.pm_cap = S;
    }
    const int nt = (int)g.opt.threads;
    const size_t smem = 4ull * (wheel_pattern_words((int)g.opt.wheel) + Z / 32 + 4);
    const void *fn = slice_kernel_ptr((int)g.opt.wheel, nt);
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fill_params(cp, sbits, *g.h_params);
    Tables t = make_tables();
    CK(cudaMemcpyAsync(g.d_params, g.h_params, sizeof(RangeParams), cudaMemcpyHostToDevice, g.stream));
    CK(launch_clear(g.stream, g.d_params, g.d_recs, g.d_ctrl, 1, 4 * g.sms));
    const uint64_t nseg = ((cp.n_total - 1) >> sbits) + 1;
    begin_progress(nseg, cp.n_total, S);
    const uint32_t chunk = (uint32_t)std::min<uint64_t>(1ull << 14, 1ull << g.seg_bits);
    uint64_t launches = 1;
    for (uint64_t s = 0; s < nseg; s++) {
        NvtxRange nv("gb: plain segment");
        const uint64_t k0 = s << sbits;
        const uint32_t cnt = (uint32_t)std::min<uint64_t>(S, cp.n_total - k0);
        const uint64_t n_lo = cp.n0 + 2 * k0;
        const uint64_t h = n_lo >> 1;
        const bool neg = h < kb;
        const uint64_t half_abs = neg ? kb - h : h - kb;
        const uint32_t j_end = cnt + kb - 1;
        const int grid = (int)((j_end + Z - 1) / Z);
        CK(launch_slice_sieve((int)g.opt.wheel, nt, grid, smem, g.stream, half_abs, neg ? 1 : 0, j_end, Z,
                              t, g.d_gwin, (uint32_t)g.gwin_words, g.d_ctrl));
        if (pbc) {
            RangeParams ps = *g.h_params;
            ps.tile_bits = sub_bits;
            const uint32_t nsub = (uint32_t)((cnt + (1ull << sub_bits) - 1) >> sub_bits);
            CK(launch_plain_bulk(pbc, std::min<int>(bgrid, (int)nsub), bsmem, g.stream, ps, k0 >> sub_bits, nsub, t,
                                 g.d_gwin, g.d_recs, g.d_ctrl));
            launches -= 1;
        } else {
            CK(launch_plain_search(g.stream, 8 * g.sms, g.d_params, g.d_gwin, g.d_PR, n_lo, cnt, g.d_pm,
                                   g.d_ctrl));
            CK(launch_plain_reduce(g.stream, g.d_params, g.d_pm, k0, n_lo, cnt, chunk, g.d_recs, g.d_ctrl));
        }
        // the per-segment status round trip of the paper's worker loop
        CK(cudaMemcpyAsync(g.h_flags, &g.d_ctrl->flags, 4, cudaMemcpyDeviceToHost, g.stream));
        CK(cudaStreamSynchronize(g.stream));
        *(volatile unsigned long long *)g.h_progress += 1;    // one segment done
        launches += 3;
    }
    CK(launch_merge(g.stream, merge_grid_for(cp.nrec), g.d_params, g.d_recs, g.d_ctrl, g.d_parts,
                    g.d_result));
    CK(cudaMemcpyAsync(g.h_result, g.d_result, sizeof(gb_result), cudaMemcpyDeviceToHost, g.stream));
    CK(cudaStreamSynchronize(g.stream));
    CK(cudaGetLastError());
    g.stats.kernel_launches += launches + 1;
    g.stats.tiles += nseg;
    return GB_OK;
}

void release_all()
{
    g_ready = false;
    serve_stop();
    ctx_serve_end();
    if (g.gexec) { cudaGraphExecDestroy(g.gexec); g.gexec = nullptr; }
    invalidate_graphs();
    if (g.aexec) { cudaGraphExecDestroy(g.aexec); g.aexec = nullptr; }
    if (g.agraph) { cudaGraphDestroy(g.agraph); g.agraph = nullptr; }
    dev_free(&g.d_primes, 4ull * ((g.nprimes + 3) & ~3ull));
    dev_free(&g.d_recip, 8ull * ((g.nprimes + 3) & ~3ull));
    dev_free(&g.d_PR, 4ull * g.k_words);
    dev_free(&g.d_params, sizeof(RangeParams));
    dev_free(&g.d_ctrl, sizeof(Ctrl));
    dev_free(&g.d_recs, sizeof(DevRec) * g.rec_cap);
    dev_free(&g.d_parts, merge_part_bytes() * MERGE_GRID_CAP);
    dev_free(&g.d_result, sizeof(gb_result));
    dev_free(&g.d_gwin, 4 * g.gwin_words);
    dev_free(&g.d_pm, 4 * g.pm_cap);
    dev_free(&g.d_bk_counts, 4 * g.bk_tiles_cap);
    dev_free(&g.d_bk_blk, 4 * g.bk_tiles_cap * bucket_grid());
    dev_free(&g.d_bk_off, 8 * g.bk_tiles_cap);
    dev_free(&g.d_bk_ent, 4 * g.bk_ent_cap);
    dev_free(&g.d_olist, 4 * g.olist_cap);
    dev_free(&g.d_aperm, 4ull * g.aperm_len);
    dev_free(&g.d_askew, 8ull * ASKEW_ENTRIES);
    dev_free(&g.d_phase, 8ull * PH_COUNT);
    if (g.h_params) cudaFreeHost(g.h_params);
    if (g.h_result) cudaFreeHost(g.h_result);
    if (g.h_flags) cudaFreeHost(g.h_flags);
    g_progress_ptr = nullptr;
    if (g.h_progress) cudaFreeHost(g.h_progress);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.ev0) cudaEventDestroy(g.ev0);
    if (g.ev1) cudaEventDestroy(g.ev1);
    Options keep = g.opt;
    g = Ctx{};
    g.opt = keep;
}

// The window search bound: the caller's P_max unless "search_pmax" sets a
// different one.  It only decides which n take the slow path; n_slow still
// counts p_min > P_max, so the records do not depend on it.
uint32_t search_pmax()
{
    return g.opt.search_pmax > 0 ? (uint32_t)g.opt.search_pmax : g.p_max;
}

// Candidate words: bit i of word t <-> p = 2(32t + i) + 1, set iff p is an
// odd prime <= the search bound; stored bit-reversed for the clz search.
int build_candidates()
{
    const uint32_t ps = search_pmax();
    const uint32_t K = (ps + 1) / 2;
    const uint32_t kw = (K + 31) / 32;
    std::vector<uint32_t> cand = host_odd_primes(std::max<uint32_t>(ps, 3));
    std::vector<uint32_t> PR(kw, 0);
    for (uint32_t p : cand) {
        if (p > ps) break;
        uint32_t i = (p - 1) / 2;
        PR[i / 32] |= 1u << (i % 32);
    }
    for (auto &w : PR) w = bitrev32(w);
    dev_free(&g.d_PR, 4ull * g.k_words);
    g.k_words = 0;
    int rc;
    if ((rc = dev_alloc(&g.d_PR, 4ull * kw))) return rc;
    g.k_words = kw;
    CK(cudaMemcpy(g.d_PR, PR.data(), 4ull * kw, cudaMemcpyHostToDevice));
    invalidate_graphs();
    return GB_OK;
}

int init_locked(uint32_t p_max, uint32_t seg_bits)
{
    if (p_max < 2 || p_max > (1u << 20)) { set_error("p_max must be in [2, 2^20]"); return GB_EINVAL; }
    if (seg_bits < 5 || seg_bits > 40) { set_error("seg_bits must be in [5, 40]"); return GB_EINVAL; }
    if (g.inited) release_all();
    g.opt = Options{};               // a new context starts from the default options
    fault_configure();
    CK(cudaGetDevice(&g.device));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, g.device));
    g.sms = prop.multiProcessorCount;
    snprintf(g.dev_name, sizeof g.dev_name, "%s", prop.name);
    g.smem_optin = prop.sharedMemPerBlockOptin;
    CK(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    g.p_max = p_max;
    g.seg_bits = seg_bits;
    int rc;
    if ((rc = build_candidates())) return rc;
    // bootstrap base primes <= 2^16
    g.h_small = host_odd_primes(1u << 16);
    g.nprimes = g.h_small.size();
    // padded with zeros to a multiple of four entries (four-wide loads)
    const size_t padded = (g.nprimes + 3) & ~(size_t)3;
    std::vector<uint32_t> pr_h(g.h_small);
    pr_h.resize(padded, 0u);
    std::vector<unsigned long long> rc_h(padded, 0ull);
    for (size_t i = 0; i < g.nprimes; i++) rc_h[i] = 0xFFFFFFFFFFFFFFFFull / g.h_small[i];
    if ((rc = dev_alloc(&g.d_primes, 4ull * padded))) return rc;
    if ((rc = dev_alloc(&g.d_recip, 8ull * padded))) return rc;
    CK(cudaMemcpy(g.d_primes, pr_h.data(), 4ull * padded, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g.d_recip, rc_h.data(), 8ull * padded, cudaMemcpyHostToDevice));
    g.table_limit = 1u << 16;
    if ((rc = dev_alloc(&g.d_params, sizeof(RangeParams)))) return rc;
    if ((rc = dev_alloc(&g.d_ctrl, sizeof(Ctrl)))) return rc;
    if ((rc = dev_alloc(&g.d_parts, merge_part_bytes() * MERGE_GRID_CAP))) return rc;
    if ((rc = dev_alloc(&g.d_result, sizeof(gb_result)))) return rc;
    CK(cudaMemset(g.d_ctrl, 0, sizeof(Ctrl)));
#ifdef GB_PHASE_CLOCKS
    if ((rc = dev_alloc(&g.d_phase, 8ull * PH_COUNT))) return rc;
    CK(cudaMemset(g.d_phase, 0, 8ull * PH_COUNT));
#endif
    CK(cudaMallocHost((void **)&g.h_params, sizeof(RangeParams)));
    CK(cudaMallocHost((void **)&g.h_result, sizeof(gb_result)));
    CK(cudaMallocHost((void **)&g.h_flags, 4));
    CK(cudaHostAlloc((void **)&g.h_progress, 64, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer((void **)&g.d_progress, g.h_progress, 0));
    *g.h_progress = 0;
    g_progress_ptr = g.h_progress;
    memset(&g.stats, 0, sizeof g.stats);
    g.inited = true;
    g_ready = true;
    if (g.opt.base_limit > 0 && (rc = ensure_table((uint64_t)g.opt.base_limit))) return rc;
    return GB_OK;
}

struct OptDesc {
    const char *key;
    int64_t Options::*field;
    int64_t lo, hi;
};

const OptDesc kOpts[] = {
    {"tile_bits", &Options::tile_bits, 10, 20},
    {"threads", &Options::threads, 256, 1024},
    {"ctas_per_sm", &Options::ctas_per_sm, 0, 8},
    {"wheel", &Options::wheel, 7, 13},
    {"pattern_max", &Options::pattern_max, 7, 61},
    {"tier_b_min", &Options::tier_b_min, 3, 1 << 16},
    {"base_limit", &Options::base_limit, 0, 0xFFFFFFFFll},
    {"mem_budget_mb", &Options::mem_budget_mb, 16, 1 << 22},
    {"plain_seg_bits", &Options::plain_seg_bits, 20, 30},
    {"plain_slice_bits", &Options::plain_slice_bits, 12, 20},
    {"plain_search_chunks", &Options::plain_search_chunks, 0, 8},
    {"use_graph", &Options::use_graph, 0, 1},
    {"slow_cap", &Options::slow_cap, 6, 24},
    {"timeout_ms", &Options::timeout_ms, 1, 1ll << 40},
    {"serve_batch_tiles", &Options::serve_batch_tiles, 1, 1 << 24},
    {"time_kernel", &Options::time_kernel, 0, 1},
    {"bucket_min", &Options::bucket_min, 0, 1 << 28},
    {"bucket_chunk_tiles", &Options::bucket_chunk_tiles, 1, 8192},
    {"search_pmax", &Options::search_pmax, 0, 1 << 20},
    {"search_chunks", &Options::search_chunks, 0, 8},
    {"autotune", &Options::autotune, 0, 1},
    {"builder_warps", &Options::builder_warps, 0, 16},
    {"debug_smem_limit", &Options::debug_smem_limit, 0, 1 << 20},
};

}  // namespace

// ---------------------------------------------------------------------------
// hooks used by the serving loop (gb_serve.cpp)
// ---------------------------------------------------------------------------
namespace gbk {
std::recursive_mutex &ctx_mutex() { return g_mu; }
bool ctx_ready() { return g_ready.load(); }
// Options are plain aligned 64-bit values: read without the context lock so
// that gb_submit never waits for a running batch.
int64_t ctx_option(const char *key)
{
    for (const auto &o : kOpts)
        if (!strcmp(o.key, key)) return __atomic_load_n(&(g.opt.*o.field), __ATOMIC_RELAXED);
    return 0;
}
int ctx_verify(uint64_t lo, uint64_t hi, gb_result *out)
{
    CallPlan cp;
    int rc = run_persistent(lo, hi, cp);
    if (rc) { if (out) { empty_result(out); out->status = rc; } return rc; }
    if (!cp.n_total) { empty_result(out); finish_stats(cp, gb_result{}); return GB_OK; }
    if (out) *out = *g.h_result;
    finish_stats(cp, *g.h_result);
    return g.h_result->status;
}
void ctx_error(const char *msg) { set_error("%s", msg); }
gb_stats_t &ctx_stats() { return g.stats; }
size_t ctx_device_bytes() { return g.device_bytes; }

// ---- serving engine state (device side of gb_submit / gb_poll) -------------
namespace {
struct ServeDev {
    bool ready = false;
    int max_slots = 0, max_items = 0;
    cudaStream_t st = nullptr, cp = nullptr;     // batches; harvest copies
    cudaEvent_t ev[2] = {nullptr, nullptr};
    SlotDev *d_slots = nullptr, *h_slots = nullptr;
    unsigned long long *d_items[2] = {nullptr, nullptr}, *h_items[2] = {nullptr, nullptr};
    Ctrl *d_ctrl = nullptr;
    const void *fn = nullptr;
    int nt = 0, grid = 0, wheel = 13;           // the serving kernel's thread count and WHEEL
    size_t smem = 0;
    // bucket pre-pass of served requests: own stream, per-slot arrays from the
    // stream-ordered pool, released after the request's last batch
    cudaStream_t pp = nullptr;
    cudaEvent_t ev_prep = nullptr;
    unsigned int *d_cnt = nullptr, *d_blk = nullptr;
    unsigned long long *h_total = nullptr;
    std::vector<unsigned long long *> bk_off;
    std::vector<uint32_t *> bk_ent;
    // open-mask slots of the serving kernel (its batches run one after another)
    uint32_t *d_olist = nullptr;
    size_t olist_cap = 0;
    uint32_t olist_wcap = 0;
};
ServeDev sv;
constexpr uint32_t SERVE_BUCKET_MAX_TILES = 8192;
}  // namespace

int ctx_serve_begin(int max_slots, int max_items)
{
    if (sv.ready) return GB_OK;
    int rc;
    sv.max_slots = max_slots;
    sv.max_items = max_items;
    CK(cudaStreamCreateWithFlags(&sv.st, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&sv.cp, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&sv.ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&sv.ev[1], cudaEventDisableTiming));
    if ((rc = dev_alloc(&sv.d_slots, sizeof(SlotDev) * max_slots))) return rc;
    CK(cudaStreamCreateWithFlags(&sv.pp, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&sv.ev_prep, cudaEventDisableTiming));
    if ((rc = dev_alloc(&sv.d_cnt, 4ull * (SERVE_BUCKET_MAX_TILES + 1)))) return rc;
    if ((rc = dev_alloc(&sv.d_blk, 4ull * (SERVE_BUCKET_MAX_TILES + 1) * bucket_grid()))) return rc;
    CK(cudaMallocHost((void **)&sv.h_total, 8));
    sv.bk_off.assign(max_slots, nullptr);
    sv.bk_ent.assign(max_slots, nullptr);
    if ((rc = dev_alloc(&sv.d_ctrl, sizeof(Ctrl)))) return rc;
    CK(cudaMallocHost((void **)&sv.h_slots, sizeof(SlotDev) * max_slots));
    for (int b = 0; b < 2; b++) {
        if ((rc = dev_alloc(&sv.d_items[b], 8ull * max_items))) return rc;
        CK(cudaMallocHost((void **)&sv.h_items[b], 8ull * max_items));
    }
    // kernel configuration: the context's, when a serving instantiation exists
    sv.nt = (int)g.opt.threads;
    int wheel = (int)g.opt.wheel, bc = (int)g.opt.search_chunks;
    sv.fn = serve_kernel_ptr(wheel, sv.nt, bc);
    if (!sv.fn) { sv.nt = 1024; bc = 6; wheel = 13; sv.fn = serve_kernel_ptr(13, 1024, 6); }
    sv.wheel = wheel;                               // its tables and pattern block follow it
    sv.smem = persistent_smem((uint32_t)g.opt.tile_bits, wheel);
    if ((rc = occupancy_grid(sv.fn, sv.nt, sv.smem, &sv.grid))) return rc;
    // open-mask slots of the search (both forms use them)
    sv.olist_wcap = olist_slice(sv.nt);
    sv.olist_cap = (size_t)sv.grid * (size_t)(sv.nt / 32) * sv.olist_wcap;
    if ((rc = dev_alloc(&sv.d_olist, 4 * sv.olist_cap))) return rc;
    (void)bc;
    sv.ready = true;
    return GB_OK;
}

void ctx_serve_end()
{
    if (!sv.ready) return;
    cudaStreamSynchronize(sv.pp);
    cudaStreamSynchronize(sv.st);
    cudaStreamSynchronize(sv.cp);
    for (size_t i = 0; i < sv.bk_off.size(); i++) {
        if (sv.bk_off[i]) cudaFreeAsync(sv.bk_off[i], sv.st);
        if (sv.bk_ent[i]) cudaFreeAsync(sv.bk_ent[i], sv.st);
    }
    cudaStreamSynchronize(sv.st);
    dev_free(&sv.d_cnt, 4ull * (SERVE_BUCKET_MAX_TILES + 1));
    dev_free(&sv.d_blk, 4ull * (SERVE_BUCKET_MAX_TILES + 1) * bucket_grid());
    if (sv.h_total) cudaFreeHost(sv.h_total);
    if (sv.ev_prep) cudaEventDestroy(sv.ev_prep);
    if (sv.pp) cudaStreamDestroy(sv.pp);
    dev_free(&sv.d_slots, sizeof(SlotDev) * sv.max_slots);
    dev_free(&sv.d_ctrl, sizeof(Ctrl));
    dev_free(&sv.d_olist, 4 * sv.olist_cap);
    for (int b = 0; b < 2; b++) {
        dev_free(&sv.d_items[b], 8ull * sv.max_items);
        if (sv.h_items[b]) cudaFreeHost(sv.h_items[b]);
        if (sv.ev[b]) cudaEventDestroy(sv.ev[b]);
    }
    if (sv.h_slots) cudaFreeHost(sv.h_slots);
    if (sv.st) cudaStreamDestroy(sv.st);
    if (sv.cp) cudaStreamDestroy(sv.cp);
    sv = ServeDev{};
}

// Validate a request and make sure the base-prime table covers it.  The
// caller has no batch in flight when the table may have to grow.
int ctx_serve_plan(uint64_t lo, uint64_t hi, ServePlan *sp)
{
    CallPlan cp;
    int rc = plan_range(lo, hi, cp);
    if (rc) return rc;
    sp->n0 = cp.n0;
    sp->n_total = cp.n_total;
    sp->ntiles = cp.ntiles;
    if (!cp.n_total) return GB_OK;
    if (cp.n_total >= (1ull << SERVE_SLOT_SHIFT)) {
        set_error("a served request must hold fewer than 2^40 even n");
        return GB_EINVAL;
    }
    return ensure_table(isqrt_host(cp.n0 + 2 * (cp.n_total - 1)));
}

bool ctx_serve_needs_table(uint64_t lo, uint64_t hi)
{
    CallPlan cp;
    if (plan_range(lo, hi, cp) || !cp.n_total) return false;
    return isqrt_host(cp.n0 + 2 * (cp.n_total - 1)) > g.table_limit;
}

// Upper estimate of the bucket bytes a request needs (admission accounting):
// hits = n * sum over bucketed primes of 1/p ~ n * ln(ln sqrt(hi) / ln B),
// 4 bytes each, plus 8 bytes of offsets per tile; 0 when no bucket is used.
uint64_t ctx_serve_bucket_estimate(uint64_t lo, uint64_t hi)
{
    CallPlan cp;
    if (plan_range(lo, hi, cp) || !cp.n_total) return 0;
    const uint64_t root = isqrt_host(cp.n0 + 2 * (cp.n_total - 1));
    const uint64_t B = bucket_bound();
    if (root < B || cp.ntiles > SERVE_BUCKET_MAX_TILES) return 0;
    const double w = std::log(std::log((double)root) / std::log((double)B)) + 0.01;
    return (uint64_t)(4.0 * 1.2 * w * (double)cp.n_total * (1.0 + 32.0 * g.k_words / (1ull << g.opt.tile_bits))) +
           8ull * (cp.ntiles + 1) + 4096;
}

// Write the request's params into its slot; when its base primes reach the
// bucket bound, run the bucket pre-pass for all its tiles on the prep stream
// (the next batch waits for it).  *bucket_bytes receives what it holds.
int ctx_serve_init_slot(int slot, const ServePlan &sp, uint64_t *bucket_bytes)
{
    *bucket_bytes = 0;
    SlotDev &h = sv.h_slots[slot];
    memset(&h, 0, sizeof h);
    CallPlan cp;
    cp.n0 = sp.n0;
    cp.n_total = sp.n_total;
    cp.ntiles = sp.ntiles;
    cp.nrec = 1;
    fill_params(cp, (uint32_t)g.opt.tile_bits, h.prm);
    h.prm.rec_bits = SERVE_SLOT_SHIFT;
    const uint64_t root = isqrt_host(cp.n0 + 2 * (cp.n_total - 1));
    const uint64_t B = bucket_bound();
    if (root < B || cp.ntiles > SERVE_BUCKET_MAX_TILES) {
        CK(cudaMemcpyAsync(&sv.d_slots[slot], &h, sizeof h, cudaMemcpyHostToDevice, sv.st));
        return GB_OK;
    }
    const uint32_t nt = (uint32_t)cp.ntiles;
    h.prm.bk_prime0 = count_odd_primes_below(B);
    Tables t = make_tables(sv.wheel);
    unsigned long long *off = nullptr;
    uint32_t *ent = nullptr;
    CK(cudaMemcpyAsync(&sv.d_slots[slot], &h, sizeof h, cudaMemcpyHostToDevice, sv.pp));
    CK(cudaMallocAsync((void **)&off, 8ull * (nt + 1), sv.pp));
    CK(cudaMemsetAsync(sv.d_cnt, 0, 4ull * nt, sv.pp));
    CK(launch_bucket_prepass(sv.pp, (int)bucket_grid(), &sv.d_slots[slot].prm, t, h.prm.bk_prime0, 0, nt, sv.d_cnt,
                             off, sv.d_blk, nullptr, 0, 0, nullptr));
    CK(cudaMemcpyAsync(sv.h_total, off + nt, 8, cudaMemcpyDeviceToHost, sv.pp));
    CK(cudaStreamSynchronize(sv.pp));
    const unsigned long long total = *sv.h_total;
    CK(cudaMallocAsync((void **)&ent, 4ull * total + 16, sv.pp));
    CK(launch_bucket_prepass(sv.pp, (int)bucket_grid(), &sv.d_slots[slot].prm, t, h.prm.bk_prime0, 0, nt, sv.d_cnt,
                             off, sv.d_blk, ent, 1, total, &sv.d_slots[slot].ctl));
    h.prm.bk_off = off;
    h.prm.bk_ent = ent;
    CK(cudaMemcpyAsync(&sv.d_slots[slot].prm, &h.prm, sizeof h.prm, cudaMemcpyHostToDevice, sv.pp));
    CK(cudaEventRecord(sv.ev_prep, sv.pp));
    CK(cudaStreamWaitEvent(sv.st, sv.ev_prep, 0));
    sv.bk_off[slot] = off;
    sv.bk_ent[slot] = ent;
    *bucket_bytes = 8ull * (nt + 1) + 4ull * total + 16;
    g.stats.kernel_launches += 3;
    return GB_OK;
}

// Give back a finished request's bucket arrays (stream-ordered after its
// last batch, which has completed).
void ctx_serve_release_slot(int slot)
{
    if (slot < 0 || slot >= (int)sv.bk_off.size()) return;
    if (sv.bk_off[slot]) cudaFreeAsync(sv.bk_off[slot], sv.st);
    if (sv.bk_ent[slot]) cudaFreeAsync(sv.bk_ent[slot], sv.st);
    sv.bk_off[slot] = nullptr;
    sv.bk_ent[slot] = nullptr;
}

unsigned long long *ctx_serve_items(int buf) { return sv.h_items[buf]; }

int ctx_serve_launch(int buf, size_t n)
{
    NvtxRange nv("gb: serving batch launch");
    CK(cudaMemcpyAsync(sv.d_items[buf], sv.h_items[buf], 8ull * n, cudaMemcpyHostToDevice, sv.st));
    CK(cudaMemsetAsync(sv.d_ctrl, 0, sizeof(Ctrl), sv.st));
    Tables t = make_tables(sv.wheel);
    t.olist = sv.d_olist;
    t.olist_wcap = sv.olist_wcap;
    t.olist_ctas = sv.d_olist ? (uint32_t)sv.grid : 0u;
    CK(launch_serve(sv.fn, sv.nt, sv.grid, sv.smem, sv.st, sv.d_items[buf], n, sv.d_slots, t, sv.d_ctrl));
    CK(cudaEventRecord(sv.ev[buf], sv.st));
    g.stats.kernel_launches += 1;
    g.stats.tiles += n;
    return GB_OK;
}

// Wait for batch buf; later copies on the harvest stream are ordered after
// it.  Touches only the serving streams and buffers, so the caller does not
// hold the context lock.
int ctx_serve_wait(int buf, int64_t timeout_ms)
{
    if (timeout_ms >= 0) {
        // bounded wait: poll the batch's event, give up after timeout_ms
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            cudaError_t q = cudaEventQuery(sv.ev[buf]);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) CK(q);
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
                set_error("serving batch did not finish within %lld ms", (long long)timeout_ms);
                return GB_ETIMEOUT;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
    CK(cudaStreamWaitEvent(sv.cp, sv.ev[buf], 0));
    CK(cudaStreamSynchronize(sv.cp));
    return GB_OK;
}

// Copy a finished request's record out (its last batch has completed);
// called without the context lock.
int ctx_serve_fetch(int slot, const ServePlan &sp, gb_result *out)
{
    // the record and the request's own control block are adjacent in its slot
    static_assert(offsetof(SlotDev, ctl) == offsetof(SlotDev, acc) + sizeof(DevRec), "slot layout");
    DevRec *h = &sv.h_slots[slot].acc;
    CK(cudaMemcpyAsync(h, &sv.d_slots[slot].acc, sizeof(DevRec) + sizeof(Ctrl), cudaMemcpyDeviceToHost, sv.cp));
    CK(cudaStreamSynchronize(sv.cp));
    const unsigned int flags = sv.h_slots[slot].ctl.flags;
    memset(out, 0, sizeof *out);
    out->n_first = sp.n0;
    out->n_count = h->n_count;
    out->max_pmin = h->key >> KEY_SHIFT;
    out->argmax_n = h->key ? sp.n0 + 2 * (KEY_KMASK - (h->key & KEY_KMASK)) : 0;
    out->sum_pmin = h->sum;
    out->wsum_pmin = h->wsum;
    for (int b = 0; b < HIST_BINS; b++) out->hist[b] = h->hist[b];
    out->n_slow = h->n_slow;
    const unsigned long long ci = h->ce_inv > sv.h_slots[slot].ctl.ce_inv ? h->ce_inv : sv.h_slots[slot].ctl.ce_inv;
    out->counterexample_n = ci ? ~ci : 0;
    int st = GB_OK;
    if (flags & F_INTERNAL) st = GB_EINTERNAL;
    else if (flags & F_SLOWCAP) st = GB_ESLOWPATH_LIMIT;
    else if (flags & F_OVERFLOW) st = GB_EOVERFLOW;
    else if (out->counterexample_n) st = GB_COUNTEREXAMPLE;
    out->status = st;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g.stats.calls++;
    g.stats.n_verified += sp.n_total;
    g.stats.n_slow += out->n_slow;
    return GB_OK;
}

size_t ctx_serve_slot_bytes() { return sizeof(SlotDev); }
}  // namespace gbk

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gb_init(uint32_t p_max, uint32_t seg_bits)
{
    serve_stop();                    // before the context lock: the loop takes it
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    int rc = init_locked(p_max, seg_bits);
    if (rc && g.inited) release_all();
    return rc;
}

int gb_set_option(const char *key, int64_t value)
{
    if (!key) { set_error("gb_set_option: null key"); return GB_EINVAL; }
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    for (const auto &o : kOpts) {
        if (strcmp(o.key, key)) continue;
        if (value < o.lo || value > o.hi) {
            set_error("option %s out of range [%lld, %lld]", key, (long long)o.lo, (long long)o.hi);
            return GB_EINVAL;
        }
        if (!strcmp(key, "threads") && value != 256 && value != 512 && value != 768 && value != 1024) {
            set_error("threads must be 256, 512, 768 or 1024");
            return GB_EINVAL;
        }
        if (!strcmp(key, "builder_warps") && value != 0 && value != 8 && value != 12 && value != 16) {
            set_error("builder_warps must be 0 (single-role kernel), 8, 12 or 16");
            return GB_EINVAL;
        }
        if (!strcmp(key, "bucket_min") && value != 0 && value < 64) {
            set_error("bucket_min must be 0 (automatic) or at least 64");
            return GB_EINVAL;
        }
        if ((!strcmp(key, "search_chunks") || !strcmp(key, "plain_search_chunks")) && value != 0 && value != 4 &&
            value != 6 && value != 8) {
            set_error("search_chunks must be 0 (per-n search), 4, 6 or 8");
            return GB_EINVAL;
        }
        if (!strcmp(key, "wheel") && value != 7 && value != 13) {
            set_error("wheel must be 7 or 13");
            return GB_EINVAL;
        }
        if (!strcmp(key, "search_pmax") && value != 0 && value < 2) {
            set_error("search_pmax must be 0 (= P_max) or in [2, 2^20]");
            return GB_EINVAL;
        }
        g.opt.*o.field = value;
        invalidate_graphs();
        if (!strcmp(key, "base_limit") && g.inited && value > 0) return ensure_table((uint64_t)value);
        if (!strcmp(key, "search_pmax") && g.inited) return build_candidates();
        return GB_OK;
    }
    set_error("unknown option '%s'", key);
    return GB_EINVAL;
}

int gb_get_option(const char *key, int64_t *value)
{
    if (!key || !value) return GB_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    for (const auto &o : kOpts)
        if (!strcmp(o.key, key)) { *value = g.opt.*o.field; return GB_OK; }
    if (!strcmp(key, "p_max")) { *value = g.p_max; return GB_OK; }
    if (!strcmp(key, "k_words")) { *value = g.k_words; return GB_OK; }
    if (!strcmp(key, "last_kernel_us")) {
        // duration of the last timed persistent kernel (time_kernel = 1); the
        // stream it ran on must have completed
        float ms = 0.f;
        if (!g.ev_pending || cudaEventElapsedTime(&ms, g.ev0, g.ev1) != cudaSuccess) {
            cudaGetLastError();
            *value = -1;
            return GB_OK;
        }
        *value = (int64_t)(ms * 1000.0f);
        return GB_OK;
    }
    if (!strcmp(key, "seg_bits")) { *value = g.seg_bits; return GB_OK; }
    // bounds checks of the GB_DEBUG build: whether this library has them, and
    // the site and byte offset of the first failure of the last range call
    // (0 if none; reading one waits for the context's work)
    if (!strcmp(key, "debug_build")) {
#ifdef GB_DEBUG
        *value = 1;
#else
        *value = 0;
#endif
        return GB_OK;
    }
    if (!strcmp(key, "debug_bounds_site") || !strcmp(key, "debug_bounds_offset")) {
        *value = 0;
        if (!g.d_ctrl) return GB_OK;
        Ctrl hc;
        if (cudaStreamSynchronize(g.stream) != cudaSuccess ||
            cudaMemcpy(&hc, g.d_ctrl, sizeof hc, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return GB_OK;
        }
        *value = !strcmp(key, "debug_bounds_site") ? hc.dbg_site : hc.dbg_off;
        return GB_OK;
    }
    // per-phase cycle sums of the last range call (builds with GB_PHASE_CLOCKS;
    // -1 otherwise); reading one waits for the context's work
    static const char *phase_keys[PH_COUNT] = {"phase_fill", "phase_mark", "phase_search", "phase_reduce",
                                               "phase_warp_bulk", "phase_warp_tail", "phase_claim",
                                               "phase_warp_tier_a", "phase_warp_tier_b"};
    for (int k = 0; k < PH_COUNT; k++) {
        if (strcmp(key, phase_keys[k])) continue;
        *value = -1;
        if (!g.d_phase) return GB_OK;
        unsigned long long v[PH_COUNT];
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(v, g.d_phase, sizeof v, cudaMemcpyDeviceToHost));
        *value = (int64_t)v[k];
        return GB_OK;
    }
    if (!strcmp(key, "sms")) { *value = g.sms; return GB_OK; }
    set_error("unknown option '%s'", key);
    return GB_EINVAL;
}

void gb_shutdown(void)
{
    serve_stop();                    // before the context lock: the loop takes it
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (g.inited) release_all();
}

int gb_verify_range(uint64_t lo, uint64_t hi, gb_result *out)
{
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!g.inited) { set_error("gb_init has not been called"); return GB_EINVAL; }
    if (!out) { set_error("gb_verify_range: null result pointer"); return GB_EINVAL; }
    return ctx_verify(lo, hi, out);
}

int gb_verify_range_segments(uint64_t lo, uint64_t hi, gb_seg_record *buf, size_t cap,
                             size_t *n_written, gb_result *out)
{
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!g.inited) { set_error("gb_init has not been called"); return GB_EINVAL; }
    CallPlan cp;
    int rc = run_persistent(lo, hi, cp);
    if (rc) { if (out) { empty_result(out); out->status = rc; } return rc; }
    if (!cp.n_total) {
        if (n_written) *n_written = 0;
        empty_result(out);
        return GB_OK;
    }
    if ((rc = copy_records(cp, buf, cap, n_written))) return rc;
    if (out) *out = *g.h_result;
    finish_stats(cp, *g.h_result);
    return g.h_result->status;
}

// What the tile indices of a claim block mean: the range's even-n grid, the
// tile and record sizes and P_max.  Callers that share a block must agree on
// all of them, or tiles would cover different n and records would not merge.
uint64_t claim_fingerprint(const CallPlan &cp)
{
    uint64_t h = 0x6a09e667f3bcc909ull;                // splitmix64-style mixing of the fields
    const uint64_t v[5] = {cp.n0, cp.n_total, (uint64_t)g.opt.tile_bits, (uint64_t)g.seg_bits, (uint64_t)g.p_max};
    for (uint64_t x : v) {
        h += x + 0x9e3779b97f4a7c15ull;
        h = (h ^ (h >> 30)) * 0xbf58476d1ce4e5b9ull;
        h = (h ^ (h >> 27)) * 0x94d049bb133111ebull;
        h ^= h >> 31;
    }
    return h ? h : 1;                                  // 0 marks a block no caller has used
}

// Cooperative form: the tiles of [lo, hi) are claimed from claim->next_tile, a
// counter in host memory that every cooperating caller (process, GPU) passes;
// this caller's records and result cover only the tiles it claimed.
int run_persistent_claimed(uint64_t lo, uint64_t hi, gb_claim_t *claim, CallPlan &cp)
{
    int rc = plan_range(lo, hi, cp);
    if (rc) return rc;
    if (!cp.n_total) return GB_OK;
    // the first caller stamps the block; the others must match it
    uint64_t expected = 0;
    const uint64_t fp = claim_fingerprint(cp);
    if (!__atomic_compare_exchange_n(&claim->fingerprint, &expected, fp, false, __ATOMIC_ACQ_REL,
                                     __ATOMIC_ACQUIRE) &&
        expected != fp) {
        set_error("gb_verify_range_claimed: the claim block belongs to another range or configuration "
                  "(range, tile_bits, seg_bits and P_max must match every other caller's)");
        return GB_EINVAL;
    }
    if ((rc = prepare_common(cp))) return rc;
    if (needs_buckets(cp)) {
        set_error("gb_verify_range_claimed: the range needs the bucket pre-pass (sqrt(n) at or above "
                  "bucket_min); split it with gb_verify_range instead");
        return GB_EINVAL;
    }
    begin_progress(cp.ntiles, cp.n_total, 1ull << g.opt.tile_bits);
    const uint32_t tile_bits = (uint32_t)g.opt.tile_bits;
    const int nt = (int)g.opt.threads;
    const size_t smem = range_smem(tile_bits);
    const void *fn = range_kernel();
    int grid = 0;
    if ((rc = ctx_grid(fn, nt, smem, &grid))) return rc;
    bool registered = false;
    cudaError_t e = cudaHostRegister(claim, sizeof *claim, cudaHostRegisterMapped | cudaHostRegisterPortable);
    if (e == cudaSuccess) registered = true;
    else if (e == cudaErrorHostMemoryAlreadyRegistered) cudaGetLastError();
    else return cuda_status(e, "cudaHostRegister(claim counter)");
    unsigned long long *d_claim = nullptr;
    e = cudaHostGetDevicePointer((void **)&d_claim, &claim->next_tile, 0);
    if (e == cudaSuccess) {
        fill_params(cp, tile_bits, *g.h_params);
        g.h_params->claim = d_claim;
        e = cudaMemcpyAsync(g.d_params, g.h_params, sizeof(RangeParams), cudaMemcpyHostToDevice, g.stream);
    }
    Tables t = make_tables();
    if (e == cudaSuccess) e = launch_clear(g.stream, g.d_params, g.d_recs, g.d_ctrl, 1, 4 * g.sms);
    if (e == cudaSuccess)
        e = launch_range_kernel(fn, nt, grid, smem, g.stream, g.d_params, t, g.d_recs, g.d_ctrl);
    if (e == cudaSuccess)
        e = launch_merge(g.stream, merge_grid_for(cp.nrec), g.d_params, g.d_recs, g.d_ctrl, g.d_parts, g.d_result);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g.h_result, g.d_result, sizeof(gb_result), cudaMemcpyDeviceToHost, g.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g.stream);
    if (registered) cudaHostUnregister(claim);
    if (e != cudaSuccess) return cuda_status(e, "claimed launch");
    g.stats.kernel_launches += 3;
    return GB_OK;
}

int gb_verify_range_claimed(uint64_t lo, uint64_t hi, gb_claim_t *claim, gb_seg_record *buf, size_t cap,
                            size_t *n_written, gb_result *out)
{
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!g.inited) { set_error("gb_init has not been called"); return GB_EINVAL; }
    if (!claim) { set_error("gb_verify_range_claimed: claim counter is NULL"); return GB_EINVAL; }
    CallPlan cp;
    int rc = run_persistent_claimed(lo, hi, claim, cp);
    if (rc) { if (out) { empty_result(out); out->status = rc; } return rc; }
    if (!cp.n_total) {
        if (n_written) *n_written = 0;
        empty_result(out);
        return GB_OK;
    }
    if ((rc = copy_records(cp, buf, cap, n_written))) return rc;
    if (out) *out = *g.h_result;
    finish_stats(cp, *g.h_result);
    return g.h_result->status;
}

int gb_verify_range_plain(uint64_t lo, uint64_t hi, gb_seg_record *buf, size_t cap,
                          size_t *n_written, gb_result *out)
{
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!g.inited) { set_error("gb_init has not been called"); return GB_EINVAL; }
    CallPlan cp;
    int rc = run_plain(lo, hi, cp);
    if (rc) { if (out) { empty_result(out); out->status = rc; } return rc; }
    if (!cp.n_total) {
        if (n_written) *n_written = 0;
        empty_result(out);
        return GB_OK;
    }
    if ((rc = copy_records(cp, buf, cap, n_written))) return rc;
    if (out) *out = *g.h_result;
    finish_stats(cp, *g.h_result);
    return g.h_result->status;
}

int gb_verify_range_async(uint64_t lo, uint64_t hi, gb_result *dev_out, void *stream)
{
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    if (!g.inited) { set_error("gb_init has not been called"); return GB_EINVAL; }
    if (!dev_out) { set_error("gb_verify_range_async: null result pointer"); return GB_EINVAL; }
    cudaStream_t st = stream ? (cudaStream_t)stream : g.stream;
    CallPlan cp;
    int rc = plan_range(lo, hi, cp);
    if (rc) return rc;
    if (!cp.n_total) {
        gb_result z;
        empty_result(&z);
        CK(cudaMemcpyAsync(dev_out, &z, sizeof z, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return GB_OK;
    }
    if ((rc = prepare_common(cp))) return rc;
    if ((rc = maybe_autotune(cp))) return rc;          // synchronises while it tunes
    begin_progress(cp.ntiles, cp.n_total, 1ull << g.opt.tile_bits);
    const uint32_t tile_bits = (uint32_t)g.opt.tile_bits;
    const int nt = (int)g.opt.threads;
    const size_t smem = range_smem(tile_bits);
    int grid = 0;
    if ((rc = ctx_grid(range_kernel(), nt, smem, &grid))) return rc;
    if (needs_buckets(cp)) {
        // the pre-pass sizes its buffers on the host, so this form synchronises
        rc = run_persistent_buckets(cp, grid, smem, merge_grid_for(cp.nrec), dev_out, st, false);
        if (rc) return rc;
        g.stats.calls++;
        g.stats.n_verified += cp.n_total;
        return GB_OK;
    }
    RangeParams p;
    fill_params(cp, tile_bits, p);
    const int mg = merge_grid_for(cp.nrec);
    const bool timed = g.opt.time_kernel != 0;
    if (g.opt.use_graph) {
        // the params travel as an argument of the graph's first kernel, so no
        // host buffer outlives the call
        if ((rc = async_graph(cp, p, dev_out, grid, smem, mg))) return rc;
        // timing events around the replay on the caller's stream (an event
        // recorded inside a graph cannot be timed): the kernel plus the clear
        // and merge launches before and after it, a few microseconds
        if (timed) {
            if (!g.ev0) CK(cudaEventCreate(&g.ev0));
            if (!g.ev1) CK(cudaEventCreate(&g.ev1));
            CK(cudaEventRecord(g.ev0, st));
        }
        {
            NvtxRange nv("gb: graph replay (async)");
            CK(cudaGraphLaunch(g.aexec, st));
        }
        if (timed) {
            CK(cudaEventRecord(g.ev1, st));
            g.ev_pending = true;
        }
        g.stats.graph_replays++;
    } else {
        CK(launch_set_params(st, g.d_params, p));
        if ((rc = enqueue_persistent(st, cp, dev_out, grid, smem, mg, timed))) return rc;
    }
    g.stats.kernel_launches += 4;
    g.stats.tiles += cp.ntiles;
    g.stats.calls++;
    g.stats.n_verified += cp.n_total;
    return GB_OK;
}

int gb_progress(gb_progress_t *out)
{
    if (!out) return GB_EINVAL;
    const unsigned long long *p = g_progress_ptr.load();
    if (!p) { set_error("gb_init has not been called"); return GB_EINVAL; }
    memset(out, 0, sizeof *out);
    out->tiles_total = g_progress_total.load();
    out->tiles_done = std::min<uint64_t>(*(const volatile unsigned long long *)p, out->tiles_total);
    out->n_total = g_progress_ntotal.load();
    // every tile but the last holds tile_n even n
    const unsigned long long tn = g_progress_tile_n.load();
    out->n_done = out->tiles_done == out->tiles_total ? out->n_total
                                                      : std::min<uint64_t>(out->tiles_done * tn, out->n_total);
    out->elapsed_s = 1e-9 * (double)(steady_ns() - g_progress_t0.load());
    out->n_per_s = out->elapsed_s > 0.0 ? (double)out->n_done / out->elapsed_s : 0.0;
    out->eta_s = out->n_per_s > 0.0 ? (double)(out->n_total - out->n_done) / out->n_per_s : -1.0;
    return GB_OK;
}

int gb_stats(gb_stats_t *out)
{
    if (!out) return GB_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    *out = g.stats;
    serve_fill_stats(out);
    out->base_prime_count = g.nprimes ? g.nprimes + 1 : 0;   // + the prime 2
    out->base_prime_limit = g.table_limit;
    out->device_bytes = g.device_bytes;
    return GB_OK;
}

const char *gb_last_error(void)
{
    static thread_local std::string copy;
    std::lock_guard<std::mutex> lk(g_err_mu);
    copy = g_err;
    return copy.c_str();
}

}  // extern "C"
