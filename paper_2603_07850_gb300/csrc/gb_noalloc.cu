// gb_noalloc.cu -- gb_verify_range_noalloc: range verification that never
// allocates device memory.
//
// Who needs it: programs that cannot call cudaMalloc at the point where they
// want a verification -- for example an application whose GPU memory is
// wholly reserved by another allocator (a framework's caching pool), where a
// stray cudaMalloc fails or fragments the pool, or a latency-critical loop
// where cudaMalloc/cudaFree would stall on an implicit device
// synchronisation.  gb_init allocates (tables, records, buffers), so such a
// caller cannot use the ordinary entry points.
//
// How: every byte of working memory -- the base-prime table, the candidate
// words, the launch parameters, the control block, the records and the merge
// partials -- lives in one file-scope static __device__ array of fixed size
// (NA_SCRATCH_BYTES, about 3.7 MB).  Every GPU that loads this library holds
// that array until the process exits.  Host code never uses the array's name
// as a device address: the address is obtained once per device with
// cudaGetSymbolAddress while that device is current, checked, and passed to
// the kernels.
//
// The kernels are the library's own persistent pipeline (clear -> persistent
// -> merge), launched on the scratch; only the small table-building kernels
// below are specific to this file.
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "gb_kernels.h"
#include "gb_serve.h"
#include "gb_types.h"

using namespace gbk;

namespace {

// ---- fixed limits of the no-allocation entry point -------------------------
constexpr uint32_t NA_TABLE_LIMIT = 1u << 20;     // base primes <= 2^20, so n < 2^40
constexpr uint32_t NA_NPRIMES = 82024;            // odd primes <= 2^20 (pi(2^20) - 1)
static_assert(NA_NPRIMES % 4 == 0, "the marking loads primes four at a time");
constexpr uint32_t NA_MAX_KWORDS = 1024;          // P_max <= 2^16
constexpr uint32_t NA_MAX_RECORDS = 8192;
constexpr uint32_t NA_MERGE_GRID = 512;
constexpr size_t NA_PART_SLOT = 320;              // >= sizeof(MergePart)
// the per-n search in one loop: the other searches need open-mask slots
// (128 KB per CTA)
constexpr int NA_TILE_BITS = 20, NA_THREADS = 512, NA_WHEEL = 13;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_PRIMES = 0;
constexpr size_t OFF_RECIP = al(OFF_PRIMES + 4ull * NA_NPRIMES);
constexpr size_t OFF_PR = al(OFF_RECIP + 8ull * NA_NPRIMES);
constexpr size_t OFF_PARAMS = al(OFF_PR + 4ull * NA_MAX_KWORDS);
constexpr size_t OFF_CTRL = al(OFF_PARAMS + sizeof(RangeParams));
constexpr size_t OFF_RECS = al(OFF_CTRL + sizeof(Ctrl));
constexpr size_t OFF_PARTS = al(OFF_RECS + sizeof(DevRec) * NA_MAX_RECORDS);
constexpr size_t NA_SCRATCH_BYTES = al(OFF_PARTS + NA_PART_SLOT * NA_MERGE_GRID);

// The scratch.  Its name is a host-side stand-in in host code; only the
// address from cudaGetSymbolAddress may be handed to a kernel.
static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

// One-CTA builder of the odd primes <= 2^20 and their reciprocals: an odd-only
// bitset of 2^19 bits in shared memory, crossed off by the odd primes below
// 2^10 (found by trial division), then compacted in order.
__global__ void __launch_bounds__(1024) na_table_kernel(unsigned char *scr, unsigned int *count_out)
{
    extern __shared__ uint32_t bits[];                // 2^14 words
    __shared__ uint32_t s_scan[1024];
    constexpr uint32_t NWORDS = NA_TABLE_LIMIT / 64;  // odd q < 2^20: 2^19 bits
    // bit 0 (q = 1) starts cleared, so no thread writes word 0 except by the
    // atomic crossing-off below
    for (uint32_t w = threadIdx.x; w < NWORDS; w += 1024) bits[w] = w ? 0xffffffffu : 0xfffffffeu;
    __syncthreads();
    for (uint32_t p = 3 + 2 * threadIdx.x; p < 1024; p += 2048) {
        bool prime = true;
        for (uint32_t d = 3; d * d <= p; d += 2)
            if (p % d == 0) { prime = false; break; }
        if (!prime) continue;
        for (uint32_t q = p * p; q < NA_TABLE_LIMIT; q += 2 * p) {
            uint32_t j = q >> 1;
            atomicAnd(&bits[j >> 5], ~(1u << (j & 31)));
        }
    }
    __syncthreads();
    // each thread owns 16 consecutive words; block-wide exclusive scan
    const uint32_t w0 = threadIdx.x * 16;
    uint32_t c = 0;
    for (int i = 0; i < 16; i++) c += __popc(bits[w0 + i]);
    s_scan[threadIdx.x] = c;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0u;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t pos = s_scan[threadIdx.x] - c;
    uint32_t *primes = reinterpret_cast<uint32_t *>(scr + OFF_PRIMES);
    unsigned long long *recip = reinterpret_cast<unsigned long long *>(scr + OFF_RECIP);
    for (int i = 0; i < 16; i++) {
        uint32_t w = bits[w0 + i];
        while (w) {
            int b = __ffs(w) - 1;
            w &= w - 1;
            uint32_t q = 2u * (32u * (w0 + i) + b) + 1u;
            if (pos < NA_NPRIMES) {
                primes[pos] = q;
                recip[pos] = 0xFFFFFFFFFFFFFFFFull / q;
            }
            pos++;
        }
    }
    if (threadIdx.x == 1023) *count_out = pos;
}

// Candidate words for p_max: bit i of word t <-> p = 64t + 2i + 1 is an odd
// prime <= p_max, stored bit-reversed (the search reads them with clz).
__global__ void __launch_bounds__(1024) na_cand_kernel(unsigned char *scr, uint32_t p_max, uint32_t k_words)
{
    __shared__ uint32_t w[NA_MAX_KWORDS];
    const uint32_t *primes = reinterpret_cast<const uint32_t *>(scr + OFF_PRIMES);
    uint32_t *PR = reinterpret_cast<uint32_t *>(scr + OFF_PR);
    for (uint32_t i = threadIdx.x; i < k_words; i += 1024) w[i] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < NA_NPRIMES; i += 1024) {
        uint32_t p = primes[i];
        if (p > p_max) continue;
        uint32_t b = (p - 1) >> 1;
        atomicOr(&w[b >> 5], 1u << (b & 31));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k_words; i += 1024) PR[i] = __brev(w[i]);
}

__global__ void na_empty_result(gb_result *out)
{
    if (threadIdx.x == 0) {
        unsigned long long *p = reinterpret_cast<unsigned long long *>(out);
        for (size_t i = 0; i < sizeof(gb_result) / 8; i++) p[i] = 0ull;
    }
}

struct DeviceScratch {
    unsigned char *ptr = nullptr;   // device address of g_na_scratch on this device
    bool ready = false;
};

std::mutex na_mu;
std::vector<DeviceScratch> na_dev;

// Once per device, with that device current: look up the scratch address and
// build the base-prime table into it.  Synchronises the stream once.
int na_setup(int dev, cudaStream_t st, unsigned char **out)
{
    if ((int)na_dev.size() <= dev) na_dev.resize(dev + 1);
    DeviceScratch &d = na_dev[dev];
    if (d.ready) { *out = d.ptr; return GB_OK; }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        gbk::ctx_error("gb_verify_range_noalloc: cudaGetSymbolAddress failed");
        return GB_ECUDA;
    }
    unsigned char *scr = static_cast<unsigned char *>(p);
    if (merge_part_bytes() > NA_PART_SLOT) {
        gbk::ctx_error("gb_verify_range_noalloc: merge partial larger than its scratch slot");
        return GB_EINTERNAL;
    }
    const int smem = (int)(4 * (NA_TABLE_LIMIT / 64));
    e = cudaFuncSetAttribute(na_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    // the prime count lands in the control-block slot, read back once
    unsigned int *cnt_dev = reinterpret_cast<unsigned int *>(scr + OFF_CTRL);
    if (e == cudaSuccess) {
        na_table_kernel<<<1, 1024, smem, st>>>(scr, cnt_dev);
        e = cudaGetLastError();
    }
    unsigned int cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, cnt_dev, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        gbk::ctx_error(cudaGetErrorString(e));
        return GB_ECUDA;
    }
    if (cnt != NA_NPRIMES) {
        gbk::ctx_error("gb_verify_range_noalloc: base-prime table has the wrong size");
        return GB_EINTERNAL;
    }
    d.ptr = scr;
    d.ready = true;
    *out = scr;
    return GB_OK;
}

uint64_t isqrt_u64_host(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 31; b >= 0; b--) {
        uint64_t c = r | (1ull << b);
        if (c <= x / c) r = c;
    }
    return r;
}

}  // namespace

extern "C" int gb_verify_range_noalloc(uint64_t lo, uint64_t hi, uint32_t p_max, uint32_t seg_bits,
                                       gb_result *dev_out, void *stream)
{
    if (!dev_out) { gbk::ctx_error("gb_verify_range_noalloc: null result pointer"); return GB_EINVAL; }
    if (p_max < 2 || p_max > (1u << 16)) {
        gbk::ctx_error("gb_verify_range_noalloc: p_max must be in [2, 2^16]");
        return GB_EINVAL;
    }
    if (seg_bits < 5 || seg_bits > 40) {
        gbk::ctx_error("gb_verify_range_noalloc: seg_bits must be in [5, 40]");
        return GB_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the even-n grid of the range
    uint64_t n0 = lo < 4 ? 4 : lo;
    bool empty = false;
    if (n0 & 1) {
        if (n0 == UINT64_MAX) empty = true; else n0++;
    }
    uint64_t n_total = 0;
    if (!empty && n0 < hi) {
        uint64_t n_last = (hi - 1) & ~1ull;
        if (n_last >= n0) n_total = (n_last - n0) / 2 + 1;
    }
    std::lock_guard<std::mutex> lk(na_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        gbk::ctx_error("gb_verify_range_noalloc: no current CUDA device");
        return GB_ECUDA;
    }
    unsigned char *scr = nullptr;
    int rc = na_setup(dev, st, &scr);
    if (rc) return rc;
    if (!n_total) {
        na_empty_result<<<1, 32, 0, st>>>(dev_out);
        return cudaGetLastError() == cudaSuccess ? GB_OK : GB_ECUDA;
    }
    const uint64_t n_last = n0 + 2 * (n_total - 1);
    if (isqrt_u64_host(n_last) >= NA_TABLE_LIMIT) {
        gbk::ctx_error("gb_verify_range_noalloc: n must stay below 2^40 (base primes <= 2^20)");
        return GB_EINVAL;
    }
    const uint64_t nrec = ((n_total - 1) >> seg_bits) + 1;
    if (nrec > NA_MAX_RECORDS) {
        gbk::ctx_error("gb_verify_range_noalloc: the range needs more than 8192 records; "
                           "use a larger seg_bits");
        return GB_EINVAL;
    }
    const uint32_t k_words = ((p_max + 1) / 2 + 31) / 32;
    RangeParams p{};
    p.n0 = n0;
    p.n_total = n_total;
    p.ntiles = ((n_total - 1) >> NA_TILE_BITS) + 1;
    p.nrec = nrec;
    p.p_slow_start = (p_max + 1ull) | 1ull;
    p.tile_bits = NA_TILE_BITS;
    p.rec_bits = seg_bits;
    p.k_words = k_words;
    p.p_max = p_max;
    p.slow_cap_log2 = 24;
    p.bk_prime0 = 0xffffffffu;      // n < 2^40: every base prime is below the bucket bound
    p.tile0 = 0;
    p.tile_end = p.ntiles;
    // tables view of the scratch (wheel 13, in-register masks up to 31, lane
    // per prime from 4096 on: index 10 = first prime above 31, 563 = number
    // of odd primes below 4096)
    Tables t{};
    t.primes = reinterpret_cast<const uint32_t *>(scr + OFF_PRIMES);
    t.recip = reinterpret_cast<const unsigned long long *>(scr + OFF_RECIP);
    t.PR = reinterpret_cast<const uint32_t *>(scr + OFF_PR);
    t.nprimes = NA_NPRIMES;
    t.iA0 = 10;
    t.iB0 = 563;
    t.pat_lo = 2;
    t.pat_hi = 7;
    t.k_words = k_words;
    RangeParams *d_params = reinterpret_cast<RangeParams *>(scr + OFF_PARAMS);
    Ctrl *d_ctrl = reinterpret_cast<Ctrl *>(scr + OFF_CTRL);
    DevRec *d_recs = reinterpret_cast<DevRec *>(scr + OFF_RECS);
    void *d_parts = scr + OFF_PARTS;
    const size_t smem = 4ull * (wheel_pattern_words(NA_WHEEL) + ((k_words + 3) & ~3u) +
                                ((((1ull << NA_TILE_BITS) + 32ull * k_words) / 32 + 2 + 3) & ~3ull));
    // the per-n search in one loop: the scratch holds no open-mask slots
    const void *fn = persistent_one_loop_ptr_512();
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NA_THREADS, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    // every call clears what must start at zero: the control block always,
    // the records whenever tiles share a record (clear_kernel decides)
    if (e == cudaSuccess) {
        na_cand_kernel<<<1, 1024, 0, st>>>(scr, p_max, k_words);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_set_params(st, d_params, p);
    const int clear_records = NA_TILE_BITS < (int)seg_bits ? 1 : 0;
    if (e == cudaSuccess) e = launch_clear(st, d_params, d_recs, d_ctrl, clear_records, clear_records ? 4 * sms : 1);
    if (e == cudaSuccess)
        e = launch_range_kernel(fn, NA_THREADS, per_sm * sms, smem, st, d_params, t, d_recs, d_ctrl);
    if (e == cudaSuccess) {
        uint64_t mg = (nrec + 255) / 256;
        if (mg > NA_MERGE_GRID) mg = NA_MERGE_GRID;
        if (mg < 1) mg = 1;
        e = launch_merge(st, (int)mg, d_params, d_recs, d_ctrl, d_parts, dev_out);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        gbk::ctx_error(cudaGetErrorString(e));
        return GB_ECUDA;
    }
    return GB_OK;
}
