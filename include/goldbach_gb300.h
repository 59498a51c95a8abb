/*
 * goldbach_gb300.h -- C ABI of libgoldbach_gb300.so
 *
 * Exhaustive verification of the binary Goldbach conjecture over ranges of
 * even integers on one GB300 (sm_103a), by a segmented double sieve that
 * stays on the device (paper: "A Lock-Free, Fully GPU-Resident Architecture
 * for the Verification of Goldbach's Conjecture", arXiv 2603.07850).
 *
 * For every even n with max(lo, 4) <= n < hi the library computes
 *
 *     p_min(n) = min { p prime : n - p prime }          (paper, Sec. 1)
 *
 * and reduces the values to per-segment records: the maximum p_min, the
 * smallest n attaining it, a histogram of floor(log2 p_min), and wrapping
 * 64-bit sums.  Candidates p <= P_max are searched in a bit-packed sieve
 * window built in shared memory (paper, Sec. 3.1); any n whose p_min exceeds
 * P_max is finished on the GPU by an exact slow path (deterministic
 * Miller-Rabin, paper Sec. 3.4) -- there is no CPU fallback.
 *
 * Conventions (paper, Sec. 3.4 "Graceful error handling"): every call
 * returns a status code instead of aborting; 0 is success, negative values
 * are errors, positive values are informational.  The text of the last
 * error is available from gb_last_error().
 *
 * Ownership: the library owns every device allocation (base-prime tables,
 * sieve state, records) and its CUDA streams.  The caller owns every struct
 * and buffer passed by pointer.  All pointers are host pointers unless a
 * function says "device".
 *
 * Range: hi is exclusive and may be as large as 2^64 - 1 (UINT64_MAX), so
 * the largest even n that can be verified is 2^64 - 2; all sieve arithmetic
 * is guarded against 64-bit wrap (paper, Sec. 3.4 "Sieve arithmetic").
 *
 * Threading: gb_verify_range* calls are serialised on one library context.
 * gb_submit/gb_poll are thread-safe and may be called while a
 * gb_verify_range* call runs on another thread.
 */
#ifndef GOLDBACH_GB300_H
#define GOLDBACH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GB_OK                 0
#define GB_PENDING            1   /* gb_poll: request not finished yet          */
#define GB_COUNTEREXAMPLE     2   /* an n with no prime pair was found          */
#define GB_EINVAL            -1   /* bad argument, or gb_init not called         */
#define GB_ENOMEM            -2   /* device memory budget or allocation failed   */
#define GB_ECUDA             -3   /* a CUDA runtime call or kernel failed        */
#define GB_ETIMEOUT          -4   /* a bounded wait ran out                      */
#define GB_ESLOWPATH_LIMIT   -5   /* slow path hit its per-n iteration cap       */
#define GB_EOVERFLOW         -6   /* p_min too large for the record encoding     */
#define GB_EINTERNAL         -7   /* a device-side consistency check failed      */

/* ---- results ----------------------------------------------------------- */

/* Aggregate over a whole range (caller-owned, filled by the library). */
typedef struct {
    uint64_t n_first;          /* first even n covered (max(lo,4) rounded up) */
    uint64_t n_count;          /* number of even n covered                     */
    uint64_t max_pmin;         /* max p_min over the range                     */
    uint64_t argmax_n;         /* smallest n with p_min(n) == max_pmin         */
    uint64_t sum_pmin;         /* sum of p_min, mod 2^64                       */
    uint64_t wsum_pmin;        /* sum of p_min * (k + 1) mod 2^64, k = (n - n_first) / 2 */
    uint64_t hist[64];         /* hist[b] = #n with floor(log2 p_min) == b     */
    uint64_t n_slow;           /* #n with p_min > P_max (finished by the slow path) */
    uint64_t counterexample_n; /* smallest counterexample found, 0 if none     */
    int32_t  status;           /* same value the call returned                 */
    int32_t  reserved;
    uint64_t submit_ns;        /* served requests: host steady-clock time of gb_submit, else 0 */
    uint64_t done_ns;          /* served requests: time the result reached the host, else 0 */
} gb_result;

/* One report segment: 2^seg_bits consecutive even n (the last one of a range
 * may be shorter), counted from the range's n_first.  wsum_pmin uses k
 * relative to this record's own n_first. */
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
} gb_seg_record;

/* Counters since gb_init. */
typedef struct {
    uint64_t calls;            /* completed gb_verify_range* calls              */
    uint64_t tiles;            /* sieve tiles processed                         */
    uint64_t n_verified;       /* even n verified                               */
    uint64_t n_slow;           /* n finished by the slow path                   */
    uint64_t kernel_launches;  /* kernels launched by the library              */
    uint64_t graph_replays;    /* CUDA-graph replays of the persistent pipeline */
    uint64_t requests_submitted;
    uint64_t requests_completed;
    uint64_t requests_rejected;/* refused by the memory-budget admission check  */
    uint64_t base_prime_count; /* primes resident in the base table            */
    uint64_t base_prime_limit; /* the table holds every prime <= this          */
    uint64_t device_bytes;     /* device memory currently held by the library  */
} gb_stats_t;

/* Measured throughput of the units the verifier is bound by, in lane
 * operations per second over the whole GPU (see gb_measure_peaks). */
typedef struct {
    double int_logic_ops;      /* lop3 and shf (the INT32 logic/shift path)     */
    double int_mad_ops;        /* integer multiply-add (mad.lo.u32)             */
    double popc_ops;           /* popc                                          */
    double smem_atomic_ops;    /* shared-memory atomicAnd, no bank conflicts    */
    uint32_t sms;              /* multiprocessors of the measured GPU           */
    uint32_t reserved;
} gb_peaks_t;

/* ---- lifecycle ----------------------------------------------------------- */

/*
 * gb_init -- create the library context on the current CUDA device.
 *
 *   p_max    : candidate bound P_max (paper Sec. 3.3, "P_SMALL"): the sieve
 *              search tries every odd prime p <= p_max; n with a larger p_min
 *              go to the GPU slow path.  2 <= p_max <= 2^20.
 *   seg_bits : report granularity, log2 of even n per gb_seg_record,
 *              5 <= seg_bits <= 40 (paper Alg. 1 processes the range in
 *              segments; here the record size is independent of the tile
 *              size the kernels use).
 *
 * Builds the small-candidate table and the base primes <= 2^16 on the
 * device.  Calling gb_init again re-initialises (gb_shutdown first); every
 * gb_init starts from the default options.
 * Returns GB_OK, GB_EINVAL, GB_ENOMEM or GB_ECUDA.
 */
int gb_init(uint32_t p_max, uint32_t seg_bits);

/*
 * gb_set_option -- tune the context.  The paper tunes a run with command-line
 * flags and compile-time constants (Sec. 3.5: --gpus, --start, --progress,
 * --batch-size; the segment size SEG_SIZE and the candidate bound P_SMALL of
 * the reproducibility checklist); here the equivalents are context options,
 * set between calls.  Keys (value range):
 *   "tile_bits"     log2 even n per sieve tile, 10..20 (default 20; at most 19
 *                   with the pipelined kernel and P_max = 2^16, whose CTA
 *                   holds two windows)
 *   "threads"       threads per CTA: 256, 512, 768 or 1024 (default 1024; the
 *                   single-role kernel has 768-thread builds for wheel 13 with
 *                   search_chunks 0, 6 and 8)
 *   "builder_warps" 0 = single-role persistent kernel (every warp builds the
 *                   window, then every warp searches it); 8, 12 or 16 = the
 *                   pipelined kernel, in which that many warps build the next
 *                   tile's window while the other warps search the current
 *                   one (instantiated: 8 of 1024 or 768 threads, 12 or 16 of
 *                   1024; wheel 13 only) (default 0)
 *   "ctas_per_sm"   persistent CTAs per SM, 1..4 (default: as many as fit)
 *   "wheel"         largest wheel prime pre-sieved by pattern: 7 or 13 (default 13)
 *   "pattern_max"   largest prime cleared by in-register patterns, 13..61 (default 31)
 *   "base_limit"    build base primes up to this value now (<= 2^32 - 1)
 *   "mem_budget_mb" device-memory budget for serving admission (default 8192)
 *   "plain_seg_bits" log2 even n per segment of the plain form, 20..30 (default 26)
 *   "use_graph"     1 = replay a captured CUDA graph (default), 0 = direct launches
 *   "slow_cap"      log2 of the slow-path candidate cap per n, 6..24 (default 24)
 *   "timeout_ms"    bound for device-side waits and gb_poll defaults (default 600000)
 *   "tier_b_min"    smallest prime crossed off lane-per-prime (default 8192)
 *   "plain_slice_bits" log2 window bits per CTA in the plain sieve kernel (default 18)
 *   "plain_search_chunks" search of the plain form: 0 = the per-n search kernel
 *                   writing a p_min array that a reduce kernel folds (default);
 *                   4, 6 or 8 = one launch of the bit-parallel search and
 *                   reduction per segment, reading the global window
 *   "time_kernel"   1 = time the persistent kernel with CUDA events (default 0)
 *   "search_chunks" bit-parallel search over the candidates p < 64 * this: 4, 6 or 8
 *                   (default 4); 0 = one lane per n (wheel 7 allows 0, 4, 8)
 *   "serve_batch_tiles" tiles per serving launch (default 1024)
 *   "autotune"      1 = before the first call of each range class (GPU, P_max,
 *                   log2 of the largest n), time the kernel configurations on a
 *                   probe at the top of the range and keep the fastest (tile_bits,
 *                   threads, search_chunks, pattern_max, search_pmax, tier_b_min,
 *                   wheel, builder_warps, bucket_min, bucket_chunk_tiles;
 *                   combinations with no kernel build are
 *                   skipped, and a pipelined one takes the largest tile that
 *                   fits shared memory); the choice is
 *                   cached, and saved to the file named by GB_TUNE_CACHE if set
 *                   (one line per range class: key and ten values, in the
 *                   order listed here).  A range that needs the bucket
 *                   pre-pass is probed with it, and bucket_min and
 *                   bucket_chunk_tiles are tuned too.
 *                   The tuning call synchronises.  Results never depend on it.
 *   "search_pmax"   bound of the in-window candidate search, 0 = P_max (default 0);
 *                   n with p_min above it take the slow path, but n_slow and
 *                   every other output still refer to P_max
 *   "bucket_min"    smallest base prime handled by the bucket pre-pass,
 *                   0 = four window spans, 4 (S + K) (default), else 64 .. 2^28
 *   "bucket_chunk_tiles" tiles per bucket pre-pass chunk, 1..8192 (default 2048)
 *   "debug_smem_limit" only in the library built with GB_DEBUG
 *                   (libgoldbach_gb300_debug.so), whose kernels check every
 *                   access to a sieve window in shared memory: the checks
 *                   then allow only the first this many bytes of the
 *                   dynamic shared memory, 0 = all of it (default).  A
 *                   failed check skips its access and the call fails with
 *                   GB_EINTERNAL; a lower limit makes checks fail on
 *                   accesses that are still inside the allocation, to test
 *                   that path.  Ignored by the ordinary library.
 * Returns GB_OK or GB_EINVAL (unknown key or value out of range).
 */
int gb_set_option(const char *key, int64_t value);

/* gb_get_option -- read back an option, or one of the read-only values
 * "p_max", "seg_bits", "k_words", "sms", "last_kernel_us" (duration of the
 * last range kernel timed with time_kernel = 1, -1 if none; for
 * gb_verify_range_async the events bracket its graph replay, so the clear
 * and merge launches, a few microseconds, are included; call it after the
 * work has completed) and "phase_fill", "phase_mark", "phase_search",
 * "phase_reduce", "phase_warp_bulk", "phase_warp_tail", "phase_claim" (clock64
 * cycle sums of the last range call, only in the library built with
 * GB_PHASE_CLOCKS, -1 otherwise; reading one waits for the device),
 * "debug_build" (1 in the library built with GB_DEBUG, else 0) and
 * "debug_bounds_site", "debug_bounds_offset" (that library: the site, 1..8,
 * and the byte offset in dynamic shared memory of the first failed bounds
 * check of the last range call, 0 if none; reading one waits for the
 * device; a serving request's failure shows in its own status only).
 * GB_EINVAL for an unknown key. */
int gb_get_option(const char *key, int64_t *value);

/* gb_shutdown -- stop the serving thread, let in-flight work finish and free
 * every device allocation and stream (the clean release the paper's error
 * handling provides for failed GPU workers, Sec. 3.4).  Safe to call when
 * gb_init has not been called. */
void gb_shutdown(void);

/* ---- range verification ------------------------------------------------------ */

/*
 * gb_verify_range -- verify every even n with max(lo,4) <= n < hi with the
 * persistent fused kernel (CTAs claim tiles from a device atomic counter,
 * the device form of the paper's lock-free pool, Sec. 3.2 / Alg. 1), and
 * write the aggregate to *out (host pointer).
 *
 * A range with no even n >= 4 is valid and returns n_count = 0.
 * Returns GB_OK, GB_COUNTEREXAMPLE (out->counterexample_n set), or an error.
 */
int gb_verify_range(uint64_t lo, uint64_t hi, gb_result *out);

/*
 * gb_verify_range_segments -- as gb_verify_range, and also copy the
 * per-segment records (2^seg_bits even n each) into buf[0..cap).
 * *n_written receives the number of records the range has (which may
 * exceed cap; only cap are written).  out may be NULL.
 */
int gb_verify_range_segments(uint64_t lo, uint64_t hi, gb_seg_record *buf, size_t cap,
                             size_t *n_written, gb_result *out);

/* Claim block shared by the callers of gb_verify_range_claimed: host memory
 * that all of them can see (for example a shared-memory mapping), zeroed
 * before the first call. */
typedef struct {
    uint64_t next_tile;        /* next tile to claim; the kernels bump it with system-scope atomics */
    uint64_t fingerprint;      /* set by the first caller: which range and configuration the tiles
                                * index; 0 until then */
} gb_claim_t;

/*
 * gb_verify_range_claimed -- cooperative form of gb_verify_range_segments:
 * several callers (processes, on one or several GPUs) verify [lo, hi)
 * together by claiming its tiles from claim->next_tile.  This is the paper's
 * lock-free work pool (Sec. 3.2, Alg. 1: workers take the next segment with
 * an atomic increment of a shared counter) shared across devices.  Every
 * caller must pass the same lo, hi and use the same seg_bits, tile_bits and
 * P_max: the first caller stamps claim->fingerprint with them (atomic
 * compare-and-swap) and a caller whose values differ is refused with
 * GB_EINVAL before it claims anything.  The autotuner is not run.  This
 * caller's records and result cover only the tiles it claimed (the other
 * records are zero).  The callers' records merge record by record: counts,
 * sums and histograms add, and the largest p_min with its smallest n wins.
 * That gives exactly the records of one gb_verify_range_segments call.
 * *claim is registered as mapped host memory for the duration of the call
 * unless it already is.  A range that needs the bucket pre-pass (sqrt(n) at
 * or above bucket_min) is refused with GB_EINVAL.  Otherwise returns as
 * gb_verify_range_segments.
 */
int gb_verify_range_claimed(uint64_t lo, uint64_t hi, gb_claim_t *claim, gb_seg_record *buf, size_t cap,
                            size_t *n_written, gb_result *out);

/*
 * gb_verify_range_plain -- the plain per-segment form kept as the baseline
 * the persistent kernel is measured against: a host loop that, per segment,
 * launches a sieve kernel (bitset written to global memory), a search
 * kernel and a reduction kernel, then reads a 4-byte status back and
 * synchronises (paper Alg. 1).  Same outputs as gb_verify_range.
 */
int gb_verify_range_plain(uint64_t lo, uint64_t hi, gb_seg_record *buf, size_t cap,
                          size_t *n_written, gb_result *out);

/*
 * gb_verify_range_async -- enqueue gb_verify_range's work on a caller
 * stream without synchronising.  dev_out is a DEVICE pointer to a gb_result
 * that receives the aggregate when the stream reaches that point; stream is
 * a cudaStream_t (NULL = the library's own stream).  The caller must not
 * enqueue another call on the context until this one has completed on the
 * device (the context's scratch is reused).  Returns GB_OK once enqueued;
 * device-side status lands in dev_out->status.
 */
int gb_verify_range_async(uint64_t lo, uint64_t hi, gb_result *dev_out, void *stream);

/*
 * gb_verify_range_noalloc -- gb_verify_range for callers that cannot
 * allocate device memory.  (This entry point has no counterpart in the
 * paper; it is a deployment convenience.)
 *
 * Some programs must not call cudaMalloc where they verify a range: their
 * GPU memory may be wholly reserved by another allocator (a framework's
 * caching pool, where a stray allocation fails or fragments the pool), or
 * they run a latency-critical loop in which cudaMalloc/cudaFree would stall
 * on an implicit device synchronisation.  gb_init allocates, so such callers
 * use this function instead; it needs no gb_init and allocates nothing.
 *
 * All working memory (base primes <= 2^20, candidate words, parameters,
 * control block, records, merge partials) is one static device array of
 * about 3.7 MB that every GPU loading this library holds until the process
 * exits.  Limits, rejected with GB_EINVAL and a message in gb_last_error():
 *   2 <= p_max <= 2^16;  5 <= seg_bits <= 40;  every n < 2^40;
 *   at most 8192 records of 2^seg_bits even n (pick seg_bits accordingly).
 *
 *   dev_out : DEVICE pointer to a gb_result, written when the stream gets
 *             there (status in dev_out->status).
 *   stream  : cudaStream_t to enqueue on (NULL = the default stream).
 *
 * The first call on each device does a one-time set-up with that device
 * current: it looks up the scratch address, builds the base-prime table in
 * it and synchronises the stream.  Make that first call before any stream
 * capture.  Later calls only enqueue work.  Every call reuses the same
 * scratch (and clears what must start at zero), so calls that overlap on the
 * GPU race: serialise them, e.g. on one stream.
 * Returns GB_OK once enqueued, GB_EINVAL, GB_ECUDA or GB_EINTERNAL.
 */
int gb_verify_range_noalloc(uint64_t lo, uint64_t hi, uint32_t p_max, uint32_t seg_bits,
                            gb_result *dev_out, void *stream);

/* ---- serving (continuous batching) ------------------------------------------ */

/*
 * gb_submit -- enqueue a range request [lo, hi) and return a ticket at once.
 * The paper runs one range per invocation and lets independent jobs take
 * disjoint ranges (Sec. 3.5, --start); a request here is such a range, and
 * many of them share the GPU.  A scheduler thread admits requests while the
 * device-memory budget allows (the paper's pre-launch VRAM check, Sec. 3.5,
 * applied per request), interleaves their tiles in the persistent pool
 * (Sec. 3.2's claim-the-next-segment pool, over the tiles of every admitted
 * request) and finishes each request independently, with its own status.
 * *ticket is caller-owned.  Returns GB_OK, GB_EINVAL (NULL ticket, gb_init
 * not called) or GB_ENOMEM (the request alone exceeds the budget).
 */
int gb_submit(uint64_t lo, uint64_t hi, uint64_t *ticket);

/*
 * gb_poll -- wait up to timeout_ms (0 = do not wait, < 0 = wait forever) for
 * a ticket.  Returns GB_PENDING while unfinished; otherwise the request's
 * status (status codes as for gb_verify_range, paper Sec. 3.4), with *out
 * (caller-owned, may be NULL) filled and the ticket released.  A request's
 * status comes only from its own tiles.  GB_EINVAL for an unknown ticket.
 */
int gb_poll(uint64_t ticket, gb_result *out, int32_t timeout_ms);

/* ---- introspection --------------------------------------------------------- */

/* Progress of one gb_verify_range* call (see gb_progress). */
typedef struct {
    uint64_t tiles_done;       /* tiles finished (segments for the plain form)  */
    uint64_t tiles_total;      /* tiles of the call                             */
    uint64_t n_done;           /* even n in the finished tiles                  */
    uint64_t n_total;          /* even n of the call                            */
    double   elapsed_s;        /* host time since the call started              */
    double   n_per_s;          /* n_done / elapsed_s (0 before the first tile)  */
    double   eta_s;            /* (n_total - n_done) / n_per_s, -1 before the first tile */
} gb_progress_t;

/*
 * gb_progress -- progress of the gb_verify_range* call that is running (or
 * finished last): tiles and even n done, the rate so far and the estimated
 * time left.  This is the paper's progress monitor (Sec. 3.2: a host thread
 * reports the rate and remaining time while the GPUs work; Sec. 3.5, the
 * --progress option).  Callable from any thread while the call runs, without
 * waiting for it: the kernels count finished tiles into mapped host memory.
 * `out` is caller-owned.  Returns GB_OK, or GB_EINVAL if out is NULL or
 * gb_init has not been called.
 */
int gb_progress(gb_progress_t *out);

/*
 * gb_stats -- counters since gb_init (gb_stats_t): calls, tiles, even n
 * verified, slow-path n, kernel launches and graph replays, served
 * requests, base-table size and device bytes held.  The throughput
 * statistics the paper's progress monitor prints (Sec. 3.2) and the launch
 * counts its profiling section reports (Sec. 4.3) come from these.  `out` is
 * caller-owned.  Returns GB_OK, or GB_EINVAL if out is NULL.
 */
int gb_stats(gb_stats_t *out);

/*
 * gb_measure_peaks -- run the microbenchmarks behind the measured roofline on
 * the current CUDA device: INT32 logic/shift, integer multiply-add, popcount
 * and conflict-free shared-memory atomicAnd.  Each is a full-occupancy kernel
 * (two 1,024-thread CTAs per SM) with eight independent chains per thread,
 * timed with CUDA events (best of three after a warm-up launch; about 0.1 s
 * in all).  Needs no gb_init and holds no memory afterwards.  `out` is
 * caller-owned.  Returns GB_OK, GB_EINVAL (out is NULL) or GB_ECUDA.
 */
int gb_measure_peaks(gb_peaks_t *out);

/*
 * gb_last_error -- text of the last error any call reported (paper Sec. 3.4:
 * a failure is reported with a description instead of ending the process).
 * The string belongs to the library and stays valid on the calling thread
 * until its next gb_last_error call.  Empty when no error has occurred.
 */
const char *gb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GOLDBACH_GB300_H */
