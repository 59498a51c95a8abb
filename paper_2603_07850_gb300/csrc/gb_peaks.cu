// gb_peaks.cu -- microbenchmarks of the units the verifier is bound by: INT32
// logic/shift, integer multiply-add, popcount and conflict-free shared-memory
// atomicAnd.  Each kernel keeps eight independent dependency chains per thread
// in inline PTX (one instruction per counted operation, nothing for the
// compiler to merge or drop) on a full SM load, and is timed with CUDA events.
// The figures are the denominators of the measured roofline fractions.
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/goldbach_gb300.h"

namespace {

constexpr int PK_THREADS = 1024;
constexpr int PK_CHAINS = 8;

// 8 chains x (lop3 + shf) per iteration
__global__ void __launch_bounds__(PK_THREADS) pk_logic(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = seed * (threadIdx.x + 1u) + 0x9e3779b9u * (uint32_t)k;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) {
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(a[(k + 1) % PK_CHAINS]), "r"(i));
            asm volatile("shf.l.wrap.b32 %0, %0, %0, 7;" : "+r"(a[k]));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x ^= a[k];
    if (x == seed) sink[blockIdx.x] = x;                 // keeps every chain live
}

// 8 chains x mad.lo per iteration
__global__ void __launch_bounds__(PK_THREADS) pk_imad(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = seed * (threadIdx.x + 1u) + (uint32_t)k;
    const uint32_t m = seed | 1u;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++)
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(i));
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x ^= a[k];
    if (x == seed) sink[blockIdx.x] = x;
}

// 8 chains x (popc + add) per iteration; counted: the popcounts
__global__ void __launch_bounds__(PK_THREADS) pk_popc(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) a[k] = seed * (threadIdx.x + 1u) + 0x85ebca6bu * (uint32_t)k;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++) {
            uint32_t c;
            asm volatile("popc.b32 %0, %1;" : "=r"(c) : "r"(a[k]));
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(c + i));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x ^= a[k];
    if (x == seed) sink[blockIdx.x] = x;
}

// 8 atomicAnd per iteration, lane l of a warp on bank l (no conflicts)
__global__ void __launch_bounds__(PK_THREADS) pk_smem_and(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    __shared__ uint32_t s[PK_CHAINS * PK_THREADS];
    for (int k = 0; k < PK_CHAINS; k++) s[k * PK_THREADS + threadIdx.x] = 0xffffffffu;
    __syncthreads();
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; k++)
            atomicAnd(&s[k * PK_THREADS + threadIdx.x], ~(1u << ((i + (uint32_t)k) & 31u)) | seed);
    }
    __syncthreads();
    if (s[threadIdx.x] == seed + 1u) sink[blockIdx.x] = s[threadIdx.x];
}

// Lane operations per second of one kernel: best of `reps` timed launches.
double time_kernel(void (*k)(uint32_t, uint32_t, uint32_t *), int grid, uint32_t iters, double ops_per_iter,
                   uint32_t *sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, cudaError_t *err)
{
    double best = 0.0;
    for (int r = 0; r <= reps; r++) {
        cudaEventRecord(e0, st);
        k<<<grid, PK_THREADS, 0, st>>>(iters, 0x2545f491u, sink);
        cudaEventRecord(e1, st);
        if ((*err = cudaEventSynchronize(e1)) != cudaSuccess) return 0.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms <= 0.f) continue;               // the first launch warms up
        const double v = (double)grid * PK_THREADS * iters * ops_per_iter / (ms * 1e-3);
        if (v > best) best = v;
    }
    return best;
}

}  // namespace

extern "C" int gb_measure_peaks(gb_peaks_t *out)
{
    if (!out) return GB_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return GB_ECUDA;
    const int grid = 2 * sms;                            // two 1,024-thread CTAs per SM
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t *sink = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess &&
        (e = cudaMalloc((void **)&sink, 4ull * grid)) == cudaSuccess) {
        out->sms = (uint32_t)sms;
        out->int_logic_ops = time_kernel(pk_logic, grid, 1u << 15, 2.0 * PK_CHAINS, sink, st, e0, e1, 3, &e);
        if (e == cudaSuccess)
            out->int_mad_ops = time_kernel(pk_imad, grid, 1u << 15, PK_CHAINS, sink, st, e0, e1, 3, &e);
        if (e == cudaSuccess)
            out->popc_ops = time_kernel(pk_popc, grid, 1u << 14, PK_CHAINS, sink, st, e0, e1, 3, &e);
        if (e == cudaSuccess)
            out->smem_atomic_ops = time_kernel(pk_smem_and, grid, 1u << 13, PK_CHAINS, sink, st, e0, e1, 3, &e);
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return e == cudaSuccess ? GB_OK : GB_ECUDA;
}
