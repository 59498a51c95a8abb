// gb_kernels.h -- host-callable launch wrappers for the kernels in gb_kernels.cu.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#include "gb_types.h"

namespace gbk {

// bc: 0 = per-n search, 2..4 = bit-parallel search over p < 64 bc (wheel 7: bc 0 or 3)
const void *persistent_kernel_ptr(int wheel, int nt, int bc);
// defined in gb_persist_<NT>.cu
const void *persistent_ptr_256(int wheel, int bc);
const void *persistent_ptr_512(int wheel, int bc);
const void *persistent_ptr_768(int wheel, int bc);
// wheel 13, 512 threads, per-n search in one loop: needs no open-mask slots
const void *persistent_one_loop_ptr_512();
const void *persistent_ptr_1024(int wheel, int bc);
const void *serve_ptr_512(int wheel, int bc);
// pipelined kernel (window-building and searching warps, two window buffers):
// np building warps out of nt threads; nullptr when not instantiated.
// Defined in gb_pipe_8.cu / gb_pipe_16.cu; wheel 13 only.
const void *pipe_kernel_ptr(int wheel, int np, int nt, int bc);
const void *pipe_ptr_8(int nt, int bc);
const void *pipe_ptr_16(int np, int nt, int bc);
// launch a persistent or pipelined range kernel given by its pointer
cudaError_t launch_range_kernel(const void *fn, int nt, int grid, size_t smem, cudaStream_t st,
                                const RangeParams *prm, const Tables &t, DevRec *recs, Ctrl *ctrl);
const void *serve_ptr_1024(int wheel, int bc);
// serving work-list kernel; nullptr when (wheel, nt, bc) has no instantiation
const void *serve_kernel_ptr(int wheel, int nt, int bc);
cudaError_t launch_serve(const void *fn, int nt, int grid, size_t smem, cudaStream_t st,
                         const unsigned long long *items, unsigned long long n_items, SlotDev *slots,
                         const Tables &t, Ctrl *ctrl);
const void *slice_kernel_ptr(int wheel, int nt);
uint32_t wheel_pattern_words(int wheel);
size_t merge_part_bytes();
uint32_t table_blocks(uint32_t nwords);

cudaError_t launch_clear(cudaStream_t st, const RangeParams *prm, DevRec *recs, Ctrl *ctrl,
                         int clear_records, int grid);
cudaError_t launch_merge(cudaStream_t st, int grid, const RangeParams *prm, const DevRec *recs,
                         Ctrl *ctrl, void *parts, gb_result *out);
cudaError_t launch_slice_sieve(int wheel, int nt, int grid, size_t smem, cudaStream_t st,
                               unsigned long long half_abs, int neg, uint32_t j_end, uint32_t Z,
                               const Tables &t, uint32_t *gwin, uint32_t gwords, Ctrl *ctrl);
cudaError_t launch_plain_search(cudaStream_t st, int grid, const RangeParams *prm,
                                const uint32_t *gwin, const uint32_t *PR, unsigned long long n_lo,
                                uint32_t cnt, uint32_t *pm, Ctrl *ctrl);
// plain form, bit-parallel search (1,024 threads, bc = 4, 6 or 8): sub-tiles
// [tile_first, tile_first + nsub) of 2^prm.tile_bits n, window from gwin
const void *plain_bulk_ptr(int bc);
cudaError_t launch_plain_bulk(int bc, int grid, size_t smem, cudaStream_t st, const RangeParams &prm,
                              unsigned long long tile_first, uint32_t nsub, const Tables &t, const uint32_t *gwin,
                              DevRec *recs, Ctrl *ctrl);
cudaError_t launch_plain_reduce(cudaStream_t st, const RangeParams *prm, const uint32_t *pm,
                                unsigned long long k_seg0, unsigned long long n_lo, uint32_t cnt,
                                uint32_t chunk, DevRec *recs, Ctrl *ctrl);
cudaError_t launch_table_compact(cudaStream_t st, const uint32_t *bits, uint32_t nwords,
                                 uint32_t *block_counts, unsigned long long *block_offsets,
                                 unsigned long long limit, uint32_t *primes,
                                 unsigned long long *recip, int count_only);

}  // namespace gbk

namespace gbk {
cudaError_t launch_set_params(cudaStream_t st, RangeParams *dst, const RangeParams &p);
// the kernel launch_set_params runs (its arguments: RangeParams *dst, RangeParams p)
const void *set_params_kernel_ptr();
// phase 0: count hits per tile and per (block, tile) with grid blocks of
// 256 threads, scan the tiles into off, turn blk into each block's first
// entry per tile; phase 1: fill the entries, staged, with grid / 4 blocks of
// 1,024 threads (each takes the primes of four count blocks).  counts holds
// nt entries (zeroed by the caller), off nt + 1, blk grid * nt; grid is a
// multiple of 4 and nt at most 8,192.
cudaError_t launch_bucket_prepass(cudaStream_t st, int grid, const RangeParams *prm, const Tables &t,
                                  uint32_t i0, unsigned long long t0, uint32_t nt, unsigned int *counts,
                                  unsigned long long *off, unsigned int *blk, uint32_t *ent, int phase,
                                  unsigned long long cap, Ctrl *ctrl);
}
