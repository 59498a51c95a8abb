// gb_serve.h -- the serving loop (gb_submit / gb_poll) and the hooks it uses
// from the library context.
#pragma once
#include <stdint.h>
#include <mutex>

#include "../../include/goldbach_gb300.h"
#include "gb_types.h"

namespace gbk {
// provided by gb_capi.cu
std::recursive_mutex &ctx_mutex();
bool ctx_ready();
int64_t ctx_option(const char *key);
int ctx_verify(uint64_t lo, uint64_t hi, gb_result *out);
void ctx_error(const char *msg);
gb_stats_t &ctx_stats();
size_t ctx_device_bytes();
struct ServePlan {
    uint64_t n0, n_total, ntiles;
};
int ctx_serve_begin(int max_slots, int max_items);
void ctx_serve_end();
int ctx_serve_plan(uint64_t lo, uint64_t hi, ServePlan *sp);
bool ctx_serve_needs_table(uint64_t lo, uint64_t hi);
uint64_t ctx_serve_bucket_estimate(uint64_t lo, uint64_t hi);
int ctx_serve_init_slot(int slot, const ServePlan &sp, uint64_t *bucket_bytes);
void ctx_serve_release_slot(int slot);
unsigned long long *ctx_serve_items(int buf);
int ctx_serve_launch(int buf, size_t n);
// timeout_ms < 0: wait without bound
int ctx_serve_wait(int buf, int64_t timeout_ms);
// a finished request's result, its status from its own flags
int ctx_serve_fetch(int slot, const ServePlan &sp, gb_result *out);
size_t ctx_serve_slot_bytes();
// provided by gb_serve.cpp
void serve_stop();
void serve_fill_stats(gb_stats_t *out);
}  // namespace gbk
