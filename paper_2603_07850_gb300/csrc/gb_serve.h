// gb_serve.h -- the serving loop (gb_submit / gb_poll) and the hooks it uses
// from the library context.
#pragma once
#include <stdint.h>
#include <mutex>

#include "../../include/goldbach_gb300.h"

namespace gbk {
// provided by gb_capi.cu
std::recursive_mutex &ctx_mutex();
bool ctx_ready();
int64_t ctx_option(const char *key);
int ctx_verify(uint64_t lo, uint64_t hi, gb_result *out);
void ctx_error(const char *msg);
gb_stats_t &ctx_stats();
size_t ctx_device_bytes();
// provided by gb_serve.cpp
void serve_stop();
void serve_fill_stats(gb_stats_t *out);
}  // namespace gbk
