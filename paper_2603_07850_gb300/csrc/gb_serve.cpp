// gb_serve.cpp -- request loop behind gb_submit / gb_poll: continuous batching
// over the persistent pool.
//
// gb_submit only enqueues on the host and returns a ticket.  One scheduler
// thread runs the loop:
//   admit   : move pending requests into free device slots while the device
//             memory budget allows (base-prime table the request needs +
//             one slot per active request); a request whose table alone is
//             over budget is rejected with GB_ENOMEM;
//   batch   : take tiles round-robin from every active request into a work
//             list (at most serve_batch_tiles items) and launch one persistent
//             serving kernel over it -- tiles of different requests share the
//             launch and overlap on the device;
//   harvest : with two batches in flight, wait for the older one and hand out
//             the requests whose last tile it held; their slots free up for
//             requests that arrived meanwhile.
// The records of a request depend only on its range, so a result is the same
// alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gb_serve.h"

namespace gbk {
namespace {

constexpr int MAX_SLOTS = 1024;

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0, lo = 0, hi = 0;
    ServePlan sp{};
    int slot = -1;
    uint64_t next_tile = 0;
    uint64_t table_bytes = 0;
    uint64_t bucket_est = 0, bucket_bytes = 0;  // bucket pre-pass: estimate, then actual
    bool done = false;
    gb_result res{};
    int status = GB_PENDING;
    uint64_t submit_ns = 0;
};

struct Batch {
    int buf;
    std::vector<uint64_t> finishing;          // requests whose last tile is in it
};

struct Serve {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> active;              // admitted, tiles left to issue or in flight
    std::map<uint64_t, Req> reqs;
    std::vector<int> free_slots;
    std::thread worker;
    bool running = false, stop = false;
    uint64_t next_id = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0;
    size_t max_items = 0;                      // capacity of each work-list buffer
    uint64_t live_bucket_bytes = 0;            // bucket arrays of admitted requests
};

Serve s;

// Device bytes of the base-prime table needed for sqrt(hi): primes up to the
// next 2^k - 1, 12 bytes each (prime + reciprocal), pi(L) <= 1.26 L / ln L.
uint64_t table_bytes_for(uint64_t hi)
{
    double r = std::sqrt((double)hi);
    double L = 1.0;
    while (L - 1.0 < r && L < 4294967296.0) L *= 2.0;
    L -= 1.0;
    if (L < 65536.0) return 0;
    return (uint64_t)(12.0 * 1.26 * L / std::log(L));
}

// Free a request's slot and its bucket arrays (caller holds s.mu).
void release(Req &r)
{
    if (r.slot < 0) return;
    {
        std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
        ctx_serve_release_slot(r.slot);
    }
    s.live_bucket_bytes -= std::min(s.live_bucket_bytes, r.bucket_bytes);
    r.bucket_bytes = 0;
    s.free_slots.push_back(r.slot);
    r.slot = -1;
}

void finish(Req &r, int status, const gb_result *res)
{
    if (res) r.res = *res;
    else memset(&r.res, 0, sizeof r.res);
    r.res.status = status;
    r.res.submit_ns = r.submit_ns;
    r.res.done_ns = now_ns();
    r.status = status;
    r.done = true;
    s.completed++;
}

void worker_loop()
{
    std::deque<Batch> inflight;
    int next_buf = 0;
    const uint64_t budget = (uint64_t)ctx_option("mem_budget_mb") << 20;
    const size_t slot_bytes = ctx_serve_slot_bytes();
    for (;;) {
        std::vector<uint64_t> batch_items;
        Batch nb{next_buf, {}};
        bool drain = false;
        {
            std::unique_lock<std::mutex> lk(s.mu);
            if (inflight.empty())
                s.cv_work.wait(lk, [] { return s.stop || !s.pending.empty() || !s.active.empty(); });
            if (s.stop) break;
            // ---- admit ---------------------------------------------------------
            while (!s.pending.empty() && !s.free_slots.empty()) {
                Req &r = s.reqs.at(s.pending.front());
                uint64_t tb = 0;
                for (uint64_t id : s.active) tb = std::max(tb, s.reqs.at(id).table_bytes);
                tb = std::max(tb, r.table_bytes);
                if (tb + (s.active.size() + 1) * slot_bytes + s.live_bucket_bytes + r.bucket_est > budget)
                    break;                                             // wait for room
                bool grow;
                {
                    std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
                    grow = ctx_serve_needs_table(r.lo, r.hi);
                }
                if (grow && !inflight.empty()) { drain = true; break; }   // grow with nothing in flight
                int rc;
                {
                    std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
                    rc = ctx_serve_plan(r.lo, r.hi, &r.sp);
                    if (rc == GB_OK && r.sp.n_total) {
                        r.slot = s.free_slots.back();
                        rc = ctx_serve_init_slot(r.slot, r.sp, &r.bucket_bytes);
                        if (rc == GB_OK) s.live_bucket_bytes += r.bucket_bytes;
                    }
                }
                s.pending.pop_front();
                if (rc != GB_OK || !r.sp.n_total) {
                    if (r.slot >= 0) release(r);
                    finish(r, rc, nullptr);
                    s.cv_done.notify_all();
                    continue;
                }
                s.free_slots.pop_back();
                s.active.push_back(r.id);
            }
            // ---- build the next batch round-robin over active requests ---------
            const size_t cap = std::min((size_t)ctx_option("serve_batch_tiles"), s.max_items);
            if (!drain && inflight.size() < 2) {
                unsigned long long *items = ctx_serve_items(next_buf);
                bool any = true;
                while (batch_items.size() < cap && any) {
                    any = false;
                    for (uint64_t id : s.active) {
                        Req &r = s.reqs.at(id);
                        if (r.next_tile >= r.sp.ntiles) continue;
                        items[batch_items.size()] =
                            ((unsigned long long)r.slot << SERVE_SLOT_SHIFT) | r.next_tile;
                        batch_items.push_back(id);
                        r.next_tile++;
                        any = true;
                        if (r.next_tile == r.sp.ntiles) nb.finishing.push_back(id);
                        if (batch_items.size() >= cap) break;
                    }
                }
            }
        }
        // ---- launch ------------------------------------------------------------
        if (!batch_items.empty()) {
            int rc;
            {
                std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
                rc = ctx_serve_launch(next_buf, batch_items.size());
            }
            if (rc != GB_OK) {
                std::lock_guard<std::mutex> lk(s.mu);
                for (uint64_t id : s.active) {
                    Req &r = s.reqs.at(id);
                    release(r);
                    finish(r, rc, nullptr);
                }
                s.active.clear();
                s.cv_done.notify_all();
                continue;
            }
            inflight.push_back(nb);
            next_buf ^= 1;
        }
        // ---- harvest the oldest batch when two are in flight, when draining,
        //      or when there is nothing more to launch ---------------------------
        if (!inflight.empty() && (inflight.size() == 2 || drain || batch_items.empty())) {
            Batch b = inflight.front();
            inflight.pop_front();
            // no context lock while waiting; bounded by the timeout_ms option
            const int rc = ctx_serve_wait(b.buf, ctx_option("timeout_ms"));
            if (rc == GB_ETIMEOUT) {
                // report at once: every admitted and every pending request fails.
                // Their slots are taken now: gb_poll may erase a finished request.
                std::vector<std::pair<int, uint64_t>> held;
                {
                    std::lock_guard<std::mutex> lk(s.mu);
                    for (uint64_t id : s.active) {
                        Req &r = s.reqs.at(id);
                        held.emplace_back(r.slot, r.bucket_bytes);
                        r.slot = -1;
                        finish(r, GB_ETIMEOUT, nullptr);
                    }
                    for (uint64_t id : s.pending) finish(s.reqs.at(id), GB_ETIMEOUT, nullptr);
                    s.pending.clear();
                    s.active.clear();
                    s.cv_done.notify_all();
                }
                // then let the device finish before any slot or buffer is reused
                ctx_serve_wait(b.buf, -1);
                for (auto &o : inflight) ctx_serve_wait(o.buf, -1);
                inflight.clear();
                std::lock_guard<std::mutex> lk(s.mu);
                for (auto &h : held) {
                    Req tmp;
                    tmp.slot = h.first;
                    tmp.bucket_bytes = h.second;
                    release(tmp);
                }
                continue;
            }
            std::vector<std::pair<uint64_t, gb_result>> out;
            for (uint64_t id : b.finishing) {
                ServePlan sp;
                int slot;
                {
                    std::lock_guard<std::mutex> lk(s.mu);
                    const Req &rq = s.reqs.at(id);      // unfinished: gb_poll cannot erase it
                    sp = rq.sp;
                    slot = rq.slot;
                }
                gb_result res{};
                int frc = rc;
                if (frc == GB_OK) frc = ctx_serve_fetch(slot, sp, &res);
                if (frc != GB_OK) { memset(&res, 0, sizeof res); res.status = frc; }
                out.emplace_back(id, res);
            }
            std::lock_guard<std::mutex> lk(s.mu);
            for (auto &pr : out) {
                Req &r = s.reqs.at(pr.first);
                release(r);
                for (size_t i = 0; i < s.active.size(); i++)
                    if (s.active[i] == r.id) { s.active.erase(s.active.begin() + i); break; }
                finish(r, pr.second.status, &pr.second);
            }
            s.cv_done.notify_all();
        }
    }
    // stopping: let in-flight batches finish before the context goes away
    std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
    for (auto &b : inflight) ctx_serve_wait(b.buf, -1);
}

int ensure_worker()
{
    if (s.running) return GB_OK;
    int rc;
    {
        std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
        s.max_items = (size_t)std::max<int64_t>(ctx_option("serve_batch_tiles"), 4096);
        rc = ctx_serve_begin(MAX_SLOTS, (int)s.max_items);
    }
    if (rc) return rc;
    s.free_slots.clear();
    for (int i = MAX_SLOTS - 1; i >= 0; i--) s.free_slots.push_back(i);
    s.stop = false;
    s.worker = std::thread(worker_loop);
    s.running = true;
    return GB_OK;
}

}  // namespace

void serve_stop()
{
    {
        std::lock_guard<std::mutex> lk(s.mu);
        if (!s.running) return;
        s.stop = true;
    }
    s.cv_work.notify_all();
    if (s.worker.joinable()) s.worker.join();
    std::lock_guard<std::mutex> lk(s.mu);
    s.running = false;
    s.pending.clear();
    s.active.clear();
    s.reqs.clear();
    s.free_slots.clear();
    s.cv_done.notify_all();
}

void serve_fill_stats(gb_stats_t *out)
{
    std::lock_guard<std::mutex> lk(s.mu);
    out->requests_submitted = s.submitted;
    out->requests_completed = s.completed;
    out->requests_rejected = s.rejected;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

int gb_submit(uint64_t lo, uint64_t hi, uint64_t *ticket)
{
    if (!ticket) { ctx_error("gb_submit: null ticket pointer"); return GB_EINVAL; }
    if (!ctx_ready()) { ctx_error("gb_init has not been called"); return GB_EINVAL; }
    const uint64_t budget = (uint64_t)ctx_option("mem_budget_mb") << 20;
    std::lock_guard<std::mutex> lk(s.mu);
    int rc = ensure_worker();
    if (rc) return rc;
    Req r;
    r.id = s.next_id++;
    r.lo = lo;
    r.hi = hi;
    r.table_bytes = table_bytes_for(hi);
    r.bucket_est = ctx_serve_bucket_estimate(lo, hi);
    r.submit_ns = now_ns();
    if (r.table_bytes + r.bucket_est + ctx_serve_slot_bytes() > budget) {
        s.rejected++;
        ctx_error("gb_submit: the request's base-prime table and buckets exceed the memory budget");
        return GB_ENOMEM;
    }
    s.reqs[r.id] = r;
    s.pending.push_back(r.id);
    s.submitted++;
    *ticket = r.id;
    s.cv_work.notify_one();
    return GB_OK;
}

int gb_poll(uint64_t ticket, gb_result *out, int32_t timeout_ms)
{
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) { ctx_error("gb_poll: unknown ticket"); return GB_EINVAL; }
    auto ready = [&] { auto j = s.reqs.find(ticket); return j == s.reqs.end() || j->second.done; };
    if (timeout_ms < 0) s.cv_done.wait(lk, ready);
    else if (timeout_ms > 0) s.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    it = s.reqs.find(ticket);
    if (it == s.reqs.end()) { ctx_error("gb_poll: the serving loop was shut down"); return GB_EINVAL; }
    if (!it->second.done) return GB_PENDING;
    if (out) *out = it->second.res;
    int st = it->second.status;
    s.reqs.erase(it);
    return st;
}

}  // extern "C"
