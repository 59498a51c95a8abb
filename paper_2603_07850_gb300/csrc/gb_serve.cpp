// gb_serve.cpp -- request loop behind gb_submit / gb_poll.
//
// gb_submit only enqueues on the host and returns a ticket.  A scheduler
// thread admits requests against the device-memory budget and runs them on
// the library context; gb_poll waits (bounded) for a ticket's result.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "gb_serve.h"

namespace gbk {
namespace {

struct Req {
    uint64_t id, lo, hi;
    bool done = false;
    gb_result res{};
    int status = GB_PENDING;
};

struct Serve {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    std::thread worker;
    bool running = false, stop = false;
    uint64_t next_id = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0;
};

Serve s;

void worker_loop()
{
    for (;;) {
        uint64_t id;
        uint64_t lo, hi;
        {
            std::unique_lock<std::mutex> lk(s.mu);
            s.cv_work.wait(lk, [] { return s.stop || !s.queue.empty(); });
            if (s.stop) return;
            id = s.queue.front();
            s.queue.pop_front();
            lo = s.reqs[id].lo;
            hi = s.reqs[id].hi;
        }
        gb_result r{};
        int rc;
        {
            std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
            rc = ctx_ready() ? ctx_verify(lo, hi, &r) : GB_EINVAL;
        }
        {
            std::lock_guard<std::mutex> lk(s.mu);
            auto it = s.reqs.find(id);
            if (it != s.reqs.end()) {
                it->second.res = r;
                it->second.res.status = rc;
                it->second.status = rc;
                it->second.done = true;
            }
            s.completed++;
        }
        s.cv_done.notify_all();
    }
}

void ensure_worker()
{
    if (s.running) return;
    s.stop = false;
    s.worker = std::thread(worker_loop);
    s.running = true;
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
    s.queue.clear();
    s.reqs.clear();
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
    if (!ticket) return GB_EINVAL;
    {
        std::lock_guard<std::recursive_mutex> ck(ctx_mutex());
        if (!ctx_ready()) { ctx_error("gb_init has not been called"); return GB_EINVAL; }
    }
    std::lock_guard<std::mutex> lk(s.mu);
    ensure_worker();
    uint64_t id = s.next_id++;
    Req r;
    r.id = id; r.lo = lo; r.hi = hi;
    s.reqs[id] = r;
    s.queue.push_back(id);
    s.submitted++;
    *ticket = id;
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
    if (it == s.reqs.end()) return GB_EINVAL;
    if (!it->second.done) return GB_PENDING;
    if (out) *out = it->second.res;
    int st = it->second.status;
    s.reqs.erase(it);
    return st;
}

}  // extern "C"
