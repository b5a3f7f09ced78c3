// ns_serve.cu -- streaming service: windows arrive from host threads, are
// admitted as slots and HBM budget free up, build concurrently on the device,
// and are summed into the resident traffic matrix in submission order.
//
// Per window (ticket t):
//   slot stream:  H2D copy of src/dst, A_t (hash path), A_t's statistics
//   accumulate stream (one, in ticket order): wait for t's build,
//                 A += A_t, statistics of A, D2H of both records
// A completion thread waits on each ticket's last event in ticket order and
// publishes the result.  Builds of different windows overlap; only the
// accumulate step is serialized, and it runs in ticket order, so a window's
// results do not depend on what else is in flight.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_kernels.h"

using namespace ns;

namespace {

using Clock = std::chrono::steady_clock;

double now_us() {
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t built = nullptr, done = nullptr;
    Buf d_src, d_dst;
    Buf d_stats;                  // 2 x ns_stats: per window, running
    ns_stats* h_stats = nullptr;  // pinned, 2 records
    ns_matrix* At = nullptr;
    u64 reserved = 0;  // bytes charged against the budget while in use
    bool busy = false;
};

struct Request {
    u64 ticket;
    const uint32_t* src;
    const uint32_t* dst;
    u64 n;
    u64 window_id;
    double t_submit;
};

struct Result {
    ns_stats per_window{};
    ns_stats running{};
    ns_stream_timing timing{};
    ns_status status = NS_OK;
    std::string message;  // error text, handed to the waiting thread
    bool done = false;
};

struct InFlight {
    u64 ticket;
    int slot;
    double t_submit, t_admit;
    u64 window_id;
};

// Device bytes a window of n packets needs while in flight: its two columns,
// A_t's tables at the context's load bound and its statistics.
u64 window_bytes(u64 n, double load) {
    const u64 want = (u64)std::ceil((double)n / load);
    u64 cap = 1024;
    while (cap < want) cap <<= 1;
    return 8 * n + (cap + 1) * (sizeof(LinkSlot) + 2 * sizeof(NodeSlot)) + 2 * sizeof(ns_stats) + sizeof(DevStats);
}

}  // namespace

struct ns_server {
    ns_ctx* ctx = nullptr;
    ns_matrix* acc = nullptr;
    int device = 0;
    int max_slots = 8;
    u64 max_queue = 32;
    u64 budget = 0;
    u64 in_use = 0;  // bytes charged by in-flight windows
    cudaStream_t acc_stream = nullptr;
    std::vector<Slot> slots;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_complete;
    std::deque<Request> queue;
    std::deque<InFlight> inflight;
    std::map<u64, Result> results;
    u64 next_ticket = 1;
    bool stopping = false;
    std::thread sched, completer;
};

namespace {

// Input buffers grow to the next power of two of the window, so that a slot
// regrows at most once per doubling and the pool's freed blocks fit other
// slots' next growth.
u64 slot_input_bytes(u64 n) {
    u64 b = 1ull << 16;
    while (b < n * sizeof(uint32_t)) b <<= 1;
    return b;
}

// A slot's stream, events, pinned result buffer, window matrix and device
// statistics.  ns_server_create sets up every slot, so that none of these
// (cudaMallocHost in particular, which can wait for the device) runs while
// windows are being served.
ns_status slot_setup(ns_server* S, Slot& sl) {
    if (sl.stream) return NS_OK;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.built, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&sl.h_stats, 2 * sizeof(ns_stats)) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "server: slot set-up failed");
    }
    ns_status st = ns_matrix_create(S->ctx, &sl.At);
    if (st != NS_OK) return st;
    AllocScope alloc(S->ctx->pool, sl.stream, true);
    st = buf_reserve(sl.d_stats, 2 * sizeof(ns_stats));
    if (st == NS_OK) st = buf_reserve(sl.d_src, slot_input_bytes(0));
    if (st == NS_OK) st = buf_reserve(sl.d_dst, slot_input_bytes(0));
    return st;
}

// Frees every slot's memory, streams and events.  Every window has
// completed.  A slot's memory comes from the context's pool in stream order
// on the slot's stream, so it is freed there while that stream still exists;
// the stream is destroyed afterwards.
void slots_release(ns_server* S) {
    for (auto& sl : S->slots) {
        if (sl.At) {
            touch(sl.At, sl.stream);
            ns_matrix_free(sl.At);
            sl.At = nullptr;
        }
        buf_free_on(sl.d_src, sl.stream);
        buf_free_on(sl.d_dst, sl.stream);
        buf_free_on(sl.d_stats, sl.stream);
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
            cudaEventDestroy(sl.built);
            cudaEventDestroy(sl.done);
            sl.stream = nullptr;
        }
        if (sl.h_stats) cudaFreeHost(sl.h_stats);
        sl.h_stats = nullptr;
    }
}

ns_status slot_prepare(ns_server* S, Slot& sl, u64 n) {
    ns_status st = slot_setup(S, sl);
    if (st != NS_OK) return st;
    // The slot's buffers are (re)allocated on its own stream.  A slot is only
    // prepared while idle (its previous window has completed), so freeing the
    // old buffers there is safe, and it stalls no other slot.
    AllocScope alloc(S->ctx->pool, sl.stream, true);
    if (sl.d_src.bytes < n * sizeof(uint32_t)) st = buf_reserve(sl.d_src, slot_input_bytes(n));
    if (st == NS_OK && sl.d_dst.bytes < n * sizeof(uint32_t)) st = buf_reserve(sl.d_dst, slot_input_bytes(n));
    return st;
}

// Issues one admitted window's GPU work.  Scheduler thread only.
ns_status launch_window(ns_server* S, Slot& sl, const Request& r) {
    ns_status st = slot_prepare(S, sl, r.n);
    if (st != NS_OK) return st;
    // A_t's tables, too, grow on the slot's stream
    AllocScope alloc(S->ctx->pool, sl.stream, true);
    if (r.n) {
        if (cudaMemcpyAsync(sl.d_src.p, r.src, r.n * sizeof(uint32_t), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess ||
            cudaMemcpyAsync(sl.d_dst.p, r.dst, r.n * sizeof(uint32_t), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess) {
            cudaGetLastError();
            return set_fail(NS_ERR_CUDA, "server: input copy failed");
        }
    }
    st = build_hash(S->ctx, (const uint32_t*)sl.d_src.p, (const uint32_t*)sl.d_dst.p, r.n, sl.At, sl.stream);
    if (st != NS_OK) return st;
    ns_stats* d_pw = (ns_stats*)sl.d_stats.p;
    st = ns_network_stats_async(S->ctx, sl.At, d_pw, sl.stream);
    if (st != NS_OK) return st;
    if (cudaEventRecord(sl.built, sl.stream) != cudaSuccess ||
        cudaStreamWaitEvent(S->acc_stream, sl.built, 0) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "server: event failed");
    }
    st = ns_accumulate(S->ctx, S->acc, sl.At, S->acc_stream);
    if (st != NS_OK) return st;
    st = ns_network_stats_async(S->ctx, S->acc, d_pw + 1, S->acc_stream);
    if (st != NS_OK) return st;
    if (cudaMemcpyAsync(sl.h_stats, d_pw, 2 * sizeof(ns_stats), cudaMemcpyDeviceToHost, S->acc_stream) != cudaSuccess ||
        cudaEventRecord(sl.done, S->acc_stream) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "server: result copy failed");
    }
    return NS_OK;
}

void scheduler_loop(ns_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_sched.wait(lk, [&] {
            if (S->stopping && S->queue.empty()) return true;
            if (S->queue.empty()) return false;
            // FIFO admission keeps the accumulation in ticket order
            const Request& r = S->queue.front();
            bool free_slot = false;
            for (auto& sl : S->slots) free_slot |= !sl.busy;
            // the resident aggregate counts against the budget too
            const u64 resident = S->acc->links.bytes + S->acc->rows.bytes + S->acc->cols.bytes;
            return free_slot && (S->in_use == 0 || resident + S->in_use + window_bytes(r.n, S->ctx->cfg.hash_load) <= S->budget);
        });
        if (S->queue.empty()) return;  // stopping
        Request r = S->queue.front();
        S->queue.pop_front();
        int si = 0;
        while (S->slots[si].busy) ++si;
        Slot& sl = S->slots[si];
        sl.busy = true;
        sl.reserved = window_bytes(r.n, S->ctx->cfg.hash_load);
        S->in_use += sl.reserved;
        const double t_admit = now_us();
        lk.unlock();
        const u64 resident = S->acc->links.bytes + S->acc->rows.bytes + S->acc->cols.bytes;
        ns_status st = (sl.reserved + resident > S->budget)
                           ? set_fail(NS_ERR_OOM, "server: window does not fit the HBM budget")
                           : launch_window(S, sl, r);
        lk.lock();
        if (st != NS_OK) {
            Result& res = S->results[r.ticket];
            res.status = st;
            res.message = ns_last_error();
            res.done = true;
            res.timing.submit_us = r.t_submit;
            res.timing.admit_us = t_admit;
            res.timing.complete_us = now_us();
            sl.busy = false;
            S->in_use -= sl.reserved;
            sl.reserved = 0;
            S->cv_done.notify_all();
            S->cv_sched.notify_all();
            continue;
        }
        S->inflight.push_back({r.ticket, si, r.t_submit, t_admit, r.window_id});
        S->cv_complete.notify_all();
    }
}

void completion_loop(ns_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_complete.wait(lk, [&] { return !S->inflight.empty() || (S->stopping && S->queue.empty()); });
        if (S->inflight.empty()) {
            if (S->stopping && S->queue.empty()) return;
            continue;
        }
        InFlight f = S->inflight.front();
        Slot& sl = S->slots[f.slot];
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(sl.done);
        const double t_done = now_us();
        lk.lock();
        S->inflight.pop_front();
        Result& res = S->results[f.ticket];
        if (e != cudaSuccess) {
            cudaGetLastError();
            res.status = set_fail(NS_ERR_CUDA, "server: window failed on the device");
            res.message = ns_last_error();
        } else {
            res.per_window = sl.h_stats[0];
            res.running = sl.h_stats[1];
        }
        res.timing.submit_us = f.t_submit;
        res.timing.admit_us = f.t_admit;
        res.timing.complete_us = t_done;
        res.timing.window_id = f.window_id;
        res.done = true;
        sl.busy = false;
        S->in_use -= sl.reserved;
        sl.reserved = 0;
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
}

}  // namespace

extern "C" {

ns_status ns_server_create(ns_ctx* c, ns_matrix* acc, ns_server** out) {
    if (!c || !acc || !out) return set_fail(NS_ERR_INVALID, "ns_server_create: NULL argument");
    DeviceGuard device_guard(c->device);
    if (acc->ctx != c) return set_fail(NS_ERR_INVALID, "ns_server_create: acc belongs to another context");
    *out = nullptr;
    {
        const ns_status pst = context_pool(c);
        if (pst != NS_OK) return pst;
    }
    ns_server* S = new ns_server();
    S->ctx = c;
    S->acc = acc;
    S->device = c->device;
    S->max_slots = c->cfg.max_slots > 0 ? c->cfg.max_slots : 8;
    S->max_queue = 4 * (u64)S->max_slots + 16;
    S->budget = c->cfg.hbm_budget_bytes;
    S->slots.resize(S->max_slots);
    cudaSetDevice(c->device);
    if (cudaStreamCreateWithFlags(&S->acc_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return set_fail(NS_ERR_CUDA, "ns_server_create: stream creation failed");
    }
    // every slot is set up now, not on its first window
    for (auto& sl : S->slots) {
        const ns_status st = slot_setup(S, sl);
        if (st != NS_OK) {
            slots_release(S);
            cudaStreamDestroy(S->acc_stream);
            delete S;
            return st;
        }
    }
    S->sched = std::thread(scheduler_loop, S);
    S->completer = std::thread(completion_loop, S);
    *out = S;
    return NS_OK;
}

ns_status ns_server_reserve(ns_server* S, uint64_t max_window) {
    if (!S) return set_fail(NS_ERR_INVALID, "ns_server_reserve: NULL server");
    DeviceGuard device_guard(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->queue.empty() || !S->inflight.empty())
        return set_fail(NS_ERR_BUSY, "ns_server_reserve: windows in flight");
    for (auto& sl : S->slots) {
        if (sl.busy) return set_fail(NS_ERR_BUSY, "ns_server_reserve: windows in flight");
        ns_status st = slot_prepare(S, sl, max_window);
        if (st == NS_OK) st = ns_matrix_reserve(sl.At, max_window, sl.stream);
        if (st != NS_OK) return st;
        if (cudaStreamSynchronize(sl.stream) != cudaSuccess) {
            cudaGetLastError();
            return set_fail(NS_ERR_CUDA, "ns_server_reserve: slot set-up failed");
        }
    }
    return NS_OK;
}

ns_status ns_server_clear(ns_server* S) {
    if (!S) return set_fail(NS_ERR_INVALID, "ns_server_clear: NULL server");
    DeviceGuard device_guard(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->queue.empty() || !S->inflight.empty())
        return set_fail(NS_ERR_BUSY, "ns_server_clear: windows in flight");
    // The scheduler pops a request and marks its slot busy under the lock,
    // then issues the window's work (accumulation into acc included) without
    // it; the request joins the in-flight list only afterwards.  A busy slot
    // therefore means a window may be touching acc right now.
    for (const auto& sl : S->slots)
        if (sl.busy) return set_fail(NS_ERR_BUSY, "ns_server_clear: windows in flight");
    ns_status st = ns_matrix_clear(S->acc, S->acc_stream);
    if (st != NS_OK) return st;
    if (cudaStreamSynchronize(S->acc_stream) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "ns_server_clear: clear failed");
    }
    return NS_OK;
}

void ns_server_destroy(ns_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_sched.notify_all();
    S->cv_complete.notify_all();
    S->sched.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
    }
    S->cv_complete.notify_all();
    S->completer.join();
    cudaSetDevice(S->device);
    cudaStreamSynchronize(S->acc_stream);
    for (auto& sl : S->slots)
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    slots_release(S);
    cudaStreamDestroy(S->acc_stream);
    delete S;
}

ns_status ns_stream_submit(ns_server* S, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n,
                           uint64_t window_id, uint64_t* ticket) {
    if (!S || !ticket) return set_fail(NS_ERR_INVALID, "ns_stream_submit: NULL argument");
    if (n > 0 && (!h_src || !h_dst)) return set_fail(NS_ERR_INVALID, "ns_stream_submit: NULL input with n > 0");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return set_fail(NS_ERR_STATE, "ns_stream_submit: server is stopping");
    if (S->queue.size() >= S->max_queue) return set_fail(NS_ERR_BUSY, "ns_stream_submit: queue full, retry later");
    const u64 t = S->next_ticket++;
    S->queue.push_back({t, h_src, h_dst, n, window_id, now_us()});
    S->results[t] = Result{};
    *ticket = t;
    S->cv_sched.notify_all();
    return NS_OK;
}

ns_status ns_stream_poll(ns_server* S, uint64_t ticket, int* done) {
    if (!S || !done) return set_fail(NS_ERR_INVALID, "ns_stream_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return set_fail(NS_ERR_INVALID, "ns_stream_poll: unknown ticket");
    *done = it->second.done ? 1 : 0;
    return NS_OK;
}

ns_status ns_stream_wait(ns_server* S, uint64_t ticket, ns_stats* per_window, ns_stats* running, int64_t timeout_us,
                         ns_stream_timing* timing) {
    if (!S) return set_fail(NS_ERR_INVALID, "ns_stream_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return set_fail(NS_ERR_INVALID, "ns_stream_wait: unknown ticket");
    auto ready = [&] { return S->results[ticket].done; };
    if (timeout_us < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return set_fail(NS_ERR_TIMEOUT, "ns_stream_wait: timed out");
    }
    Result res = S->results[ticket];
    S->results.erase(ticket);
    if (per_window) *per_window = res.per_window;
    if (running) *running = res.running;
    if (timing) *timing = res.timing;
    if (res.status != NS_OK) return set_fail(res.status, res.message.c_str());
    return NS_OK;
}

}  // extern "C"
