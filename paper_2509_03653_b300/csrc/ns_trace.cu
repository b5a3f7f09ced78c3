// ns_trace.cu -- per-kernel timing (the library's tracing subsystem).
//
// When tracing is on, every kernel a context launches on a stream that is not
// being captured into a graph is bracketed by two CUDA events on that stream;
// ns_trace_read waits for the recorded events and returns, per kernel name,
// the launch count and the total and largest elapsed time.
#include <cstring>
#include <map>
#include <string>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_kernels.h"

namespace ns {

cudaEvent_t tracer_event(Tracer* t) {
    if (t->used == t->pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        t->pool.push_back(e);
    }
    return t->pool[t->used++];
}

TraceScope::TraceScope(Tracer* tr, const char* nm, cudaStream_t st) : t(tr), name(nm), s(st), a(nullptr) {
    if (!t || !t->on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    a = tracer_event(t);
    if (a && cudaEventRecord(a, s) != cudaSuccess) {
        cudaGetLastError();
        a = nullptr;
    }
}

TraceScope::~TraceScope() {
    if (!a) return;
    cudaEvent_t b = tracer_event(t);
    if (!b || cudaEventRecord(b, s) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    t->recs.push_back({name, a, b});
}

void tracer_destroy(Tracer* t) {
    for (cudaEvent_t e : t->pool) cudaEventDestroy(e);
    t->pool.clear();
    t->recs.clear();
    t->used = 0;
}

}  // namespace ns

extern "C" {

ns_status ns_trace_enable(ns_ctx* c, int on) {
    if (!c) return ns::set_fail(NS_ERR_INVALID, "ns_trace_enable: NULL context");
    c->tracer.on = on != 0;
    return NS_OK;
}

ns_status ns_trace_read(ns_ctx* c, ns_trace_entry* out, int cap, int* count) {
    if (!c || !count || (cap > 0 && !out)) return ns::set_fail(NS_ERR_INVALID, "ns_trace_read: NULL argument");
    ns::DeviceGuard device_guard(c->device);
    struct Agg {
        uint64_t n = 0;
        double total = 0, mx = 0;
    };
    std::map<std::string, Agg> agg;
    ns_status st = NS_OK;
    for (const auto& r : c->tracer.recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            st = ns::set_fail(NS_ERR_CUDA, "ns_trace_read: event query failed");
            continue;
        }
        Agg& g = agg[r.name];
        g.n += 1;
        g.total += ms;
        if (ms > g.mx) g.mx = ms;
    }
    c->tracer.recs.clear();
    c->tracer.used = 0;
    int i = 0;
    for (const auto& kv : agg) {
        if (i < cap) {
            memset(&out[i], 0, sizeof(ns_trace_entry));
            strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.n;
            out[i].total_ms = kv.second.total;
            out[i].max_ms = kv.second.mx;
        }
        ++i;
    }
    *count = i;
    return st;
}

ns_status ns_diag_wait_timeout(int which, ns_stream_t stream) {
    if (which < 0 || which > 2) return ns::set_fail(NS_ERR_INVALID, "ns_diag_wait_timeout: which must be 0, 1 or 2");
    cudaStream_t s = (cudaStream_t)stream;
    ns::AllocScope alloc(nullptr, s);
    ns::Buf b;
    ns_status st = ns::buf_reserve(b, sizeof(ns::DevStats) + 64);
    if (st != NS_OK) return st;
    ns::DevStats h{};
    ns::DevStats* d = (ns::DevStats*)b.p;
    ns::u64* status_word = (ns::u64*)((char*)b.p + sizeof(ns::DevStats));
    if (cudaMemsetAsync(b.p, 0, sizeof(ns::DevStats) + 64, s) != cudaSuccess) {
        cudaGetLastError();
        ns::buf_free(b);
        return ns::set_fail(NS_ERR_CUDA, "ns_diag_wait_timeout: memset failed");
    }
    ns::launch_diag_wait(which, status_word, d, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ns::buf_free(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ns::set_fail(NS_ERR_CUDA, "ns_diag_wait_timeout: launch failed");
    }
    if (h.err & ns::ERR_TIMEOUT) return ns::set_fail(NS_ERR_TIMEOUT, "bounded device wait gave up (as intended)");
    return ns::set_fail(NS_ERR_STATE, "ns_diag_wait_timeout: the wait did not report a timeout");
}

}  // extern "C"

namespace {

// Fastest of `reps` timed launches (after one warm-up) of launch(r) on s.
template <typename F>
ns_status time_best(const char* what, int reps, cudaStream_t s, F launch, double* best_us) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return ns::fail_fmt(NS_ERR_CUDA, "%s: event creation failed", what);
    }
    ns_status st = NS_OK;
    float best = 1e30f;
    for (int r = 0; r <= reps; ++r) {  // the first run warms up
        cudaEventRecord(e0, s);
        launch(r);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            st = ns::fail_fmt(NS_ERR_CUDA, "%s: launch failed", what);
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == NS_OK) *best_us = best * 1e3;
    return st;
}

}  // namespace

extern "C" {

ns_status ns_diag_random_atomics(uint64_t table_words, uint64_t threads, int reps, double* best_us,
                                 ns_stream_t stream) {
    if (!best_us || reps < 1 || table_words < 1024 || (table_words & (table_words - 1)) || threads == 0)
        return ns::set_fail(NS_ERR_INVALID, "ns_diag_random_atomics: bad argument (table_words a power of two >= 1024)");
    cudaStream_t s = (cudaStream_t)stream;
    ns::AllocScope alloc(nullptr, s);
    ns::Buf a, b, c;
    ns_status st = ns::buf_reserve(a, table_words * 8);
    if (st == NS_OK) st = ns::buf_reserve(b, table_words * 8);
    if (st == NS_OK) st = ns::buf_reserve(c, table_words * 8);
    if (st == NS_OK) {
        cudaMemsetAsync(a.p, 0, table_words * 8, s);
        cudaMemsetAsync(b.p, 0, table_words * 8, s);
        cudaMemsetAsync(c.p, 0, table_words * 8, s);
        st = time_best("ns_diag_random_atomics", reps, s, [&](int r) {
            ns::launch_diag_rand3((ns::u64*)a.p, (ns::u64*)b.p, (ns::u64*)c.p, table_words - 1, threads,
                                  0x5EEDull + (ns::u64)r * 7919, s);
        }, best_us);
    }
    ns::buf_free(a);
    ns::buf_free(b);
    ns::buf_free(c);
    return st;
}

ns_status ns_diag_random_claims(uint64_t table_slots, uint64_t threads, int mode, int reps, double* best_us,
                                ns_stream_t stream) {
    if (!best_us || reps < 1 || table_slots < 1024 || (table_slots & (table_slots - 1)) || threads == 0 ||
        mode < NS_DIAG_CLAIM || mode > NS_DIAG_CLAIM_STALE)
        return ns::set_fail(NS_ERR_INVALID, "ns_diag_random_claims: bad argument (table_slots a power of two >= "
                                            "1024, mode 0..2)");
    cudaStream_t s = (cudaStream_t)stream;
    ns::AllocScope alloc(nullptr, s);
    ns::Buf a, b, c, sink;
    const ns::u64 bytes = table_slots * 16;
    ns_status st = ns::buf_reserve(a, bytes);
    if (st == NS_OK) st = ns::buf_reserve(b, bytes);
    if (st == NS_OK) st = ns::buf_reserve(c, bytes);
    if (st == NS_OK) st = ns::buf_reserve(sink, 16);
    if (st == NS_OK) {
        // empty slots, or (stale mode) every slot holding an old entry
        const int fill = mode == NS_DIAG_CLAIM_STALE ? 0x11 : 0;
        cudaMemsetAsync(a.p, fill, bytes, s);
        cudaMemsetAsync(b.p, fill, bytes, s);
        cudaMemsetAsync(c.p, fill, bytes, s);
        st = time_best("ns_diag_random_claims", reps, s, [&](int r) {
            ns::launch_diag_claims((ns::u64*)a.p, (ns::u64*)b.p, (ns::u64*)c.p, table_slots - 1, threads,
                                   0xC1A1ull + (ns::u64)r * 7919, mode, (ns::u64*)sink.p, s);
        }, best_us);
    }
    ns::buf_free(a);
    ns::buf_free(b);
    ns::buf_free(c);
    ns::buf_free(sink);
    return st;
}

}  // extern "C"
