// ns_slide.cu -- per-window and sliding-window statistics beside the running
// sum (the windows' matrices A_t are time-indexed, Table 2 caption).
//
// A slider keeps the matrices of the last K windows in a ring.  Each push
// builds the new window's A_t into the ring slot of the oldest one, writes
// A_t's quantities, and re-forms the sliding sum A_{t-K+1} + ... + A_t from
// the ring by accumulation into a cleared matrix.  Re-forming (instead of
// subtracting the window that leaves) keeps every quantity exact with the
// same kernels as the running sum: counts only grow inside one accumulation,
// so its maxima are the incremental ones; a subtraction would lower counts
// and invalidate the maxima.  The cost is K accumulations of window-sized
// matrices per push.
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"

using namespace ns;

struct ns_slider {
    ns_ctx* ctx = nullptr;
    std::vector<ns_matrix*> ring;  // K window matrices
    ns_matrix* sum = nullptr;      // the sliding sum, re-formed on every push
    uint64_t pushed = 0;
};

extern "C" {

ns_status ns_slider_create(ns_ctx* c, uint32_t windows, ns_slider** out) {
    if (!c || !out) return set_fail(NS_ERR_INVALID, "ns_slider_create: NULL argument");
    DeviceGuard device_guard(c->device);
    if (windows == 0) return set_fail(NS_ERR_INVALID, "ns_slider_create: windows == 0");
    *out = nullptr;
    ns_slider* x = new ns_slider();
    x->ctx = c;
    ns_status st = NS_OK;
    for (uint32_t i = 0; i < windows && st == NS_OK; ++i) {
        ns_matrix* m = nullptr;
        st = ns_matrix_create(c, &m);
        if (st == NS_OK) x->ring.push_back(m);
    }
    if (st == NS_OK) st = ns_matrix_create(c, &x->sum);
    if (st != NS_OK) {
        ns_slider_free(x);
        return st;
    }
    *out = x;
    return NS_OK;
}

void ns_slider_free(ns_slider* x) {
    if (!x) return;
    for (ns_matrix* m : x->ring) ns_matrix_free(m);
    if (x->sum) ns_matrix_free(x->sum);
    delete x;
}

ns_status ns_slider_push(ns_ctx* c, ns_slider* x, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                         ns_stats* d_window, ns_stats* d_sliding, ns_stream_t stream) {
    if (!c || !x) return set_fail(NS_ERR_INVALID, "ns_slider_push: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    if (x->ctx != c) return set_fail(NS_ERR_INVALID, "ns_slider_push: slider belongs to another context");
    const size_t K = x->ring.size();
    ns_matrix* at = x->ring[x->pushed % K];
    ns_status st = ns_window_build(c, d_src, d_dst, n, at, stream);
    if (st == NS_OK && d_window) st = ns_network_stats_async(c, at, d_window, stream);
    if (st != NS_OK) return st;
    ++x->pushed;
    // the sliding sum of the windows in the ring (all of them once K have been pushed)
    st = ns_matrix_clear(x->sum, stream);
    const uint64_t live = x->pushed < K ? x->pushed : K;
    for (uint64_t i = 0; i < live && st == NS_OK; ++i) st = ns_accumulate(c, x->sum, x->ring[i], stream);
    if (st == NS_OK && d_sliding) st = ns_network_stats_async(c, x->sum, d_sliding, stream);
    return st;
}

ns_status ns_slider_matrix(const ns_slider* x, const ns_matrix** out) {
    if (!x || !out) return set_fail(NS_ERR_INVALID, "ns_slider_matrix: NULL argument");
    *out = x->sum;
    return NS_OK;
}

}  // extern "C"
