// ns_api_internal.h -- host-side objects behind the opaque ns_ctx / ns_matrix.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <map>
#include <string>

#include "ns.h"
#include "ns_kernels.h"

namespace ns {

// Makes `device` current for the guard's scope and gives the calling thread
// its own current device back afterwards, so that an entry point works on
// its context's GPU whichever device the caller had current.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != device && cudaSetDevice(device) != cudaSuccess) cudaGetLastError();
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev && cudaSetDevice(prev) != cudaSuccess)
            cudaGetLastError();
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// A grow-only device allocation.  Inside a stream-private allocation scope
// (the AllocScope below; the serving slots) buffers come from the context's
// memory pool and are allocated, grown and freed in stream order on the
// scope's stream, which stalls no other stream; elsewhere they come from
// cudaMalloc and go back with cudaFree, which waits for the device.
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    bool pooled = false;  // from the context's pool: freed with cudaFreeAsync
};

// The pool and stream that buf_reserve / buf_free use on this host thread,
// set by an entry point for its duration (nested scopes restore the outer
// one).  Only a scope that declares its buffers private to its stream (every
// earlier use of them is on that stream or has completed) allocates from the
// pool in stream order; elsewhere growth frees the old memory with cudaFree,
// which waits for every reader on any stream.
struct AllocScope {
    cudaMemPool_t prev_pool;
    cudaStream_t prev_stream;
    bool prev_private;
    AllocScope(cudaMemPool_t pool, cudaStream_t s, bool stream_private = false);
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
};
cudaStream_t alloc_stream();
// Frees b on stream s (after the work enqueued there so far).
void buf_free_on(Buf& b, cudaStream_t s);

enum { FMT_EMPTY = 0, FMT_HASH = 1, FMT_LIST = 2 };

ns_status buf_reserve(Buf& b, size_t bytes);
ns_status fail_fmt(ns_status s, const char* fmt, ...);
ns_status to_hash(ns_matrix* m, u64 extra, cudaStream_t s);
// The path ns_window_build takes for n packets (NS_PATH_SORT or NS_PATH_HASH).
int resolve_path(const ns_ctx* c, u64 n);
// The sort-path build of n packets into `out` (its sorted nonzero list and
// statistics).  split: -1 = the context's rule, 0 = off, 1 = on; tile: -1 =
// the context's rule, else the digit passes' tile shape; digits: -1 = the
// context's rule, else the digit plan (kDigits8, kDigitsWide).
ns_status build_sort(ns_ctx* c, const uint32_t* src, const uint32_t* dst, u64 n, ns_matrix* out, cudaStream_t s,
                     int split = -1, int tile = -1, int digits = -1);
// The sort variant a build of n packets takes: split (0/1), tile shape, digit plan.
void resolve_sort(const ns_ctx* c, u64 n, int* split, int* tile, int* digits);
ns_status check_launch();
HashView hash_view(const ns_matrix* m);
void buf_free(Buf& b);
ns_status check_launch();
ns_status set_fail(ns_status s, const char* msg);
// Reads the matrix's statistics record (blocking); the device error word
// comes back as a status.
ns_status read_stats(const ns_matrix* m, cudaStream_t s, DevStats* out);
// Creates the context's memory pool (for stream-private allocation scopes)
// if it has none yet.
ns_status context_pool(ns_ctx* c);
// Sizes the context's look-back status words for sorts of up to n elements.
ns_status sort_scratch(ns_ctx* c, u64 n);
// Hash path: out := A_t.  cache: -1 = the context's rule, 0 = off, 1 = on.
ns_status build_hash(ns_ctx* c, const uint32_t* src, const uint32_t* dst, u64 n, ns_matrix* out,
                     cudaStream_t s, int cache = -1);

// Autotuner cache file (ns_tuner.cu): entries keyed "<gpu>|<kind>|<shape>",
// each a one-line JSON object kept as text.
std::string gpu_name(int device);
std::map<std::string, std::string> tuner_load(const std::string& path);
void tuner_store(const std::string& path, const std::map<std::string, std::string>& m);
bool json_number(const std::string& obj, const char* name, double* v);
bool json_string(const std::string& obj, const char* name, std::string* v);

}  // namespace ns

struct ns_ctx {
    int device = 0;
    int sms = 148;
    ns_config cfg{};
    std::string tuner_cache;
    // ns_path_tune's choices by floor(log2 n): path (NS_PATH_SORT / NS_PATH_HASH)
    // and, for the hash path, whether inserts stage hot keys in shared memory
    struct PathChoice {
        int path;
        bool cta_cache;
        int split;  // sort path: 1 split, 0 not, -1 the size rule
        int tile;   // sort path: digit-pass tile shape (0..kSortTileShapes-1), -1 the default
        int digits; // sort path: digit plan (kDigits8, kDigitsWide), -1 the default
    };
    std::map<int, PathChoice> path_choice;
    ns::SortScratch sc{};
    ns::Buf ghist, offs, tcount, counters, status;
    ns::Buf k64[2], pos, psum, k32[2], v64[2], xk, xv;
    cudaMemPool_t pool = nullptr;  // the serving slots' memory (created with the first server)
    // The stream of the last call that used the context's scratch.  Calls
    // without a stream (creation) allocate on the legacy default stream and
    // wait for it.
    cudaStream_t last_stream = nullptr;
    ns::Buf stage[2];  // device copies of host columns (ns_window_build_host)
    ns::Buf split;     // the hot-key split's device state
    ns::Buf colsplit;  // the hot-destination split's device state
    bool last_split = false;  // the last sort-path build split
    bool last_colsplit = false;  // the last sort-path build split its column side
    ns::DevStats* host_stats = nullptr;  // pinned
    ns::Tracer tracer;
};

// A traffic matrix.  Hash format: link/row/column tables with incrementally
// maintained statistics.  List format: A's nonzeros sorted by key, with the
// statistics computed by the sort path.  In both, the statistics record's
// unique-links field is the number of nonzeros.
struct ns_matrix {
    ns_ctx* ctx = nullptr;
    int device = 0;  // the context's device (kept here: a matrix may be freed after its context)
    int fmt = ns::FMT_EMPTY;
    ns::Buf links, rows, cols;
    uint64_t link_cap = 0, node_cap = 0;
    ns::Buf keys, counts;
    ns::Buf stats;       // ns::DevStats
    uint64_t bound = 0;       // host-side upper bound on the number of nonzeros
    uint64_t node_limit = 0;  // caller's bound on sources and destinations (0 = none)
    cudaStream_t last_stream = nullptr;  // the stream of the last call that enqueued work on it
};

namespace ns {
// Records that a call enqueues work on m on stream s (ns_matrix_free frees
// the matrix's buffers on the last such stream).
inline void touch(ns_matrix* m, cudaStream_t s) {
    if (m) m->last_stream = s;
}
inline void touch(const ns_matrix* m, cudaStream_t s) { touch(const_cast<ns_matrix*>(m), s); }
// An entry point's scope: its context's device, and its pool and stream for
// buffer allocation; also records the stream as the context's last.
struct CallScope {
    DeviceGuard dev;
    AllocScope alloc;
    CallScope(ns_ctx* c, cudaStream_t s) : dev(c->device), alloc(c->pool, s) { c->last_stream = s; }
};
}  // namespace ns
