// ns_api_internal.h -- host-side objects behind the opaque ns_ctx / ns_matrix.
#pragma once

#include <cstdint>
#include <string>

#include "ns.h"
#include "ns_kernels.h"

namespace ns {

// A grow-only device allocation.
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

enum { FMT_EMPTY = 0, FMT_HASH = 1, FMT_LIST = 2 };

ns_status buf_reserve(Buf& b, size_t bytes);
ns_status fail_fmt(ns_status s, const char* fmt, ...);
ns_status to_hash(ns_matrix* m, u64 extra, cudaStream_t s);
ns_status check_launch();
HashView hash_view(const ns_matrix* m);
void buf_free(Buf& b);
ns_status check_launch();
ns_status set_fail(ns_status s, const char* msg);

}  // namespace ns

struct ns_ctx {
    int device = 0;
    int sms = 148;
    ns_config cfg{};
    std::string tuner_cache;
    ns::SortScratch sc{};
    ns::Buf ghist, offs, tcount, counters, status;
    ns::Buf k64[2], pos, psum, k32[2], v64[2], xk, xv;
    ns::DevStats* host_stats = nullptr;  // pinned
    ns::Tracer tracer;
};

// A traffic matrix.  Hash format: link/row/column tables with incrementally
// maintained statistics.  List format: A's nonzeros sorted by key, with the
// statistics computed by the sort path.  In both, the statistics record's
// unique-links field is the number of nonzeros.
struct ns_matrix {
    ns_ctx* ctx = nullptr;
    int fmt = ns::FMT_EMPTY;
    ns::Buf links, rows, cols;
    uint64_t link_cap = 0, node_cap = 0;
    ns::Buf keys, counts;
    ns::Buf stats;       // ns::DevStats
    uint64_t bound = 0;       // host-side upper bound on the number of nonzeros
    uint64_t node_limit = 0;  // caller's bound on sources and destinations (0 = none)
};
