// ns_api.cu -- the C ABI (include/ns.h): contexts, matrices, path selection,
// capacity planning and error reporting around the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_kernels.h"

using namespace ns;

namespace {

thread_local std::string g_err;

ns_status fail(ns_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return fail(NS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(call)                    \
    do {                             \
        ns_status st_ = (call);      \
        if (st_ != NS_OK) return st_; \
    } while (0)

u64 next_pow2(u64 x) {
    u64 p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

namespace ns {

namespace {
thread_local cudaMemPool_t t_pool = nullptr;
thread_local cudaStream_t t_stream = nullptr;
thread_local bool t_private = false;
}  // namespace

AllocScope::AllocScope(cudaMemPool_t pool, cudaStream_t s, bool stream_private)
    : prev_pool(t_pool), prev_stream(t_stream), prev_private(t_private) {
    t_pool = pool;
    t_stream = s;
    t_private = stream_private;
}
AllocScope::~AllocScope() {
    t_pool = prev_pool;
    t_stream = prev_stream;
    t_private = prev_private;
}
cudaStream_t alloc_stream() { return t_stream; }

ns_status buf_reserve(Buf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return NS_OK;
    const cudaStream_t s = t_stream;
    // Growing inside a CUDA graph capture would make the new buffer the
    // graph's own (or fail): refuse with a clear error.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (cs != cudaStreamCaptureStatusNone)
        return fail(NS_ERR_STATE, "a buffer must grow (to %zu bytes) while its stream is being captured; "
                                  "run the call once before the capture", bytes);
    // Stream-private scopes (every earlier use of their buffers is on their
    // stream or complete) allocate from the context's pool in stream order;
    // all others use cudaMalloc / cudaFree, which wait for the device.
    const bool pooled = t_private && t_pool;
    if (b.p) {
        if (b.pooled) {
            if (!t_private) cudaDeviceSynchronize();  // earlier readers on other streams are done
            cudaFreeAsync(b.p, s);
        } else {
            cudaFree(b.p);
        }
        b.p = nullptr;
        b.bytes = 0;
        b.pooled = false;
    }
    if (bytes == 0) return NS_OK;
    const cudaError_t e = pooled ? cudaMallocFromPoolAsync(&b.p, bytes, t_pool, s) : cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(NS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    b.pooled = pooled;
    return NS_OK;
}

void buf_free_on(Buf& b, cudaStream_t s) {
    if (b.p) {
        if (!b.pooled) {
            cudaFree(b.p);
        } else if (cudaFreeAsync(b.p, s) != cudaSuccess) {
            // the stream is gone: wait for the device, then free on the legacy stream
            cudaGetLastError();
            cudaDeviceSynchronize();
            cudaFreeAsync(b.p, nullptr);
        }
        cudaGetLastError();
    }
    b.p = nullptr;
    b.bytes = 0;
    b.pooled = false;
}

void buf_free(Buf& b) { buf_free_on(b, t_stream); }

ns_status set_fail(ns_status s, const char* msg) { return fail(s, "%s", msg); }

ns_status fail_fmt(ns_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

ns_status check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(NS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return NS_OK;
}

HashView hash_view(const ns_matrix* m) {
    HashView v;
    v.links = (LinkSlot*)m->links.p;
    v.link_mask = m->link_cap - 1;
    v.rows = (NodeSlot*)m->rows.p;
    v.row_mask = m->node_cap - 1;
    v.cols = (NodeSlot*)m->cols.p;
    v.col_mask = m->node_cap - 1;
    v.stats = (DevStats*)m->stats.p;
    return v;
}

// Smallest power-of-two capacity (>= 1024) holding `items` at load <= load.
u64 table_cap(u64 items, double load) {
    return next_pow2(std::max<u64>((u64)std::ceil((double)items / load), 1024));
}

// Sets the matrix's active table capacities for at least `links` nonzeros at
// the context's load bound, and for at least min(links, node_limit) sources and as many
// destinations (sources, destinations <= links; node_limit is the caller's
// optional promise, 0 = none).  Allocations only grow; a smaller active
// capacity reuses them, so clearing and scanning cost what this window needs.
// Contents are undefined until cleared.
ns_status hash_alloc(ns_matrix* m, u64 links) {
    const double load = m->ctx->cfg.hash_load;
    const u64 cap = table_cap(links, load);
    const u64 nodes = m->node_limit ? std::min<u64>(links, m->node_limit) : links;
    const u64 ncap = table_cap(nodes, load);
    TRY(buf_reserve(m->links, (cap + 1) * sizeof(LinkSlot)));
    TRY(buf_reserve(m->rows, (ncap + 1) * sizeof(NodeSlot)));
    TRY(buf_reserve(m->cols, (ncap + 1) * sizeof(NodeSlot)));
    m->link_cap = cap;
    m->node_cap = ncap;
    return NS_OK;
}

ns_status hash_clear(ns_matrix* m, cudaStream_t s) {
    CK(cudaMemsetAsync(m->links.p, 0, (m->link_cap + 1) * sizeof(LinkSlot), s));
    CK(cudaMemsetAsync(m->rows.p, 0, (m->node_cap + 1) * sizeof(NodeSlot), s));
    CK(cudaMemsetAsync(m->cols.p, 0, (m->node_cap + 1) * sizeof(NodeSlot), s));
    CK(cudaMemsetAsync(m->stats.p, 0, sizeof(DevStats), s));
    return NS_OK;
}

// Reads the matrix's statistics record (blocking) into the context's pinned
// buffer and returns the device error word as a status.
ns_status read_stats(const ns_matrix* m, cudaStream_t s, DevStats* out) {
    ns_ctx* c = m->ctx;
    CK(cudaMemcpyAsync(c->host_stats, m->stats.p, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = *c->host_stats;
    if (out->err & ERR_TIMEOUT) return fail(NS_ERR_TIMEOUT, "a device-side wait gave up (look-back)");
    if (out->err & ERR_CAPACITY) return fail(NS_ERR_CAPACITY, "a hash probe sequence exceeded its bound");
    return NS_OK;
}

// Makes room in a hash-format accumulator for `extra` more nonzeros.  Uses
// the host-side bound first; only when that is exhausted does it read the
// true count and, if needed, rehash into larger tables.
ns_status hash_grow(ns_matrix* m, u64 extra, cudaStream_t s) {
    const u64 limit = (u64)((double)m->link_cap * m->ctx->cfg.hash_load);
    if (m->bound + extra <= limit) return NS_OK;
    DevStats ds;
    TRY(read_stats(m, s, &ds));
    const u64 actual = ds.v[S_LINKS];
    m->bound = actual;
    if (actual + extra <= limit) return NS_OK;
    // rehash: rebuild rows/cols/statistics from the link entries
    ns_matrix tmp;
    tmp.ctx = m->ctx;
    tmp.device = m->device;
    tmp.stats = m->stats;
    tmp.node_limit = m->node_limit;
    TRY(hash_alloc(&tmp, actual + extra));
    CK(cudaMemsetAsync(tmp.links.p, 0, (tmp.link_cap + 1) * sizeof(LinkSlot), s));
    CK(cudaMemsetAsync(tmp.rows.p, 0, (tmp.node_cap + 1) * sizeof(NodeSlot), s));
    CK(cudaMemsetAsync(tmp.cols.p, 0, (tmp.node_cap + 1) * sizeof(NodeSlot), s));
    CK(cudaMemsetAsync(m->stats.p, 0, sizeof(DevStats), s));
    {
        TraceScope ts(&m->ctx->tracer, "k_insert_slots", s);
        launch_insert_slots((const LinkSlot*)m->links.p, m->link_cap, hash_view(&tmp), m->ctx->sms, s);
    }
    TRY(check_launch());
    CK(cudaStreamSynchronize(s));
    buf_free(m->links);
    buf_free(m->rows);
    buf_free(m->cols);
    m->links = tmp.links;
    m->rows = tmp.rows;
    m->cols = tmp.cols;
    m->link_cap = tmp.link_cap;
    m->node_cap = tmp.node_cap;
    tmp.links = tmp.rows = tmp.cols = Buf{};
    tmp.stats = Buf{};
    return NS_OK;
}

// Turns an accumulator into hash format (empty, or from its sorted list).
ns_status to_hash(ns_matrix* m, u64 extra, cudaStream_t s) {
    touch(m, s);
    if (m->fmt == FMT_HASH) return hash_grow(m, extra, s);
    ns_ctx* c = m->ctx;
    const u64 have = (m->fmt == FMT_LIST) ? m->bound : 0;
    TRY(hash_alloc(m, have + extra));
    if (m->fmt == FMT_LIST && have > 0) {
        // the list length lives in the statistics record, which is rebuilt:
        // keep a copy for the insert kernel
        TRY(buf_reserve(c->counters, 16 * sizeof(u64)));
        u64* nnz_copy = (u64*)c->counters.p + 15;
        CK(cudaMemcpyAsync(nnz_copy, &((DevStats*)m->stats.p)->v[S_LINKS], sizeof(u64),
                           cudaMemcpyDeviceToDevice, s));
        TRY(hash_clear(m, s));
        TraceScope ts(&c->tracer, "k_insert_list", s);
        launch_insert_list((const u64*)m->keys.p, (const u64*)m->counts.p, have, nnz_copy,
                           hash_view(m), c->sms, s);
        TRY(check_launch());
    } else {
        TRY(hash_clear(m, s));
        m->bound = 0;
    }
    m->fmt = FMT_HASH;
    return NS_OK;
}

ns_status context_pool(ns_ctx* c) {
    if (c->pool) return NS_OK;
    // keeps freed memory for reuse until the context is destroyed
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        c->pool = nullptr;
        return fail(NS_ERR_CUDA, "memory pool creation failed");
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    return NS_OK;
}

ns_status sort_scratch(ns_ctx* c, u64 n) {
    const u64 tiles = sort_tiles(std::max<u64>(n, 1));
    const u64 words = tiles * (u64)sort_radix(c->sc.digit_plan);
    if (c->status.bytes < words * sizeof(u64)) {
        TRY(buf_reserve(c->status, words * sizeof(u64)));
        CK(cudaMemsetAsync(c->status.p, 0, words * sizeof(u64), alloc_stream()));
        c->sc.tag = 0;
    }
    c->sc.status = (u64*)c->status.p;
    c->sc.status_words = c->status.bytes / sizeof(u64);
    return NS_OK;
}

// Whether a sort-path build of n packets takes the hot-key split: the
// context's setting, else ns_path_tune's measurement for the size, else on
// from 2^23 packets.  Below 2^16 packets the sample would be too small.
constexpr int kAutoSplitLog2 = 23;
bool use_split(const ns_ctx* c, u64 n) {
    if (n < (1ull << 16) || c->cfg.sort_split == NS_SPLIT_OFF) return false;
    if (c->cfg.sort_split == NS_SPLIT_ON) return true;
    const int lg = 63 - __builtin_clzll(n);
    const auto it = c->path_choice.find(lg);
    if (it != c->path_choice.end() && it->second.split >= 0) return it->second.split != 0;
    return lg >= kAutoSplitLog2;
}

// Sort path: A_t's sorted nonzero list and its statistics.
// The digit passes' tile shape for n packets: the context's setting, else
// ns_path_tune's measurement for the size, else 512 threads x 16 keys.
int resolve_tile(const ns_ctx* c, u64 n) {
    if (c->cfg.sort_tile != NS_TILE_AUTO) return c->cfg.sort_tile - 1;
    const auto it = c->path_choice.find(n ? 63 - __builtin_clzll(n) : 0);
    if (it != c->path_choice.end() && it->second.tile >= 0) return it->second.tile;
    return 0;
}

// The digit plan of the digit passes over 64-bit keys for n packets: the
// context's setting, else ns_path_tune's measurement for the size, else
// eight 8-bit passes.
int resolve_digits(const ns_ctx* c, u64 n) {
    if (c->cfg.sort_digits != NS_DIGITS_AUTO) return c->cfg.sort_digits == NS_DIGITS_WIDE ? kDigitsWide : kDigits8;
    const auto it = c->path_choice.find(n ? 63 - __builtin_clzll(n) : 0);
    if (it != c->path_choice.end() && it->second.digits >= 0) return it->second.digits;
    return kDigits8;
}

void resolve_sort(const ns_ctx* c, u64 n, int* split, int* tile, int* digits) {
    if (split) *split = use_split(c, n) ? 1 : 0;
    if (tile) *tile = resolve_tile(c, n);
    if (digits) *digits = resolve_digits(c, n);
}

// split: -1 = use_split's rule, 0 = no split, 1 = split (from 2^16 packets);
// tile: -1 = resolve_tile's rule, else the digit passes' tile shape;
// digits: -1 = resolve_digits's rule, else the digit plan.
ns_status build_sort(ns_ctx* c, const uint32_t* src, const uint32_t* dst, u64 n, ns_matrix* out,
                     cudaStream_t s, int split, int tile, int digits) {
    touch(out, s);
    c->sc.tile_shape = tile < 0 ? resolve_tile(c, n) : tile;
    c->sc.digit_plan = digits < 0 ? resolve_digits(c, n) : digits;
    out->fmt = FMT_LIST;
    out->bound = n;
    CK(cudaMemsetAsync(out->stats.p, 0, sizeof(DevStats), s));
    if (n == 0) return NS_OK;
    TRY(buf_reserve(out->keys, n * sizeof(u64)));
    TRY(buf_reserve(out->counts, n * sizeof(u64)));
    TRY(sort_scratch(c, n));
    TRY(buf_reserve(c->k64[0], n * sizeof(u64)));
    TRY(buf_reserve(c->k64[1], n * sizeof(u64)));
    TRY(buf_reserve(c->pos, (n + 1) * sizeof(u64)));
    TRY(buf_reserve(c->psum, (n + 1) * sizeof(u64)));
    // Below 2^32 packets every count fits 32 bits, and the column side sorts
    // single words (dst << 32 | count) by their upper half; otherwise it
    // sorts (dst, count) pairs.
    const bool packed_cols = n < (1ull << 32) && c->cfg.column_sort != NS_COLSORT_PAIRS;
    TRY(buf_reserve(c->v64[0], n * sizeof(u64)));
    if (!packed_cols) {
        TRY(buf_reserve(c->k32[0], n * sizeof(u32)));
        TRY(buf_reserve(c->k32[1], n * sizeof(u32)));
        TRY(buf_reserve(c->v64[1], n * sizeof(u64)));
    }
    TRY(buf_reserve(c->counters, 16 * sizeof(u64)));
    DevStats* st = (DevStats*)out->stats.p;
    u64* nnz = &st->v[S_LINKS];
    u64* runs_out = (u64*)c->counters.p;

    // links: sort packed keys, then runs of equal keys (Table 2 row 3);
    // with the split, the heaviest sampled links are counted apart and only
    // the other packets are sorted
    u64* kb[2] = {(u64*)c->k64[0].p, (u64*)c->k64[1].p};
    c->last_split = split < 0 ? use_split(c, n) : (split != 0 && n >= (1ull << 16));
    if (c->last_split) {
        TRY(buf_reserve(c->split, split_state_bytes()));
        sort_links_split(src, dst, n, kb, (u64*)c->v64[0].p, (u64*)c->pos.p, c->split.p, (u64*)out->keys.p,
                         (u64*)out->counts.p, c->sc, st, c->sms, s);
    } else {
        const int r = radix_sort_packets(src, dst, kb, n, c->sc, st, s);
        launch_runs(RUN_U64, false, kb[r], nullptr, n, nullptr, (u64*)out->keys.p,
                    (u64*)c->pos.p, nullptr, nnz, c->sc, st, s);
        launch_run_stats(RS_LINKS, (const u64*)c->pos.p, nullptr, nnz, n, (u64*)out->counts.p,
                         st, c->sms, &c->tracer, s);
    }
    // rows: runs of equal src over the source-major list (rows 5-9)
    u64* packed = packed_cols ? (u64*)c->v64[0].p : nullptr;
    launch_runs(RUN_SRC_OF_U64, true, out->keys.p, (const u64*)out->counts.p, n, nnz, nullptr,
                (u64*)c->pos.p, (u64*)c->psum.p, runs_out, c->sc, st, s, packed);
    launch_run_stats(RS_ROWS, (const u64*)c->pos.p, (const u64*)c->psum.p, runs_out, n,
                     nullptr, st, c->sms, &c->tracer, s);
    c->last_colsplit = packed_cols && c->last_split;
    if (c->last_colsplit) {
        // columns with the hot-destination split: the heaviest sampled
        // destinations are counted apart, only the other words are sorted
        TRY(buf_reserve(c->colsplit, col_split_state_bytes()));
        col_split_runs(packed, nnz, n, kb, (u64*)c->pos.p, (u64*)c->psum.p, c->colsplit.p, runs_out + 1, c->sc, st,
                       c->sms, s);
        return check_launch();
    }
    if (packed_cols) {
        // columns: the words (dst << 32 | count) sorted by dst, then runs of
        // equal dst (the reverse operations)
        const int r2 = radix_sort_hi32(packed, nnz, kb, n, c->sc, st, s);
        launch_runs(RUN_HI_OF_PACKED, true, kb[r2], nullptr, n, nnz, nullptr, (u64*)c->pos.p,
                    (u64*)c->psum.p, runs_out + 1, c->sc, st, s);
        launch_run_stats(RS_COLS, (const u64*)c->pos.p, (const u64*)c->psum.p, runs_out + 1, n,
                         nullptr, st, c->sms, &c->tracer, s);
        return check_launch();
    }
    // columns: (dst, count) sorted by dst, then runs (the reverse operations)
    u32* ck[2] = {(u32*)c->k32[0].p, (u32*)c->k32[1].p};
    u64* cv[2] = {(u64*)c->v64[0].p, (u64*)c->v64[1].p};
    const int r2 = radix_sort_dst_pairs((const u64*)out->keys.p, (const u64*)out->counts.p,
                                        nnz, ck, cv, n, c->sc, st, s);
    launch_runs(RUN_U32, true, ck[r2], cv[r2], n, nnz, nullptr, (u64*)c->pos.p,
                (u64*)c->psum.p, runs_out + 1, c->sc, st, s);
    launch_run_stats(RS_COLS, (const u64*)c->pos.p, (const u64*)c->psum.p, runs_out + 1, n,
                     nullptr, st, c->sms, &c->tracer, s);
    return check_launch();
}

// The per-CTA cache pays off when each CTA sees many packets (skewed keys
// then repeat inside it); a single 2^17-packet window gives each CTA ~256.
int floor_log2(u64 n) { return n ? 63 - __builtin_clzll(n) : 0; }

bool use_cta_cache(const ns_ctx* c, u64 n) {
    if (c->cfg.cta_cache == NS_CACHE_ON) return true;
    if (c->cfg.cta_cache == NS_CACHE_OFF) return false;
    const auto it = c->path_choice.find(floor_log2(n));
    if (it != c->path_choice.end() && it->second.path == NS_PATH_HASH) return it->second.cta_cache;
    return n >= (1ull << 22);
}

// Sizes from which NS_PATH_AUTO takes the sort path when the context has no
// tuned choice for that size: floor(log2 n) >= kAutoSortLog2.  Measured on a
// B300 over Zipf(1.2) and RMAT windows of 2^14..2^30 packets: the hash path is
// faster up to 2^22, the sort path from 2^24 on (1.3x at 2^26, 1.8-2.4x at 2^30).
constexpr int kAutoSortLog2 = 24;

std::string path_key(int device, int lg) {
    char buf[32];
    snprintf(buf, sizeof buf, "|path|n2^%d", lg);
    return gpu_name(device) + buf;
}

// Tuned choices for this GPU from the context's cache file.
void load_path_choices(ns_ctx* c) {
    const std::string prefix = gpu_name(c->device) + "|path|n2^";
    for (const auto& kv : tuner_load(c->tuner_cache)) {
        if (kv.first.compare(0, prefix.size(), prefix) != 0) continue;
        const int lg = atoi(kv.first.c_str() + prefix.size());
        std::string p;
        double cache = 0, split = -1, tile = -1, digits = -1;
        if (lg < 0 || lg > 40 || !json_string(kv.second, "path", &p)) continue;
        json_number(kv.second, "cta_cache", &cache);
        json_number(kv.second, "sort_split", &split);
        json_number(kv.second, "sort_tile", &tile);
        json_number(kv.second, "sort_digits", &digits);
        const int sp = split < 0 ? -1 : (split != 0 ? 1 : 0);
        const int tl = (tile >= 0 && tile < kSortTileShapes) ? (int)tile : -1;
        const int dg = (digits >= 0 && digits < kDigitPlans) ? (int)digits : -1;
        if (p == "sort") c->path_choice[lg] = {NS_PATH_SORT, false, sp, tl, dg};
        if (p == "hash") c->path_choice[lg] = {NS_PATH_HASH, cache != 0, sp, tl, dg};
    }
}

int resolve_path(const ns_ctx* c, u64 n) {
    if (c->cfg.path != NS_PATH_AUTO) return c->cfg.path;
    const int lg = floor_log2(n);
    const auto it = c->path_choice.find(lg);
    if (it != c->path_choice.end()) return it->second.path;
    return lg >= kAutoSortLog2 ? NS_PATH_SORT : NS_PATH_HASH;
}

ns_status build_hash(ns_ctx* c, const uint32_t* src, const uint32_t* dst, u64 n, ns_matrix* out,
                     cudaStream_t s, int cache) {
    touch(out, s);
    TRY(hash_alloc(out, n));
    TRY(hash_clear(out, s));
    out->fmt = FMT_HASH;
    out->bound = n;
    if (n == 0) return NS_OK;
    TraceScope ts(&c->tracer, "k_insert_packets", s);
    launch_insert_packets(src, dst, n, hash_view(out), c->sms, cache < 0 ? use_cta_cache(c, n) : cache != 0, s);
    return check_launch();
}

}  // namespace ns

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

const char* ns_last_error(void) { return g_err.c_str(); }

const char* ns_status_string(ns_status s) {
    switch (s) {
        case NS_OK: return "NS_OK";
        case NS_ERR_INVALID: return "NS_ERR_INVALID";
        case NS_ERR_OOM: return "NS_ERR_OOM";
        case NS_ERR_CAPACITY: return "NS_ERR_CAPACITY";
        case NS_ERR_CUDA: return "NS_ERR_CUDA";
        case NS_ERR_TIMEOUT: return "NS_ERR_TIMEOUT";
        case NS_ERR_BUSY: return "NS_ERR_BUSY";
        case NS_ERR_STATE: return "NS_ERR_STATE";
        case NS_ERR_IO: return "NS_ERR_IO";
    }
    return "NS_ERR_?";
}

ns_status ns_create(ns_ctx** out, const ns_config* cfg, int device) {
    if (!out) return fail(NS_ERR_INVALID, "ns_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(NS_ERR_INVALID, "ns_create: no CUDA device %d", device);
    ns_config c{};
    if (cfg) c = *cfg;
    if (c.path < NS_PATH_AUTO || c.path > NS_PATH_HASH)
        return fail(NS_ERR_INVALID, "ns_create: unknown path %d", c.path);
    if (c.cta_cache < NS_CACHE_AUTO || c.cta_cache > NS_CACHE_OFF)
        return fail(NS_ERR_INVALID, "ns_create: unknown cta_cache %d", c.cta_cache);
    if (c.column_sort < NS_COLSORT_AUTO || c.column_sort > NS_COLSORT_PAIRS)
        return fail(NS_ERR_INVALID, "ns_create: unknown column_sort %d", c.column_sort);
    if (c.sort_split < NS_SPLIT_AUTO || c.sort_split > NS_SPLIT_OFF)
        return fail(NS_ERR_INVALID, "ns_create: unknown sort_split %d", c.sort_split);
    if (c.sort_tile < NS_TILE_AUTO || c.sort_tile > NS_TILE_256X16)
        return fail(NS_ERR_INVALID, "ns_create: unknown sort_tile %d", c.sort_tile);
    if (c.sort_digits < NS_DIGITS_AUTO || c.sort_digits > NS_DIGITS_WIDE)
        return fail(NS_ERR_INVALID, "ns_create: unknown sort_digits %d", c.sort_digits);
    if (c.hash_load == 0.0) c.hash_load = 0.5;
    if (!(c.hash_load >= 0.05 && c.hash_load <= 0.9))
        return fail(NS_ERR_INVALID, "ns_create: hash_load %g outside [0.05, 0.9]", c.hash_load);
    DeviceGuard device_guard(device);
    CK(cudaSetDevice(device));
    ns_ctx* x = new ns_ctx();
    x->device = device;
    x->cfg = c;
    if (x->cfg.hbm_budget_bytes == 0) x->cfg.hbm_budget_bytes = 64ull << 30;
    if (x->cfg.max_slots <= 0) x->cfg.max_slots = 8;
    x->tuner_cache = c.tuner_cache ? c.tuner_cache : "";
    x->cfg.tuner_cache = nullptr;
    load_path_choices(x);
    cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, device);
    x->sc.sms = x->sms;
    AllocScope alloc(nullptr, nullptr);
    // digit histograms and bucket starts of either digit plan: eight passes
    // of 256 digits, or the wide plan's 1024 + 6 x 512; then the first
    // pass's cursors
    ns_status st = buf_reserve(x->ghist, 4096 * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x->offs, (4096 + 1024) * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x->tcount, 16 * sizeof(u32));
    if (st == NS_OK) st = buf_reserve(x->counters, 16 * sizeof(u64));
    if (st == NS_OK && cudaMallocHost((void**)&x->host_stats, sizeof(DevStats)) != cudaSuccess)
        st = fail(NS_ERR_OOM, "cudaMallocHost failed");
    if (st == NS_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = check_launch();
    if (st != NS_OK) {
        ns_destroy(x);
        return st;
    }
    x->sc.ghist = (u64*)x->ghist.p;
    x->sc.offs = (u64*)x->offs.p;
    x->sc.tile_counters = (u32*)x->tcount.p;
    x->sc.tag = 0;
    x->sc.status = nullptr;
    x->sc.status_words = 0;
    x->sc.tr = &x->tracer;
    *out = x;
    return NS_OK;
}

void ns_destroy(ns_ctx* c) {
    if (!c) return;
    DeviceGuard device_guard(c->device);
    // The context's scratch may have been used on several streams: wait for
    // the device, then free it; the pool gives its memory back once every
    // buffer allocated from it has been freed.
    cudaDeviceSynchronize();
    Buf* all[] = {&c->ghist, &c->offs, &c->tcount, &c->counters, &c->status, &c->k64[0], &c->k64[1],
                  &c->pos, &c->psum, &c->k32[0], &c->k32[1], &c->v64[0], &c->v64[1], &c->xk, &c->xv,
                  &c->stage[0], &c->stage[1], &c->split, &c->colsplit};
    for (Buf* b : all) buf_free_on(*b, c->last_stream);
    if (c->host_stats) cudaFreeHost(c->host_stats);  // used only by blocking reads, all complete
    tracer_destroy(&c->tracer);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaGetLastError();
    delete c;
}

ns_status ns_sync(ns_ctx* c, ns_stream_t stream) {
    if (!c) return fail(NS_ERR_INVALID, "ns_sync: NULL context");
    DeviceGuard device_guard(c->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return check_launch();
}

ns_status ns_matrix_create(ns_ctx* c, ns_matrix** out) {
    if (!c || !out) return fail(NS_ERR_INVALID, "ns_matrix_create: NULL argument");
    DeviceGuard device_guard(c->device);
    AllocScope alloc(c->pool, nullptr);
    ns_matrix* m = new ns_matrix();
    m->ctx = c;
    m->device = c->device;
    m->last_stream = nullptr;
    ns_status st = buf_reserve(m->stats, sizeof(DevStats));
    if (st == NS_OK && (cudaMemsetAsync(m->stats.p, 0, sizeof(DevStats), nullptr) != cudaSuccess ||
                        cudaStreamSynchronize(nullptr) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(NS_ERR_CUDA, "ns_matrix_create: clearing the statistics record failed");
    }
    if (st != NS_OK) {
        ns_matrix_free(m);
        return st;
    }
    *out = m;
    return NS_OK;
}

ns_status ns_matrix_reserve(ns_matrix* m, uint64_t max_links, ns_stream_t stream) {
    if (!m) return fail(NS_ERR_INVALID, "ns_matrix_reserve: NULL matrix");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(m->ctx, s);
    touch(m, s);
    if (m->fmt == FMT_EMPTY) {
        TRY(hash_alloc(m, max_links));
        TRY(hash_clear(m, s));
        m->fmt = FMT_HASH;
        m->bound = 0;
        return NS_OK;
    }
    if (m->fmt == FMT_HASH) return hash_grow(m, max_links > m->bound ? max_links - m->bound : 0, s);
    return NS_OK;
}

ns_status ns_matrix_reserve_ex(ns_matrix* m, uint64_t max_links, uint64_t max_nodes, ns_stream_t stream) {
    if (!m) return fail(NS_ERR_INVALID, "ns_matrix_reserve_ex: NULL matrix");
    DeviceGuard device_guard(m->device);
    if (m->fmt != FMT_EMPTY) return fail(NS_ERR_STATE, "ns_matrix_reserve_ex: matrix is not empty");
    m->node_limit = max_nodes;
    return ns_matrix_reserve(m, max_links, stream);
}

ns_status ns_matrix_clear(ns_matrix* m, ns_stream_t stream) {
    if (!m) return fail(NS_ERR_INVALID, "ns_matrix_clear: NULL matrix");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(m->ctx, s);
    touch(m, s);
    if (m->fmt == FMT_HASH) {
        TRY(hash_clear(m, s));
    } else {
        CK(cudaMemsetAsync(m->stats.p, 0, sizeof(DevStats), s));
        if (m->fmt == FMT_LIST) m->fmt = FMT_EMPTY;
    }
    m->bound = 0;
    return NS_OK;
}

void ns_matrix_free(ns_matrix* m) {
    if (!m) return;
    DeviceGuard device_guard(m->device);
    // behind the matrix's pending work on the stream it was last used on;
    // the host does not wait
    const cudaStream_t s = m->last_stream;
    buf_free_on(m->links, s);
    buf_free_on(m->rows, s);
    buf_free_on(m->cols, s);
    buf_free_on(m->keys, s);
    buf_free_on(m->counts, s);
    buf_free_on(m->stats, s);
    delete m;
}

ns_status ns_matrix_nnz(const ns_matrix* m, uint64_t* h_nnz, ns_stream_t stream) {
    if (!m || !h_nnz) return fail(NS_ERR_INVALID, "ns_matrix_nnz: NULL argument");
    DeviceGuard device_guard(m->device);
    DevStats ds;
    ns_status st = read_stats(m, (cudaStream_t)stream, &ds);
    *h_nnz = ds.v[S_LINKS];
    return st;
}

ns_status ns_matrix_export(const ns_matrix* m, uint64_t* d_keys, uint64_t* d_counts, uint64_t cap,
                           uint64_t* h_nnz, ns_stream_t stream) {
    if (!m || !h_nnz) return fail(NS_ERR_INVALID, "ns_matrix_export: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(m->ctx, s);
    touch(m, s);
    DevStats ds;
    TRY(read_stats(m, s, &ds));
    const u64 nnz = ds.v[S_LINKS];
    *h_nnz = nnz;
    if (nnz == 0) return NS_OK;
    if (!d_keys || !d_counts) return fail(NS_ERR_INVALID, "ns_matrix_export: NULL output with nnz > 0");
    if (cap < nnz) return fail(NS_ERR_CAPACITY, "ns_matrix_export: cap %llu < nnz %llu",
                               (unsigned long long)cap, (unsigned long long)nnz);
    ns_ctx* c = m->ctx;
    if (m->fmt == FMT_LIST) {
        CK(cudaMemcpyAsync(d_keys, m->keys.p, nnz * sizeof(u64), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(d_counts, m->counts.p, nnz * sizeof(u64), cudaMemcpyDeviceToDevice, s));
    } else {
        TRY(sort_scratch(c, nnz));
        TRY(buf_reserve(c->xk, nnz * sizeof(u64)));
        TRY(buf_reserve(c->xv, nnz * sizeof(u64)));
        TRY(buf_reserve(c->k64[0], nnz * sizeof(u64)));
        TRY(buf_reserve(c->v64[0], nnz * sizeof(u64)));
        TRY(buf_reserve(c->counters, 16 * sizeof(u64)));
        u64* cnt = (u64*)c->counters.p + 2;
        CK(cudaMemsetAsync(cnt, 0, sizeof(u64), s));
        DevStats* st = (DevStats*)m->stats.p;
        TraceScope ts(&c->tracer, "k_compact_links", s);
        launch_compact_links((const LinkSlot*)m->links.p, m->link_cap, (u64*)c->xk.p,
                             (u64*)c->xv.p, cnt, nnz, st, c->sms, s);
        u64* kb[2] = {(u64*)c->k64[0].p, (u64*)d_keys};
        u64* vb[2] = {(u64*)c->v64[0].p, (u64*)d_counts};
        const int r = radix_sort_pairs64((const u64*)c->xk.p, (const u64*)c->xv.p, cnt, kb, vb,
                                         nnz, c->sc, st, s);
        if (r != 1) return fail(NS_ERR_STATE, "export: unexpected sort parity");
        TRY(check_launch());
    }
    DevStats after;
    return read_stats(m, s, &after);
}

ns_status ns_window_build(ns_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                          ns_matrix* out, ns_stream_t stream) {
    if (!c || !out) return fail(NS_ERR_INVALID, "ns_window_build: NULL context or matrix");
    CallScope scope(c, (cudaStream_t)stream);
    if (n > 0 && (!d_src || !d_dst)) return fail(NS_ERR_INVALID, "ns_window_build: NULL input with n > 0");
    if (n >= (1ull << 40)) return fail(NS_ERR_INVALID, "ns_window_build: n too large");
    if (out->ctx != c) return fail(NS_ERR_INVALID, "ns_window_build: matrix belongs to another context");
    if (resolve_path(c, n) == NS_PATH_SORT) return build_sort(c, d_src, d_dst, n, out, (cudaStream_t)stream);
    return build_hash(c, d_src, d_dst, n, out, (cudaStream_t)stream);
}

ns_status ns_window_build_host(ns_ctx* c, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n,
                               ns_matrix* out, ns_stats* h_stats, ns_stream_t stream) {
    if (!c || !out) return fail(NS_ERR_INVALID, "ns_window_build_host: NULL context or matrix");
    CallScope scope(c, (cudaStream_t)stream);
    if (n > 0 && (!h_src || !h_dst)) return fail(NS_ERR_INVALID, "ns_window_build_host: NULL input with n > 0");
    if (n >= (1ull << 40)) return fail(NS_ERR_INVALID, "ns_window_build_host: n too large");
    if (out->ctx != c) return fail(NS_ERR_INVALID, "ns_window_build_host: matrix belongs to another context");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t* d_src = nullptr;
    const uint32_t* d_dst = nullptr;
    if (n > 0) {
        TRY(buf_reserve(c->stage[0], n * sizeof(uint32_t)));
        TRY(buf_reserve(c->stage[1], n * sizeof(uint32_t)));
        CK(cudaMemcpyAsync(c->stage[0].p, h_src, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->stage[1].p, h_dst, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        d_src = (const uint32_t*)c->stage[0].p;
        d_dst = (const uint32_t*)c->stage[1].p;
    }
    TRY(ns_window_build(c, d_src, d_dst, n, out, stream));
    if (h_stats) return ns_network_stats(c, out, h_stats, stream);
    CK(cudaStreamSynchronize(s));
    return check_launch();
}

ns_status ns_path_tune(ns_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n, ns_stream_t stream,
                       int* chosen, float* sort_ms, float* hash_ms) {
    if (!c) return fail(NS_ERR_INVALID, "ns_path_tune: NULL context");
    CallScope scope(c, (cudaStream_t)stream);
    if (n == 0) return fail(NS_ERR_INVALID, "ns_path_tune: n == 0");
    if (!d_src || !d_dst) return fail(NS_ERR_INVALID, "ns_path_tune: NULL input");
    if (n >= (1ull << 40)) return fail(NS_ERR_INVALID, "ns_path_tune: n too large");
    cudaStream_t s = (cudaStream_t)stream;
    // candidates: the sort path without and with the hot-key split (only the
    // forced one if the context fixes sort_split; no split below 2^16
    // packets), then the hash path without and with per-CTA caches (only the
    // forced one if the context fixes cta_cache)
    struct Cand {
        int path, cache, split, tile, digits;
        float ms;
    };
    std::vector<Cand> cand;
    const bool can_split = n >= (1ull << 16);
    std::vector<int> splits, tiles, plans;
    if (c->cfg.sort_split != NS_SPLIT_ON || !can_split) splits.push_back(0);
    if (c->cfg.sort_split != NS_SPLIT_OFF && can_split) splits.push_back(1);
    for (int t = 0; t < kSortTileShapes; ++t)
        if (c->cfg.sort_tile == NS_TILE_AUTO || c->cfg.sort_tile - 1 == t) tiles.push_back(t);
    if (c->cfg.sort_digits != NS_DIGITS_WIDE) plans.push_back(kDigits8);
    if (c->cfg.sort_digits != NS_DIGITS_8) plans.push_back(kDigitsWide);
    for (int sp : splits)
        for (int dg : plans)
            for (int t : tiles) cand.push_back({NS_PATH_SORT, 0, sp, t, dg, 1e30f});
    const size_t n_sort = cand.size();
    if (c->cfg.cta_cache != NS_CACHE_ON) cand.push_back({NS_PATH_HASH, 0, -1, -1, -1, 1e30f});
    if (c->cfg.cta_cache != NS_CACHE_OFF) cand.push_back({NS_PATH_HASH, 1, -1, -1, -1, 1e30f});
    ns_matrix* m = nullptr;
    TRY(ns_matrix_create(c, &m));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ns_status st = NS_OK;
    for (Cand& k : cand) {
        // the first build of each candidate sizes its scratch and tables;
        // the next two are timed
        for (int rep = 0; rep < 3 && st == NS_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = k.path == NS_PATH_SORT ? build_sort(c, d_src, d_dst, n, m, s, k.split, k.tile, k.digits)
                                        : build_hash(c, d_src, d_dst, n, m, s, k.cache);
            cudaEventRecord(e1, s);
            if (st != NS_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = check_launch();
                if (st == NS_OK) st = fail(NS_ERR_CUDA, "ns_path_tune: event wait failed");
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) k.ms = std::min(k.ms, ms);
        }
        if (st != NS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ns_matrix_free(m);
    TRY(st);
    const Cand* best = &cand[0];
    const Cand* best_sort = &cand[0];
    float best_hash = 1e30f, split_ms = -1, plain_ms = -1, d8_ms = -1, wide_ms = -1;
    for (size_t i = 0; i < cand.size(); ++i) {
        const Cand& k = cand[i];
        if (k.ms < best->ms) best = &k;
        if (i < n_sort && k.ms < best_sort->ms) best_sort = &k;
        if (k.path == NS_PATH_HASH) best_hash = std::min(best_hash, k.ms);
        if (k.path == NS_PATH_SORT) {
            float& r = k.split ? split_ms : plain_ms;  // the best tile and plan of each
            if (r < 0 || k.ms < r) r = k.ms;
            float& q = k.digits == kDigitsWide ? wide_ms : d8_ms;  // the best split and tile of each plan
            if (q < 0 || k.ms < q) q = k.ms;
        }
    }
    const int lg = floor_log2(n);
    // the sort path's choices are kept for the size whichever path wins
    c->path_choice[lg] = {best->path, best->cache != 0, best_sort->split, best_sort->tile, best_sort->digits};
    if (chosen) *chosen = best->path;
    if (sort_ms) *sort_ms = best_sort->ms;
    if (hash_ms) *hash_ms = best_hash;
    auto cache = tuner_load(c->tuner_cache);
    char val[384];
    snprintf(val, sizeof val,
             "{\"path\": \"%s\", \"cta_cache\": %d, \"sort_split\": %d, \"sort_tile\": %d, \"sort_digits\": %d, "
             "\"sort_ms\": %.4f, \"hash_ms\": %.4f, \"sort_split_ms\": %.4f, \"sort_plain_ms\": %.4f, "
             "\"sort_digits8_ms\": %.4f, \"sort_wide_ms\": %.4f}",
             best->path == NS_PATH_SORT ? "sort" : "hash", best->cache, best_sort->split, best_sort->tile,
             best_sort->digits, best_sort->ms, best_hash, split_ms, plain_ms, d8_ms, wide_ms);
    cache[path_key(c->device, lg)] = val;
    tuner_store(c->tuner_cache, cache);
    return NS_OK;
}

ns_status ns_sort_split_info(ns_ctx* c, int* used, uint64_t* hot_keys, uint64_t* cold_packets,
                             ns_stream_t stream) {
    if (!c) return fail(NS_ERR_INVALID, "ns_sort_split_info: NULL context");
    DeviceGuard device_guard(c->device);
    if (used) *used = c->last_split ? 1 : 0;
    u64 h = 0, cold = 0;
    if (c->last_split && c->split.p) {
        const cudaError_t e = split_info(c->split.p, &h, &cold, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(NS_ERR_CUDA, "ns_sort_split_info: %s", cudaGetErrorString(e));
        }
    }
    if (hot_keys) *hot_keys = h;
    if (cold_packets) *cold_packets = cold;
    return NS_OK;
}

ns_status ns_column_split_info(ns_ctx* c, int* used, uint64_t* hot_destinations, uint64_t* cold_words,
                               ns_stream_t stream) {
    if (!c) return fail(NS_ERR_INVALID, "ns_column_split_info: NULL context");
    DeviceGuard device_guard(c->device);
    if (used) *used = c->last_colsplit ? 1 : 0;
    u64 h = 0, cold = 0;
    if (c->last_colsplit && c->colsplit.p) {
        const cudaError_t e = col_split_info(c->colsplit.p, &h, &cold, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(NS_ERR_CUDA, "ns_column_split_info: %s", cudaGetErrorString(e));
        }
    }
    if (hot_destinations) *hot_destinations = h;
    if (cold_words) *cold_words = cold;
    return NS_OK;
}

ns_status ns_path_resolve(const ns_ctx* c, uint64_t n, int* path) {
    if (!c || !path) return fail(NS_ERR_INVALID, "ns_path_resolve: NULL argument");
    *path = resolve_path(c, n);
    return NS_OK;
}

ns_status ns_sort_resolve(const ns_ctx* c, uint64_t n, int* split, int* tile, int* digits) {
    if (!c) return fail(NS_ERR_INVALID, "ns_sort_resolve: NULL context");
    int sp = 0, tl = 0, dg = 0;
    resolve_sort(c, n, &sp, &tl, &dg);
    if (split) *split = sp;
    if (tile) *tile = NS_TILE_512X16 + tl;
    if (digits) *digits = dg == kDigitsWide ? NS_DIGITS_WIDE : NS_DIGITS_8;
    return NS_OK;
}

ns_status ns_accumulate(ns_ctx* c, ns_matrix* acc, const ns_matrix* add, ns_stream_t stream) {
    if (!c || !acc || !add) return fail(NS_ERR_INVALID, "ns_accumulate: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    touch(acc, (cudaStream_t)stream);
    touch(add, (cudaStream_t)stream);
    if (acc == add) return fail(NS_ERR_INVALID, "ns_accumulate: acc and add must be distinct");
    if (acc->ctx != c || add->ctx != c) return fail(NS_ERR_INVALID, "ns_accumulate: foreign matrix");
    cudaStream_t s = (cudaStream_t)stream;
    if (add->fmt == FMT_EMPTY || add->bound == 0) {
        if (acc->fmt == FMT_EMPTY) return NS_OK;
    }
    TRY(to_hash(acc, add->bound, s));
    if (add->fmt == FMT_HASH) {
        TraceScope ts(&c->tracer, "k_insert_slots", s);
        launch_insert_slots((const LinkSlot*)add->links.p, add->link_cap, hash_view(acc), c->sms, s,
                            c->cfg.cta_cache != NS_CACHE_OFF);
    } else if (add->fmt == FMT_LIST && add->bound > 0) {
        TraceScope ts(&c->tracer, "k_insert_list", s);
        launch_insert_list((const u64*)add->keys.p, (const u64*)add->counts.p, add->bound,
                           &((const DevStats*)add->stats.p)->v[S_LINKS], hash_view(acc), c->sms, s);
    }
    acc->bound += add->bound;
    return check_launch();
}

ns_status ns_window_ingest(ns_ctx* c, ns_matrix* acc, const uint32_t* d_src, const uint32_t* d_dst,
                           uint64_t n, ns_stream_t stream) {
    if (!c || !acc) return fail(NS_ERR_INVALID, "ns_window_ingest: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    touch(acc, (cudaStream_t)stream);
    if (n > 0 && (!d_src || !d_dst)) return fail(NS_ERR_INVALID, "ns_window_ingest: NULL input with n > 0");
    if (acc->ctx != c) return fail(NS_ERR_INVALID, "ns_window_ingest: foreign matrix");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(to_hash(acc, n, s));
    if (n == 0) return NS_OK;
    TraceScope ts(&c->tracer, "k_insert_packets", s);
    launch_insert_packets(d_src, d_dst, n, hash_view(acc), c->sms, use_cta_cache(c, n), s, true);
    acc->bound += n;
    return check_launch();
}

ns_status ns_window_ingest_stats(ns_ctx* c, ns_matrix* acc, const uint32_t* d_src, const uint32_t* d_dst,
                                 uint64_t n, ns_stats* d_out, ns_stream_t stream) {
    if (!c || !acc || !d_out) return fail(NS_ERR_INVALID, "ns_window_ingest_stats: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    touch(acc, (cudaStream_t)stream);
    if (n > 0 && (!d_src || !d_dst))
        return fail(NS_ERR_INVALID, "ns_window_ingest_stats: NULL input with n > 0");
    if (acc->ctx != c) return fail(NS_ERR_INVALID, "ns_window_ingest_stats: foreign matrix");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(to_hash(acc, n, s));
    {
        TraceScope ts(&c->tracer, "k_insert_packets", s);
        launch_insert_packets_snapshot(d_src, d_dst, n, hash_view(acc), (u64*)d_out, c->sms,
                                       use_cta_cache(c, n), s);
    }
    acc->bound += n;
    return check_launch();
}

ns_status ns_network_stats(ns_ctx* c, const ns_matrix* m, ns_stats* h_out, ns_stream_t stream) {
    if (!c || !m || !h_out) return fail(NS_ERR_INVALID, "ns_network_stats: NULL argument");
    DeviceGuard device_guard(c->device);
    DevStats ds;
    ns_status st = read_stats(m, (cudaStream_t)stream, &ds);
    static_assert(sizeof(ns_stats) == S_NFIELDS * sizeof(uint64_t), "ns_stats layout");
    memcpy(h_out, ds.v, sizeof(ns_stats));
    return st;
}

ns_status ns_network_stats_async(ns_ctx* c, const ns_matrix* m, ns_stats* d_out, ns_stream_t stream) {
    if (!c || !m || !d_out) return fail(NS_ERR_INVALID, "ns_network_stats_async: NULL argument");
    DeviceGuard device_guard(c->device);
    touch(m, (cudaStream_t)stream);
    TraceScope ts(&c->tracer, "k_stats_out", (cudaStream_t)stream);
    launch_stats_out((const DevStats*)m->stats.p, (u64*)d_out, (cudaStream_t)stream);
    return check_launch();
}

}  // extern "C"
