// ns_batch.cu -- batched windows (persistent segmented launches) and the
// autotuner that picks their launch parameters.
//
// A batch is a list of independent windows laid end to end in two uint32
// columns, window w being packets [off[w], off[w+1]).  Each window gets its
// own link/row/column tables, carved from one arena at per-window offsets;
// per-window statistics come out of the same incremental inserts the hash
// path uses.  Windows are grouped into chunks whose tables fit the arena; a
// chunk costs one memset of its tables, one persistent insert launch and, if
// the caller passed an accumulator, one launch adding the chunk's distinct
// links into it.  Nothing here blocks or allocates after ns_batch_create, so
// a run can be captured into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_kernels.h"

using namespace ns;

struct ns_batch {
    ns_ctx* ctx = nullptr;
    int device = 0;  // the context's device (kept here: a batch may be freed after its context)
    uint64_t max_windows = 0, max_packets = 0;
    ns_batch_params params{4096, 8, 0.5, 1};
    Buf meta;                  // win_off, tile_off, tab_off, tab_cap: 4 x (max_windows + 1) u64
    u64* h_meta = nullptr;       // pinned staging of the same
    Buf links, rows, cols;     // the arena
    uint64_t arena_slots = 0;  // slots per table kind
    Buf wstats;                // DevStats x max_windows
    Buf counter;               // tile counters, one per chunk
    Buf dscal;                 // device-planned runs: total tiles, total slots, error flag
    cudaStream_t last_stream = nullptr;  // the stream the batch last ran on
    uint64_t max_chunks = 0;
};

namespace {

u64 pow2_at_least(u64 x) {
    u64 p = 1;
    while (p < x) p <<= 1;
    return p;
}

// table capacity of one window: power of two, load <= max_load, >= 64 slots
u64 window_cap(u64 n, double max_load) {
    const double want = std::ceil((double)n / max_load);
    return pow2_at_least(std::max<u64>((u64)want, 64));
}

struct Chunk {
    u64 w0, w1;      // windows [w0, w1)
    u64 slots;       // arena slots used (per table kind)
    u64 tiles;
    u64 packets;
};

// ---- tuner cache entries of kind "batch": {"T": t, "per_sm": c, "load": l, "cache": k}

std::string tuner_key(int device, u64 windows, u64 packets) {
    const int wb = windows ? (int)std::log2((double)windows) : 0;
    const int mb = (windows && packets) ? (int)std::log2((double)packets / (double)windows) : 0;
    char buf[64];
    snprintf(buf, sizeof buf, "|batch|windows2^%d|mean2^%d", wb, mb);
    return gpu_name(device) + buf;
}

bool params_parse(const std::string& obj, ns_batch_params* p) {
    double t, c, l, k = 1;
    if (!json_number(obj, "T", &t) || !json_number(obj, "per_sm", &c) || !json_number(obj, "load", &l)) return false;
    json_number(obj, "cache", &k);
    *p = ns_batch_params{(uint32_t)t, (uint32_t)c, l, (uint32_t)k};
    return true;
}

std::string params_format(const ns_batch_params& p) {
    char buf[160];
    snprintf(buf, sizeof buf, "{\"T\": %u, \"per_sm\": %u, \"load\": %.3f, \"cache\": %u}", p.tile_packets,
             p.ctas_per_sm, p.max_load, p.cta_cache);
    return buf;
}

bool params_ok(const ns_batch_params& p) {
    return p.tile_packets >= 256 && p.tile_packets <= (1u << 20) && (p.tile_packets % 32) == 0 &&
           p.ctas_per_sm >= 1 && p.ctas_per_sm <= 32 && p.max_load > 0.05 && p.max_load <= 0.9 && p.cta_cache <= 1;
}

ns_status plan(ns_batch* b, const uint64_t* h_off, u64 W, std::vector<Chunk>& chunks) {
    chunks.clear();
    u64* win_off = b->h_meta;
    u64* tile_off = win_off + (b->max_windows + 1);
    u64* tab_off = tile_off + (b->max_windows + 1);
    u64* tab_cap = tab_off + (b->max_windows + 1);
    const u64 T = b->params.tile_packets;
    Chunk cur{0, 0, 0, 0, 0};
    for (u64 w = 0; w < W; ++w) {
        const u64 n = h_off[w + 1] - h_off[w];
        const u64 cap = window_cap(n, b->params.max_load);
        if (cap + 1 > b->arena_slots)
            return fail_fmt(NS_ERR_CAPACITY, "ns_batch_run: window %llu (%llu packets) needs %llu table slots, "
                            "the arena holds %llu", (unsigned long long)w, (unsigned long long)n,
                            (unsigned long long)(cap + 1), (unsigned long long)b->arena_slots);
        if (cur.slots + cap + 1 > b->arena_slots) {
            chunks.push_back(cur);
            cur = Chunk{w, w, 0, 0, 0};
        }
        win_off[w] = h_off[w];
        tile_off[w] = cur.tiles;  // relative to the chunk's first window
        tab_off[w] = cur.slots;
        tab_cap[w] = cap;
        cur.slots += cap + 1;
        cur.tiles += (n + T - 1) / T;
        cur.packets += n;
        cur.w1 = w + 1;
    }
    win_off[W] = W ? h_off[W] : 0;
    if (W) chunks.push_back(cur);
    // tile offsets are relative to each chunk's first window; the kernel's
    // binary search never reads the entry after a chunk's last window (the
    // chunk's tile total is passed separately)
    if (chunks.size() > b->max_chunks) return fail_fmt(NS_ERR_CAPACITY, "ns_batch_run: too many chunks");
    return NS_OK;
}

// ---- device-side planning (ns_batch_run_device) ------------------------------

__device__ __forceinline__ u64 window_cap_dev(u64 n, double max_load) {
    const double want = ceil((double)n / max_load);
    u64 x = (u64)want > 64 ? (u64)want : 64;
    u64 p = 1;
    while (p < x) p <<= 1;
    return p;
}

// One CTA: the same plan as the host's for one chunk, from offsets in device
// memory -- each window's table capacity, its tile and table offsets
// (exclusive scans over the windows), and the totals.  If the offsets do not
// start at 0, decrease, exceed max_packets, or the tables do not fit the
// arena in one chunk, the plan is empty and the error flag is set.
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads) k_batch_plan(const u64* __restrict__ off, u64 W, u32 T, double max_load,
                                                            u64 arena_slots, u64 max_packets, u64* __restrict__ win_off,
                                                            u64* __restrict__ tile_off, u64* __restrict__ tab_off,
                                                            u64* __restrict__ tab_cap, u64* __restrict__ scal) {
    __shared__ u64 wt[kPlanThreads / 32], wsl[kPlanThreads / 32];
    __shared__ u64 carry_t, carry_s;
    __shared__ u32 bad;
    const u32 lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry_t = carry_s = 0;
        bad = off[0] != 0;
    }
    __syncthreads();
    for (u64 base = 0; base < W; base += kPlanThreads) {
        const u64 w = base + threadIdx.x;
        u64 tiles = 0, slots = 0, cap = 0;
        if (w < W) {
            const u64 a = off[w], b = off[w + 1];
            if (b < a) atomicOr(&bad, 1u);
            const u64 n = b >= a ? b - a : 0;
            cap = window_cap_dev(n, max_load);
            tiles = (n + T - 1) / T;
            slots = cap + 1;
        }
        // inclusive scans within the warp, then over the warps
        u64 it = tiles, is = slots;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 yt = __shfl_up_sync(0xFFFFFFFFu, it, o), ys = __shfl_up_sync(0xFFFFFFFFu, is, o);
            if (lane >= (u32)o) {
                it += yt;
                is += ys;
            }
        }
        if (lane == 31) {
            wt[wi] = it;
            wsl[wi] = is;
        }
        __syncthreads();
        u64 bt = carry_t, bs = carry_s;
        for (u32 q = 0; q < wi; ++q) {
            bt += wt[q];
            bs += wsl[q];
        }
        if (w < W) {
            win_off[w] = off[w];
            tile_off[w] = bt + it - tiles;
            tab_off[w] = bs + is - slots;
            tab_cap[w] = cap;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 0; q < kPlanThreads / 32; ++q) {
                carry_t += wt[q];
                carry_s += wsl[q];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const u64 total = off[W];
        win_off[W] = total;
        tile_off[W] = carry_t;
        const bool ok = !bad && total <= max_packets && carry_s <= arena_slots;
        scal[0] = ok ? carry_t : 0;  // total tiles (none when the plan is refused)
        scal[1] = ok ? carry_s : 0;  // arena slots in use
        scal[2] = ok ? 0 : 1;        // error flag
    }
}

// Clears the arena's slots [0, scal[1]) in all three tables.
__global__ void k_arena_clear(LinkSlot* links, NodeSlot* rows, NodeSlot* cols, const u64* __restrict__ scal) {
    const u64 n = scal[1];
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        reinterpret_cast<uint4*>(links)[i] = z;
        reinterpret_cast<uint4*>(rows)[i] = z;
        reinterpret_cast<uint4*>(cols)[i] = z;
    }
}

}  // namespace

extern "C" {

ns_status ns_batch_create(ns_ctx* c, uint64_t max_windows, uint64_t max_packets, ns_batch** out) {
    if (!c || !out) return set_fail(NS_ERR_INVALID, "ns_batch_create: NULL argument");
    DeviceGuard device_guard(c->device);
    AllocScope alloc(c->pool, nullptr);
    if (max_windows == 0) return set_fail(NS_ERR_INVALID, "ns_batch_create: max_windows == 0");
    *out = nullptr;
    ns_batch* b = new ns_batch();
    b->ctx = c;
    b->device = c->device;
    b->max_windows = max_windows;
    b->max_packets = max_packets;
    // tuned parameters for this shape, if the cache has them
    const auto cache = tuner_load(c->tuner_cache);
    const auto it = cache.find(tuner_key(c->device, max_windows, max_packets));
    ns_batch_params cached;
    if (it != cache.end() && params_parse(it->second, &cached) && params_ok(cached)) b->params = cached;
    // arena: enough for every window at the smallest load the tuner tries,
    // capped by the context's HBM budget
    const double min_load = 0.5;
    const u64 need = (u64)std::ceil(2.0 * (double)max_packets / min_load) + 65 * max_windows;
    const u64 budget_slots = c->cfg.hbm_budget_bytes / (sizeof(LinkSlot) + 2 * sizeof(NodeSlot));
    b->arena_slots = std::max<u64>(std::min(need, budget_slots), 1024);
    b->max_chunks = max_windows;
    ns_status st = buf_reserve(b->meta, 4 * (max_windows + 1) * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(b->links, b->arena_slots * sizeof(LinkSlot));
    if (st == NS_OK) st = buf_reserve(b->rows, b->arena_slots * sizeof(NodeSlot));
    if (st == NS_OK) st = buf_reserve(b->cols, b->arena_slots * sizeof(NodeSlot));
    if (st == NS_OK) st = buf_reserve(b->wstats, max_windows * sizeof(DevStats));
    if (st == NS_OK) st = buf_reserve(b->counter, max_windows * sizeof(u32));
    if (st == NS_OK) st = buf_reserve(b->dscal, 4 * sizeof(u64));
    if (st == NS_OK && cudaMemsetAsync(b->dscal.p, 0, 4 * sizeof(u64), nullptr) != cudaSuccess) {
        cudaGetLastError();
        st = set_fail(NS_ERR_CUDA, "ns_batch_create: clearing the device scalars failed");
    }
    if (st == NS_OK && cudaMallocHost((void**)&b->h_meta, 4 * (max_windows + 1) * sizeof(u64)) != cudaSuccess) {
        cudaGetLastError();
        st = set_fail(NS_ERR_OOM, "ns_batch_create: pinned staging allocation failed");
    }
    if (st == NS_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) {
        cudaGetLastError();
        st = set_fail(NS_ERR_CUDA, "ns_batch_create: allocation failed");
    }
    b->last_stream = nullptr;
    if (st != NS_OK) {
        ns_batch_free(b);
        return st;
    }
    *out = b;
    return NS_OK;
}

void ns_batch_free(ns_batch* b) {
    if (!b) return;
    DeviceGuard device_guard(b->device);
    // behind the batch's work on the stream it last ran on; the pinned
    // staging is read by copies on that stream, so it waits for them
    const cudaStream_t s = b->last_stream;
    buf_free_on(b->meta, s);
    buf_free_on(b->links, s);
    buf_free_on(b->rows, s);
    buf_free_on(b->cols, s);
    buf_free_on(b->wstats, s);
    buf_free_on(b->counter, s);
    buf_free_on(b->dscal, s);
    if (b->h_meta) {
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            cudaDeviceSynchronize();
        }
        cudaFreeHost(b->h_meta);
    }
    delete b;
}

ns_status ns_batch_get_params(const ns_batch* b, ns_batch_params* out) {
    if (!b || !out) return set_fail(NS_ERR_INVALID, "ns_batch_get_params: NULL argument");
    *out = b->params;
    return NS_OK;
}

ns_status ns_batch_set_params(ns_batch* b, const ns_batch_params* p) {
    if (!b || !p) return set_fail(NS_ERR_INVALID, "ns_batch_set_params: NULL argument");
    if (!params_ok(*p)) return set_fail(NS_ERR_INVALID, "ns_batch_set_params: parameters out of range");
    if (p->max_load < 0.5 - 1e-9) return set_fail(NS_ERR_INVALID, "ns_batch_set_params: max_load below 0.5");
    b->params = *p;
    return NS_OK;
}

ns_status ns_batch_run(ns_ctx* c, ns_batch* b, const uint32_t* d_src, const uint32_t* d_dst,
                       const uint64_t* h_offsets, uint64_t windows, ns_stats* d_window_stats, ns_matrix* acc,
                       ns_stream_t stream) {
    if (!c || !b || !h_offsets || !d_window_stats) return set_fail(NS_ERR_INVALID, "ns_batch_run: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    b->last_stream = (cudaStream_t)stream;
    touch(acc, (cudaStream_t)stream);
    if (b->ctx != c || (acc && acc->ctx != c)) return set_fail(NS_ERR_INVALID, "ns_batch_run: foreign object");
    if (windows > b->max_windows) return set_fail(NS_ERR_INVALID, "ns_batch_run: more windows than the batch plan");
    if (windows == 0) return NS_OK;
    if (h_offsets[0] != 0) return set_fail(NS_ERR_INVALID, "ns_batch_run: offsets must start at 0");
    for (u64 w = 0; w < windows; ++w)
        if (h_offsets[w + 1] < h_offsets[w]) return set_fail(NS_ERR_INVALID, "ns_batch_run: offsets decrease");
    const u64 total = h_offsets[windows];
    if (total > b->max_packets) return set_fail(NS_ERR_INVALID, "ns_batch_run: more packets than the batch plan");
    if (total > 0 && (!d_src || !d_dst)) return set_fail(NS_ERR_INVALID, "ns_batch_run: NULL input");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Chunk> chunks;
    ns_status st = plan(b, h_offsets, windows, chunks);
    if (st != NS_OK) return st;
    // An empty aggregate over a batch in the sort path's range is the
    // matrix of the batch's packets, which lie back to back in the columns:
    // one sort-path build of them replaces adding every window's table.
    const bool acc_by_sort = acc && acc->bound == 0 && resolve_path(c, total) == NS_PATH_SORT;
    if (acc_by_sort) {
        st = build_sort(c, d_src, d_dst, total, acc, s);
        if (st != NS_OK) return st;
    } else if (acc) {
        st = to_hash(acc, total, s);
        if (st != NS_OK) return st;
    }
    const u64 M1 = b->max_windows + 1;
    u64* dm = (u64*)b->meta.p;
    if (cudaMemcpyAsync(dm, b->h_meta, 4 * M1 * sizeof(u64), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(b->wstats.p, 0, windows * sizeof(DevStats), s) != cudaSuccess ||
        cudaMemsetAsync(b->counter.p, 0, chunks.size() * sizeof(u32), s) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "ns_batch_run: staging copy failed");
    }
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const Chunk& ch = chunks[ci];
        if (cudaMemsetAsync(b->links.p, 0, ch.slots * sizeof(LinkSlot), s) != cudaSuccess ||
            cudaMemsetAsync(b->rows.p, 0, ch.slots * sizeof(NodeSlot), s) != cudaSuccess ||
            cudaMemsetAsync(b->cols.p, 0, ch.slots * sizeof(NodeSlot), s) != cudaSuccess) {
            cudaGetLastError();
            return set_fail(NS_ERR_CUDA, "ns_batch_run: clearing the arena failed");
        }
        BatchDev B;
        B.src = d_src;
        B.dst = d_dst;
        B.win_off = dm + ch.w0;
        B.tile_off = dm + M1 + ch.w0;
        B.tab_off = dm + 2 * M1 + ch.w0;
        B.tab_cap = dm + 3 * M1 + ch.w0;
        B.links = (LinkSlot*)b->links.p;
        B.rows = (NodeSlot*)b->rows.p;
        B.cols = (NodeSlot*)b->cols.p;
        B.wstats = (DevStats*)b->wstats.p + ch.w0;
        B.W = ch.w1 - ch.w0;
        B.T = b->params.tile_packets;
        {
            TraceScope ts(&c->tracer, "k_batch_insert", s);
            launch_batch_insert(B, (u32*)b->counter.p + ci, ch.tiles, c->sms, (int)b->params.ctas_per_sm,
                                b->params.cta_cache != 0, s);
        }
        if (acc && !acc_by_sort) {
            // every window's link slots, side slots included (a side slot's
            // key field is 0, which is the key it holds)
            TraceScope ts(&c->tracer, "k_insert_slots", s);
            launch_insert_slots((const LinkSlot*)b->links.p, ch.slots - 1, hash_view(acc), c->sms, s,
                                b->params.cta_cache != 0);
        }
    }
    {
        TraceScope ts(&c->tracer, "k_batch_stats_out", s);
        launch_batch_stats_out((const DevStats*)b->wstats.p, windows, (u64*)d_window_stats, c->sms, s);
    }
    if (acc && !acc_by_sort) acc->bound += total;  // (the sort-path build set its own)
    return check_launch();
}

ns_status ns_batch_run_device(ns_ctx* c, ns_batch* b, const uint32_t* d_src, const uint32_t* d_dst,
                              const uint64_t* d_offsets, uint64_t windows, ns_stats* d_window_stats, ns_matrix* acc,
                              ns_stream_t stream) {
    if (!c || !b || !d_offsets || !d_window_stats)
        return set_fail(NS_ERR_INVALID, "ns_batch_run_device: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    b->last_stream = (cudaStream_t)stream;
    touch(acc, (cudaStream_t)stream);
    if (b->ctx != c || (acc && acc->ctx != c)) return set_fail(NS_ERR_INVALID, "ns_batch_run_device: foreign object");
    if (windows > b->max_windows)
        return set_fail(NS_ERR_INVALID, "ns_batch_run_device: more windows than the batch plan");
    if (windows == 0) return NS_OK;
    if (b->max_packets > 0 && (!d_src || !d_dst)) return set_fail(NS_ERR_INVALID, "ns_batch_run_device: NULL input");
    cudaStream_t s = (cudaStream_t)stream;
    if (acc) {
        // room for the largest batch the plan allows (the host does not see the offsets)
        const ns_status st = to_hash(acc, b->max_packets, s);
        if (st != NS_OK) return st;
    }
    const u64 M1 = b->max_windows + 1;
    u64* dm = (u64*)b->meta.p;
    u64* scal = (u64*)b->dscal.p;
    if (cudaMemsetAsync(b->wstats.p, 0, windows * sizeof(DevStats), s) != cudaSuccess ||
        cudaMemsetAsync(b->counter.p, 0, sizeof(u32), s) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "ns_batch_run_device: clearing failed");
    }
    {
        TraceScope ts(&c->tracer, "k_batch_plan", s);
        k_batch_plan<<<1, kPlanThreads, 0, s>>>((const u64*)d_offsets, windows, b->params.tile_packets,
                                                b->params.max_load, b->arena_slots, b->max_packets, dm, dm + M1,
                                                dm + 2 * M1, dm + 3 * M1, scal);
    }
    {
        TraceScope ts(&c->tracer, "k_arena_clear", s);
        k_arena_clear<<<c->sms * 8, 256, 0, s>>>((LinkSlot*)b->links.p, (NodeSlot*)b->rows.p, (NodeSlot*)b->cols.p,
                                                 scal);
    }
    BatchDev B;
    B.src = d_src;
    B.dst = d_dst;
    B.win_off = dm;
    B.tile_off = dm + M1;
    B.tab_off = dm + 2 * M1;
    B.tab_cap = dm + 3 * M1;
    B.links = (LinkSlot*)b->links.p;
    B.rows = (NodeSlot*)b->rows.p;
    B.cols = (NodeSlot*)b->cols.p;
    B.wstats = (DevStats*)b->wstats.p;
    B.W = windows;
    B.T = b->params.tile_packets;
    const u64 tile_bound = b->max_packets / B.T + windows + 1;
    {
        TraceScope ts(&c->tracer, "k_batch_insert", s);
        launch_batch_insert(B, (u32*)b->counter.p, tile_bound, c->sms, (int)b->params.ctas_per_sm,
                            b->params.cta_cache != 0, s, scal);
    }
    if (acc) {
        TraceScope ts(&c->tracer, "k_insert_slots", s);
        launch_insert_slots((const LinkSlot*)b->links.p, b->arena_slots - 1, hash_view(acc), c->sms, s,
                            b->params.cta_cache != 0, scal + 1);
    }
    {
        TraceScope ts(&c->tracer, "k_batch_stats_out", s);
        launch_batch_stats_out((const DevStats*)b->wstats.p, windows, (u64*)d_window_stats, c->sms, s);
    }
    if (acc) acc->bound += b->max_packets;
    return check_launch();
}

ns_status ns_batch_sync(ns_batch* b, ns_stream_t stream) {
    if (!b) return set_fail(NS_ERR_INVALID, "ns_batch_sync: NULL batch");
    DeviceGuard device_guard(b->device);
    u64 flag = 0;
    if (cudaMemcpyAsync(&flag, (const u64*)b->dscal.p + 2, sizeof(u64), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "ns_batch_sync: the batch's work failed");
    }
    if (flag)
        return set_fail(NS_ERR_CAPACITY, "ns_batch_run_device: offsets that do not start at 0 or decrease, more "
                                         "packets than the plan, or tables that do not fit the arena at once");
    return NS_OK;
}

ns_status ns_batch_tune(ns_ctx* c, ns_batch* b, const uint32_t* d_src, const uint32_t* d_dst,
                        const uint64_t* h_offsets, uint64_t windows, ns_stats* d_scratch_stats, ns_stream_t stream,
                        ns_batch_params* chosen) {
    if (!c || !b || !d_scratch_stats) return set_fail(NS_ERR_INVALID, "ns_batch_tune: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    b->last_stream = (cudaStream_t)stream;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned Ts[] = {2048, 4096, 16384};
    const unsigned Cs[] = {4, 8, 16};
    const double Ls[] = {0.5, 0.7};
    const unsigned Ks[] = {0, 1};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return set_fail(NS_ERR_CUDA, "ns_batch_tune: event creation failed");
    }
    const ns_batch_params saved = b->params;
    ns_batch_params best = saved;
    float best_ms = 1e30f;
    ns_status st = NS_OK;
    for (unsigned T : Ts)
        for (unsigned C : Cs)
            for (double L : Ls)
                for (unsigned K : Ks) {
                b->params = ns_batch_params{T, C, L, K};
                float ms_min = 1e30f;
                for (int rep = 0; rep < 3 && st == NS_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    st = ns_batch_run(c, b, d_src, d_dst, h_offsets, windows, d_scratch_stats, nullptr, stream);
                    cudaEventRecord(e1, s);
                    if (st != NS_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaGetLastError();
                        st = set_fail(NS_ERR_CUDA, "ns_batch_tune: timing failed");
                        break;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_min = std::min(ms_min, ms);  // first run warms up
                }
                if (st != NS_OK) break;
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best = b->params;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NS_OK) {
        b->params = saved;
        return st;
    }
    b->params = best;
    if (chosen) *chosen = best;
    auto cache = tuner_load(c->tuner_cache);
    cache[tuner_key(c->device, b->max_windows, b->max_packets)] = params_format(best);
    tuner_store(c->tuner_cache, cache);
    return NS_OK;
}

}  // extern "C"
