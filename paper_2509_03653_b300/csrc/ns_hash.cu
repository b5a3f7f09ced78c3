// ns_hash.cu -- hash-path kernels: build and accumulate the traffic matrix A
// in open-addressing tables in HBM, keeping the per-source and
// per-destination aggregates and the Table 2 scalars up to date as each
// (key, count) item lands.
//
// Per item (key = src << 32 | dst, count c):
//   link  A(i,j) += c        -> new link iff the slot's old count was 0
//   row   A1(i)  += c, |A|_0 1 (i) += [new link]   (Table 2 rows 6, 8)
//   col   1^T A (j) += c, 1^T |A|_0 (j) += [new link]  (the reverse ops)
// All counts only grow, so each maximum in Table 2 (rows 4, 7, 9 and their
// reverses) equals the largest value any atomic add returned plus its
// increment; counts of sources / destinations / links grow by one exactly
// when an add finds the old value 0.  Every quantity therefore stays exact
// however the items are ordered or interleaved.
#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

constexpr int kInsertThreads = 256;

struct BlockStats {
    u64 sum[4];  // valid, links, srcs, dsts
    u64 mx[5];   // max link, max src pk, max src fo, max dst pk, max dst fi
};

__device__ __forceinline__ LinkSlot* find_link(const HashView& M, u64 key) {
    if (key == 0) return &M.links[M.link_mask + 1];
    u64 i = mix64(key) & M.link_mask;
    for (u32 p = 0; p < kMaxProbes; ++p) {
        u64 old = atomicCAS(&M.links[i].key, 0ull, key);
        if (old == 0ull || old == key) return &M.links[i];
        i = (i + 1) & M.link_mask;
    }
    set_error(M.stats, ERR_CAPACITY);
    return nullptr;
}

__device__ __forceinline__ NodeSlot* find_node(NodeSlot* tbl, u64 mask, u32 id, DevStats* st) {
    const u64 id1 = (u64)id + 1;
    u64 i = mix32(id) & mask;
    for (u32 p = 0; p < kMaxProbes; ++p) {
        u64 old = atomicCAS(&tbl[i].id1, 0ull, id1);
        if (old == 0ull || old == id1) return &tbl[i];
        i = (i + 1) & mask;
    }
    set_error(st, ERR_CAPACITY);
    return nullptr;
}

__device__ __forceinline__ void smax(u64* p, u64 v) {
    if (v > *reinterpret_cast<volatile u64*>(p)) atomicMax(p, v);
}

// One item per lane; every lane of the warp must call this.  With `dedup`
// set (raw packets, c == 1), lanes holding equal keys are merged first so a
// hot link costs one atomic per warp instead of one per packet.
__device__ __forceinline__ void insert_item(const HashView& M, bool valid, u64 key, u64 c, bool dedup,
                                            BlockStats& bs) {
    const u32 FULL = 0xFFFFFFFFu;
    const u32 lane = lane_id();
    const u32 vmask = __ballot_sync(FULL, valid);
    if (vmask == 0) return;
    bool lead = valid;
    u64 cs = c;
    if (dedup) {
        u32 peers = __match_any_sync(FULL, key) & vmask;
        if (valid) {
            lead = (lane == (u32)(__ffs(peers) - 1));
            cs = (u64)__popc(peers) * c;
        }
    }
    bool newlink = false, newsrc = false, newdst = false;
    u64 cnt_new = 0, rpk = 0, rdeg = 0, cpk = 0, cdeg = 0;
    if (lead) {
        LinkSlot* s = find_link(M, key);
        if (s) {
            u64 prev = atomicAdd(&s->count, cs);
            newlink = (prev == 0);
            cnt_new = prev + cs;
        }
        NodeSlot* r = find_node(M.rows, M.row_mask, (u32)(key >> 32), M.stats);
        NodeSlot* q = find_node(M.cols, M.col_mask, (u32)key, M.stats);
        if (r) {
            u64 p = atomicAdd(&r->packets, cs);
            newsrc = (p == 0);
            rpk = p + cs;
        }
        if (q) {
            u64 p = atomicAdd(&q->packets, cs);
            newdst = (p == 0);
            cpk = p + cs;
        }
        if (newlink) {
            if (r) rdeg = atomicAdd(&r->degree, 1ull) + 1;
            if (q) cdeg = atomicAdd(&q->degree, 1ull) + 1;
        }
    }
    // warp totals -> block accumulators
    const u32 nl = __popc(__ballot_sync(FULL, newlink));
    const u32 nsrc = __popc(__ballot_sync(FULL, newsrc));
    const u32 ndst = __popc(__ballot_sync(FULL, newdst));
    u64 vs = lead ? cs : 0;
    if (!dedup) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vs += __shfl_xor_sync(FULL, vs, o);
    } else {
        vs = (u64)__popc(vmask) * c;
    }
    if (lane == 0) {
        atomicAdd(&bs.sum[0], vs);
        if (nl) atomicAdd(&bs.sum[1], (u64)nl);
        if (nsrc) atomicAdd(&bs.sum[2], (u64)nsrc);
        if (ndst) atomicAdd(&bs.sum[3], (u64)ndst);
    }
    if (lead) {
        smax(&bs.mx[0], cnt_new);
        smax(&bs.mx[1], rpk);
        smax(&bs.mx[2], rdeg);
        smax(&bs.mx[3], cpk);
        smax(&bs.mx[4], cdeg);
    }
}

__device__ __forceinline__ void block_stats_init(BlockStats& bs) {
    if (threadIdx.x < 4) bs.sum[threadIdx.x] = 0;
    if (threadIdx.x < 5) bs.mx[threadIdx.x] = 0;
}

__device__ __forceinline__ void block_stats_flush(BlockStats& bs, DevStats* st) {
    if (threadIdx.x == 0) {
        if (bs.sum[0]) atomicAdd(&st->v[S_VALID], bs.sum[0]);
        if (bs.sum[1]) atomicAdd(&st->v[S_LINKS], bs.sum[1]);
        if (bs.sum[2]) atomicAdd(&st->v[S_SRCS], bs.sum[2]);
        if (bs.sum[3]) atomicAdd(&st->v[S_DSTS], bs.sum[3]);
        if (bs.mx[0]) atomicMax(&st->v[S_MAX_LINK], bs.mx[0]);
        if (bs.mx[1]) atomicMax(&st->v[S_MAX_SRC_PK], bs.mx[1]);
        if (bs.mx[2]) atomicMax(&st->v[S_MAX_SRC_FO], bs.mx[2]);
        if (bs.mx[3]) atomicMax(&st->v[S_MAX_DST_PK], bs.mx[3]);
        if (bs.mx[4]) atomicMax(&st->v[S_MAX_DST_FI], bs.mx[4]);
    }
}

// Raw packets: two uint32 columns (the paper's src and dst), count 1 each.
__global__ void __launch_bounds__(kInsertThreads) k_insert_packets(const u32* __restrict__ src,
                                                                   const u32* __restrict__ dst, u64 n,
                                                                   HashView M) {
    __shared__ BlockStats bs;
    block_stats_init(bs);
    __syncthreads();
    const u64 stride = (u64)gridDim.x * blockDim.x;
    // warp-uniform trip count so that every lane reaches the warp intrinsics
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    for (u64 b = warp_base; b < n; b += stride) {
        const u64 i = b + lane_id();
        const bool valid = i < n;
        u64 key = 0;
        if (valid) key = ((u64)__ldg(src + i) << 32) | (u64)__ldg(dst + i);
        insert_item(M, valid, key, 1, true, bs);
    }
    __syncthreads();
    block_stats_flush(bs, M.stats);
}

// Entries of another hash matrix: its link table slots (count > 0 = occupied;
// slot `cap` holds key 0).  Keys are unique, so no merging is needed.
__global__ void __launch_bounds__(kInsertThreads) k_insert_slots(const LinkSlot* __restrict__ in,
                                                                 u64 in_cap, HashView M) {
    __shared__ BlockStats bs;
    block_stats_init(bs);
    __syncthreads();
    const u64 total = in_cap + 1;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    for (u64 b = warp_base; b < total; b += stride) {
        const u64 i = b + lane_id();
        u64 key = 0, c = 0;
        if (i < total) {
            LinkSlot s = in[i];
            c = s.count;
            key = (i == in_cap) ? 0ull : s.key;
        }
        insert_item(M, c > 0, key, c, false, bs);
    }
    __syncthreads();
    block_stats_flush(bs, M.stats);
}

// Entries of a sorted-list matrix (keys[i], counts[i]), i < n.
__global__ void __launch_bounds__(kInsertThreads) k_insert_list(const u64* __restrict__ keys,
                                                                const u64* __restrict__ counts, u64 n_arg,
                                                                const u64* __restrict__ n_dev,
                                                                HashView M) {
    __shared__ BlockStats bs;
    block_stats_init(bs);
    __syncthreads();
    const u64 n = n_dev ? *n_dev : n_arg;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    for (u64 b = warp_base; b < n; b += stride) {
        const u64 i = b + lane_id();
        u64 key = 0, c = 0;
        if (i < n) {
            key = keys[i];
            c = counts[i];
        }
        insert_item(M, c > 0, key, c, false, bs);
    }
    __syncthreads();
    block_stats_flush(bs, M.stats);
}

// Occupied link slots -> dense (key, count) list in arbitrary order; the
// caller sorts it.  out_n receives the number written.
__global__ void __launch_bounds__(256) k_compact_links(const LinkSlot* __restrict__ in, u64 cap,
                                                       u64* __restrict__ out_keys,
                                                       u64* __restrict__ out_counts, u64* out_n,
                                                       u64 out_cap, DevStats* st) {
    const u32 FULL = 0xFFFFFFFFu;
    const u64 total = cap + 1;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    for (u64 b = warp_base; b < total; b += stride) {
        const u64 i = b + lane_id();
        LinkSlot s = {0, 0};
        if (i < total) s = in[i];
        const bool occ = s.count > 0;
        const u32 m = __ballot_sync(FULL, occ);
        if (!m) continue;
        u64 base = 0;
        if (lane_id() == 0) base = atomicAdd(out_n, (u64)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (occ) {
            u64 pos = base + __popc(m & lanemask_lt());
            if (pos < out_cap) {
                out_keys[pos] = (i == cap) ? 0ull : s.key;
                out_counts[pos] = s.count;
            } else {
                set_error(st, ERR_CAPACITY);
            }
        }
    }
}

__global__ void k_stats_out(const DevStats* __restrict__ st, u64* __restrict__ out) {
    if (threadIdx.x < S_NFIELDS) out[threadIdx.x] = st->v[threadIdx.x];
}

int grid_for(u64 n, int threads, int sms, int per_sm) {
    u64 want = (n + threads - 1) / threads;
    u64 cap = (u64)sms * per_sm;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace

void launch_insert_packets(const u32* src, const u32* dst, u64 n, const HashView& M,
                           int sms, cudaStream_t s) {
    if (n == 0) return;
    k_insert_packets<<<grid_for(n, kInsertThreads, sms, 8), kInsertThreads, 0, s>>>(src, dst, n, M);
}

void launch_insert_slots(const LinkSlot* in, u64 in_cap, const HashView& M, int sms,
                         cudaStream_t s) {
    k_insert_slots<<<grid_for(in_cap + 1, kInsertThreads, sms, 8), kInsertThreads, 0, s>>>(in, in_cap,
                                                                                            M);
}

void launch_insert_list(const u64* keys, const u64* counts, u64 n_bound,
                        const u64* n_dev, const HashView& M, int sms, cudaStream_t s) {
    if (n_bound == 0) return;
    k_insert_list<<<grid_for(n_bound, kInsertThreads, sms, 8), kInsertThreads, 0, s>>>(
        (const u64*)keys, (const u64*)counts, n_bound, (const u64*)n_dev, M);
}

void launch_compact_links(const LinkSlot* in, u64 cap, u64* out_keys, u64* out_counts,
                          u64* out_n, u64 out_cap, DevStats* st, int sms, cudaStream_t s) {
    k_compact_links<<<grid_for(cap + 1, 256, sms, 8), 256, 0, s>>>(in, cap, out_keys, out_counts,
                                                                   (u64*)out_n, out_cap, st);
}

void launch_stats_out(const DevStats* st, u64* out, cudaStream_t s) {
    k_stats_out<<<1, 32, 0, s>>>(st, (u64*)out);
}

}  // namespace ns
