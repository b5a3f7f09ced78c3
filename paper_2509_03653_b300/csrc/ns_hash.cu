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
#include <algorithm>

#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

constexpr int kInsertThreads = 256;

struct BlockStats {
    u64 sum[4];  // valid, links, srcs, dsts
    u64 mx[5];   // max link, max src pk, max src fo, max dst pk, max dst fi
};

constexpr u64 kNoSlot = ~0ull;

// Home slot of a link key; key 0 lives in the extra slot [cap].
__device__ __forceinline__ u64 link_home(const HashView& M, u64 key) {
    return key == 0 ? M.link_mask + 1 : (mix64(key) & M.link_mask);
}
// Home slot of a node id; id 0xFFFFFFFF lives in the extra slot [cap].
__device__ __forceinline__ u64 node_home(u64 mask, u32 id) {
    return id == 0xFFFFFFFFu ? mask + 1 : (mix32(id) & mask);
}

// 128-bit compare-and-swap (PTX atom.cas.b128, sm_90 and later): one
// atomic claims an empty 16-byte slot and writes both of its words.
struct W128 {
    u64 lo, hi;
};
__device__ __forceinline__ W128 cas128(void* p, u64 cmp_lo, u64 cmp_hi, u64 new_lo, u64 new_hi) {
    W128 r;
    asm volatile(
        "{\n\t.reg .b128 d, c, v;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.cas.relaxed.gpu.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(r.lo), "=l"(r.hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
        : "memory");
    return r;
}

// Result of adding c to the entry of a key: the slot and the entry's value
// before the addition (0 = the entry was created by this call).
struct Upsert {
    u64 slot;
    u64 prev;
};

// Link table: {key, count}.  An empty slot is {0, 0}; a claim writes {key, c}
// in one 128-bit CAS, so a slot never holds a key with count 0.  Key 0 lives
// in the extra slot [cap] and is only ever added to.
__device__ __noinline__ Upsert link_probe(const HashView& M, u64 key, u64 c, u64 i) {
    for (u32 p = 1; p < kMaxProbes; ++p) {
        i = (i + 1) & M.link_mask;
        const W128 o = cas128(&M.links[i], 0ull, 0ull, key, c);
        if (o.lo == 0ull) return {i, 0ull};
        if (o.lo == key) return {i, atomicAdd(&M.links[i].count, c)};
    }
    set_error(M.stats, ERR_CAPACITY);
    return {kNoSlot, 1ull};
}

// Node table: {id + 1 (u32), degree (u32), packets}; claims write
// {id + 1, degree 0, packets c}.  Id 0xFFFFFFFF lives in the extra slot [cap].
__device__ __noinline__ Upsert node_probe(NodeSlot* tbl, u64 mask, u32 id1, u64 c, u64 i, DevStats* st) {
    for (u32 p = 1; p < kMaxProbes; ++p) {
        i = (i + 1) & mask;
        const W128 o = cas128(&tbl[i], 0ull, 0ull, (u64)id1, c);
        if ((u32)o.lo == 0u) return {i, 0ull};
        if ((u32)o.lo == id1) return {i, atomicAdd(&tbl[i].packets, c)};
    }
    set_error(st, ERR_CAPACITY);
    return {kNoSlot, 1ull};
}

__device__ __forceinline__ void smax(u64* p, u64 v) {
    if (v > *reinterpret_cast<volatile u64*>(p)) atomicMax(p, v);
}

// degree increment that refuses to wrap past 2^32 - 1
__device__ __forceinline__ u64 degree_inc(NodeSlot* s, DevStats* st) {
    const u32 old = atomicAdd(&s->degree, 1u);
    if (old == 0xFFFFFFFFu) set_error(st, ERR_CAPACITY);
    return (u64)old + 1;
}

// ---- CTA-level caches for skewed keys --------------------------------------
//
// With skewed traffic (Zipf, RMAT hubs) a few links, sources and destinations
// take most of the updates, and thousands of atomics on one global address
// serialize.  Each CTA keeps small shared-memory tables of links, rows and
// columns (bounded probing; an item that finds no room goes to the global
// tables directly).  Cached counts are added to the global tables once per CTA
// at the flush.  Whether a cached link is new is only known at its flush, so
// the degree increments of its row and column are applied there.
constexpr int kCache = 512;
constexpr int kCacheProbes = 4;

struct CtaCache {
    u64 lkey[kCache];
    u64 lcnt[kCache];
    u32 rid[kCache];   // id + 1, 0 = empty
    u32 rdeg[kCache];
    u64 rpk[kCache];
    u32 cid[kCache];
    u32 cdeg[kCache];
    u64 cpk[kCache];
};

__device__ __forceinline__ void cache_clear(CtaCache& C) {
    for (int i = threadIdx.x; i < kCache; i += blockDim.x) {
        C.lkey[i] = 0;
        C.lcnt[i] = 0;
        C.rid[i] = 0;
        C.rdeg[i] = 0;
        C.rpk[i] = 0;
        C.cid[i] = 0;
        C.cdeg[i] = 0;
        C.cpk[i] = 0;
    }
}

// slot of `key` in the link cache (claimed if absent), or -1 if no room
__device__ __forceinline__ int lcache_slot(CtaCache& C, u64 key) {
    u32 h = (u32)(mix64(key) >> 40) & (kCache - 1);
    for (int p = 0; p < kCacheProbes; ++p) {
        const u64 old = atomicCAS(&C.lkey[h], 0ull, key);
        if (old == 0ull || old == key) return (int)h;
        h = (h + 1) & (kCache - 1);
    }
    return -1;
}

__device__ __forceinline__ int ncache_slot(u32* ids, u32 id) {
    if (id == 0xFFFFFFFFu) return -1;  // the side-slot id is never cached
    u32 h = (u32)(mix32(id) >> 40) & (kCache - 1);
    for (int p = 0; p < kCacheProbes; ++p) {
        const u32 old = atomicCAS(&ids[h], 0u, id + 1);
        if (old == 0u || old == id + 1) return (int)h;
        h = (h + 1) & (kCache - 1);
    }
    return -1;
}

// Global node update with `pk` packets and `deg` new partners at once.
// Returns the values before the update (prev packets, prev degree).
struct NodePrev {
    u64 pk;
    u64 deg;
    bool ok;
};
__device__ __noinline__ NodePrev node_add(NodeSlot* tbl, u64 mask, u32 id, u64 pk, u32 deg, DevStats* st) {
    u64 i = node_home(mask, id);
    if (id != 0xFFFFFFFFu) {
        const u32 id1 = id + 1;
        for (u32 p = 0;; ++p) {
            if (p >= kMaxProbes) {
                set_error(st, ERR_CAPACITY);
                return {0, 0, false};
            }
            const W128 o = cas128(&tbl[i], 0ull, 0ull, (u64)id1 | ((u64)deg << 32), pk);
            if ((u32)o.lo == 0u) return {0, 0, true};
            if ((u32)o.lo == id1) break;
            i = (i + 1) & mask;
        }
    }
    NodePrev r{0, 0, true};
    if (pk) r.pk = atomicAdd(&tbl[i].packets, pk);
    else r.pk = 1;  // unchanged; not a new node
    if (deg) {
        const u32 old = atomicAdd(&tbl[i].degree, deg);
        if ((u64)old + deg > 0xFFFFFFFFull) set_error(st, ERR_CAPACITY);
        r.deg = old;
    }
    return r;
}

// Adds one new partner to a node: in the cache if the node is there (or fits),
// else in the global table.  Returns the node's degree after the increment if
// it was applied globally (0 if cached: the flush reports it).
__device__ __forceinline__ u64 degree_add_cached(u32* cids, u32* cdeg, NodeSlot* tbl, u64 mask, u32 id,
                                                 DevStats* st) {
    const int s = ncache_slot(cids, id);
    if (s >= 0) {
        atomicAdd(&cdeg[s], 1u);
        return 0;
    }
    const NodePrev r = node_add(tbl, mask, id, 0, 1, st);
    return r.ok ? r.deg + 1 : 0;
}

// One item per lane; every lane of the warp must call this.  With `dedup`
// set (raw packets, c == 1), lanes holding equal keys are merged first so a
// hot link costs one atomic per warp instead of one per packet.
//
// Without a cache, two dependent round trips to L2 per item: (1) the three
// 128-bit claims of the link, row and column home slots, issued together --
// a new entry is complete after this, and whether the link is new is known;
// (2) the count additions of entries that already existed and, for a new
// link, the degree increments of its row and column, again issued together.
// With a cache, the parts that find room in it stay in shared memory.
template <bool CACHE, bool SNAP>
__device__ __forceinline__ void insert_item(const HashView& M, bool valid, u64 key, u64 c, bool dedup,
                                            BlockStats& bs, CtaCache* C) {
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
        const u32 sid = (u32)(key >> 32), did = (u32)key;
        const bool lside = (key == 0), rside = (sid == 0xFFFFFFFFu), cside = (did == 0xFFFFFFFFu);
        int lc = -1, rc = -1, cc = -1;
        if constexpr (CACHE) {
            if (!lside) lc = lcache_slot(*C, key);
            rc = ncache_slot(C->rid, sid);
            cc = ncache_slot(C->cid, did);
            if (lc >= 0) atomicAdd(&C->lcnt[lc], cs);
            if (rc >= 0) atomicAdd(&C->rpk[rc], cs);
            if (cc >= 0) atomicAdd(&C->cpk[cc], cs);
        }
        const bool ldir = lc < 0, rdir = rc < 0, cdir = cc < 0;
        const u64 li0 = link_home(M, key);
        const u64 ri0 = node_home(M.row_mask, sid);
        const u64 ci0 = node_home(M.col_mask, did);
        // round trip 1
        W128 lo = {0, 0}, ro = {0, 0}, co = {0, 0};
        if (ldir && !lside) lo = cas128(&M.links[li0], 0ull, 0ull, key, cs);
        if (rdir && !rside) ro = cas128(&M.rows[ri0], 0ull, 0ull, (u64)(sid + 1), cs);
        if (cdir && !cside) co = cas128(&M.cols[ci0], 0ull, 0ull, (u64)(did + 1), cs);
        // classify: 0 = created, 1 = existing entry found, 2 = probe on
        const int lk = lside ? 1 : (lo.lo == 0ull ? 0 : (lo.lo == key ? 1 : 2));
        const int rk = rside ? 1 : ((u32)ro.lo == 0u ? 0 : ((u32)ro.lo == sid + 1 ? 1 : 2));
        const int ck = cside ? 1 : ((u32)co.lo == 0u ? 0 : ((u32)co.lo == did + 1 ? 1 : 2));
        Upsert L = {li0, 0}, R = {ri0, 0}, Cl = {ci0, 0};
        if (ldir && lk == 2) L = link_probe(M, key, cs, li0);
        if (rdir && rk == 2) R = node_probe(M.rows, M.row_mask, sid + 1, cs, ri0, M.stats);
        if (cdir && ck == 2) Cl = node_probe(M.cols, M.col_mask, did + 1, cs, ci0, M.stats);
        // a found link cannot have count 0, so "new" is known now
        newlink = ldir && ((lk == 0) || (lk == 2 && L.slot != kNoSlot && L.prev == 0));
        // round trip 2.  With SNAP, a node found at its home slot by the
        // claim returned its contents: when the link is new, one 128-bit CAS
        // from that snapshot adds the packets and the partner together
        // (falling back to two additions if another update got there first).
        // That pays when inserts go to a large resident matrix whose nodes
        // are rarely updated twice at once; in small per-window tables with
        // hot nodes the CAS mostly fails and costs a third round trip.
        if (ldir && lk == 1) L.prev = atomicAdd(&M.links[li0].count, cs);
        if (ldir && lside) newlink = (L.prev == 0);  // the key-0 slot is only added to
        bool rdone = false, cdone = false;
        if (SNAP && newlink && rdir && rk == 1 && !rside && (u32)(ro.lo >> 32) != 0xFFFFFFFFu) {
            const W128 w = cas128(&M.rows[ri0], ro.lo, ro.hi, ro.lo + (1ull << 32), ro.hi + cs);
            if (w.lo == ro.lo && w.hi == ro.hi) {
                R.prev = ro.hi;
                rdeg = (ro.lo >> 32) + 1;
                rdone = true;
            }
        }
        if (SNAP && newlink && cdir && ck == 1 && !cside && (u32)(co.lo >> 32) != 0xFFFFFFFFu) {
            const W128 w = cas128(&M.cols[ci0], co.lo, co.hi, co.lo + (1ull << 32), co.hi + cs);
            if (w.lo == co.lo && w.hi == co.hi) {
                Cl.prev = co.hi;
                cdeg = (co.lo >> 32) + 1;
                cdone = true;
            }
        }
        if (rdir && rk == 1 && !rdone) R.prev = atomicAdd(&M.rows[ri0].packets, cs);
        if (cdir && ck == 1 && !cdone) Cl.prev = atomicAdd(&M.cols[ci0].packets, cs);
        if (newlink) {
            if (rdir) {
                if (R.slot != kNoSlot && !rdone) rdeg = degree_inc(&M.rows[R.slot], M.stats);
            } else {
                atomicAdd(&C->rdeg[rc], 1u);
            }
            if (cdir) {
                if (Cl.slot != kNoSlot && !cdone) cdeg = degree_inc(&M.cols[Cl.slot], M.stats);
            } else {
                atomicAdd(&C->cdeg[cc], 1u);
            }
        }
        newsrc = rdir && (R.slot != kNoSlot) && R.prev == 0;
        newdst = cdir && (Cl.slot != kNoSlot) && Cl.prev == 0;
        if (ldir) cnt_new = L.prev + cs;
        if (rdir) rpk = R.prev + cs;
        if (cdir) cpk = Cl.prev + cs;
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

// Moves a CTA's cached counts into the global tables; whole CTA, after a
// barrier.  Links first: a link found new adds a partner to its row and
// column, in the cache when they are there.  Then rows and columns.  Leaves
// the cache empty.
__device__ void cache_flush(const HashView& M, CtaCache& C, BlockStats& bs) {
    __syncthreads();
    for (int i = threadIdx.x; i < kCache; i += blockDim.x) {
        const u64 key = C.lkey[i];
        if (key == 0) continue;
        const u64 cnt = C.lcnt[i];
        const u64 h0 = link_home(M, key);
        Upsert L;
        const W128 o = cas128(&M.links[h0], 0ull, 0ull, key, cnt);
        if (o.lo == 0ull) L = {h0, 0};
        else if (o.lo == key) L = {h0, atomicAdd(&M.links[h0].count, cnt)};
        else L = link_probe(M, key, cnt, h0);
        if (L.slot == kNoSlot) continue;
        smax(&bs.mx[0], L.prev + cnt);
        if (L.prev == 0) {
            atomicAdd(&bs.sum[1], 1ull);
            const u64 rd = degree_add_cached(C.rid, C.rdeg, M.rows, M.row_mask, (u32)(key >> 32), M.stats);
            const u64 cd = degree_add_cached(C.cid, C.cdeg, M.cols, M.col_mask, (u32)key, M.stats);
            if (rd) smax(&bs.mx[2], rd);
            if (cd) smax(&bs.mx[4], cd);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCache; i += blockDim.x) {
        if (C.rid[i]) {
            const u64 pk = C.rpk[i];
            const u32 dg = C.rdeg[i];
            const NodePrev r = node_add(M.rows, M.row_mask, C.rid[i] - 1, pk, dg, M.stats);
            if (r.ok) {
                if (pk && r.pk == 0) atomicAdd(&bs.sum[2], 1ull);
                if (pk) smax(&bs.mx[1], r.pk + pk);
                if (dg) smax(&bs.mx[2], r.deg + dg);
            }
        }
        if (C.cid[i]) {
            const u64 pk = C.cpk[i];
            const u32 dg = C.cdeg[i];
            const NodePrev r = node_add(M.cols, M.col_mask, C.cid[i] - 1, pk, dg, M.stats);
            if (r.ok) {
                if (pk && r.pk == 0) atomicAdd(&bs.sum[3], 1ull);
                if (pk) smax(&bs.mx[3], r.pk + pk);
                if (dg) smax(&bs.mx[4], r.deg + dg);
            }
        }
    }
    __syncthreads();
    cache_clear(C);
    __syncthreads();
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

// After every CTA has flushed, the last one to finish copies the nine
// quantities to `out` (the classic last-block pattern: each CTA's atomics are
// fenced before it counts itself done).  The counter lives in the statistics
// record and is reset by the last CTA for the next launch.
__device__ __forceinline__ void last_block_snapshot(DevStats* st, u64* out) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const u64 done = atomicAdd(&st->pad[0], 1ull);
        last = (done == (u64)gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < S_NFIELDS) {
        __threadfence();
        out[threadIdx.x] = atomicAdd(&st->v[threadIdx.x], 0ull);
    }
    if (last && threadIdx.x == 0) st->pad[0] = 0;
}

// Raw packets: two uint32 columns (the paper's src and dst), count 1 each.
// With `out` set, the statistics after this launch are written there.
template <bool CACHE, bool SNAP>
__global__ void __launch_bounds__(kInsertThreads) k_insert_packets(const u32* __restrict__ src,
                                                                   const u32* __restrict__ dst, u64 n,
                                                                   HashView M, u64* __restrict__ out) {
    __shared__ BlockStats bs;
    extern __shared__ __align__(16) unsigned char cache_smem[];  // sized sizeof(CtaCache) when CACHE
    CtaCache* C = CACHE ? reinterpret_cast<CtaCache*>(cache_smem) : nullptr;
    block_stats_init(bs);
    if constexpr (CACHE) cache_clear(*C);
    __syncthreads();
    const u64 stride = (u64)gridDim.x * blockDim.x;
    // warp-uniform trip count so that every lane reaches the warp intrinsics
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    // When launched as a programmatic dependent of the previous window's
    // launch, this grid may start before that one has finished: let the next
    // launch start too, read this window's packets (which do not depend on
    // the previous grid), and only then wait for the previous grid's writes to
    // the tables and statistics.  Without such a launch the wait returns at once.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    u64 b = warp_base;
    u64 key = 0;
    bool valid = false;
    if (b < n) {
        const u64 i = b + lane_id();
        valid = i < n;
        if (valid) key = ((u64)__ldg(src + i) << 32) | (u64)__ldg(dst + i);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (; b < n; b += stride) {
        if (b != warp_base) {
            const u64 i = b + lane_id();
            valid = i < n;
            key = valid ? (((u64)__ldg(src + i) << 32) | (u64)__ldg(dst + i)) : 0ull;
        }
        insert_item<CACHE, SNAP>(M, valid, key, 1, true, bs, C);
    }
    if constexpr (CACHE) cache_flush(M, *C, bs);
    __syncthreads();
    block_stats_flush(bs, M.stats);
    if (out) last_block_snapshot(M.stats, out);
}

// Entries of another hash matrix: its link table slots (count > 0 = occupied;
// slot `cap` holds key 0).  Keys are unique, so no merging is needed.
template <bool CACHE>
__global__ void __launch_bounds__(kInsertThreads) k_insert_slots(const LinkSlot* __restrict__ in,
                                                                 u64 in_cap, HashView M,
                                                                 const u64* __restrict__ total_dev) {
    __shared__ BlockStats bs;
    extern __shared__ __align__(16) unsigned char cache_smem[];  // sized sizeof(CtaCache) when CACHE
    CtaCache* C = CACHE ? reinterpret_cast<CtaCache*>(cache_smem) : nullptr;
    block_stats_init(bs);
    if constexpr (CACHE) cache_clear(*C);
    __syncthreads();
    // slots [0, total): the table's cap + 1, or a count on the device (an
    // arena of tables whose extra slots hold key 0 in their key fields)
    const u64 total = total_dev ? *total_dev : in_cap + 1;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 warp_base = ((u64)blockIdx.x * blockDim.x) + (threadIdx.x & ~31u);
    for (u64 b = warp_base; b < total; b += stride) {
        const u64 i = b + lane_id();
        u64 key = 0, c = 0;
        if (i < total) {
            LinkSlot s = in[i];
            c = s.count;
            key = (i == total - 1) ? 0ull : s.key;
        }
        insert_item<CACHE, false>(M, c > 0, key, c, false, bs, C);
    }
    if constexpr (CACHE) cache_flush(M, *C, bs);
    __syncthreads();
    block_stats_flush(bs, M.stats);
}

// Entries of a sorted-list matrix (keys[i], counts[i]), i < n.
template <bool CACHE>
__global__ void __launch_bounds__(kInsertThreads) k_insert_list(const u64* __restrict__ keys,
                                                                const u64* __restrict__ counts, u64 n_arg,
                                                                const u64* __restrict__ n_dev,
                                                                HashView M) {
    __shared__ BlockStats bs;
    extern __shared__ __align__(16) unsigned char cache_smem[];  // sized sizeof(CtaCache) when CACHE
    CtaCache* C = CACHE ? reinterpret_cast<CtaCache*>(cache_smem) : nullptr;
    block_stats_init(bs);
    if constexpr (CACHE) cache_clear(*C);
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
        insert_item<CACHE, false>(M, c > 0, key, c, false, bs, C);
    }
    if constexpr (CACHE) cache_flush(M, *C, bs);
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

// ---- batched windows ------------------------------------------------------
//
// Many independent windows in one persistent launch: CTAs take tiles of T
// packets from an atomic counter in window-major order (so the tables in use
// at any moment belong to a few windows and stay in L2), find the tile's
// window by binary search over the tile prefix, and insert its packets into
// that window's own tables, carved from one arena at per-window offsets.
// Each tile flushes its block totals into its window's statistics record.
template <bool CACHE>
__global__ void __launch_bounds__(kInsertThreads) k_batch_insert(BatchDev B, u32* tile_counter, u64 total_tiles_arg,
                                                                 const u64* __restrict__ total_dev) {
    const u64 total_tiles = total_dev ? *total_dev : total_tiles_arg;
    __shared__ BlockStats bs;
    __shared__ u64 s_tile, s_w, s_p0, s_p1;
    extern __shared__ __align__(16) unsigned char cache_smem[];  // sized sizeof(CtaCache) when CACHE
    CtaCache* C = CACHE ? reinterpret_cast<CtaCache*>(cache_smem) : nullptr;
    if constexpr (CACHE) cache_clear(*C);
    const u32 lane = lane_id();
    for (;;) {
        if (threadIdx.x == 0) {
            const u64 tile = atomicAdd(tile_counter, 1u);
            s_tile = tile;
            if (tile < total_tiles) {
                // largest w with tile_off[w] <= tile (windows without tiles are skipped)
                u64 lo = 0, hi = B.W;  // invariant: tile_off[lo] <= tile < tile_off[hi]
                while (hi - lo > 1) {
                    const u64 mid = (lo + hi) >> 1;
                    if (B.tile_off[mid] <= tile) lo = mid;
                    else hi = mid;
                }
                const u64 p0 = B.win_off[lo] + (tile - B.tile_off[lo]) * (u64)B.T;
                const u64 pe = B.win_off[lo + 1];
                s_w = lo;
                s_p0 = p0;
                s_p1 = (p0 + B.T < pe) ? p0 + B.T : pe;
            }
        }
        block_stats_init(bs);
        __syncthreads();
        if (s_tile >= total_tiles) break;
        const u64 w = s_w, p0 = s_p0, p1 = s_p1;
        const u64 off = B.tab_off[w], cap = B.tab_cap[w];
        HashView M;
        M.links = B.links + off;
        M.link_mask = cap - 1;
        M.rows = B.rows + off;
        M.row_mask = cap - 1;
        M.cols = B.cols + off;
        M.col_mask = cap - 1;
        M.stats = B.wstats + w;
        for (u64 b = p0 + (threadIdx.x & ~31u); b < p1; b += kInsertThreads) {
            const u64 i = b + lane;
            const bool valid = i < p1;
            u64 key = 0;
            if (valid) key = ((u64)__ldg(B.src + i) << 32) | (u64)__ldg(B.dst + i);
            insert_item<CACHE, false>(M, valid, key, 1, true, bs, C);
        }
        if constexpr (CACHE) cache_flush(M, *C, bs);
        __syncthreads();
        block_stats_flush(bs, M.stats);
        __syncthreads();
    }
}

__global__ void k_batch_stats_out(const DevStats* __restrict__ wstats, u64 W, u64* __restrict__ out) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < W * S_NFIELDS; i += stride) {
        const u64 w = i / S_NFIELDS, f = i % S_NFIELDS;
        out[i] = wstats[w].v[f];
    }
}

// Diagnostic: the random-atomic ceiling for the ingest's access pattern --
// each of `threads` threads adds 1 at one pseudo-random 8-byte word of each of
// three tables (a link, a row and a column update), all three issued
// together.  No hashing, probing or statistics: only the memory traffic.
__global__ void k_diag_rand3(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= threads) return;
    const u64 h = mix64(seed ^ (i * 0x9E3779B97F4A7C15ull));
    atomicAdd(&a[h & mask], 1ull);
    atomicAdd(&b[mix64(h + 1) & mask], 1ull);
    atomicAdd(&c[mix64(h + 2) & mask], 1ull);
}

// Diagnostic: the ingest's own access structure without hashing, probing or
// statistics.  Each thread claims one pseudo-random 16-byte slot in each of
// three tables with a 128-bit CAS from the empty value {0, 0}, the three
// issued together (mode 0).  Mode 1 adds the dependent second round trip:
// an 8-byte add on the row and column slots after the claims return.  Mode
// 2 models claims of stale slots (what a per-slot epoch tag in place of a
// table clear needs): the CAS from {0, 0} finds a stale entry, a second CAS
// from the value it returned claims the slot, then mode 1's second round
// trip.  The results feed a store that practically never happens (it keeps
// them live without contention on one address).
__global__ void k_diag_claims(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed, int mode, u64* sink) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= threads) return;
    const u64 h = mix64(seed ^ (i * 0x9E3779B97F4A7C15ull));
    const u64 ia = h & mask, ib = mix64(h + 1) & mask, ic = mix64(h + 2) & mask;
    const u64 key = h | 1;
    W128 x = cas128(&a[2 * ia], 0ull, 0ull, key, 1ull);
    W128 y = cas128(&b[2 * ib], 0ull, 0ull, key, 1ull);
    W128 z = cas128(&c[2 * ic], 0ull, 0ull, key, 1ull);
    if (mode == 2) {
        x = cas128(&a[2 * ia], x.lo, x.hi, key, 1ull);
        y = cas128(&b[2 * ib], y.lo, y.hi, key, 1ull);
        z = cas128(&c[2 * ic], z.lo, z.hi, key, 1ull);
    }
    u64 r = x.lo + y.lo + z.lo;
    if (mode >= 1) {
        r += atomicAdd(&b[2 * ib + 1], 1ull);
        r += atomicAdd(&c[2 * ic + 1], 1ull);
    }
    if (r == ~0ull) sink[0] = i;
}

int grid_for(u64 n, int threads, int sms, int per_sm) {
    u64 want = (n + threads - 1) / threads;
    u64 cap = (u64)sms * per_sm;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace

void launch_insert_packets(const u32* src, const u32* dst, u64 n, const HashView& M,
                           int sms, bool cache, cudaStream_t s, bool snap) {
    if (n == 0) return;
    const int grid = grid_for(n, kInsertThreads, sms, 8);
    const size_t smem = cache ? sizeof(CtaCache) : 0;
    if (cache && snap) k_insert_packets<true, true><<<grid, kInsertThreads, smem, s>>>(src, dst, n, M, nullptr);
    else if (cache) k_insert_packets<true, false><<<grid, kInsertThreads, smem, s>>>(src, dst, n, M, nullptr);
    else if (snap) k_insert_packets<false, true><<<grid, kInsertThreads, smem, s>>>(src, dst, n, M, nullptr);
    else k_insert_packets<false, false><<<grid, kInsertThreads, smem, s>>>(src, dst, n, M, nullptr);
}

void launch_insert_packets_snapshot(const u32* src, const u32* dst, u64 n, const HashView& M,
                                    u64* out, int sms, bool cache, cudaStream_t s) {
    if (n == 0) {
        launch_stats_out(M.stats, out, s);
        return;
    }
    // programmatic dependent launch: overlaps this launch's start and packet
    // loads with the tail of the previous kernel on the stream
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid_for(n, kInsertThreads, sms, 8));
    cfg.blockDim = dim3(kInsertThreads);
    cfg.dynamicSmemBytes = cache ? sizeof(CtaCache) : 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cache) cudaLaunchKernelEx(&cfg, k_insert_packets<true, true>, src, dst, n, M, out);
    else cudaLaunchKernelEx(&cfg, k_insert_packets<false, true>, src, dst, n, M, out);
}

void launch_insert_slots(const LinkSlot* in, u64 in_cap, const HashView& M, int sms,
                         cudaStream_t s, bool cache, const u64* total_dev) {
    const int grid = grid_for(in_cap + 1, kInsertThreads, sms, 8);
    if (cache) k_insert_slots<true><<<grid, kInsertThreads, sizeof(CtaCache), s>>>(in, in_cap, M, total_dev);
    else k_insert_slots<false><<<grid, kInsertThreads, 0, s>>>(in, in_cap, M, total_dev);
}

void launch_insert_list(const u64* keys, const u64* counts, u64 n_bound,
                        const u64* n_dev, const HashView& M, int sms, cudaStream_t s) {
    if (n_bound == 0) return;
    k_insert_list<true><<<grid_for(n_bound, kInsertThreads, sms, 8), kInsertThreads, sizeof(CtaCache), s>>>(
        (const u64*)keys, (const u64*)counts, n_bound, (const u64*)n_dev, M);
}

void launch_compact_links(const LinkSlot* in, u64 cap, u64* out_keys, u64* out_counts,
                          u64* out_n, u64 out_cap, DevStats* st, int sms, cudaStream_t s) {
    k_compact_links<<<grid_for(cap + 1, 256, sms, 8), 256, 0, s>>>(in, cap, out_keys, out_counts,
                                                                   (u64*)out_n, out_cap, st);
}

void launch_batch_insert(const BatchDev& B, u32* tile_counter, u64 total_tiles, int sms, int per_sm,
                         bool cache, cudaStream_t s, const u64* total_dev) {
    if (total_tiles == 0) return;
    const u64 grid = std::min<u64>(total_tiles, (u64)sms * (u64)per_sm);
    if (cache)
        k_batch_insert<true><<<(unsigned)grid, kInsertThreads, sizeof(CtaCache), s>>>(B, tile_counter, total_tiles,
                                                                                      total_dev);
    else k_batch_insert<false><<<(unsigned)grid, kInsertThreads, 0, s>>>(B, tile_counter, total_tiles, total_dev);
}

void launch_batch_stats_out(const DevStats* wstats, u64 W, u64* out, int sms, cudaStream_t s) {
    if (W == 0) return;
    k_batch_stats_out<<<grid_for(W * S_NFIELDS, 256, sms, 4), 256, 0, s>>>(wstats, W, out);
}

void launch_diag_rand3(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed, cudaStream_t s) {
    k_diag_rand3<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, b, c, mask, threads, seed);
}

void launch_diag_claims(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed, int mode, u64* sink,
                        cudaStream_t s) {
    k_diag_claims<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, b, c, mask, threads, seed, mode, sink);
}

void launch_stats_out(const DevStats* st, u64* out, cudaStream_t s) {
    k_stats_out<<<1, 32, 0, s>>>(st, (u64*)out);
}

}  // namespace ns
