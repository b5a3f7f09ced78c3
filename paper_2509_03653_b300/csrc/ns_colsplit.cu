// ns_colsplit.cu -- the sort path's hot-destination split for the column
// side.
//
// The column quantities (unique destinations, largest destination packet
// count, largest fan-in; the reverses of Table 2 rows 5, 7 and 9) come from
// one word per link, dst << 32 | count, grouped by destination.  Under skewed
// traffic a few destinations hold most of the links (Zipf(1.2) over 2^24
// addresses, 2^26 packets: the 8,000 largest fan-ins cover 57% of the links),
// and sorting their words only to add them up is wasted work.  So:
//
//   1. sample: 64 evenly spaced blocks of the column words (a quarter of
//      them, kCSampleMax at most), destinations only, sorted by destination
//      (four digit passes) and cut into runs: a destination's run length is
//      its sampled fan-in;
//   2. select: the destinations seen at least kCMinSample times, the most
//      frequent first, up to kCHotMax (12,288) of them, go into a cuckoo
//      table (2 buckets x 4 slots of 32-bit destinations); one that finds no
//      slot stays cold, and so does 0xFFFFFFFF (it marks a free slot);
//   3. split: one pass over the words.  A word of a hot destination adds 1
//      to the destination's link count and its count to the destination's
//      packets in the CTA's shared memory; every other word is appended to
//      the cold buffer.  At the end each CTA adds its counts to the global
//      per-slot counts;
//   4. the cold words are sorted by destination and cut into runs, which
//      give the cold destinations' quantities as before;
//   5. the hot destinations' quantities are folded in: each adds one
//      destination, and its packets and links enter the two maxima.
//
// Exact for any hot set: a destination is either hot, and all its words are
// counted in the table, or cold, and all its words are sorted.  Every hot
// destination occurs among the words (the sample is drawn from them).
#include <algorithm>
#include <cstddef>

#include "ns_api_internal.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

constexpr int kCWays = 4;
constexpr int kCBuckets = 4096;
constexpr int kCBucketBits = 12;
static_assert((1 << kCBucketBits) == kCBuckets, "bucket bits");
constexpr int kCSlots = kCBuckets * kCWays;
constexpr int kCHotMax = kCSlots / 4 * 3;  // table load <= 3/4
constexpr u32 kDEmpty = 0xFFFFFFFFu;       // a free slot (never a hot destination)
constexpr int kCSampleBlocks = 64;
constexpr u64 kCSampleMax = 1ull << 22;
constexpr u32 kCBins = 2048;               // sampled fan-ins, the last bin holding >= kCBins - 1
constexpr u32 kCMinSample = 4;
static_assert(kCSampleMax / (kCBins - 1) < (u64)kCHotMax, "the top bin alone never exceeds the hot set");

// Device-side state of one column split (one allocation per context).
struct ColDev {
    u32 table[kCSlots];     // slot -> hot destination (kDEmpty = free); bucket b = slots [4b, 4b + 4)
    u64 links[kCSlots];     // the slot destination's words (its fan-in)
    u64 packets[kCSlots];   // the sum of their counts
    u32 cand[kCHotMax];     // candidates, any order
    u32 hist[kCBins];       // sampled destinations by run length
    u64 m;                  // sample size
    u64 H;                  // candidates collected, then the hot destinations placed
    u64 thresh;             // least sampled fan-in of a hot destination
    u64 cold;               // cold words
    u64 R_sample;           // distinct sampled destinations
};

__device__ __forceinline__ u32 dst_mix(u32 d) {
    const u32 x = d * 0x9E3779B1u;
    return x ^ (x >> 16);
}
__device__ __forceinline__ u32 dst_bucket1(u32 x) { return x >> (32 - kCBucketBits); }
__device__ __forceinline__ u32 dst_bucket2(u32 x, u32 b1) {
    const u32 b = (x * 0x85EBCA6Bu) >> (32 - kCBucketBits);
    return b == b1 ? b ^ 1u : b;
}

// Slot of destination d in a table (shared or global), or -1.  The two
// buckets are read as two 16-byte loads.
__device__ __forceinline__ int dst_find(const u32* table, u32 d) {
    if (d == kDEmpty) return -1;
    const u32 x = dst_mix(d);
    const u32 b1 = dst_bucket1(x), b2 = dst_bucket2(x, b1);
    const uint4 p = reinterpret_cast<const uint4*>(table)[b1];
    const uint4 q = reinterpret_cast<const uint4*>(table)[b2];
    int slot = -1;
    slot = p.x == d ? (int)(4 * b1 + 0) : slot;
    slot = p.y == d ? (int)(4 * b1 + 1) : slot;
    slot = p.z == d ? (int)(4 * b1 + 2) : slot;
    slot = p.w == d ? (int)(4 * b1 + 3) : slot;
    slot = q.x == d ? (int)(4 * b2 + 0) : slot;
    slot = q.y == d ? (int)(4 * b2 + 1) : slot;
    slot = q.z == d ? (int)(4 * b2 + 2) : slot;
    slot = q.w == d ? (int)(4 * b2 + 3) : slot;
    return slot;
}

// 1. The sample: words [b * (R / 64), + blen) of each block b, destination
// only (dst << 32); its size m goes to cd->m for the sort.
__global__ void k_col_sample_gather(const u64* __restrict__ words, const u64* __restrict__ R_ptr, ColDev* cd,
                                    u64* __restrict__ out) {
    const u64 R = *R_ptr;
    const u64 q = (R / 4) / kCSampleBlocks * kCSampleBlocks;
    const u64 m = q < kCSampleMax ? q : kCSampleMax;
    const u64 blen = m / kCSampleBlocks;
    const u64 stride = R / kCSampleBlocks;
    if (blockIdx.x == 0 && threadIdx.x == 0) cd->m = m;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (u64)gridDim.x * blockDim.x) {
        const u64 p = (i / blen) * stride + (i % blen);
        out[i] = words[p] & 0xFFFFFFFF00000000ull;
    }
}

// 2a. Sampled destinations by run length (only lengths >= kCMinSample).
__global__ void __launch_bounds__(1024) k_col_hist(const u64* __restrict__ pos, ColDev* cd) {
    __shared__ u32 h[kCBins];
    for (u32 i = threadIdx.x; i < kCBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const u64 R = cd->R_sample;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (u64)gridDim.x * blockDim.x) {
        const u64 len = pos[r + 1] - pos[r];
        if (len >= kCMinSample) atomicAdd(&h[len < kCBins - 1 ? len : kCBins - 1], 1u);
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < kCBins; i += blockDim.x)
        if (h[i]) atomicAdd(&cd->hist[i], h[i]);
}

// 2b. The least sampled fan-in t >= kCMinSample such that at most kCHotMax
// destinations reach it (none: 2^64 - 1).  One CTA: suffix sums of the bins,
// then the largest bin whose suffix is over the limit.
constexpr int kCPickThreads = 1024;
static_assert(kCBins == 2 * kCPickThreads, "two bins per thread");
__global__ void __launch_bounds__(kCPickThreads) k_col_pick(ColDev* cd) {
    __shared__ u64 S[kCBins + 1];
    __shared__ u32 cut;
    const u32 t = threadIdx.x;
    for (u32 b = t; b < kCBins; b += kCPickThreads) S[b] = cd->hist[b];
    if (t == 0) {
        S[kCBins] = 0;
        cut = 0;
    }
    __syncthreads();
    for (u32 o = 1; o < kCBins; o <<= 1) {
        u64 v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const u32 b = t + q * kCPickThreads;
            v[q] = b + o < kCBins ? S[b + o] : 0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) S[t + q * kCPickThreads] += v[q];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const u32 b = t + q * kCPickThreads;
        if (b >= kCMinSample && S[b] > (u64)kCHotMax) atomicMax(&cut, b + 1);
    }
    __syncthreads();
    if (t == 0) {
        const u32 L = cut ? cut : kCMinSample;
        cd->thresh = (L < kCBins && S[L] > 0) ? (u64)L : ~0ull;
    }
}

// 2c. The candidates, in any order.
__global__ void k_col_collect(const u64* __restrict__ heads, const u64* __restrict__ pos, ColDev* cd) {
    const u64 R = cd->R_sample, t = cd->thresh;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (u64)gridDim.x * blockDim.x) {
        const u32 d = (u32)(heads[r] >> 32);
        if (d == kDEmpty || pos[r + 1] - pos[r] < t) continue;
        const u64 i = atomicAdd(&cd->H, 1ull);
        if (i < (u64)kCHotMax) cd->cand[i] = d;
    }
}

// 2d. One CTA (the table in dynamic shared memory): each candidate takes a
// free slot of its first bucket, else of
// its second (compare-and-swap in shared memory).  A candidate that finds
// both full stays cold; a copy of a destination already placed stops (every
// copy probes the same slots in the same order).  Then the table goes to
// global memory and the counts start at zero.
constexpr int kCTableThreads = 1024;
__global__ void __launch_bounds__(kCTableThreads, 1) k_col_table(ColDev* cd) {
    extern __shared__ __align__(16) u32 table[];  // [kCSlots]
    for (int i = threadIdx.x; i < kCSlots; i += kCTableThreads) table[i] = kDEmpty;
    __syncthreads();
    const u64 H = cd->H < (u64)kCHotMax ? cd->H : (u64)kCHotMax;
    for (u64 i = threadIdx.x; i < H; i += kCTableThreads) {
        const u32 d = cd->cand[i];
        const u32 x = dst_mix(d);
        const u32 b1 = dst_bucket1(x), b2 = dst_bucket2(x, b1);
        bool done = false;
        for (int q = 0; q < 2 * kCWays && !done; ++q) {
            const u32 slot = 4 * (q < kCWays ? b1 : b2) + (q & (kCWays - 1));
            const u32 old = atomicCAS(&table[slot], kDEmpty, d);
            done = old == kDEmpty || old == d;
        }
    }
    __shared__ u32 placed;
    if (threadIdx.x == 0) placed = 0;
    __syncthreads();
    u32 mine = 0;
    for (int i = threadIdx.x; i < kCSlots; i += kCTableThreads) {
        cd->table[i] = table[i];
        cd->links[i] = 0;
        cd->packets[i] = 0;
        mine += table[i] != kDEmpty ? 1u : 0u;
    }
    if (mine) atomicAdd(&placed, mine);
    __syncthreads();
    if (threadIdx.x == 0) cd->H = placed;  // the hot destinations
}

// 3. The split.  One CTA of 1024 threads per SM holds the table and its
// 32-bit counts (192 KB) and runs as eight independent 128-thread groups
// (named barriers), each taking chunks of 1024 words (chunk b * 8 + g, then
// every gridDim.x * 8 chunks).  The column words are only used below 2^32
// packets, so no destination's packets or links reach 2^32 and 32-bit
// counts are exact; every kCDrainChunks of its own chunks a group still
// drains all counts to the global ones (atomic exchange; the other groups
// keep adding), which keeps each count below 2^31 between drains.
constexpr int kCSplitThreads = 1024;
constexpr int kCGroupThreads = 128;
constexpr int kCGroups = kCSplitThreads / kCGroupThreads;
constexpr int kCItems = 8;
constexpr u64 kCChunk = (u64)kCGroupThreads * kCItems;
constexpr u64 kCDrainChunks = (1ull << 31) / (2 * kCGroups * kCChunk);
struct ColSmem {
    u32 table[kCSlots];
    u32 links[kCSlots];
    u32 pk[kCSlots];
    u32 wsum[kCGroups][kCGroupThreads / 32];
    u64 base[kCGroups];
};

__device__ __forceinline__ void col_group_sync(u32 g) {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kCGroupThreads) : "memory");
}

__device__ __forceinline__ void col_drain(ColSmem& sm, ColDev* cd, u32 tg) {
    for (int i = tg; i < kCSlots; i += kCGroupThreads) {
        const u32 l = atomicExch(&sm.links[i], 0u);
        const u32 p = atomicExch(&sm.pk[i], 0u);
        if (l) atomicAdd(reinterpret_cast<unsigned long long*>(&cd->links[i]), (unsigned long long)l);
        if (p) atomicAdd(reinterpret_cast<unsigned long long*>(&cd->packets[i]), (unsigned long long)p);
    }
}

__global__ void __launch_bounds__(kCSplitThreads, 1) k_col_split(const u64* __restrict__ words,
                                                                 const u64* __restrict__ R_ptr, bool vec, ColDev* cd,
                                                                 u64* __restrict__ cold) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColSmem& sm = *reinterpret_cast<ColSmem*>(smem_raw);
    const u32 ALL = 0xFFFFFFFFu;
    const u32 lane = threadIdx.x & 31, t = threadIdx.x;
    const u32 g = t / kCGroupThreads, tg = t % kCGroupThreads, w = tg >> 5;
    for (int i = t; i < kCSlots; i += kCSplitThreads) {
        sm.table[i] = cd->table[i];
        sm.links[i] = 0;
        sm.pk[i] = 0;
    }
    __syncthreads();
    const u64 n = *R_ptr;
    const u32 lt = lanemask_lt();
    const u64 step = (u64)gridDim.x * kCGroups * kCChunk;
    u64 since_drain = 0;  // the same in every thread of the group
    for (u64 base = ((u64)blockIdx.x * kCGroups + g) * kCChunk; base < n; base += step) {
        if (++since_drain == kCDrainChunks) {
            since_drain = 0;
            col_drain(sm, cd, tg);
        }
        const u64 nb = base + step;
        if (vec && tg == 0 && nb + kCChunk <= n) bulk_prefetch_l2(words + nb, (u32)(kCChunk * 8));
        u64 wd[kCItems];
        u32 valid = 0;
        if (vec && n - base >= kCChunk) {
            valid = (1u << kCItems) - 1;
#pragma unroll
            for (int h = 0; h < kCItems / 2; ++h) {
                const u64 i = base + (u64)h * (2 * kCGroupThreads) + 2 * tg;
                const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(words + i));
                wd[2 * h + 0] = a.x;
                wd[2 * h + 1] = a.y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < kCItems; ++u) {
                const u64 i = base + (u64)u * kCGroupThreads + tg;
                wd[u] = i < n ? __ldg(words + i) : 0;
                valid |= (i < n ? 1u : 0u) << u;
            }
        }
        u32 coldm = 0;
#pragma unroll
        for (int u = 0; u < kCItems; ++u) {
            if (!((valid >> u) & 1u)) continue;
            const int slot = dst_find(sm.table, (u32)(wd[u] >> 32));
            if (slot >= 0) {
                atomicAdd(&sm.links[slot], 1u);
                atomicAdd(&sm.pk[slot], (u32)wd[u]);
            } else {
                coldm |= 1u << u;
            }
        }
        u32 bal[kCItems];
        u32 wtot = 0;
#pragma unroll
        for (int u = 0; u < kCItems; ++u) {
            bal[u] = __ballot_sync(ALL, (coldm >> u) & 1u);
            wtot += __popc(bal[u]);
        }
        if (lane == 0) sm.wsum[g][w] = wtot;
        col_group_sync(g);
        if (w == 0) {  // exclusive scan of the warp counts, and the group's reservation
            constexpr u32 kW = kCGroupThreads / 32;
            const u32 v = lane < kW ? sm.wsum[g][lane] : 0u;
            u32 x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(ALL, x, o);
                if (lane >= (u32)o) x += y;
            }
            const u32 run = __shfl_sync(ALL, x, 31);
            if (lane < kW) sm.wsum[g][lane] = x - v;
            if (lane == 0) sm.base[g] = run ? atomicAdd(reinterpret_cast<unsigned long long*>(&cd->cold),
                                                        (unsigned long long)run)
                                            : 0;
        }
        col_group_sync(g);
        u64 off = sm.base[g] + sm.wsum[g][w];
#pragma unroll
        for (int u = 0; u < kCItems; ++u) {
            if ((coldm >> u) & 1u) cold[off + __popc(bal[u] & lt)] = wd[u];
            off += __popc(bal[u]);
        }
        col_group_sync(g);  // wsum and base are rewritten by the group's next chunk
    }
    __syncthreads();
    for (int i = t; i < kCSlots; i += kCSplitThreads) {
        const u32 l = sm.links[i], p = sm.pk[i];
        if (l) atomicAdd(reinterpret_cast<unsigned long long*>(&cd->links[i]), (unsigned long long)l);
        if (p) atomicAdd(reinterpret_cast<unsigned long long*>(&cd->packets[i]), (unsigned long long)p);
    }
}

// 5. The hot destinations' share of the column quantities: each one with a
// word adds a destination, and its packets and links enter the maxima.
__global__ void __launch_bounds__(256) k_col_hot_stats(const ColDev* cd, DevStats* st) {
    __shared__ u64 sh_n, sh_pk, sh_fi;
    if (threadIdx.x == 0) sh_n = sh_pk = sh_fi = 0;
    __syncthreads();
    u64 cnt = 0, pk = 0, fi = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kCSlots; i += gridDim.x * blockDim.x) {
        const u64 l = cd->links[i];
        if (cd->table[i] != kDEmpty && l > 0) {
            ++cnt;
            pk = max(pk, cd->packets[i]);
            fi = max(fi, l);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        pk = max(pk, __shfl_xor_sync(0xFFFFFFFFu, pk, o));
        fi = max(fi, __shfl_xor_sync(0xFFFFFFFFu, fi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(reinterpret_cast<unsigned long long*>(&sh_n), (unsigned long long)cnt);
        if (pk) atomicMax(reinterpret_cast<unsigned long long*>(&sh_pk), (unsigned long long)pk);
        if (fi) atomicMax(reinterpret_cast<unsigned long long*>(&sh_fi), (unsigned long long)fi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sh_n) atomicAdd(&st->v[S_DSTS], sh_n);
        if (sh_pk) atomicMax(&st->v[S_MAX_DST_PK], sh_pk);
        if (sh_fi) atomicMax(&st->v[S_MAX_DST_FI], sh_fi);
    }
}

}  // namespace

u64 col_split_state_bytes() { return sizeof(ColDev); }

// The column side with the hot-destination split; see the top of this file.
// words: R = *nnz column words (dst << 32 | count) of a window of fewer than
// 2^32 packets, 16-byte aligned or not;
// n: an upper bound on R that sizes kb (two buffers of n entries), pos and
// psum (n + 1 entries each); state: col_split_state_bytes() of device
// memory; runs_out: the cold runs' count.  Writes the three column fields of
// st (after the caller's other fields: run statistics set the destination
// count, the hot ones add to it).
void col_split_runs(const u64* words, const u64* nnz, u64 n, u64* kb[2], u64* pos, u64* psum, void* state,
                    u64* runs_out, SortScratch& sc, DevStats* st, int sms, cudaStream_t s) {
    ColDev* cd = (ColDev*)state;
    Tracer* tr = sc.tr;
    cudaMemsetAsync(&cd->hist, 0, sizeof(ColDev) - offsetof(ColDev, hist), s);
    // 1. sample (into kb[1]), sorted by destination, in runs (heads into psum)
    const u64 mb = std::min<u64>(kCSampleMax, n);
    {
        TraceScope ts(tr, "k_col_sample_gather", s);
        k_col_sample_gather<<<sms * 4, 256, 0, s>>>(words, nnz, cd, kb[1]);
    }
    const int r = radix_sort_hi32(kb[1], &cd->m, kb, mb, sc, st, s, "k_onesweep<column sample>");
    launch_runs(RUN_U64, false, kb[r], nullptr, mb, &cd->m, psum, pos, nullptr, &cd->R_sample, sc, st, s);
    // 2. the hot destinations and their table
    {
        TraceScope ts(tr, "k_col_hist", s);
        k_col_hist<<<sms, 1024, 0, s>>>(pos, cd);
    }
    {
        TraceScope ts(tr, "k_col_pick", s);
        k_col_pick<<<1, kCPickThreads, 0, s>>>(cd);
    }
    {
        TraceScope ts(tr, "k_col_collect", s);
        k_col_collect<<<sms * 2, 256, 0, s>>>(psum, pos, cd);
    }
    {
        TraceScope ts(tr, "k_col_table", s);
        const size_t tsmem = sizeof(u32) * kCSlots;
        resident_ctas_of((const void*)k_col_table, kCTableThreads, tsmem);  // sets its shared-memory size
        k_col_table<<<1, kCTableThreads, tsmem, s>>>(cd);
    }
    // 3. the split: hot destinations counted, cold words into kb[1]
    {
        const size_t smem = sizeof(ColSmem);
        const int grid = resident_ctas_of((const void*)k_col_split, kCSplitThreads, smem);
        const u64 chunks = (n + kCGroups * kCChunk - 1) / (kCGroups * kCChunk);
        const bool vec = ((uintptr_t)words & 15) == 0;
        TraceScope ts(tr, "k_col_split", s);
        k_col_split<<<(unsigned)std::max<u64>(1, std::min<u64>(chunks, (u64)grid)), kCSplitThreads, smem, s>>>(
            words, nnz, vec, cd, kb[1]);
    }
    // 4. the cold words by destination, in runs, and their statistics
    const int r2 = radix_sort_hi32(kb[1], &cd->cold, kb, n, sc, st, s);
    launch_runs(RUN_HI_OF_PACKED, true, kb[r2], nullptr, n, &cd->cold, nullptr, pos, psum, runs_out, sc, st, s);
    launch_run_stats(RS_COLS, pos, psum, runs_out, n, nullptr, st, sms, tr, s);
    // 5. the hot destinations folded in
    {
        TraceScope ts(tr, "k_col_hot_stats", s);
        k_col_hot_stats<<<(kCSlots + 255) / 256, 256, 0, s>>>(cd, st);
    }
}

// Hot destinations and cold words of the last column split (blocking read).
cudaError_t col_split_info(const void* state, u64* hot, u64* cold, cudaStream_t s) {
    const ColDev* cd = (const ColDev*)state;
    u64 v[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&v[0], &cd->H, sizeof(u64), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v[1], &cd->cold, sizeof(u64), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (hot) *hot = v[0];
    if (cold) *cold = v[1];
    return e;
}

}  // namespace ns
