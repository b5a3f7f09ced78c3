// ns_split.cu -- the sort path's hot-key split.
//
// Under skewed traffic a small set of links carries a large share of the
// packets (Zipf(1.2) over 2^24 addresses per column: the 6144 heaviest of
// ~1.5e8 distinct links carry about half of 2^30 packets, the 60,000
// heaviest about 62%).  Sorting their
// copies is wasted work: every copy travels through all eight digit passes
// only to be counted by the run kernel.  So, before the sort:
//
//   1. sample: 64 evenly spaced blocks of consecutive packets (a quarter of
//      the window, kSampleMax packets at most) are packed into keys, each
//      scrambled by an invertible multiplication, sorted by the upper half of
//      the scrambled word alone (four digit passes) and cut into runs of
//      equal words with the sort path's own kernels.  Only the grouping
//      matters here: two distinct keys interleave only if their scrambled
//      upper halves coincide, which splits their sample counts and at worst
//      keeps them out of the hot set;
//   2. select: the keys seen most often in the sample become the hot set,
//      in two tiers.  Tier 1: the keys seen at least kMinHotSample times,
//      the most frequent first, up to kHotMax of them, go into a cuckoo
//      table of 4 kHotMax / 3 slots that each CTA of the split holds in
//      shared memory.  Tier 2 ("warm"): the next ones, seen at least
//      kMinWarmSample times, up to kWarmMax of them, go into a larger cuckoo
//      table in global memory (small enough to stay in L2).  A key that
//      finds no slot in its tier stays cold.  The keys of both tables,
//      sorted, form the hot list;
//   3. split: one pass over all packets.  A packet whose key is in tier 1
//      adds 1 to its CTA's count of that key; one whose key is in tier 2
//      adds 1 to the key's global count (an L2 atomic); every other ("cold")
//      key is appended to the cold-key buffer (warp-compacted, one global
//      reservation per CTA chunk, in no particular order).  At the end each
//      CTA adds its tier-1 counts to the global per-slot counts;
//   4. the cold keys are sorted (LSD onesweep, the count read on the device)
//      and cut into runs;
//   5. merge: the cold runs and the hot list (disjoint key sets, both
//      ascending) are merged into A's sorted nonzero list; each element's
//      place is its own rank plus the number of keys of the other set below
//      it.  The whole-matrix quantities come out of the same pass.
//
// The result does not depend on which keys are hot: any hot set gives the
// same list, since a key's count is the sum of its hot and cold occurrences
// and a hot key has no cold occurrence.  The sample only decides how much
// work the split saves.  Every hot key occurs in the input (the sample is
// drawn from it), so every hot count is at least 1.  Each hot key holds
// exactly one slot in one of the two tables, however often it appears among
// the candidates, and the hot list is read from the tables' slots, so no key
// is listed twice.
#include <algorithm>
#include <cstddef>

#include "ns_api_internal.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

// The hot table: bucketized cuckoo hashing.  kBuckets buckets of kWays
// key slots; a key lives in one of its two buckets, so a lookup reads two
// 32-byte buckets (four 16-byte loads) and compares eight slots, with no
// data-dependent loop.  Keys that cannot be placed (insertion gives up
// after kMaxKicks evictions) simply stay cold.
#ifndef NS_HOT_BUCKETS
#define NS_HOT_BUCKETS 2048
#endif
constexpr int kWays = 4;
constexpr int kBuckets = NS_HOT_BUCKETS;  // a power of two
constexpr int kBucketBits = kBuckets == 1024 ? 10 : kBuckets == 2048 ? 11 : kBuckets == 4096 ? 12 : 0;
static_assert(kBucketBits && (1 << kBucketBits) == kBuckets, "kBuckets: 1024, 2048 or 4096");
constexpr int kHotSlots = kBuckets * kWays;
constexpr int kHotMax = kHotSlots / 4 * 3;  // hot keys at most: table load <= 3/4
constexpr int kHotPad = kHotSlots;          // candidates plus room for the left-over ones (>= kHotMax)
constexpr int kMaxKicks = 500;
constexpr u64 kEmpty = ~0ull;  // an empty slot (never a hot key)
constexpr int kSampleBlocks = 64;
#ifndef NS_SAMPLE_LOG2
#define NS_SAMPLE_LOG2 23
#endif
constexpr u64 kSampleMax = 1ull << NS_SAMPLE_LOG2;
constexpr u32 kHotBins = 2048;      // sample run lengths, the last bin holding >= kHotBins - 1
constexpr u32 kMinHotSample = 4;    // fewest sample occurrences of a tier-1 key
static_assert(kSampleMax / (kHotBins - 1) < (u64)kHotMax, "the top bin alone never exceeds the hot set");

// Tier 2: kWarmBuckets buckets of kWays slots in global memory, at most
// kWarmMax keys (load <= 5/8, placed without evictions).  Any multiple of
// 256 buckets: a key's bucket is a 32-bit hash scaled to [0, kWarmBuckets)
// (multiply-high), so the count is set by the shared memory the split
// kernel has left for tier 2's fingerprint words, not by a power of two.
#ifndef NS_WARM_BUCKETS
#define NS_WARM_BUCKETS 31232
#endif
constexpr int kWarmBuckets = NS_WARM_BUCKETS;  // 0 turns tier 2 off
static_assert(kWarmBuckets >= 0 && kWarmBuckets % 256 == 0, "kWarmBuckets: a multiple of 256");
constexpr int kWarmSlots = kWarmBuckets * kWays;
constexpr int kWarmMax = kWarmSlots / 8 * 5;
constexpr u32 kMinWarmSample = 2;   // fewest sample occurrences of a tier-2 key
constexpr int kListMax = kHotMax + kWarmMax;
constexpr int kArr = kWarmSlots > 0 ? kWarmSlots : 1;  // array extents of an absent tier 2
constexpr int kWarmArr = kWarmMax > 0 ? kWarmMax : 1;
constexpr int kIndexStride = 8;     // the merge's shared-memory index holds every 8th hot-list key
constexpr int kIndexMax = (kListMax + kIndexStride - 1) / kIndexStride;

// Device-side state of one split (one allocation per context).
struct SplitDev {
    u64 table[kHotSlots];       // tier-1 slot -> key (kEmpty = free); bucket b = slots [4b, 4b + 4)
    u64 slot_count[kHotSlots];  // packets of the slot's key
    u64 hot[kHotMax];           // tier-1 candidates, any order
    u64 table2[kArr];           // tier-2 slot -> key (kEmpty = free)
    u64 count2[kArr];           // packets of the tier-2 slot's key
    u32 fpw2[kWarmBuckets > 0 ? kWarmBuckets : 1];  // tier-2 fingerprints, one word per bucket
    u64 warm[kWarmArr];         // tier-2 candidates, any order
    u64 list[kListMax];         // the hot list: the keys of both tables, ascending after the sort
    u32 hist[kHotBins];         // sample keys by run length
    u64 H1;                     // tier-1 keys (collected, then placed)
    u64 W;                      // tier-2 candidates collected
    u64 W2;                     // tier-2 keys placed
    u64 H;                      // hot-list length (H1 + W2)
    u64 thresh;                 // least sample count of a tier-1 key
    u64 thresh2;                // least sample count of a tier-2 key
    u64 cold;                   // cold packets
    u64 R_sample;               // distinct sample keys
    u64 R_cold;                 // distinct cold keys
};

// A 32-bit mix of the key (32-bit multiplies only), and from it the key's
// two buckets (never the same one) and, in ns_split's filter, its
// fingerprint.  Weak hashing only costs hot keys (a key that finds no slot
// stays cold), never exactness.
__device__ __forceinline__ u32 key_mix(u64 key) {
    const u32 x = (u32)key * 0x9E3779B1u ^ (u32)(key >> 32) * 0x85EBCA77u;
    return x ^ (x >> 16);
}
__device__ __forceinline__ u32 bucket1(u64 key) { return key_mix(key) >> (32 - kBucketBits); }
__device__ __forceinline__ u32 bucket2_of_mix(u32 x, u32 b1) {
    const u32 b = (x * 0xC2B2AE3Du) >> (32 - kBucketBits);
    return b == b1 ? b ^ 1u : b;
}
__device__ __forceinline__ u32 bucket2(u64 key, u32 b1) { return bucket2_of_mix(key_mix(key), b1); }
// The two tier-2 buckets of a key (from the same mix, other multipliers,
// scaled to the bucket count), never the same one.
__device__ __forceinline__ u32 warm_bucket1(u32 x) { return __umulhi(x * 0x85EBCA6Bu, (u32)kWarmBuckets); }
__device__ __forceinline__ u32 warm_bucket2(u32 x, u32 b1) {
    const u32 b = __umulhi(x * 0xCC9E2D51u, (u32)kWarmBuckets);
    return b != b1 ? b : (b + 1 == (u32)kWarmBuckets ? 0u : b + 1);
}

// Slot of `key` in the table, or -1.  kEmpty, the mark of a free slot, is
// never a hot key (it would otherwise match a free slot).
__device__ __forceinline__ int hot_find(const u64* table, u64 key) {
    if (key == kEmpty) return -1;
    const u32 b1 = bucket1(key), b2 = bucket2(key, b1);
    const ulonglong2* t = reinterpret_cast<const ulonglong2*>(table);
    const ulonglong2 a0 = t[2 * b1], a1 = t[2 * b1 + 1], c0 = t[2 * b2], c1 = t[2 * b2 + 1];
    int slot = -1;
    slot = a0.x == key ? (int)(4 * b1 + 0) : slot;
    slot = a0.y == key ? (int)(4 * b1 + 1) : slot;
    slot = a1.x == key ? (int)(4 * b1 + 2) : slot;
    slot = a1.y == key ? (int)(4 * b1 + 3) : slot;
    slot = c0.x == key ? (int)(4 * b2 + 0) : slot;
    slot = c0.y == key ? (int)(4 * b2 + 1) : slot;
    slot = c1.x == key ? (int)(4 * b2 + 2) : slot;
    slot = c1.y == key ? (int)(4 * b2 + 3) : slot;
    return slot;
}

// 8-bit fingerprint of a key (never 0, which marks a free slot); the split
// kernel filters with the fingerprints of the key's two buckets -- one
// 32-bit word each, byte w for slot w -- and reads a full key only where a
// fingerprint matches.
__device__ __forceinline__ u32 fingerprint_of_mix(u32 x) {
    const u32 f = (x * 0x27D4EB2Fu) >> 24;
    return f ? f : 1u;
}
__device__ __forceinline__ u32 fingerprint(u64 key) { return fingerprint_of_mix(key_mix(key)); }

// hot_find with the fingerprint filter (shared-memory tables of the split
// kernel): two 4-byte loads for almost every cold key, plus one 8-byte load
// per fingerprint match.  A byte of a bucket word equal to the fingerprint
// is found with the zero-byte test on (word ^ fingerprint x 4): bit 8w+7 of
// (v - 0x01010101) & ~v & 0x80808080 is set for every zero byte w of v (and
// possibly for a byte above a zero byte, a false candidate the key compare
// rejects).  A false candidate can be a free slot, whose key field holds
// kEmpty, so the key kEmpty (never hot) is refused before any compare.
__device__ __forceinline__ u32 zero_bytes(u32 v) { return (v - 0x01010101u) & ~v & 0x80808080u; }

// x: key_mix(key); f4: its fingerprint in all four bytes.
__device__ __forceinline__ int hot_find_fp(const u32* fpw, const u64* table, u64 key, u32 x, u32 f4) {
    const u32 b1 = x >> (32 - kBucketBits), b2 = bucket2_of_mix(x, b1);
    // bit 8w+7: slot w of b1 may match; bit 8w+6: slot w of b2 may match
    u32 cand = zero_bytes(fpw[b1] ^ f4) | (zero_bytes(fpw[b2] ^ f4) >> 1);
    if (cand == 0 || key == kEmpty) return -1;
    // almost always one candidate: check it without a loop
    u32 bit = __ffs(cand) - 1;
    u32 slot = 4 * ((bit & 1) ? b1 : b2) + (bit >> 3);
    if (table[slot] == key) return (int)slot;
    cand &= cand - 1;
    while (cand) {
        bit = __ffs(cand) - 1;
        cand &= cand - 1;
        slot = 4 * ((bit & 1) ? b1 : b2) + (bit >> 3);
        if (table[slot] == key) return (int)slot;
    }
    return -1;
}

// Slot of `key` in the tier-2 table, or -1: the same fingerprint filter
// over the two tier-2 buckets, read through the read-only path.
__device__ __forceinline__ int warm_find(const u32* __restrict__ fpw, const u64* __restrict__ table, u64 key) {
    if (kWarmBuckets == 0 || key == kEmpty) return -1;
    const u32 x = key_mix(key);
    const u32 b1 = warm_bucket1(x), b2 = warm_bucket2(x, b1);
    const u32 f4 = fingerprint_of_mix(x) * 0x01010101u;
    u32 cand = zero_bytes(__ldg(fpw + b1) ^ f4) | (zero_bytes(__ldg(fpw + b2) ^ f4) >> 1);
    while (cand) {
        const u32 bit = __ffs(cand) - 1;
        cand &= cand - 1;
        const u32 slot = 4 * ((bit & 1) ? b1 : b2) + (bit >> 3);
        if (__ldg(table + slot) == key) return (int)slot;
    }
    return -1;
}

__device__ __forceinline__ u64 pack_key(u32 s, u32 d) { return ((u64)s << 32) | (u64)d; }

// The sample's scramble: multiplication by an odd constant modulo 2^64 (a
// bijection whose upper half depends on every bit of the key), and its
// inverse (the constant's multiplicative inverse modulo 2^64).
constexpr u64 kScramble = 0x9E3779B97F4A7C15ull;
constexpr u64 kUnscramble = 0xF1DE83E19937733Dull;
static_assert(kScramble * kUnscramble == 1ull, "inverse modulo 2^64");

// 1. The sample: packets [b * (n / 64), + blen) of each block b, packed and scrambled.
__global__ void k_sample_gather(const u32* __restrict__ src, const u32* __restrict__ dst, u64 n, u64 blen,
                                u64* __restrict__ out) {
    const u64 m = blen * kSampleBlocks;
    const u64 stride = n / kSampleBlocks;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (u64)gridDim.x * blockDim.x) {
        const u64 p = (i / blen) * stride + (i % blen);
        out[i] = pack_key(__ldg(src + p), __ldg(dst + p)) * kScramble;
    }
}

// 2a. Sample keys by run length (only lengths >= the least of either tier).
constexpr u32 kMinSample = kWarmBuckets > 0 ? kMinWarmSample : kMinHotSample;
__global__ void __launch_bounds__(1024) k_hot_hist(const u64* __restrict__ pos, SplitDev* sd) {
    __shared__ u32 h[kHotBins];
    for (u32 i = threadIdx.x; i < kHotBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const u64 R = sd->R_sample;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (u64)gridDim.x * blockDim.x) {
        const u64 len = pos[r + 1] - pos[r];
        if (len >= kMinSample) atomicAdd(&h[len < kHotBins - 1 ? len : kHotBins - 1], 1u);
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < kHotBins; i += blockDim.x)
        if (h[i]) atomicAdd(&sd->hist[i], h[i]);
}

// 2b. Tier 1: the least sample count t1 >= kMinHotSample such that at most
// kHotMax keys occur t1 or more times.  Tier 2 continues downwards from the
// first count that tier 1 could not take: the least t2 >= kMinWarmSample
// such that at most kWarmMax keys occur at least t2 and fewer than t1
// times.  An empty tier has threshold 2^64 - 1.  One CTA: with S[b] the
// number of sample keys seen b or more times (a suffix sum over the bins),
// tier 1 stops below the largest b with S[b] > kHotMax, tier 2 likewise
// with the counts below tier 1's.
constexpr int kPickThreads = 1024;
static_assert(kHotBins == 2 * kPickThreads, "two bins per thread");
__global__ void __launch_bounds__(kPickThreads) k_hot_pick(SplitDev* sd) {
    __shared__ u64 S[kHotBins + 1];
    __shared__ u32 cut1, cut2;  // 1 + the largest bin over the limit, 0 = none
    const u32 t = threadIdx.x;
    for (u32 b = t; b < kHotBins; b += kPickThreads) S[b] = sd->hist[b];
    if (t == 0) {
        S[kHotBins] = 0;
        cut1 = 0;
        cut2 = 0;
    }
    __syncthreads();
    for (u32 o = 1; o < (u32)kHotBins; o <<= 1) {  // S[b] += S[b + o], Hillis-Steele
        u64 v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const u32 b = t + q * kPickThreads;
            v[q] = b + o < (u32)kHotBins ? S[b + o] : 0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) S[t + q * kPickThreads] += v[q];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const u32 b = t + q * kPickThreads;
        if (b >= kMinHotSample && S[b] > (u64)kHotMax) atomicMax(&cut1, b + 1);
    }
    __syncthreads();
    // tier 1 takes the bins from L up; tier 2 looks at [kMinWarmSample, L)
    const u32 L = cut1 ? cut1 : kMinHotSample;  // cut1 = largest bin over the limit, + 1
    const u64 above = S[L];                        // keys tier 1 takes (L <= kHotBins)
    if (kWarmBuckets > 0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const u32 b = t + q * kPickThreads;
            if (b >= kMinWarmSample && b < L && S[b] - above > (u64)kWarmMax) atomicMax(&cut2, b + 1);
        }
    }
    __syncthreads();
    if (t == 0) {
        sd->thresh = (L < (u32)kHotBins && above > 0) ? (u64)L : kEmpty;
        const u32 L2 = cut2 ? cut2 : kMinWarmSample;
        sd->thresh2 = (kWarmBuckets > 0 && L2 < L && S[L2] - above > 0) ? (u64)L2 : kEmpty;
    }
}

// 2c. The candidates of each tier, in any order.
__global__ void k_hot_collect(const u64* __restrict__ heads, const u64* __restrict__ pos, SplitDev* sd) {
    const u64 R = sd->R_sample, t1 = sd->thresh, t2 = sd->thresh2;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (u64)gridDim.x * blockDim.x) {
        const u64 key = heads[r] * kUnscramble, len = pos[r + 1] - pos[r];
        if (key == kEmpty) continue;
        if (len >= t1) {
            const u64 i = atomicAdd(&sd->H1, 1ull);
            if (i < (u64)kHotMax) sd->hot[i] = key;
        } else if (len >= t2) {
            const u64 i = atomicAdd(&sd->W, 1ull);
            if (i < (u64)kWarmMax) sd->warm[i] = key;
        }
    }
}

// 2d. One CTA: places the tier-1 candidates in the cuckoo table, writes the
// keys that found a slot to the head of the hot list (in slot order; the
// list is sorted once both tiers are placed) and clears the per-slot counts.
// A candidate list may hold a key more than once (a key whose sample
// occurrences were not all adjacent); every copy probes the same slots in
// the same order, so a copy that finds its own key there stops, and each
// key holds one slot at most.
constexpr int kTableThreads = 1024;
__global__ void __launch_bounds__(kTableThreads, 1) k_hot_table(SplitDev* sd) {
    extern __shared__ __align__(16) u64 sh[];
    u64* keys = sh;              // [kHotPad]: the candidates, then the left-over ones at the end
    u64* table = sh + kHotPad;   // [kHotSlots]
    const u64 H = sd->H1 < (u64)kHotMax ? sd->H1 : (u64)kHotMax;
    for (int i = threadIdx.x; i < kHotPad; i += kTableThreads) keys[i] = (u64)i < H ? sd->hot[i] : kEmpty;
    for (int i = threadIdx.x; i < kHotSlots; i += kTableThreads) table[i] = kEmpty;
    // first, in parallel: every key takes a free slot of its first bucket,
    // else of its second (compare-and-swap on the slot); the few that find
    // both buckets full are left to the evicting insertion below
    __shared__ u32 n_left;
    if (threadIdx.x == 0) n_left = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < (int)H; i += kTableThreads) {
        const u64 key = keys[i];
        const u32 b1 = bucket1(key), b2 = bucket2(key, b1);
        bool done = false;  // placed, or found placed by another copy
        for (int q = 0; q < 2 * kWays && !done; ++q) {
            const u32 slot = 4 * (q < kWays ? b1 : b2) + (q & (kWays - 1));
            const u64 old = atomicCAS(reinterpret_cast<unsigned long long*>(&table[slot]), kEmpty, key);
            done = old == kEmpty || old == key;
        }
        if (!done) {
            // the left-over keys go after the candidates (index >= H); one
            // that finds no room there stays cold
            const u32 j = atomicAdd(&n_left, 1u);
            if ((u64)j < (u64)kHotPad - H) keys[kHotPad - 1 - j] = key;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const u32 left = (u64)n_left < (u64)kHotPad - H ? n_left : (u32)((u64)kHotPad - H);
        for (u32 i = 0; i < left; ++i) {
            u64 cur = keys[kHotPad - 1 - i];
            if (hot_find(table, cur) >= 0) continue;  // another copy is already in
            for (int kick = 0; kick < kMaxKicks && cur != kEmpty; ++kick) {
                const u32 b1 = bucket1(cur), b2 = bucket2(cur, b1);
                int free_slot = -1;
                for (int w = kWays - 1; w >= 0; --w) {
                    if (table[4 * b2 + w] == kEmpty) free_slot = (int)(4 * b2 + w);
                }
                for (int w = kWays - 1; w >= 0; --w) {
                    if (table[4 * b1 + w] == kEmpty) free_slot = (int)(4 * b1 + w);
                }
                if (free_slot >= 0) {
                    table[free_slot] = cur;
                    cur = kEmpty;
                } else {  // evict a resident of one of the two buckets
                    const u32 victim = 4 * ((kick & 1) ? b2 : b1) + (u32)((kick * 5 + (int)i) & (kWays - 1));
                    // (cur is never kEmpty here)
                    const u64 out = table[victim];
                    table[victim] = cur;
                    cur = out;
                }
            }
            // a key still in hand after kMaxKicks stays cold
        }
    }
    __syncthreads();
    // the hot list's head: the table's keys, in slot order (a block-wide
    // ordered compaction, kTableThreads slots per round)
    __shared__ u32 wcount[kTableThreads / 32];
    __shared__ u32 kept;
    if (threadIdx.x == 0) kept = 0;
    __syncthreads();
    for (int r = 0; r < kHotSlots; r += kTableThreads) {
        const int i = r + threadIdx.x;
        const bool keep = table[i] != kEmpty;
        const u32 bal = __ballot_sync(0xFFFFFFFFu, keep);
        if ((threadIdx.x & 31) == 0) wcount[threadIdx.x >> 5] = __popc(bal);
        __syncthreads();
        u32 before = kept;
        for (u32 w = 0; w < (threadIdx.x >> 5); ++w) before += wcount[w];
        if (keep) sd->list[before + __popc(bal & lanemask_lt())] = table[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 t = 0;
            for (int w = 0; w < kTableThreads / 32; ++w) t += wcount[w];
            kept += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sd->H1 = kept;
        sd->H = kept;
    }
    for (int i = threadIdx.x; i < kHotSlots; i += kTableThreads) {
        sd->table[i] = table[i];
        sd->slot_count[i] = 0;
    }
}

// 2e. Tier 2, many CTAs: each candidate takes a free slot of its first
// tier-2 bucket, else of its second (compare-and-swap), and is appended to
// the hot list after the tier-1 keys; one that finds both buckets full
// stays cold.  A key already in tier 1, or a copy that finds its own key
// placed (every copy probes the same slots in the same order), is skipped.
// The table starts all free and the counts zero.
__global__ void k_warm_insert(SplitDev* sd) {
    const u64 W = sd->W < (u64)kWarmMax ? sd->W : (u64)kWarmMax, H1 = sd->H1;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < W; i += (u64)gridDim.x * blockDim.x) {
        const u64 key = sd->warm[i];
        if (hot_find(sd->table, key) >= 0) continue;
        const u32 x = key_mix(key);
        const u32 b1 = warm_bucket1(x), b2 = warm_bucket2(x, b1);
        bool placed = false, done = false;
        for (int q = 0; q < 2 * kWays && !done; ++q) {
            const u32 slot = 4 * (q < kWays ? b1 : b2) + (q & (kWays - 1));
            const u64 old = atomicCAS(reinterpret_cast<unsigned long long*>(&sd->table2[slot]), kEmpty, key);
            placed = old == kEmpty;
            done = placed || old == key;
        }
        if (placed) sd->list[H1 + atomicAdd(&sd->W2, 1ull)] = key;
    }
}

// 2f. The tier-2 fingerprint words, and the hot list's length.
__global__ void k_warm_fp(SplitDev* sd) {
    const u32 b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < (u32)kWarmBuckets) {
        u32 w = 0;
        for (int q = 0; q < kWays; ++q) {
            const u64 k = sd->table2[kWays * b + q];
            w |= (k == kEmpty ? 0u : fingerprint(k)) << (8 * q);
        }
        sd->fpw2[b] = w;
    }
    if (b == 0) sd->H = sd->H1 + sd->W2;
}

// 3. The split.  Each CTA holds the tables once and runs as kGroups
// independent groups of kGroupThreads threads (named barriers): group g of
// CTA b takes chunks of kGroupThreads * 8 packets (chunk b * kGroups + g,
// then every gridDim.x * kGroups chunks), so that while one group waits on
// its barrier or its tier-2 loads the other keeps the SM busy.  With
// 16-byte-aligned columns a thread loads its eight packets as two 16-byte
// vectors per column.
// Counts are 32-bit in shared memory (64-bit shared atomics are not native
// and serialize badly on the hottest keys).  Every kDrainChunks of its own
// chunks a group drains all counts into the global per-slot counts (atomic
// exchange, so the other group's additions are never lost); between two
// drains no count can reach 2^31.
#ifndef NS_SPLIT_THREADS
#define NS_SPLIT_THREADS (NS_WARM_BUCKETS > 0 ? 1024 : 512)
#endif
constexpr int kSplitThreads = NS_SPLIT_THREADS;
#ifndef NS_SPLIT_GROUP
#define NS_SPLIT_GROUP 128
#endif
constexpr int kGroupThreads = NS_SPLIT_GROUP;  // 128 (eight groups) measured fastest at 2^30 packets
constexpr int kGroups = kSplitThreads / kGroupThreads;
static_assert(kGroups >= 1 && kGroups <= 15 && kGroups * kGroupThreads == kSplitThreads && kGroupThreads % 32 == 0,
              "whole warps per group; named barriers 1..15");
constexpr int kSplitItems = 8;
constexpr u64 kGroupChunk = (u64)kGroupThreads * kSplitItems;
constexpr u64 kDrainChunks = (1ull << 31) / (2 * kGroups * kGroupChunk);
struct SplitSmem {
    u64 table[kHotSlots];
    u32 count[kHotSlots];
    u32 fpw[kBuckets];  // per bucket: the fingerprints of its kWays slots
    u32 fpw2[kWarmBuckets > 0 ? kWarmBuckets : 1];  // the same for tier 2 (its keys stay in global memory)
    u32 wsum[kGroups][kGroupThreads / 32];
    u64 base[kGroups];
};

__device__ __forceinline__ void group_sync(u32 g) {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kGroupThreads) : "memory");
}

// All counts into the global ones: by one group while the other may still
// be adding (drain), or by the whole CTA at the end (flush).
__device__ __forceinline__ void split_drain(SplitSmem& sm, SplitDev* sd, u32 tg) {
    for (int i = tg; i < kHotSlots; i += kGroupThreads) {
        const u32 c = atomicExch(&sm.count[i], 0u);
        if (c) atomicAdd(reinterpret_cast<unsigned long long*>(&sd->slot_count[i]), (unsigned long long)c);
    }
}
__device__ __forceinline__ void split_flush(SplitSmem& sm, SplitDev* sd) {
    for (int i = threadIdx.x; i < kHotSlots; i += kSplitThreads) {
        const u32 c = sm.count[i];
        if (c) atomicAdd(reinterpret_cast<unsigned long long*>(&sd->slot_count[i]), (unsigned long long)c);
    }
}

__global__ void __launch_bounds__(kSplitThreads, 1024 / kSplitThreads) k_hot_split(const u32* __restrict__ src, const u32* __restrict__ dst,
                                                                 u64 n, bool vec, SplitDev* sd, u64* __restrict__ cold) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitSmem& sm = *reinterpret_cast<SplitSmem*>(smem_raw);
    const u32 lane = threadIdx.x & 31, t = threadIdx.x;
    const u32 g = t / kGroupThreads, tg = t % kGroupThreads, w = tg >> 5;  // group, thread and warp in it
    const u32 FULL = 0xFFFFFFFFu;
    for (int i = t; i < kHotSlots; i += kSplitThreads) {
        sm.table[i] = sd->table[i];
        sm.count[i] = 0;
    }
    for (int b = t; b < kBuckets; b += kSplitThreads) {
        u32 fw = 0;
        for (int q = 0; q < kWays; ++q) {
            const u64 k = sd->table[kWays * b + q];
            fw |= (k == kEmpty ? 0u : fingerprint(k)) << (8 * q);
        }
        sm.fpw[b] = fw;
    }
    for (int b = t; b < kWarmBuckets; b += kSplitThreads) sm.fpw2[b] = sd->fpw2[b];
    __syncthreads();
    const u32 lt = lanemask_lt();
    const u64* __restrict__ table2 = sd->table2;
    u64* count2 = sd->count2;
    const u64 step = (u64)gridDim.x * kGroups * kGroupChunk;
    u64 since_drain = 0;  // the same in every thread of the group
    for (u64 base = ((u64)blockIdx.x * kGroups + g) * kGroupChunk; base < n; base += step) {
        if (++since_drain == kDrainChunks) {
            since_drain = 0;
            split_drain(sm, sd, tg);
        }
        // this group's next chunk starts moving into L2 now
        const u64 nb = base + step;
        if (vec && tg == 0 && nb + kGroupChunk <= n) {
            bulk_prefetch_l2(src + nb, (u32)(kGroupChunk * 4));
            bulk_prefetch_l2(dst + nb, (u32)(kGroupChunk * 4));
        }
        u64 key[kSplitItems];
        u32 valid = 0;
        if (vec && n - base >= kGroupChunk) {
            valid = (1u << kSplitItems) - 1;
#pragma unroll
            for (int h = 0; h < kSplitItems / 4; ++h) {
                const u64 i = base + (u64)h * (4 * kGroupThreads) + 4 * tg;
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(src + i));
                const uint4 b = __ldg(reinterpret_cast<const uint4*>(dst + i));
                key[4 * h + 0] = pack_key(a.x, b.x);
                key[4 * h + 1] = pack_key(a.y, b.y);
                key[4 * h + 2] = pack_key(a.z, b.z);
                key[4 * h + 3] = pack_key(a.w, b.w);
            }
        } else {
#pragma unroll
            for (int u = 0; u < kSplitItems; ++u) {
                const u64 i = base + (u64)u * kGroupThreads + tg;
                key[u] = i < n ? pack_key(__ldg(src + i), __ldg(dst + i)) : 0;
                valid |= (i < n ? 1u : 0u) << u;
            }
        }
        // tier 1: counted in shared memory; the others are marked cold.  A
        // key missing tier 1 takes its tier-2 candidate slot from the same
        // mix and fingerprint (fingerprint words in shared memory)
        u32 coldm = 0;
        u32 cand[kSplitItems], sl[kSplitItems];
#pragma unroll
        for (int u = 0; u < kSplitItems; ++u) {
            cand[u] = 0;
            sl[u] = 0;
            if ((valid >> u) & 1u) {
                const u32 x = key_mix(key[u]);
                const u32 f4 = fingerprint_of_mix(x) * 0x01010101u;
                const int slot = hot_find_fp(sm.fpw, sm.table, key[u], x, f4);
                if (slot >= 0) {
                    atomicAdd(&sm.count[slot], 1u);
                } else {
                    coldm |= 1u << u;
                    if (kWarmBuckets > 0 && key[u] != kEmpty) {
                        const u32 b1 = warm_bucket1(x), b2 = warm_bucket2(x, b1);
                        cand[u] = zero_bytes(sm.fpw2[b1] ^ f4) | (zero_bytes(sm.fpw2[b2] ^ f4) >> 1);
                        const u32 bit = __ffs(cand[u]) - 1;
                        sl[u] = 4 * ((bit & 1) ? b1 : b2) + (bit >> 3);
                    }
                }
            }
        }
        if (kWarmBuckets > 0 && coldm) {
            // tier 2: all candidates' keys are loaded (L2) before any
            // compare; a key whose first candidate is not it checks its
            // others one by one (rare)
            u64 k2[kSplitItems];
#pragma unroll
            for (int u = 0; u < kSplitItems; ++u) k2[u] = cand[u] ? __ldg(table2 + sl[u]) : 0;
#pragma unroll
            for (int u = 0; u < kSplitItems; ++u) {
                if (!cand[u]) continue;
                int slot = k2[u] == key[u] ? (int)sl[u] : -1;
                u32 c = cand[u] & (cand[u] - 1);
                if (slot < 0 && c) {
                    const u32 x = key_mix(key[u]);
                    const u32 b1 = warm_bucket1(x), b2 = warm_bucket2(x, b1);
                    while (c && slot < 0) {
                        const u32 bit = __ffs(c) - 1;
                        c &= c - 1;
                        const u32 q = 4 * ((bit & 1) ? b1 : b2) + (bit >> 3);
                        if (__ldg(table2 + q) == key[u]) slot = (int)q;
                    }
                }
                if (slot >= 0) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(count2 + slot), 1ull);
                    coldm &= ~(1u << u);
                }
            }
        }
        u32 bal[kSplitItems];
        u32 wtot = 0;
#pragma unroll
        for (int u = 0; u < kSplitItems; ++u) {
            bal[u] = __ballot_sync(FULL, (coldm >> u) & 1u);
            wtot += __popc(bal[u]);
        }
        if (lane == 0) sm.wsum[g][w] = wtot;
        group_sync(g);
        if (w == 0) {  // exclusive scan of the warp counts (one warp), and the group's reservation
            constexpr u32 kW = kGroupThreads / 32;
            const u32 v = lane < kW ? sm.wsum[g][lane] : 0u;
            u32 x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(FULL, x, o);
                if (lane >= (u32)o) x += y;
            }
            const u32 run = __shfl_sync(FULL, x, 31);
            if (lane < kW) sm.wsum[g][lane] = x - v;
            if (lane == 0) sm.base[g] = run ? atomicAdd(&sd->cold, (u64)run) : 0;
        }
        group_sync(g);
        u64 off = sm.base[g] + sm.wsum[g][w];
#pragma unroll
        for (int u = 0; u < kSplitItems; ++u) {
            if ((coldm >> u) & 1u) cold[off + __popc(bal[u] & lt)] = key[u];
            off += __popc(bal[u]);
        }
        group_sync(g);  // wsum and base are rewritten by the group's next chunk
    }
    __syncthreads();
    split_flush(sm, sd);
}

// 5. Merge of the cold runs (heads[r], length pos[r+1] - pos[r]) with the
// hot list into keys/counts, and the whole-matrix quantities: unique links,
// valid packets and the largest count.
constexpr int kMergeThreads = 512;
__device__ __forceinline__ u64 count_below(const u64* a, u64 len, u64 key) {
    u64 lo = 0, hi = len;  // first index with a[i] >= key
    while (lo < hi) {
        const u64 mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Hot-list keys below `key`.  idx (shared memory) holds list[0], list[S],
// list[2S], ... (S = kIndexStride); if p index keys are below `key`, then
// list[0 .. (p-1)S] all are and list[pS] is not, which leaves the S - 1 keys
// between to compare (one or two cache lines of the list).
__device__ __forceinline__ u64 hot_rank(const u64* idx, u64 NI, const u64* __restrict__ list, u64 H, u64 key) {
    const u64 p = count_below(idx, NI, key);
    if (p == 0) return 0;
    const u64 b = (p - 1) * kIndexStride;
    u64 r = b + 1;
#pragma unroll
    for (int q = 1; q < kIndexStride; ++q) r += (b + q < H && __ldg(list + b + q) < key) ? 1 : 0;
    return r;
}

// Each warp takes kMergeRounds x 32 consecutive elements at a time and
// issues all their loads before any search, so that HBM latency is paid
// once per group rather than once per element.  The hot keys below a cold
// key of the group are those below the group's first key (lo) plus those
// below it among the hot keys that fall between the group's first and last
// keys (span of them: almost always none).
constexpr int kMergeRounds = 4;
// cap: the output's capacity (the window's packets); places at or past it
// are never written (they cannot occur unless a look-back gave up).
__global__ void __launch_bounds__(kMergeThreads) k_hot_merge(const u64* __restrict__ heads, const u64* __restrict__ pos,
                                                             const SplitDev* sd, u64* __restrict__ keys_out,
                                                             u64* __restrict__ counts_out, u64 cap, DevStats* st) {
    extern __shared__ __align__(16) u64 idx[];  // [kIndexMax]
    __shared__ u64 bmax;
    const u32 FULL = 0xFFFFFFFFu, lane = threadIdx.x & 31;
    const u64 H = sd->H, RC = sd->R_cold, total = RC + H;
    const u64 NI = (H + kIndexStride - 1) / kIndexStride;
    const u64* __restrict__ list = sd->list;
    for (u64 i = threadIdx.x; i < NI; i += kMergeThreads) idx[i] = list[i * kIndexStride];
    if (threadIdx.x == 0) bmax = 0;
    __syncthreads();
    u64 mx = 0, hot_sum = 0;
    const u64 group = 32ull * kMergeRounds;
    const u64 warp0 = (((u64)blockIdx.x * kMergeThreads + threadIdx.x) >> 5) * group;
    const u64 wstride = ((u64)gridDim.x * kMergeThreads >> 5) * group;
    for (u64 base = warp0; base < total; base += wstride) {
        u64 key[kMergeRounds], c[kMergeRounds], below[kMergeRounds];
#pragma unroll
        for (int r = 0; r < kMergeRounds; ++r) {
            const u64 i = base + (u64)r * 32 + lane;
            key[r] = 0;
            c[r] = 0;
            if (i < RC) {
                key[r] = heads[i];
                c[r] = pos[i + 1] - pos[i];
            }
        }
        u64 lo = 0, hi = 0;
        if (base < RC) {  // warp-uniform
            const u64 last = min(base + group, RC) - 1;
            u64 v = 0;
            if (lane < 2) v = hot_rank(idx, NI, list, H, heads[lane == 0 ? base : last]);
            lo = __shfl_sync(FULL, v, 0);
            hi = __shfl_sync(FULL, v, 1);
        }
        // hi >= lo for ascending inputs; clamped so that a list left out of
        // order (a look-back that gave up, recorded as an error) cannot
        // send the search outside the list
        const u64 span = hi > lo ? hi - lo : 0;
#pragma unroll
        for (int r = 0; r < kMergeRounds; ++r) below[r] = lo;
        if (span > 0 && span <= 32) {
            const u64 w = lane < span ? __ldg(list + lo + lane) : 0;
            for (u32 j = 0; j < (u32)span; ++j) {
                const u64 wj = __shfl_sync(FULL, w, j);
#pragma unroll
                for (int r = 0; r < kMergeRounds; ++r) below[r] += wj < key[r] ? 1 : 0;
            }
        } else if (span > 32) {
#pragma unroll
            for (int r = 0; r < kMergeRounds; ++r) below[r] = lo + count_below(list + lo, span, key[r]);
        }
#pragma unroll
        for (int r = 0; r < kMergeRounds; ++r) {
            const u64 i = base + (u64)r * 32 + lane;
            if (i < RC) {
                const u64 at = i + below[r];
                if (at < cap) {
                    keys_out[at] = key[r];
                    counts_out[at] = c[r];
                }
                mx = c[r] > mx ? c[r] : mx;
            } else if (i < total) {
                const u64 h = i - RC, k = list[h];
                const int slot = hot_find(sd->table, k);
                u64 ch = 0;
                if (slot >= 0) {
                    ch = sd->slot_count[slot];
                } else {
                    const int s2 = warm_find(sd->fpw2, sd->table2, k);
                    ch = s2 >= 0 ? sd->count2[s2] : 0;
                }
                const u64 at = h + count_below(heads, RC, k);
                if (at < cap) {
                    keys_out[at] = k;
                    counts_out[at] = ch;
                }
                mx = ch > mx ? ch : mx;
                hot_sum += ch;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(FULL, mx, o));
        hot_sum += __shfl_xor_sync(FULL, hot_sum, o);
    }
    if (lane == 0) {
        if (mx) atomicMax(&bmax, mx);
        if (hot_sum) atomicAdd(&st->v[S_VALID], hot_sum);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bmax) atomicMax(&st->v[S_MAX_LINK], bmax);
        if (blockIdx.x == 0) {
            st->v[S_LINKS] = total;
            atomicAdd(&st->v[S_VALID], pos[RC]);  // the cold packets
        }
    }
}

}  // namespace

u64 split_state_bytes() { return sizeof(SplitDev); }

// The sort path's links with the hot-key split; see the top of this file.
// kb: the two key buffers of n entries; heads/pos: run scratch (n and n + 1
// entries); state: split_state_bytes() of device memory.  Writes A's sorted
// nonzero list to keys_out/counts_out and the links, valid-packets and
// max-link fields of st.
void sort_links_split(const u32* src, const u32* dst, u64 n, u64* kb[2], u64* heads, u64* pos, void* state,
                      u64* keys_out, u64* counts_out, SortScratch& sc, DevStats* st, int sms, cudaStream_t s) {
    SplitDev* sd = (SplitDev*)state;
    Tracer* tr = sc.tr;
    // the histogram and the scalars after it start from zero, the tier-2
    // table free and its counts zero
    cudaMemsetAsync(&sd->hist, 0, sizeof(SplitDev) - offsetof(SplitDev, hist), s);
    if (kWarmBuckets > 0) {
        cudaMemsetAsync(sd->table2, 0xFF, sizeof(sd->table2), s);
        cudaMemsetAsync(sd->count2, 0, sizeof(sd->count2), s);
    }
    // 1. sample, sorted, in runs
    const u64 m = std::min<u64>(kSampleMax, (n / 4) / kSampleBlocks * kSampleBlocks);
    const u64 blen = m / kSampleBlocks;
    {
        TraceScope ts(tr, "k_sample_gather", s);
        k_sample_gather<<<sms * 4, 256, 0, s>>>(src, dst, n, blen, kb[1]);
    }
    const int r = radix_sort_hi32(kb[1], nullptr, kb, m, sc, st, s, "k_onesweep<sample key>");
    launch_runs(RUN_U64, false, kb[r], nullptr, m, nullptr, heads, pos, nullptr, &sd->R_sample, sc, st, s);
    // 2. the hot set and its table
    {
        TraceScope ts(tr, "k_hot_hist", s);
        k_hot_hist<<<sms, 1024, 0, s>>>(pos, sd);
    }
    {
        TraceScope ts(tr, "k_hot_pick", s);
        k_hot_pick<<<1, kPickThreads, 0, s>>>(sd);
    }
    {
        TraceScope ts(tr, "k_hot_collect", s);
        k_hot_collect<<<sms * 2, 256, 0, s>>>(heads, pos, sd);
    }
    {
        TraceScope ts(tr, "k_hot_table", s);
        const size_t tsmem = sizeof(u64) * (kHotPad + kHotSlots);
        resident_ctas_of((const void*)k_hot_table, kTableThreads, tsmem);  // sets its shared-memory size
        k_hot_table<<<1, kTableThreads, tsmem, s>>>(sd);
    }
    if (kWarmBuckets > 0) {
        {
            TraceScope ts(tr, "k_warm_insert", s);
            k_warm_insert<<<(kWarmMax + 255) / 256, 256, 0, s>>>(sd);
        }
        TraceScope ts(tr, "k_warm_fp", s);
        k_warm_fp<<<(kWarmBuckets + 255) / 256, 256, 0, s>>>(sd);
    }
    {
        // the hot list ascending: both tiers' keys sorted together (kb is
        // free until the split writes the cold keys)
        // (the list holds at most the sample's distinct keys, a quarter of
        // the window, so the window's buffers bound its sort)
        const int rl = radix_sort_keys64(sd->list, &sd->H, kb, std::min<u64>(kListMax, n), sc, st, s,
                                         "k_onesweep<hot list>");
        cudaMemcpyAsync(sd->list, kb[rl], sizeof(u64) * std::min<u64>(kListMax, n), cudaMemcpyDeviceToDevice, s);
    }
    // 3. the split: hot keys counted, cold keys into kb[1]
    {
        const size_t smem = sizeof(SplitSmem);
        const int grid = resident_ctas_of((const void*)k_hot_split, kSplitThreads, smem);
        const u64 chunks = (n + kGroups * kGroupChunk - 1) / (kGroups * kGroupChunk);
        const bool vec = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0;
        TraceScope ts(tr, "k_hot_split", s);
        k_hot_split<<<(unsigned)std::min<u64>(chunks, (u64)grid), kSplitThreads, smem, s>>>(src, dst, n, vec, sd,
                                                                                            kb[1]);
    }
    // 4. the cold keys sorted (kb[1] -> kb[r2]) and in runs
    const int r2 = radix_sort_keys64(kb[1], &sd->cold, kb, n, sc, st, s, nullptr);
    launch_runs(RUN_U64, false, kb[r2], nullptr, n, &sd->cold, heads, pos, nullptr, &sd->R_cold, sc, st, s);
    // 5. merged with the hot keys
    {
        TraceScope ts(tr, "k_hot_merge", s);
        const size_t msmem = sizeof(u64) * kIndexMax;
        const int mgrid = resident_ctas_of((const void*)k_hot_merge, kMergeThreads, msmem);
        k_hot_merge<<<mgrid, kMergeThreads, msmem, s>>>(heads, pos, sd, keys_out, counts_out, n, st);
    }
}

// Hot keys and cold packets of the last split (blocking read).
cudaError_t split_info(const void* state, u64* hot_keys, u64* cold_packets, cudaStream_t s) {
    const SplitDev* sd = (const SplitDev*)state;
    u64 v[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&v[0], &sd->H, sizeof(u64), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v[1], &sd->cold, sizeof(u64), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (hot_keys) *hot_keys = v[0];
    if (cold_packets) *cold_packets = v[1];
    return e;
}

}  // namespace ns
