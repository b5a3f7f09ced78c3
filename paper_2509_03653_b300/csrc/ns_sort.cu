// ns_sort.cu -- sort-path kernels.
//
//  * LSD radix sort, 8-bit digits (64-bit keys alone may take the wide plan
//    below: one 10-bit and six 9-bit passes), "onesweep" structure: one histogram pass
//    computes every digit's global bucket offsets up front, then each digit
//    pass is a single kernel in which a CTA takes the next tile from an atomic
//    counter, ranks its keys stably in shared memory, obtains its global
//    per-digit offsets by decoupled look-back over its predecessors' published
//    counts, and scatters.  Tile ids are handed out in launch order, so every
//    predecessor a tile waits on is already resident; each wait is bounded
//    and records ERR_TIMEOUT instead of spinning forever.  The first pass of
//    a keys-only sort keeps no order within a digit: it ranks with shared
//    atomics and takes its global slots from per-digit cursors, with no
//    look-back.
//  * Run kernels: over a sorted sequence, emit each run's first position, its
//    key and the exclusive prefix sum of a value column at that position;
//    run lengths and run sums are then differences of neighbours.  This one
//    primitive yields A's nonzeros (runs of equal keys, Table 2 row 3), the
//    row aggregates (runs of equal src: A1 and |A|_0 1, rows 6 and 8) and the
//    column aggregates (runs of equal dst after a sort by dst).
//
// Status words for look-back: tag(16) | flag(2) | value(46).  The tag is a
// per-launch number, so a status array never needs clearing between launches.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

// CTAs of kernel `fn` (at `threads` threads and `smem` dynamic shared bytes)
// resident at once on the whole current GPU.  The first call for a kernel on
// a device also lets it take that much shared memory there (the attribute is
// per device).  Cached per (kernel, device); callers on several host threads
// or devices are safe.
int resident_ctas(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(fn, dev);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = 0, per_sm = 0;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    const int r = std::max(1, sms * std::max(per_sm, 1));
    cache[key] = r;
    return r;
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kRadix = 256;
#ifndef NS_ONESWEEP_NT
#define NS_ONESWEEP_NT 512
#endif
#ifndef NS_ONESWEEP_ITEMS
#define NS_ONESWEEP_ITEMS 16
#endif
// L2 prefetch distance of a digit pass, in multiples of the CTAs resident on
// the whole GPU (0 = none)
#ifndef NS_ONESWEEP_PF
#define NS_ONESWEEP_PF 1
#endif
// rank the first pass of keys-only sorts without stability
#ifndef NS_UNSTABLE_FIRST
#define NS_UNSTABLE_FIRST 1
#endif
// ranking of a stable digit pass: warp match, or per-bit ballots (passes in
// the bit mask NS_BALLOT_PASSES)
enum { RANK_MATCH = 0, RANK_BALLOT = 1, RANK_UNSTABLE = 2 };
#ifndef NS_BALLOT_PASSES
#define NS_BALLOT_PASSES 0x10
#endif
inline int pass_rank(int p) { return ((NS_BALLOT_PASSES >> p) & 1) ? RANK_BALLOT : RANK_MATCH; }
// L2 prefetch distance of the run kernels (as above)
#ifndef NS_RUNS_PF
#define NS_RUNS_PF 1
#endif

constexpr u64 kFlagAgg = 1, kFlagPrefix = 2;
#ifndef NS_LOOK_DIGITS
#define NS_LOOK_DIGITS 3
#endif
constexpr int kLookDigits = NS_LOOK_DIGITS;  // look-back window of the digit passes
constexpr u64 kValMask = (1ull << 46) - 1;

__device__ __forceinline__ u64 pack_status(u32 tag, u64 flag, u64 v) {
    return ((u64)tag << 48) | (flag << 46) | (v & kValMask);
}

// Exclusive prefix for `tile` of one counter whose per-tile status words are
// status[k * stride] (k = tile index).  Returns 0 for tile 0.
//
// With hundreds of tiles in flight, the nearest predecessor holding an
// inclusive prefix is typically a few dozen tiles back (measured: ~28 on
// 2^30 keys), so the walk reads WIN predecessors per round trip (independent
// loads) and sums aggregates until it meets a prefix.  A predecessor that has
// published nothing yet is waited for (bounded), then the walk resumes from
// it.  The digit passes read 3 words per round trip (their digit threads
// hold the tile's keys in registers: 4 or more spill, and 1 or 2 were
// slower); the run kernels walk with a whole warp (warp_lookback).
template <int WIN>
__device__ u64 lookback(u64* status, u64 stride, u64 tile, u32 tag, DevStats* st) {
    constexpr int kLookWindow = WIN;
    u64 prefix = 0;
    long long k = (long long)tile - 1;  // nearest predecessor not yet accounted for
    u32 spins = 0;
    u64 t0 = 0;
    while (k >= 0) {
        u64 sv[kLookWindow];
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) sv[q] = (k - q >= 0) ? ld_volatile(&status[(u64)(k - q) * stride]) : 0ull;
        int used = 0;
        bool go = true, done = false;
#pragma unroll
        for (int q = 0; q < kLookWindow; ++q) {
            if (go) {
                if (k - q < 0) {
                    done = true;
                    go = false;
                } else {
                    const u64 s = sv[q];
                    const u32 stag = (u32)(s >> 48);
                    const u64 flag = (s >> 46) & 3;
                    if (stag == tag && flag != 0) {
                        prefix += s & kValMask;
                        used = q + 1;
                        if (flag == kFlagPrefix) {
                            done = true;
                            go = false;
                        }
                    } else {
                        go = false;  // not published yet
                    }
                }
            }
        }
        if (done) break;
        k -= used;
        if (used > 0) continue;
        // the nearest predecessor has published nothing yet: poll that one
        // word alone (bounded) before reading a window again
        bool ready = false, gave_up = false;
        while (!ready && !gave_up) {
            const u64 s = ld_volatile(&status[(u64)k * stride]);
            if ((u32)(s >> 48) == tag && ((s >> 46) & 3) != 0) {
                ready = true;
            } else {
                const u64 now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                if (++spins > kMaxSpin || now - t0 > kWaitLimitNs) gave_up = true;
                else __nanosleep(20);
            }
        }
        if (gave_up) {
            set_error(st, ERR_TIMEOUT);
            break;
        }
        spins = 0;
        t0 = 0;
    }
    return prefix;
}

// The same walk by a whole warp (every lane must call it): lane l reads
// predecessor k - l, so one round trip covers 32 predecessors.  Aggregates
// are summed up to the nearest prefix; if an unpublished predecessor comes
// first, the aggregates before it are taken and the warp waits (bounded) for
// it.  Returns the prefix in every lane.
__device__ u64 warp_lookback(const u64* status, u64 tile, u32 tag, DevStats* st) {
    const u32 FULL = 0xFFFFFFFFu;
    const u32 lane = threadIdx.x & 31;
    u64 prefix = 0;
    long long k = (long long)tile - 1;
    u32 spins = 0;
    u64 t0 = 0;
    while (k >= 0) {
        const long long j = k - (long long)lane;
        // before tile 0 there is nothing: read as a prefix of 0
        const u64 sw = j >= 0 ? ld_volatile(&status[j]) : pack_status(tag, kFlagPrefix, 0);
        const bool ready = (u32)(sw >> 48) == tag && ((sw >> 46) & 3) != 0;
        const bool is_prefix = ready && ((sw >> 46) & 3) == kFlagPrefix;
        const u32 not_ready = __ballot_sync(FULL, !ready);
        const u32 prefixes = __ballot_sync(FULL, is_prefix);
        const u32 first_nr = not_ready ? (u32)(__ffs(not_ready) - 1) : 32u;
        const u32 first_pf = prefixes ? (u32)(__ffs(prefixes) - 1) : 32u;
        // lanes before the first unpublished one, through the first prefix
        const u32 take = first_pf < first_nr ? first_pf + 1 : first_nr;
        u64 v = lane < take ? (sw & kValMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        prefix += v;
        if (first_pf < first_nr) break;  // reached a prefix
        k -= (long long)take;
        if (take > 0) {
            spins = 0;
            t0 = 0;
            continue;
        }
        const u64 now = globaltimer_ns();
        if (t0 == 0) t0 = now;
        if (++spins > kMaxSpin || now - t0 > kWaitLimitNs) {
            if (lane == 0) set_error(st, ERR_TIMEOUT);
            break;
        }
        __nanosleep(20);
    }
    return prefix;
}

__device__ __forceinline__ u64 block_excl_scan64(u64 v, u64* wsum, u64* total) {
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u64 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (u32)o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 run = 0;
        for (int i = 0; i < kWarps; ++i) {
            u64 t = wsum[i];
            wsum[i] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return wsum[w] + x - v;
}

// ---- key loading ---------------------------------------------------------

template <typename K, int LOAD>
__device__ __forceinline__ K load_key(const SortIn& in, u64 i) {
    if constexpr (LOAD == LOAD_PACK) {
        return (K)(((u64)__ldg(in.src + i) << 32) | (u64)__ldg(in.dst + i));
    } else if constexpr (LOAD == LOAD_DST_OF) {
        return (K)(u32)(reinterpret_cast<const u64*>(in.keys)[i]);
    } else {
        return reinterpret_cast<const K*>(in.keys)[i];
    }
}

// ---- histogram of every digit pass ------------------------------------------

// Counting is bound by the shared-memory atomic pipe, and with one counter
// per bin, lanes holding different digits that share a bank replay (about
// 2.8 wavefronts per atomic on random digits).  So every lane counts into
// its own column instead: word (q, d, lane) is bank `lane`, so a warp's
// atomic never conflicts.  The word holds two 16-bit counts, digit d of pass
// q in the low half and of pass q + PASSES/2 in the high half (the added
// constant is fixed per pass).  Each half counts at most kHistRounds rounds
// of kHistUnroll keys from each of the CTA's warps (< 2^16) before the
// counts are added to the 64-bit global histogram and cleared.
constexpr int kHistThreads = 1024;
constexpr int kHistUnroll = 8;
constexpr int kHistRounds = 128;
static_assert(kHistRounds * kHistUnroll * (kHistThreads / 32) < 65536, "16-bit shared counters would wrap");

template <int PASSES>
__device__ __forceinline__ void hist_flush(u32* hs, u64* __restrict__ ghist) {
    constexpr int kPairs = PASSES / 2;
    const u32 lane = threadIdx.x & 31;
    for (int c = threadIdx.x; c < kPairs * kRadix; c += kHistThreads) {
        u32* row = hs + c * 32;
        u64 lo = 0, hi = 0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) {
            const int j = (l + lane) & 31;  // lanes start in different banks
            const u32 x = row[j];
            lo += x & 0xFFFFu;
            hi += x >> 16;
            row[j] = 0;
        }
        const int q = c / kRadix, d = c % kRadix;
        if (lo) atomicAdd(reinterpret_cast<unsigned long long*>(&ghist[q * kRadix + d]), (unsigned long long)lo);
        if (hi)
            atomicAdd(reinterpret_cast<unsigned long long*>(&ghist[(q + kPairs) * kRadix + d]), (unsigned long long)hi);
    }
}

// Loads block [blk, blk + kHistThreads * kHistUnroll) of the keys, kHistUnroll
// per thread; bit u of the result says whether k[u] is a key.  Each thread
// loads all of its keys before any is counted, so that enough loads are in
// flight to cover HBM latency; full blocks of 16-byte-aligned inputs are read
// with 16-byte loads.
template <typename K, int LOAD>
__device__ __forceinline__ u32 hist_load_block(const SortIn& in, u64 blk, u64 n, bool vec, K (&k)[kHistUnroll]) {
    const u64 per_block = (u64)kHistThreads * kHistUnroll;
    const u32 t = threadIdx.x;
    u32 valid = 0;
    if (vec && n - blk >= per_block) {
        valid = (1u << kHistUnroll) - 1;
        if constexpr (LOAD == LOAD_PACK) {
#pragma unroll
            for (int h = 0; h < kHistUnroll / 4; ++h) {
                const u64 i = blk + (u64)h * (4 * kHistThreads) + 4 * t;
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(in.src + i));
                const uint4 b = __ldg(reinterpret_cast<const uint4*>(in.dst + i));
                k[4 * h + 0] = (K)(((u64)a.x << 32) | b.x);
                k[4 * h + 1] = (K)(((u64)a.y << 32) | b.y);
                k[4 * h + 2] = (K)(((u64)a.z << 32) | b.z);
                k[4 * h + 3] = (K)(((u64)a.w << 32) | b.w);
            }
        } else if constexpr (sizeof(K) == 8) {
#pragma unroll
            for (int h = 0; h < kHistUnroll / 2; ++h) {
                const u64 i = blk + (u64)h * (2 * kHistThreads) + 2 * t;
                const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(reinterpret_cast<const u64*>(in.keys) + i));
                k[2 * h + 0] = (K)a.x;
                k[2 * h + 1] = (K)a.y;
            }
        } else {
#pragma unroll
            for (int h = 0; h < kHistUnroll / 4; ++h) {
                const u64 i = blk + (u64)h * (4 * kHistThreads) + 4 * t;
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const u32*>(in.keys) + i));
                k[4 * h + 0] = (K)a.x;
                k[4 * h + 1] = (K)a.y;
                k[4 * h + 2] = (K)a.z;
                k[4 * h + 3] = (K)a.w;
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const u64 i = blk + (u64)u * kHistThreads + t;
            k[u] = i < n ? load_key<K, LOAD>(in, i) : (K)0;
            valid |= (i < n ? 1u : 0u) << u;
        }
    }
    return valid;
}

template <typename K, int LOAD, int PASSES>
__global__ void __launch_bounds__(kHistThreads, 1) k_sort_hist(SortIn in, u64 n_arg, int begin_bit,
                                                                u64* __restrict__ ghist) {
    static_assert(PASSES % 2 == 0, "passes are counted in pairs");
    constexpr int kPairs = PASSES / 2;
    extern __shared__ __align__(16) u32 hs[];  // [kPairs][kRadix][32 lanes]
    const u64 n = in.n_dev ? *in.n_dev : n_arg;
    for (int i = threadIdx.x; i < kPairs * kRadix * 32; i += kHistThreads) hs[i] = 0;
    __syncthreads();
    u32* hl = hs + (threadIdx.x & 31);
    // The CTA takes blocks of kHistThreads * kHistUnroll consecutive keys.
    const u64 per_block = (u64)kHistThreads * kHistUnroll;
    const bool vec = in.bulk && LOAD != LOAD_DST_OF;
    int rounds = 0;
    for (u64 blk = (u64)blockIdx.x * per_block; blk < n; blk += (u64)gridDim.x * per_block) {
        K k[kHistUnroll];
        const u32 valid = hist_load_block<K, LOAD>(in, blk, n, vec, k);
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            if ((valid >> u) & 1u) {
                const u64 kb = (u64)k[u] >> begin_bit;
#pragma unroll
                for (int p = 0; p < PASSES; ++p)
                    atomicAdd(&hl[((p % kPairs) * kRadix + ((u32)(kb >> (8 * p)) & 0xFF)) * 32],
                              p < kPairs ? 1u : 0x10000u);
            }
        }
        if (++rounds == kHistRounds) {  // the same count in every thread of the CTA
            rounds = 0;
            __syncthreads();
            hist_flush<PASSES>(hs, ghist);
            __syncthreads();
        }
    }
    __syncthreads();
    hist_flush<PASSES>(hs, ghist);
}

// ---- the wide digit plan for 64-bit keys ----------------------------------------
//
// Seven passes instead of eight: a 10-bit first pass (bits 0..9, unstable,
// 1024 digits) and six stable 9-bit passes (bits 10..63, 512 digits each).
// Its histograms and bucket starts are laid out [pass 0: 1024][pass 1: 512]
// ... [pass 6: 512], 4096 entries, followed by pass 0's 1024 slot cursors.
constexpr int kWidePasses = 7;
constexpr int kWideBins = 1024 + 6 * 512;
constexpr int kWideStableRadix = 512;  // look-back status words per tile
__host__ __device__ constexpr int wide_bits(int p) { return p == 0 ? 10 : 9; }
__host__ __device__ constexpr int wide_shift(int p) { return p == 0 ? 0 : 10 + 9 * (p - 1); }
__host__ __device__ constexpr int wide_base(int p) { return p == 0 ? 0 : 1024 + 512 * (p - 1); }

// The wide plan's 4096 bins do not fit lane-private 16-bit columns in one
// CTA's shared memory (256 KB), so they are counted in two launches of 128
// KB each, group 0 for passes 0..2 and group 1 for passes 3..6.  As in
// k_sort_hist, word (slot, lane) holds two 16-bit counts and every lane counts
// into its own column; the counts are flushed every kHistRounds rounds.
//   group 0: low half of slot s = digit s of pass 0 (s < 1024); high half =
//            digit s of pass 1 (s < 512), digit s - 512 of pass 2 (s >= 512)
//   group 1: low half = digit s of pass 3 / digit s - 512 of pass 4; high
//            half = digit s of pass 5 / digit s - 512 of pass 6
constexpr int kWideSlots = 1024;
static_assert(kWideSlots == kHistThreads, "the flush gives every thread one slot");

__host__ __device__ constexpr int wide_low_pass(int g, u32 slot) { return g == 0 ? 0 : (slot < 512 ? 3 : 4); }
__host__ __device__ constexpr int wide_high_pass(int g, u32 slot) {
    return g == 0 ? (slot < 512 ? 1 : 2) : (slot < 512 ? 5 : 6);
}

template <int G>
__device__ __forceinline__ void hist_flush_wide(u32* hs, u64* __restrict__ ghist) {
    const u32 lane = threadIdx.x & 31;
    const u32 c = threadIdx.x;  // the slot
    u32* row = hs + c * 32;
    u64 lo = 0, hi = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) {
        const int j = (l + lane) & 31;  // lanes start in different banks
        const u32 x = row[j];
        lo += x & 0xFFFFu;
        hi += x >> 16;
        row[j] = 0;
    }
    unsigned long long* g = reinterpret_cast<unsigned long long*>(ghist);
    const u32 lp = wide_low_pass(G, c), hp = wide_high_pass(G, c);
    const u32 ld = G == 0 ? c : (c & 511u), hd = c & 511u;
    if (lo) atomicAdd(&g[wide_base(lp) + ld], (unsigned long long)lo);
    if (hi) atomicAdd(&g[wide_base(hp) + hd], (unsigned long long)hi);
}

template <typename K, int LOAD, int G>
__global__ void __launch_bounds__(kHistThreads, 1) k_sort_hist_wide(SortIn in, u64 n_arg, u64* __restrict__ ghist) {
    static_assert(sizeof(K) == 8, "the wide plan sorts 64-bit keys");
    extern __shared__ __align__(16) u32 hs[];  // [kWideSlots][32 lanes]
    const u64 n = in.n_dev ? *in.n_dev : n_arg;
    for (int i = threadIdx.x; i < kWideSlots * 32; i += kHistThreads) hs[i] = 0;
    __syncthreads();
    u32* hl = hs + (threadIdx.x & 31);
    const u64 per_block = (u64)kHistThreads * kHistUnroll;
    const bool vec = in.bulk;
    int rounds = 0;
    for (u64 blk = (u64)blockIdx.x * per_block; blk < n; blk += (u64)gridDim.x * per_block) {
        K k[kHistUnroll];
        const u32 valid = hist_load_block<K, LOAD>(in, blk, n, vec, k);
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            if ((valid >> u) & 1u) {
                const u64 kb = (u64)k[u];
                if constexpr (G == 0) {
                    atomicAdd(&hl[((u32)kb & 1023u) * 32], 1u);
                    atomicAdd(&hl[((u32)(kb >> wide_shift(1)) & 511u) * 32], 0x10000u);
                    atomicAdd(&hl[(512u + ((u32)(kb >> wide_shift(2)) & 511u)) * 32], 0x10000u);
                } else {
                    atomicAdd(&hl[((u32)(kb >> wide_shift(3)) & 511u) * 32], 1u);
                    atomicAdd(&hl[(512u + ((u32)(kb >> wide_shift(4)) & 511u)) * 32], 1u);
                    atomicAdd(&hl[((u32)(kb >> wide_shift(5)) & 511u) * 32], 0x10000u);
                    atomicAdd(&hl[(512u + ((u32)(kb >> wide_shift(6)) & 511u)) * 32], 0x10000u);
                }
            }
        }
        if (++rounds == kHistRounds) {  // the same count in every thread of the CTA
            rounds = 0;
            __syncthreads();
            hist_flush_wide<G>(hs, ghist);
            __syncthreads();
        }
    }
    __syncthreads();
    hist_flush_wide<G>(hs, ghist);
}

template <typename K, int LOAD, int G>
void launch_hist_wide_group(const SortIn& in, u64 n, u64* ghist, Tracer* tr, cudaStream_t s) {
    const size_t hsmem = sizeof(u32) * kWideSlots * 32;
    const int max_grid = resident_ctas((const void*)k_sort_hist_wide<K, LOAD, G>, kHistThreads, hsmem);
    const u64 blocks = (n + (u64)kHistThreads * kHistUnroll - 1) / ((u64)kHistThreads * kHistUnroll);
    const int grid = (int)std::max<u64>(1, std::min<u64>(blocks, (u64)max_grid));
    TraceScope ts(tr, "k_sort_hist", s);
    k_sort_hist_wide<K, LOAD, G><<<grid, kHistThreads, hsmem, s>>>(in, n, ghist);
}

template <typename K, int LOAD>
void launch_hist_wide(const SortIn& in, u64 n, u64* ghist, Tracer* tr, cudaStream_t s) {
    launch_hist_wide_group<K, LOAD, 0>(in, n, ghist, tr, s);
    launch_hist_wide_group<K, LOAD, 1>(in, n, ghist, tr, s);
}

// bucket starts of the wide plan: offs[wide_base(p) + d] = sum of pass p's
// ghist below d, then pass 0's slot cursors at offs[kWideBins + d]
__global__ void __launch_bounds__(1024) k_sort_offsets_wide(const u64* __restrict__ ghist, u64* __restrict__ offs) {
    __shared__ u64 wsum[32];
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int p = 0; p < kWidePasses; ++p) {
        const int r = 1 << wide_bits(p);
        const u64 v = (int)threadIdx.x < r ? ghist[wide_base(p) + threadIdx.x] : 0ull;
        u64 x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (u32)o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            u64 run = 0;
            for (int i = 0; i < 32; ++i) {
                const u64 t = wsum[i];
                wsum[i] = run;
                run += t;
            }
        }
        __syncthreads();
        const u64 e = wsum[w] + x - v;
        if ((int)threadIdx.x < r) {
            offs[wide_base(p) + threadIdx.x] = e;
            if (p == 0) offs[kWideBins + threadIdx.x] = e;
        }
        __syncthreads();
    }
}

template <typename K, int LOAD, int PASSES>
void launch_hist(const SortIn& in, u64 n, int begin_bit, u64* ghist, Tracer* tr, cudaStream_t s) {
    const size_t hsmem = sizeof(u32) * (PASSES / 2) * kRadix * 32;
    const int max_grid = resident_ctas((const void*)k_sort_hist<K, LOAD, PASSES>, kHistThreads, hsmem);
    const u64 blocks = (n + (u64)kHistThreads * kHistUnroll - 1) / ((u64)kHistThreads * kHistUnroll);
    const int grid = (int)std::max<u64>(1, std::min<u64>(blocks, (u64)max_grid));
    TraceScope ts(tr, "k_sort_hist", s);
    k_sort_hist<K, LOAD, PASSES><<<grid, kHistThreads, hsmem, s>>>(in, n, begin_bit, ghist);
}

// bucket starts: offs[p][d] = sum of ghist[p][0..d)
// and offs[8][d] = offs[0][d]: the slot cursors of a first pass ranked
// without stability
__global__ void __launch_bounds__(kThreads) k_sort_offsets(const u64* __restrict__ ghist, int passes,
                                                            u64* __restrict__ offs) {
    __shared__ u64 wsum[kWarps];
    __shared__ u64 tot;
    for (int p = 0; p < passes; ++p) {
        const u64 v = ghist[p * kRadix + threadIdx.x];
        const u64 e = block_excl_scan64(v, wsum, &tot);
        offs[p * kRadix + threadIdx.x] = e;
        if (p == 0) offs[8 * kRadix + threadIdx.x] = e;
        __syncthreads();
    }
}

// ---- one digit pass -----------------------------------------------------------
//
// One tile per CTA, tiles handed out in launch order by an atomic counter.
// The tile is staged into shared memory by the bulk-copy engine (no register
// is held while it streams in), ranked stably per warp, given its global
// per-digit offsets by decoupled look-back, placed in digit order in the same
// buffer and written out in digit runs.  With RANK_UNSTABLE (the first pass
// of a keys-only sort) the ranks come from shared atomics on the tile's digit
// counters and the global offsets from per-digit cursors instead.
// (Reserving a second tile ahead of time for double buffering was measured
// slower: successors then wait on a tile whose count cannot be published
// until its CTA gets to it.)

typedef unsigned short WCount;  // a per-warp digit count (<= 512)

// RB: digit width in bits (8, 9 or 10); only the arrays a pass uses are sized
// for its radix (stable passes: per-warp counts; unstable: tile counts)
template <typename K, bool HAS_V, int NT, int IT, int RB = 8, bool UNSTABLE = false>
struct ScatterSmem {
    static constexpr int NW = NT / 32, TILE = NT * IT, R = 1 << RB;
    K keys[TILE];  // staged tile, then the tile in digit order
    u64 vals[HAS_V ? TILE : 1];
    WCount whist[UNSTABLE ? 1 : NW][UNSTABLE ? 1 : R];  // per-warp digit counts (<= 512)
    u32 tcount[UNSTABLE ? R : 1];  // unstable ranking: the tile's digit counts, then their exclusive scan
    u64 gdelta[R];  // global position of a digit's first key minus its tile-local start
    u32 wsum[NW];
    u32 total;
    u32 tile;
    u32 abort;
    u64 bar;
};

// Stages tile [base, base + tile_n) into shared memory.  With `bulk`, thread
// 0 issues bulk copies of the 16-byte-aligned prefix and the threads load the
// ragged tail (< 4 elements); otherwise all threads load.  Packed mode stages
// the two uint32 columns side by side in the key buffer's bytes.
template <typename K, bool HAS_V, int LOAD, int NT, int IT, typename SM>
__device__ __forceinline__ bool stage_tile(const SortIn& in, SM& sm, u64 base, u32 tile_n,
                                           bool bulk, u32 parity, DevStats* st) {
    constexpr int kTile = NT * IT;
    u32* s32 = reinterpret_cast<u32*>(sm.keys);
    constexpr u32 kq = (LOAD == LOAD_PACK) ? 4u : (16u / (u32)sizeof(K));
    const u32 nb = bulk ? (tile_n & ~(kq - 1)) : 0u;
    const u32 nv = (bulk && HAS_V) ? (tile_n & ~1u) : 0u;
    if (bulk && threadIdx.x == 0) {
        u32 bytes;
        if constexpr (LOAD == LOAD_PACK) bytes = 2u * nb * 4u;
        else bytes = nb * (u32)sizeof(K) + nv * 8u;
        mbar_arrive_expect_tx(&sm.bar, bytes);
        if (nb) {
            if constexpr (LOAD == LOAD_PACK) {
                bulk_g2s(s32, in.src + base, nb * 4u, &sm.bar);
                bulk_g2s(s32 + kTile, in.dst + base, nb * 4u, &sm.bar);
            } else {
                bulk_g2s(sm.keys, reinterpret_cast<const K*>(in.keys) + base, nb * (u32)sizeof(K), &sm.bar);
            }
        }
        if constexpr (HAS_V && LOAD != LOAD_PACK) {
            if (nv) bulk_g2s(sm.vals, in.vals + base, nv * 8u, &sm.bar);
        }
    }
    for (u32 i = nb + threadIdx.x; i < tile_n; i += NT) {
        if constexpr (LOAD == LOAD_PACK) {
            s32[i] = in.src[base + i];
            s32[kTile + i] = in.dst[base + i];
        } else if constexpr (LOAD == LOAD_DST_OF) {
            sm.keys[i] = (K)(u32)(reinterpret_cast<const u64*>(in.keys)[base + i]);
        } else {
            sm.keys[i] = reinterpret_cast<const K*>(in.keys)[base + i];
        }
    }
    if constexpr (HAS_V && LOAD != LOAD_PACK) {
        for (u32 i = nv + threadIdx.x; i < tile_n; i += NT) sm.vals[i] = in.vals[base + i];
    }
    return bulk ? mbar_wait_bounded(&sm.bar, parity, st) : true;
}

// exclusive scan of one u32 per thread over an NT-thread block
template <int NT>
__device__ __forceinline__ u32 block_excl_scan_nt(u32 v, u32* wsum, u32* total) {
    constexpr int NW = NT / 32;
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (u32)o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 run = 0;
        for (int i = 0; i < NW; ++i) {
            u32 tt = wsum[i];
            wsum[i] = run;
            run += tt;
        }
        *total = run;
    }
    __syncthreads();
    return wsum[w] + x - v;
}

template <typename K, bool HAS_V, int LOAD, int NT, int IT, int RANK, int RB>
__global__ void __launch_bounds__(NT, (NT >= 1024) ? 1 : (NT >= 512) ? 2 : (NT >= 384) ? 2 : (HAS_V ? 3 : 4))
    k_onesweep(SortIn in, K* __restrict__ kout, u64* __restrict__ vout, u64 n_arg, int shift,
               const u64* __restrict__ offs, u64* __restrict__ status, u32* tile_counter, u32 tag, DevStats* st,
               u32 pf_tiles, u64* __restrict__ cursor) {
    constexpr int kWarps = NT / 32, kTile = NT * IT, kItems = IT;
    constexpr bool UNSTABLE = RANK == RANK_UNSTABLE;
    // digits of this pass; thread t handles digits [t*DPT, (t+1)*DPT)
    constexpr int R = 1 << RB, DPT = R > NT ? R / NT : 1;
    constexpr u32 kMask = (u32)R - 1;
    static_assert(R <= NT || R % NT == 0, "digits per thread must be whole");
    using Smem = ScatterSmem<K, HAS_V, NT, IT, RB, UNSTABLE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 FULL = 0xFFFFFFFFu;
    const u64 n = in.n_dev ? *in.n_dev : n_arg;
    // bulk copies only for aligned inputs, and never for the u64 -> u32 mode
    const bool bulk = in.bulk && LOAD != LOAD_DST_OF;

    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        sm.abort = 0;
    }
    u32 parity = 0;
    // Persistent: take tiles in order until none are left.  Every tile a
    // look-back waits on was taken earlier by a running CTA, and the grid
    // never outnumbers the CTAs that fit at once, so a launch for an upper
    // bound on n costs no empty CTAs.
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(tile_counter, 1u);
        if constexpr (UNSTABLE) {
            for (int i = threadIdx.x; i < R; i += NT) sm.tcount[i] = 0;
        } else {
            for (int i = threadIdx.x; i < kWarps * R; i += NT) (&sm.whist[0][0])[i] = 0;
        }
        __syncthreads();
        const u64 tile = sm.tile;
        const u64 base = tile * kTile;
        if (base >= n) break;  // no tiles left
        const u32 tile_n = (u32)((n - base) < (u64)kTile ? (n - base) : (u64)kTile);

        // Tiles are taken in order, so the tile pf_tiles ahead will be taken by
        // some CTA about one residency later: start moving it into L2 now, and
        // its staging copy then reads L2 instead of waiting on HBM.
        if (bulk && pf_tiles && threadIdx.x == 0) {
            const u64 pb = base + (u64)pf_tiles * kTile;
            if (pb < n) {
                const u64 cnt = (n - pb) < (u64)kTile ? (n - pb) : (u64)kTile;
                if constexpr (LOAD == LOAD_PACK) {
                    const u32 bytes = (u32)(cnt * 4u) & ~15u;
                    if (bytes) {
                        bulk_prefetch_l2(in.src + pb, bytes);
                        bulk_prefetch_l2(in.dst + pb, bytes);
                    }
                } else {
                    const u32 bytes = (u32)(cnt * sizeof(K)) & ~15u;
                    if (bytes) bulk_prefetch_l2(reinterpret_cast<const K*>(in.keys) + pb, bytes);
                    if constexpr (HAS_V) {
                        const u32 vb = (u32)(cnt * 8u) & ~15u;
                        if (vb) bulk_prefetch_l2(in.vals + pb, vb);
                    }
                }
            }
        }

        {
            const bool ok = stage_tile<K, HAS_V, LOAD, NT, IT>(in, sm, base, tile_n, bulk, parity, st);
            if (threadIdx.x == 0 && !ok) sm.abort = 1;
        }
        parity ^= bulk ? 1u : 0u;
        __syncthreads();
        if (sm.abort) break;  // a staging copy never completed (recorded); stop taking tiles

        // warp w owns tile items [w*kItems*32, +kItems*32), read consecutively
        K k[kItems];
        u64 v[kItems];
        u32 rank[kItems];
        const u32 w0 = w * kItems * 32;
        const u32* s32 = reinterpret_cast<const u32*>(sm.keys);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const u32 li = w0 + j * 32 + lane;
            if (li < tile_n) {
                if constexpr (LOAD == LOAD_PACK) k[j] = (K)(((u64)s32[li] << 32) | (u64)s32[kTile + li]);
                else k[j] = sm.keys[li];
                if constexpr (HAS_V) v[j] = sm.vals[li];
            } else {
                k[j] = 0;
                if constexpr (HAS_V) v[j] = 0;
            }
        }
        const u32 lt = lanemask_lt();
        if constexpr (UNSTABLE) {
            // any order within a digit: a slot from the tile's digit counter
            // (shared atomics; no item waits on the previous one's result)
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                const u32 li = w0 + j * 32 + lane;
                if (li < tile_n) rank[j] = atomicAdd(&sm.tcount[(u32)(k[j] >> shift) & kMask], 1u);
            }
        } else {
        // stable rank within the warp, item by item
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const u32 li = w0 + j * 32 + lane;
            const bool valid = li < tile_n;
            const u32 d = valid ? ((u32)(k[j] >> shift) & kMask) : (u32)R;
            u32 peers;
            if constexpr (RANK == RANK_BALLOT) {
                // the lanes agreeing with this one on every bit of d
                peers = __ballot_sync(FULL, valid);
                if (!valid) peers = ~peers;
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const bool bit = (d >> b) & 1u;
                    const u32 bal = __ballot_sync(FULL, bit);
                    peers &= bit ? bal : ~bal;
                }
            } else {
                peers = __match_any_sync(FULL, d);
            }
            u32 before = 0;
            if (valid) before = sm.whist[w][d];
            __syncwarp();
            if (valid) {
                rank[j] = before + __popc(peers & lt);
                if ((peers & lt) == 0) sm.whist[w][d] = (WCount)(before + __popc(peers));
            }
            __syncwarp();
        }
        }
        __syncthreads();

        // per digit: exclusive over warps, tile count
        const u32 d0 = threadIdx.x * DPT;
        u32 run[DPT];
        u32 trun = 0;  // this thread's digits together
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const u32 d = d0 + q;
            run[q] = 0;
            if (d < (u32)R) {
                if constexpr (UNSTABLE) {
                    run[q] = sm.tcount[d];
                } else {
#pragma unroll
                    for (int ww = 0; ww < kWarps; ++ww) {
                        const u32 c = sm.whist[ww][d];
                        sm.whist[ww][d] = (WCount)run[q];
                        run[q] += c;
                    }
                    // publish this tile's count early so successors can proceed
                    st_volatile(&status[tile * R + d], pack_status(tag, tile == 0 ? kFlagPrefix : kFlagAgg, run[q]));
                }
            }
            trun += run[q];
        }
        u32 ls = block_excl_scan_nt<NT>(trun, sm.wsum, &sm.total);
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const u32 d = d0 + q;
            if (d < (u32)R) {
                if constexpr (UNSTABLE) {
                    sm.tcount[d] = ls;  // the digit's first slot in the tile's digit order
                    // Tiles may take their places in any order: the digit's
                    // global slots come from one atomic on its cursor (which
                    // starts at the digit's bucket start) instead of a look-back.
                    const u64 g = run[q] ? atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[d]),
                                                     (unsigned long long)run[q])
                                         : 0ull;
                    sm.gdelta[d] = g - ls;  // modulo 2^64; + i below lands in range
                } else {
                    // each warp's first slot for digit d in the tile's digit order
#pragma unroll
                    for (int ww = 0; ww < kWarps; ++ww) sm.whist[ww][d] = (WCount)(sm.whist[ww][d] + ls);
                    u64 prefix = 0;
                    if (tile > 0) {
                        prefix = lookback<kLookDigits>(status + d, R, tile, tag, st);
                        st_volatile(&status[tile * R + d], pack_status(tag, kFlagPrefix, prefix + run[q]));
                    }
                    sm.gdelta[d] = offs[d] + prefix - ls;  // modulo 2^64; + i below lands in range
                }
            }
            ls += run[q];
        }
        __syncthreads();

        // place keys in tile-local digit order
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const u32 li = w0 + j * 32 + lane;
            if (li < tile_n) {
                const u32 dj = (u32)(k[j] >> shift) & kMask;
                u32 pos;
                if constexpr (UNSTABLE) pos = sm.tcount[dj] + rank[j];
                else pos = (u32)sm.whist[w][dj] + rank[j];
                if (pos < (u32)kTile) {
                    sm.keys[pos] = k[j];
                    if constexpr (HAS_V) sm.vals[pos] = v[j];
                }
            }
        }
        __syncthreads();

        // write out: consecutive smem positions of one digit go to consecutive
        // global positions
        for (u32 i = threadIdx.x; i < tile_n; i += NT) {
            const K key = sm.keys[i];
            const u32 dk = (u32)(key >> shift) & kMask;
            const u64 dst = sm.gdelta[dk] + i;
            if (dst < n) {  // always true unless a look-back gave up
                kout[dst] = key;
                if constexpr (HAS_V) vout[dst] = sm.vals[i];
            }
        }
        __syncthreads();  // the tile's shared memory is reused by the next one
    }
}

// ---- runs of a sorted sequence ------------------------------------------------

template <int KEYMODE>
__device__ __forceinline__ u64 run_key(const void* keys, u64 i) {
    if constexpr (KEYMODE == RUN_U64) return reinterpret_cast<const u64*>(keys)[i];
    else if constexpr (KEYMODE == RUN_SRC_OF_U64 || KEYMODE == RUN_HI_OF_PACKED)
        return reinterpret_cast<const u64*>(keys)[i] >> 32;
    else return reinterpret_cast<const u32*>(keys)[i];
}

// Run-kernel CTA shape: threads and keys per thread.  Keys alone take
// 8192-key tiles (fewer look-backs per key); with values, 2048-key tiles
// (the registers that stage a tile otherwise halve the resident CTAs).
#ifndef NS_RUNS_NT
#define NS_RUNS_NT 512
#endif
#ifndef NS_RUNS_VNT
#define NS_RUNS_VNT 256
#endif
#ifndef NS_RUNS_VITEMS
#define NS_RUNS_VITEMS 8
#endif
template <bool HAS_V>
struct RunShape {
    static constexpr int threads = HAS_V ? NS_RUNS_VNT : NS_RUNS_NT;
    static constexpr int items = HAS_V ? NS_RUNS_VITEMS : kItems;
    static constexpr int warps = threads / 32;
    static constexpr int tile = threads * items;
};

template <bool HAS_V>
struct RunsSmem {
    u64 key[RunShape<HAS_V>::tile + 1];  // key[0] = the element before the tile
    u64 val[HAS_V ? RunShape<HAS_V>::tile : 1];
    u32 wcnt[RunShape<HAS_V>::warps];    // heads per warp -> exclusive offsets
    u64 wsum[RunShape<HAS_V>::warps];    // value sums per warp -> exclusive offsets
    u64 cbase, sbase, tot64;
    u32 tot;
    u32 tile;
};

// For each run head i (i == 0 or key(i) != key(i-1)), in order r = 0, 1, ...:
//   pos[r] = i, psum[r] = sum of val[0..i) (if HAS_V), head_keys[r] = key(i)
// and finally pos[R] = n, psum[R] = total, *R_out = R.
//
// Warp w owns the tile's kRunItems * 32 items from 32 kRunItems w, visited as kRunItems rounds
// of 32 consecutive items, so every shared-memory access is consecutive
// across the lanes; heads are counted with ballots, value prefixes with
// shuffle scans.  Two sweeps over the tile: count, then (after the tile's
// offsets are known by look-back) write.
template <int KEYMODE, bool HAS_V>
__global__ void __launch_bounds__(RunShape<HAS_V>::threads) k_runs(const void* __restrict__ keys,
                                                    const u64* __restrict__ vals, u64 n_arg,
                                                    const u64* __restrict__ n_dev,
                                                    u64* __restrict__ head_keys, u64* __restrict__ pos,
                                                    u64* __restrict__ psum, u64* status_c,
                                                    u64* status_s, u32* tile_counter, u32 tag,
                                                    u64* R_out, DevStats* st, u64* __restrict__ pack_out,
                                                    u32 pf_tiles) {
    constexpr int kRunThreads = RunShape<HAS_V>::threads, kRunWarps = RunShape<HAS_V>::warps,
                  kRunTile = RunShape<HAS_V>::tile, kRunItems = RunShape<HAS_V>::items;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RunsSmem<HAS_V>& sm = *reinterpret_cast<RunsSmem<HAS_V>*>(smem_raw);
    const u32 FULL = 0xFFFFFFFFu;
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u64 n = n_dev ? *n_dev : n_arg;
    // Persistent: take tiles in order until none are left (a launch for an
    // upper bound on n costs no empty CTAs).
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const u64 tile = sm.tile;
        const u64 base = tile * kRunTile;
        if (base >= n) {
            // an empty sequence still needs its terminal entry
            if (n == 0 && tile == 0 && threadIdx.x == 0) {
                pos[0] = 0;
                if constexpr (HAS_V) psum[0] = 0;
                *R_out = 0;
            }
            break;
        }
        const u64 tile_n = (n - base) < (u64)kRunTile ? (n - base) : (u64)kRunTile;

        // the tile pf_tiles ahead is taken about one residency later: start
        // moving it into L2 now (pf_tiles is 0 unless the inputs are 16-byte
        // aligned)
        if (pf_tiles && threadIdx.x == 0) {
            const u64 pb = base + (u64)pf_tiles * kRunTile;
            if (pb < n) {
                const u64 cnt = (n - pb) < (u64)kRunTile ? (n - pb) : (u64)kRunTile;
                constexpr u32 ksz = KEYMODE == RUN_U32 ? 4u : 8u;
                const u32 kbytes = (u32)(cnt * ksz) & ~15u;
                if (kbytes) bulk_prefetch_l2(reinterpret_cast<const unsigned char*>(keys) + pb * ksz, kbytes);
                if constexpr (HAS_V && KEYMODE != RUN_HI_OF_PACKED) {
                    const u32 vbytes = (u32)(cnt * 8u) & ~15u;
                    if (vbytes) bulk_prefetch_l2(vals + pb, vbytes);
                }
            }
        }

        // stage the tile: all of a thread's loads are issued before any is
        // stored, so that kRunItems of them are in flight at once
        {
            u64 wd[kRunItems], vv[kRunItems];
#pragma unroll
            for (int r = 0; r < kRunItems; ++r) {
                const u32 i = threadIdx.x + r * kRunThreads;
                wd[r] = vv[r] = 0;
                if (i < tile_n) {
                    if constexpr (KEYMODE == RUN_U32) wd[r] = reinterpret_cast<const u32*>(keys)[base + i];
                    else wd[r] = reinterpret_cast<const u64*>(keys)[base + i];
                    if constexpr (HAS_V && KEYMODE != RUN_HI_OF_PACKED) vv[r] = vals[base + i];
                }
            }
#pragma unroll
            for (int r = 0; r < kRunItems; ++r) {
                const u32 i = threadIdx.x + r * kRunThreads;
                if (i < tile_n) {
                    if constexpr (KEYMODE == RUN_HI_OF_PACKED) {
                        sm.key[i + 1] = wd[r] >> 32;
                        sm.val[i] = wd[r] & 0xFFFFFFFFull;
                    } else if constexpr (KEYMODE == RUN_SRC_OF_U64) {
                        // with pack_out, also emit (dst << 32 | value) for a
                        // sort by dst (values < 2^32)
                        sm.key[i + 1] = wd[r] >> 32;
                        sm.val[i] = vv[r];
                        if (pack_out) pack_out[base + i] = (wd[r] << 32) | (vv[r] & 0xFFFFFFFFull);
                    } else {
                        sm.key[i + 1] = wd[r];
                        if constexpr (HAS_V) sm.val[i] = vv[r];
                    }
                }
            }
        }
        if (threadIdx.x == 0) sm.key[0] = base > 0 ? run_key<KEYMODE>(keys, base - 1) : ~0ull;
        __syncthreads();

        // sweep 1: heads and value sums per warp
        const u32 w0 = w * (kRunItems * 32);
        u32 cnt = 0;
        u64 vs = 0;
#pragma unroll 4
        for (int r = 0; r < kRunItems; ++r) {
            const u32 li = w0 + r * 32 + lane;
            bool h = false;
            if (li < tile_n) {
                h = (base + li == 0) || sm.key[li + 1] != sm.key[li];
                if constexpr (HAS_V) vs += sm.val[li];
            }
            cnt += __popc(__ballot_sync(FULL, h));
        }
        if constexpr (HAS_V) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vs += __shfl_xor_sync(FULL, vs, o);
        }
        if (lane == 0) {
            sm.wcnt[w] = cnt;
            if constexpr (HAS_V) sm.wsum[w] = vs;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 c = 0;
            u64 s = 0;
            for (int i = 0; i < kRunWarps; ++i) {
                const u32 tc = sm.wcnt[i];
                sm.wcnt[i] = c;
                c += tc;
                if constexpr (HAS_V) {
                    const u64 ts = sm.wsum[i];
                    sm.wsum[i] = s;
                    s += ts;
                }
            }
            sm.tot = c;
            sm.tot64 = s;
        }
        __syncthreads();
        // look-back: warp 0 for the head count, warp 1 for the value sum
        if (w == 0) {
            if (lane == 0)
                st_volatile(&status_c[tile], pack_status(tag, tile == 0 ? kFlagPrefix : kFlagAgg, sm.tot));
            u64 c = 0;
            if (tile > 0) {
                c = warp_lookback(status_c, tile, tag, st);
                if (lane == 0) st_volatile(&status_c[tile], pack_status(tag, kFlagPrefix, c + sm.tot));
            }
            if (lane == 0) sm.cbase = c;
        }
        if (HAS_V && w == 1) {
            if (lane == 0)
                st_volatile(&status_s[tile], pack_status(tag, tile == 0 ? kFlagPrefix : kFlagAgg, sm.tot64));
            u64 sv = 0;
            if (tile > 0) {
                sv = warp_lookback(status_s, tile, tag, st);
                if (lane == 0) st_volatile(&status_s[tile], pack_status(tag, kFlagPrefix, sv + sm.tot64));
            }
            if (lane == 0) sm.sbase = sv;
        }
        __syncthreads();

        // sweep 2: write heads in order
        u64 r_run = sm.cbase + sm.wcnt[w];
        u64 s_run = HAS_V ? sm.sbase + sm.wsum[w] : 0;
        const u32 lt = lanemask_lt();
#pragma unroll 4
        for (int r = 0; r < kRunItems; ++r) {
            const u32 li = w0 + r * 32 + lane;
            bool h = false;
            u64 v = 0;
            if (li < tile_n) {
                h = (base + li == 0) || sm.key[li + 1] != sm.key[li];
                if constexpr (HAS_V) v = sm.val[li];
            }
            const u32 bal = __ballot_sync(FULL, h);
            u64 vex = 0, vtot = 0;
            if constexpr (HAS_V) {
                u64 x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u64 y = __shfl_up_sync(FULL, x, o);
                    if (lane >= (u32)o) x += y;
                }
                vex = x - v;
                vtot = __shfl_sync(FULL, x, 31);
            }
            if (h) {
                const u64 rr = r_run + __popc(bal & lt);
                if (rr < n) {  // R <= n unless a look-back gave up
                    pos[rr] = base + li;
                    if constexpr (HAS_V) psum[rr] = s_run + vex;
                    if (head_keys) head_keys[rr] = sm.key[li + 1];
                }
            }
            r_run += __popc(bal);
            s_run += vtot;
        }
        if (base + tile_n == n && threadIdx.x == 0) {
            const u64 R = min(sm.cbase + sm.tot, n);
            pos[R] = n;
            if constexpr (HAS_V) psum[R] = sm.sbase + sm.tot64;
            *R_out = R;
        }
        __syncthreads();  // the tile's shared memory is reused by the next one
    }
}

// Statistics of runs r < R from neighbour differences.
//   RS_LINKS: counts[r] = pos[r+1]-pos[r]; links = R, max link, valid = n
//   RS_ROWS : sources = R, max src packets (psum diff), max fan-out (pos diff)
//   RS_COLS : destinations = R, max dst packets, max fan-in
template <int MODE>
__global__ void __launch_bounds__(256) k_run_stats(const u64* __restrict__ pos,
                                                    const u64* __restrict__ psum,
                                                    const u64* __restrict__ R_ptr,
                                                    u64* __restrict__ counts_out, DevStats* st) {
    __shared__ u64 m1, m2;
    if (threadIdx.x == 0) m1 = m2 = 0;
    __syncthreads();
    const u64 R = *R_ptr;
    u64 a = 0, b = 0;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += stride) {
        const u64 len = pos[r + 1] - pos[r];
        if constexpr (MODE == RS_LINKS) {
            counts_out[r] = len;
            a = len > a ? len : a;
        } else {
            const u64 sum = psum[r + 1] - psum[r];
            a = sum > a ? sum : a;
            b = len > b ? len : b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = max(a, __shfl_xor_sync(0xFFFFFFFFu, a, o));
        b = max(b, __shfl_xor_sync(0xFFFFFFFFu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicMax(&m1, a);
        if (b) atomicMax(&m2, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if constexpr (MODE == RS_LINKS) {
            if (m1) atomicMax(&st->v[S_MAX_LINK], m1);
            if (blockIdx.x == 0) {
                st->v[S_LINKS] = R;
                st->v[S_VALID] = pos[R];
            }
        } else if constexpr (MODE == RS_ROWS) {
            if (m1) atomicMax(&st->v[S_MAX_SRC_PK], m1);
            if (m2) atomicMax(&st->v[S_MAX_SRC_FO], m2);
            if (blockIdx.x == 0) st->v[S_SRCS] = R;
        } else {
            if (m1) atomicMax(&st->v[S_MAX_DST_PK], m1);
            if (m2) atomicMax(&st->v[S_MAX_DST_FI], m2);
            if (blockIdx.x == 0) st->v[S_DSTS] = R;
        }
    }
}

template <typename K, bool HAS_V>
constexpr const char* onesweep_name() {
    if constexpr (sizeof(K) == 4 && HAS_V) return "k_onesweep<u32 key, u64 value>";
    else if constexpr (sizeof(K) == 4) return "k_onesweep<u32 key>";
    else if constexpr (HAS_V) return "k_onesweep<u64 key, u64 value>";
    else return "k_onesweep<u64 key>";
}

template <typename K, bool HAS_V, int LOAD, int NT, int IT, int RANK, int RB>
void launch_onesweep_nt(const SortIn& in, K* kout, u64* vout, u64 n, int shift, const u64* offs, u64* status,
                        u32* tile_counter, u32 tag, DevStats* st, Tracer* tr, cudaStream_t s, u64* cursor) {
    const size_t smem = sizeof(ScatterSmem<K, HAS_V, NT, IT, RB, RANK == RANK_UNSTABLE>);
    const u32 resident = (u32)resident_ctas((const void*)k_onesweep<K, HAS_V, LOAD, NT, IT, RANK, RB>, NT, smem);
    constexpr u64 tile = (u64)NT * IT;
    const u64 tiles = (n + tile - 1) / tile;
    if (tiles == 0) return;
    const unsigned grid = (unsigned)std::min<u64>(tiles, resident);
    TraceScope ts(tr, in.trace_name ? in.trace_name : onesweep_name<K, HAS_V>(), s);
    k_onesweep<K, HAS_V, LOAD, NT, IT, RANK, RB><<<grid, NT, smem, s>>>(
        in, kout, vout, n, shift, offs, status, tile_counter, tag, st, (u32)NS_ONESWEEP_PF * resident, cursor);
}

// Keys without values use 8192-key tiles (512 threads): half the look-back
// hops and per-tile fixed work per key; pairs keep 4096-key tiles (their
// shared memory would not fit twice).  `rank` picks the ranking (RANK_*;
// RANK_UNSTABLE for keys only).
// `cursor` (RANK_UNSTABLE only): per digit, the next free global slot.
// `bits`: the pass's digit width.  8 for every sort; 64-bit keys without
// values also take the wide plan's 10-bit first pass (unstable) and 9-bit
// stable passes (warp match).
template <typename K, bool HAS_V, int LOAD, int NT, int IT>
void launch_onesweep_rank(const SortIn& in, K* kout, u64* vout, u64 n, int shift, const u64* offs, u64* status,
                          u32* tile_counter, u32 tag, DevStats* st, Tracer* tr, cudaStream_t s, int rank,
                          u64* cursor, int bits) {
    if constexpr (!HAS_V && sizeof(K) == 8) {
        if (bits == 10) {
            launch_onesweep_nt<K, HAS_V, LOAD, NT, IT, RANK_UNSTABLE, 10>(in, kout, vout, n, shift, offs, status,
                                                                           tile_counter, tag, st, tr, s, cursor);
            return;
        }
        if (bits == 9) {
            launch_onesweep_nt<K, HAS_V, LOAD, NT, IT, RANK_MATCH, 9>(in, kout, vout, n, shift, offs, status,
                                                                       tile_counter, tag, st, tr, s, nullptr);
            return;
        }
    }
    if constexpr (!HAS_V) {
        if (rank == RANK_UNSTABLE) {
            launch_onesweep_nt<K, HAS_V, LOAD, NT, IT, RANK_UNSTABLE, 8>(in, kout, vout, n, shift, offs, status,
                                                                          tile_counter, tag, st, tr, s, cursor);
            return;
        }
    }
    if (rank == RANK_BALLOT)
        launch_onesweep_nt<K, HAS_V, LOAD, NT, IT, RANK_BALLOT, 8>(in, kout, vout, n, shift, offs, status,
                                                                    tile_counter, tag, st, tr, s, nullptr);
    else
        launch_onesweep_nt<K, HAS_V, LOAD, NT, IT, RANK_MATCH, 8>(in, kout, vout, n, shift, offs, status,
                                                                   tile_counter, tag, st, tr, s, nullptr);
}

// `shape` (64-bit keys without values): the tile of a digit pass, 512
// threads x 16 keys (0, the default), 512 x 12 (1) or 256 x 16 (2).  The
// path tuner picks one per window size.
template <typename K, bool HAS_V, int LOAD>
void launch_onesweep(const SortIn& in, K* kout, u64* vout, u64 n, int shift, const u64* offs, u64* status,
                     u32* tile_counter, u32 tag, DevStats* st, Tracer* tr, cudaStream_t s, int rank,
                     u64* cursor = nullptr, int shape = 0, int bits = 8) {
    if constexpr (!HAS_V && sizeof(K) == 8) {
        if (shape == 1)
            launch_onesweep_rank<K, HAS_V, LOAD, 512, 12>(in, kout, vout, n, shift, offs, status, tile_counter, tag,
                                                          st, tr, s, rank, cursor, bits);
        else if (shape == 2)
            launch_onesweep_rank<K, HAS_V, LOAD, 256, 16>(in, kout, vout, n, shift, offs, status, tile_counter, tag,
                                                          st, tr, s, rank, cursor, bits);
        else
            launch_onesweep_rank<K, HAS_V, LOAD, NS_ONESWEEP_NT, NS_ONESWEEP_ITEMS>(
                in, kout, vout, n, shift, offs, status, tile_counter, tag, st, tr, s, rank, cursor, bits);
    } else if constexpr (!HAS_V)
        launch_onesweep_rank<K, HAS_V, LOAD, NS_ONESWEEP_NT, NS_ONESWEEP_ITEMS>(
            in, kout, vout, n, shift, offs, status, tile_counter, tag, st, tr, s, rank, cursor, 8);
    else
        launch_onesweep_rank<K, HAS_V, LOAD, 256, kItems>(in, kout, vout, n, shift, offs, status, tile_counter, tag,
                                                          st, tr, s, rank, cursor, 8);
}

template <int KEYMODE, bool HAS_V>
void launch_runs_t(const void* keys, const u64* vals, u64 n, const u64* n_dev, u64* head_keys, u64* pos, u64* psum,
                   u64* status_c, u64* status_s, u32* tile_counter, u32 tag, u64* R_out, DevStats* st,
                   Tracer* tr, cudaStream_t s, u64* pack_out) {
    constexpr int kRunThreads = RunShape<HAS_V>::threads, kRunTile = RunShape<HAS_V>::tile;
    const size_t smem = sizeof(RunsSmem<HAS_V>);
    const u32 resident = (u32)resident_ctas((const void*)k_runs<KEYMODE, HAS_V>, kRunThreads, smem);
    u64 tiles = (n + kRunTile - 1) / kRunTile;
    if (tiles == 0) tiles = 1;
    tiles = std::min<u64>(tiles, resident);
    TraceScope ts(tr, KEYMODE == RUN_U64 ? "k_runs<links>" : (KEYMODE == RUN_SRC_OF_U64 ? "k_runs<rows>" : "k_runs<cols>"),
                  s);
    const bool aligned = (((uintptr_t)keys | (uintptr_t)vals) & 15) == 0;
    const u32 pf = aligned ? (u32)NS_RUNS_PF * resident : 0u;
    k_runs<KEYMODE, HAS_V><<<(unsigned)tiles, kRunThreads, smem, s>>>(
        keys, vals, n, n_dev, head_keys, pos, psum, status_c, status_s, tile_counter, tag, R_out, st, pack_out, pf);
}

// Diagnostics: the library's bounded waits run against something nothing
// will ever signal -- a look-back status word that is never published, an
// mbarrier phase expecting bytes that no copy delivers -- so that they time
// out and record ERR_TIMEOUT.  No fault, trap or unbounded wait is involved.
__global__ void k_diag_lookback(u64* status, DevStats* st) {
    if (threadIdx.x == 0) lookback<8>(status, 1, 1, 0x7777u, st);
}

__global__ void k_diag_lookback_warp(u64* status, DevStats* st) {
    warp_lookback(status, 1, 0x7777u, st);  // tile 1 waits on status[0], never published
}

__global__ void k_diag_mbarrier(DevStats* st) {
    __shared__ u64 bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, 64);  // no copy will deliver these bytes
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, st);
}

}  // namespace

u64 sort_tiles(u64 n) { return (n + kTile - 1) / kTile; }
int resident_ctas_of(const void* fn, int threads, size_t smem) { return resident_ctas(fn, threads, smem); }
int sort_radix(int digit_plan) { return digit_plan == kDigitsWide ? kWideStableRadix : kRadix; }

// Sort n keys by bits [begin_bit, begin_bit + 8*passes).  Pass p reads
// buffer (p == 0 ? the input : bufs[(p-1)&1]) and writes bufs[p&1].
// Returns the index (0 or 1) of the buffer holding the result.  With the
// wide digit plan (sc.digit_plan), 64-bit keys alone sorted on all 64 bits
// take seven passes (10 bits, then six of 9) instead of eight.
template <typename K, bool HAS_V, int LOAD>
int radix_sort_t(const SortIn& in, K* kbuf[2], u64* vbuf[2], u64 n, int begin_bit, int passes,
                 SortScratch& sc, DevStats* st, cudaStream_t s) {
    // 64-bit keys alone, sorted on every bit, may take the wide digit plan
    const bool wide = sc.digit_plan == kDigitsWide && !HAS_V && sizeof(K) == 8 && passes == 8 && begin_bit == 0;
    cudaMemsetAsync(sc.ghist, 0, sizeof(u64) * (wide ? kWideBins : 8 * kRadix), s);
    cudaMemsetAsync(sc.tile_counters, 0, sizeof(u32) * 8, s);
    if constexpr (!HAS_V && sizeof(K) == 8) {
        if (wide) launch_hist_wide<K, LOAD>(in, n, sc.ghist, sc.tr, s);
    }
    if (!wide) {
        if (passes == 8)
            launch_hist<K, LOAD, 8>(in, n, begin_bit, sc.ghist, sc.tr, s);
        else  // 4: 32-bit keys, or one half of 64-bit ones
            launch_hist<K, LOAD, 4>(in, n, begin_bit, sc.ghist, sc.tr, s);
    }
    {
        TraceScope ts(sc.tr, "k_sort_offsets", s);
        if (wide) k_sort_offsets_wide<<<1, 1024, 0, s>>>(sc.ghist, sc.offs);
        else k_sort_offsets<<<1, kThreads, 0, s>>>(sc.ghist, passes, sc.offs);
    }
    if (wide) passes = kWidePasses;
    // a pass's tiles hold 4096 keys or more, so its status words are within
    // the first sort_tiles(n) * (its radix)
    const u64 status_used =
        std::min<u64>(sort_tiles(std::max<u64>(n, 1)) * (wide ? kWideStableRadix : kRadix), sc.status_words);
    for (int p = 0; p < passes; ++p) {
        const u32 tag = next_tag(sc, s);
        clear_status_in_capture(sc.status, status_used, s);
        if (wide) {
            SortIn mid{};
            if (p > 0) {
                mid.keys = kbuf[(p - 1) & 1];
                mid.n_dev = in.n_dev;
                mid.trace_name = in.trace_name;
                mid.bulk = ((uintptr_t)kbuf[(p - 1) & 1] & 15) == 0;
            }
            if constexpr (!HAS_V && sizeof(K) == 8) {
                if (p == 0)
                    launch_onesweep<K, HAS_V, LOAD>(in, kbuf[0], vbuf[0], n, wide_shift(0), sc.offs, sc.status,
                                                    sc.tile_counters + p, tag, st, sc.tr, s, RANK_UNSTABLE,
                                                    sc.offs + kWideBins, sc.tile_shape, wide_bits(0));
                else
                    launch_onesweep<K, HAS_V, LOAD_KEYS>(mid, kbuf[p & 1], vbuf[p & 1], n, wide_shift(p),
                                                         sc.offs + wide_base(p), sc.status, sc.tile_counters + p,
                                                         tag, st, sc.tr, s, RANK_MATCH, nullptr, sc.tile_shape,
                                                         wide_bits(p));
            }
            continue;
        }
        const int shift = begin_bit + 8 * p;
        if (p == 0) {
            // The first pass of a keys-only sort need not be stable: its
            // input order carries no information.  (Keys equal in the sorted
            // bits then come out in any order; no caller relies on theirs.)
            launch_onesweep<K, HAS_V, LOAD>(in, kbuf[0], vbuf[0], n, shift, sc.offs, sc.status,
                                            sc.tile_counters + p, tag, st, sc.tr, s,
                                            !HAS_V && NS_UNSTABLE_FIRST ? RANK_UNSTABLE : pass_rank(0),
                                            sc.offs + 8 * kRadix, sc.tile_shape);
        } else {
            SortIn mid{};
            mid.keys = kbuf[(p - 1) & 1];
            mid.vals = vbuf[(p - 1) & 1];
            mid.n_dev = in.n_dev;
            mid.trace_name = in.trace_name;
            // a caller's output buffer can be one of the ping-pong buffers:
            // stage with bulk copies only from 16-byte-aligned addresses
            mid.bulk = (((uintptr_t)kbuf[(p - 1) & 1] | (uintptr_t)vbuf[(p - 1) & 1]) & 15) == 0;
            launch_onesweep<K, HAS_V, LOAD_KEYS>(mid, kbuf[p & 1], vbuf[p & 1], n, shift, sc.offs + p * kRadix,
                                                 sc.status, sc.tile_counters + p, tag, st, sc.tr, s, pass_rank(p),
                                                 nullptr, sc.tile_shape);
        }
    }
    return (passes - 1) & 1;
}

int radix_sort_packets(const u32* src, const u32* dst, u64* kbuf[2], u64 n,
                       SortScratch& sc, DevStats* st, cudaStream_t s) {
    SortIn in{};
    in.src = src;
    in.dst = dst;
    in.bulk = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0;
    u64* vb[2] = {nullptr, nullptr};
    return radix_sort_t<u64, false, LOAD_PACK>(in, (u64**)kbuf, vb, n, 0, 8, sc, st, s);
}

int radix_sort_keys64(const u64* keys, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                      cudaStream_t s, const char* trace_name) {
    SortIn in{};
    in.keys = keys;
    in.n_dev = n_dev;
    in.bulk = ((uintptr_t)keys & 15) == 0;
    in.trace_name = trace_name;
    u64* vb[2] = {nullptr, nullptr};
    return radix_sort_t<u64, false, LOAD_KEYS>(in, kbuf, vb, n, 0, 8, sc, st, s);
}

int radix_sort_pairs64(const u64* keys, const u64* vals, const u64* n_dev,
                       u64* kbuf[2], u64* vbuf[2], u64 n, SortScratch& sc,
                       DevStats* st, cudaStream_t s) {
    SortIn in{};
    in.keys = keys;
    in.vals = (const u64*)vals;
    in.n_dev = (const u64*)n_dev;
    in.bulk = (((uintptr_t)keys | (uintptr_t)vals) & 15) == 0;
    return radix_sort_t<u64, true, LOAD_KEYS>(in, (u64**)kbuf, (u64**)vbuf, n, 0, 8, sc, st, s);
}

int radix_sort_dst_pairs(const u64* link_keys, const u64* counts, const u64* n_dev,
                         u32* kbuf[2], u64* vbuf[2], u64 n, SortScratch& sc,
                         DevStats* st, cudaStream_t s) {
    SortIn in{};
    in.keys = link_keys;
    in.vals = (const u64*)counts;
    in.n_dev = (const u64*)n_dev;
    return radix_sort_t<u32, true, LOAD_DST_OF>(in, (u32**)kbuf, (u64**)vbuf, n, 0, 4, sc, st, s);
}

int radix_sort_u32(const u32* keys, const u64* n_dev, u32* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                   cudaStream_t s) {
    SortIn in{};
    in.keys = keys;
    in.n_dev = (const u64*)n_dev;
    in.bulk = ((uintptr_t)keys & 15) == 0;
    in.trace_name = "k_onesweep<u32 key>";
    u64* vb[2] = {nullptr, nullptr};
    return radix_sort_t<u32, false, LOAD_KEYS>(in, (u32**)kbuf, vb, n, 0, 4, sc, st, s);
}

int radix_sort_lo32(const u64* keys, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                    cudaStream_t s) {
    SortIn in{};
    in.keys = keys;
    in.n_dev = (const u64*)n_dev;
    in.bulk = ((uintptr_t)keys & 15) == 0;
    in.trace_name = "k_onesweep<u64 key, low half>";
    u64* vb[2] = {nullptr, nullptr};
    return radix_sort_t<u64, false, LOAD_KEYS>(in, (u64**)kbuf, vb, n, 0, 4, sc, st, s);
}

int radix_sort_hi32(const u64* packed, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                    cudaStream_t s, const char* trace_name) {
    SortIn in{};
    in.keys = packed;
    in.n_dev = (const u64*)n_dev;
    in.bulk = ((uintptr_t)packed & 15) == 0;
    in.trace_name = trace_name ? trace_name : "k_onesweep<u64 key, by dst>";
    u64* vb[2] = {nullptr, nullptr};
    return radix_sort_t<u64, false, LOAD_KEYS>(in, (u64**)kbuf, vb, n, 32, 4, sc, st, s);
}

void launch_runs(int keymode, bool has_v, const void* keys, const u64* vals, u64 n,
                 const u64* n_dev, u64* head_keys, u64* pos, u64* psum,
                 u64* R_out, SortScratch& sc, DevStats* st, cudaStream_t s, u64* pack_out) {
    cudaMemsetAsync(sc.tile_counters + 8, 0, sizeof(u32), s);
    const u32 tag = next_tag(sc, s);
    const u64* nd = (const u64*)n_dev;
    u64* sc_c = sc.status;
    u64* sc_s = sc.status + sc.status_words / 2;
    {
        // run tiles hold 1024 keys or more: one count and one sum word each
        const u64 used = std::min<u64>((n + 1023) / 1024 + 1, sc.status_words / 2);
        clear_status_in_capture(sc_c, used, s);
        clear_status_in_capture(sc_s, used, s);
    }
    u32* tc = sc.tile_counters + 8;
    if (keymode == RUN_U64 && !has_v)
        launch_runs_t<RUN_U64, false>(keys, (const u64*)vals, n, nd, (u64*)head_keys, (u64*)pos,
                                      (u64*)psum, sc_c, sc_s, tc, tag, (u64*)R_out, st, sc.tr, s, nullptr);
    else if (keymode == RUN_SRC_OF_U64 && has_v)
        launch_runs_t<RUN_SRC_OF_U64, true>(keys, (const u64*)vals, n, nd, (u64*)head_keys, (u64*)pos,
                                            (u64*)psum, sc_c, sc_s, tc, tag, (u64*)R_out, st, sc.tr, s, pack_out);
    else if (keymode == RUN_U32 && has_v)
        launch_runs_t<RUN_U32, true>(keys, (const u64*)vals, n, nd, (u64*)head_keys, (u64*)pos,
                                     (u64*)psum, sc_c, sc_s, tc, tag, (u64*)R_out, st, sc.tr, s, nullptr);
    else if (keymode == RUN_U32 && !has_v)
        launch_runs_t<RUN_U32, false>(keys, nullptr, n, nd, (u64*)head_keys, (u64*)pos, nullptr, sc_c, sc_s, tc, tag,
                                      (u64*)R_out, st, sc.tr, s, nullptr);
    else if (keymode == RUN_HI_OF_PACKED && has_v)
        launch_runs_t<RUN_HI_OF_PACKED, true>(keys, nullptr, n, nd, (u64*)head_keys, (u64*)pos,
                                              (u64*)psum, sc_c, sc_s, tc, tag, (u64*)R_out, st, sc.tr, s, nullptr);
}

void launch_run_stats(int mode, const u64* pos, const u64* psum, const u64* R_ptr,
                      u64 bound, u64* counts_out, DevStats* st, int sms, Tracer* tr, cudaStream_t s) {
    u64 want = (bound + 255) / 256;
    u64 cap = (u64)sms * 8;
    int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    TraceScope ts(tr, mode == RS_LINKS ? "k_run_stats<links>" : (mode == RS_ROWS ? "k_run_stats<rows>" : "k_run_stats<cols>"),
                  s);
    if (mode == RS_LINKS)
        k_run_stats<RS_LINKS><<<grid, 256, 0, s>>>((const u64*)pos, (const u64*)psum,
                                                  (const u64*)R_ptr, (u64*)counts_out, st);
    else if (mode == RS_ROWS)
        k_run_stats<RS_ROWS><<<grid, 256, 0, s>>>((const u64*)pos, (const u64*)psum,
                                                 (const u64*)R_ptr, (u64*)counts_out, st);
    else
        k_run_stats<RS_COLS><<<grid, 256, 0, s>>>((const u64*)pos, (const u64*)psum,
                                                 (const u64*)R_ptr, (u64*)counts_out, st);
}

}  // namespace ns

namespace ns {
void launch_diag_wait(int which, u64* status_word, DevStats* st, cudaStream_t s) {
    if (which == 0) k_diag_lookback<<<1, 32, 0, s>>>(status_word, st);
    else if (which == 1) k_diag_mbarrier<<<1, 32, 0, s>>>(st);
    else k_diag_lookback_warp<<<1, 32, 0, s>>>(status_word, st);
}
}  // namespace ns
