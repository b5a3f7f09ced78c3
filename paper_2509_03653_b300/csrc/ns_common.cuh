// ns_common.cuh -- device-side definitions shared by the library's kernels.
//
// Data layout in HBM (all little-endian, 16-byte aligned):
//   link table  LinkSlot[cap + 1]: {key, count}; key = src << 32 | dst.
//               key 0 marks an empty slot, so the one real key equal to 0
//               (src = dst = 0) is kept in the extra slot links[cap].
//               After a kernel completes, a slot is occupied iff count > 0.
//   node tables NodeSlot[cap + 1]: {id + 1 (u32), degree (u32), packets}; an
//               id field of 0 marks an empty slot, so the id 0xFFFFFFFF (whose
//               id + 1 wraps to 0) is kept in the extra slot [cap].  Rows are
//               keyed by src, columns by dst (Table 2 rows 5-9 and their
//               reverses).  A degree is at most the matrix's number of
//               nonzeros; an increment that would pass 2^32 - 1 is reported as
//               ERR_CAPACITY instead of wrapping.
//   statistics  DevStats: the nine Table 2 quantities plus an error word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ns {

typedef unsigned long long u64;
typedef unsigned int u32;

enum : u32 { ERR_CAPACITY = 1u, ERR_TIMEOUT = 2u };

enum {
    S_VALID = 0,
    S_LINKS,
    S_SRCS,
    S_DSTS,
    S_MAX_SRC_PK,
    S_MAX_SRC_FO,
    S_MAX_DST_PK,
    S_MAX_DST_FI,
    S_MAX_LINK,
    S_NFIELDS
};

struct DevStats {
    u64 v[S_NFIELDS];
    u64 err;
    u64 pad[6];  // 128 bytes
};

struct __align__(16) LinkSlot {
    u64 key;
    u64 count;
};

struct __align__(16) NodeSlot {
    u32 id1;     // id + 1, 0 = empty
    u32 degree;  // number of distinct partners (|A|_0 1 or 1^T |A|_0)
    u64 packets; // A 1 or 1^T A
};

// Bounds on device-side loops: a probe sequence or a wait that reaches its
// bound records an error instead of continuing.  Waits are bounded in time
// (about one second of the GPU's global timer) and, as a backstop, in polls.
constexpr u32 kMaxProbes = 1u << 16;
constexpr u32 kMaxSpin = 1u << 24;
constexpr u64 kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ u64 globaltimer_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// 64-bit finalizing mixer (two multiply-xorshift rounds with odd constants).
__device__ __forceinline__ u64 mix64(u64 x) {
    x ^= x >> 32;
    x *= 0xD6E8FEB86659FD93ull;
    x ^= x >> 32;
    x *= 0xD6E8FEB86659FD93ull;
    x ^= x >> 32;
    return x;
}

__device__ __forceinline__ u64 mix32(u32 x) { return mix64((u64)x * 0x9E3779B97F4A7C15ull + 1); }

// Views of a hash-format matrix (passed by value to kernels).
struct HashView {
    LinkSlot* links;
    u64 link_mask;  // cap - 1 (cap a power of two); links[cap] is the key-0 slot
    NodeSlot* rows;
    u64 row_mask;
    NodeSlot* cols;
    u64 col_mask;
    DevStats* stats;
};

__device__ __forceinline__ void set_error(DevStats* st, u32 e) { atomicOr(&st->err, (u64)e); }

// Raw lane index / masks.
__device__ __forceinline__ u32 lane_id() {
    u32 r;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ u32 lanemask_lt() {
    u32 r;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Volatile 64-bit load/store for flags published across CTAs.
__device__ __forceinline__ u64 ld_volatile(const u64* p) {
    return *reinterpret_cast<const volatile u64*>(p);
}
__device__ __forceinline__ void st_volatile(u64* p, u64 v) { *reinterpret_cast<volatile u64*>(p) = v; }

// ---- shared-memory staging with the bulk-copy (TMA) engine ----------------
// A 1-D cp.async.bulk copy moves a contiguous global range into shared memory
// and signals an mbarrier; both addresses must be 16-byte aligned and the
// size a multiple of 16 bytes.

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// A hint to pull [src, src + bytes) from HBM into L2; src 16-byte aligned,
// bytes a multiple of 16.  Nothing waits for it.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(u64* bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for an mbarrier phase.  If the bound is reached the error is
// recorded and the wait continues, again bounded, so that no copy is still
// landing in shared memory when the CTA retires.
constexpr u32 kMaxBarrierPolls = 1u << 26;
// Returns true once the phase completed; false (with ERR_TIMEOUT recorded)
// if it did not within the bounds.
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, u32 parity, DevStats* st) {
    u64 t0 = 0;
    for (u32 i = 0; i < kMaxBarrierPolls; ++i) {
        if (mbar_test_wait(bar, parity)) return true;
        if (i > 64) {
            const u64 now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitLimitNs) break;
            __nanosleep(32);
        }
    }
    set_error(st, ERR_TIMEOUT);
    t0 = globaltimer_ns();
    for (u32 i = 0; i < kMaxBarrierPolls; ++i) {
        if (mbar_test_wait(bar, parity)) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
        __nanosleep(64);
    }
    return false;
}

}  // namespace ns
