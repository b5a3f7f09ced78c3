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

// Bounds on device-side loops: a probe sequence or a spin that reaches its
// bound records an error instead of continuing.
constexpr u32 kMaxProbes = 1u << 16;
constexpr u32 kMaxSpin = 1u << 24;

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

}  // namespace ns
