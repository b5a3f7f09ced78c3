// ns_shard.cu -- the pieces a sharded (several-GPU) traffic matrix needs from
// each rank: A's nonzeros grouped by the rank that owns their source (or
// destination), and the addition of received entries to a matrix.
//
// The decomposition: every rank aggregates its own packets; the entries are
// exchanged so that rank r holds every entry whose source r owns (its rows
// of A are then exact: row quantities are local, links, packets and sources
// add up over the ranks); a second exchange by destination owner gives rank
// r every entry of the destinations it owns (keys are unique across ranks
// after the first exchange, so each received entry is one distinct link of
// that column), whose column quantities are then local too.  The exchange
// itself is the caller's (any transport); this file only groups and adds.
#include <algorithm>
#include <vector>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_common.cuh"
#include "ns_kernels.h"

using namespace ns;

namespace {

// The owner of an address among `parts` ranks: a multiplicative hash of the
// address scaled to [0, parts).  Host and device compute the same integers.
__host__ __device__ __forceinline__ u32 owner_of(u32 addr, u32 parts) {
    const u32 h = addr * 0x9E3779B1u;
    return (u32)(((u64)h * parts) >> 32);
}

constexpr int kPartThreads = 256;
constexpr int kPartItems = 8;
constexpr u64 kPartChunk = (u64)kPartThreads * kPartItems;

__device__ __forceinline__ u32 key_owner(u64 key, int by, u32 parts) {
    return owner_of(by == NS_BY_SRC ? (u32)(key >> 32) : (u32)key, parts);
}

// Per chunk of kPartChunk entries: how many belong to `part`.
__global__ void __launch_bounds__(kPartThreads) k_part_count(const u64* __restrict__ keys, u64 n, int by, u32 parts,
                                                             u32 part, u64* __restrict__ chunk_count) {
    __shared__ u32 wsum[kPartThreads / 32];
    const u64 base = (u64)blockIdx.x * kPartChunk;
    u32 c = 0;
    for (int j = 0; j < kPartItems; ++j) {
        const u64 i = base + (u64)j * kPartThreads + threadIdx.x;
        if (i < n && key_owner(keys[i], by, parts) == part) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int w = 0; w < kPartThreads / 32; ++w) t += wsum[w];
        chunk_count[blockIdx.x] = t;
    }
}

// Exclusive scan of the chunk counts in place (one CTA); total to *total.
__global__ void k_part_scan(u64* __restrict__ chunk_count, u64 chunks, u64* __restrict__ total) {
    __shared__ u64 carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (u64 b = 0; b < chunks; b += blockDim.x) {
        const u64 i = b + threadIdx.x;
        const u64 v = i < chunks ? chunk_count[i] : 0;
        // inclusive scan of the block's values (Hillis-Steele in registers
        // and shared memory)
        __shared__ u64 buf[1024];
        buf[threadIdx.x] = v;
        __syncthreads();
        for (u32 o = 1; o < blockDim.x; o <<= 1) {
            const u64 add = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < chunks) chunk_count[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += buf[blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// The entries of `part`, in their input order, to out + chunk start.
__global__ void __launch_bounds__(kPartThreads) k_part_write(const u64* __restrict__ keys,
                                                             const u64* __restrict__ counts, u64 n, int by,
                                                             u32 parts, u32 part, const u64* __restrict__ chunk_start,
                                                             u64* __restrict__ out_keys, u64* __restrict__ out_counts) {
    __shared__ u32 wsum[kPartThreads / 32];
    __shared__ u32 run;
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u64 base = (u64)blockIdx.x * kPartChunk;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    // rounds of kPartThreads consecutive entries, in order
    for (int j = 0; j < kPartItems; ++j) {
        const u64 i = base + (u64)j * kPartThreads + threadIdx.x;
        const bool mine = i < n && key_owner(keys[i], by, parts) == part;
        const u32 bal = __ballot_sync(0xFFFFFFFFu, mine);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        u32 before = run;
        for (u32 q = 0; q < w; ++q) before += wsum[q];
        if (mine) {
            const u64 at = chunk_start[blockIdx.x] + before + __popc(bal & lanemask_lt());
            out_keys[at] = keys[i];
            out_counts[at] = counts[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 t = 0;
            for (int q = 0; q < kPartThreads / 32; ++q) t += wsum[q];
            run += t;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" {

uint32_t ns_owner(uint32_t addr, uint32_t parts) { return parts ? owner_of(addr, parts) : 0; }

ns_status ns_matrix_partition(ns_ctx* c, const ns_matrix* m, int by, uint32_t parts, uint64_t* d_keys,
                              uint64_t* d_counts, uint64_t cap, uint64_t* h_offsets, ns_stream_t stream) {
    if (!c || !m || !h_offsets) return set_fail(NS_ERR_INVALID, "ns_matrix_partition: NULL argument");
    if (by != NS_BY_SRC && by != NS_BY_DST) return set_fail(NS_ERR_INVALID, "ns_matrix_partition: unknown `by`");
    if (parts == 0) return set_fail(NS_ERR_INVALID, "ns_matrix_partition: parts == 0");
    if (m->ctx != c) return set_fail(NS_ERR_INVALID, "ns_matrix_partition: matrix belongs to another context");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(c, s);
    touch(m, s);
    uint64_t nnz = 0;
    ns_status st = ns_matrix_nnz(m, &nnz, stream);
    if (st != NS_OK) return st;
    for (uint32_t p = 0; p <= parts; ++p) h_offsets[p] = 0;
    if (nnz == 0) return NS_OK;
    if (!d_keys || !d_counts) return set_fail(NS_ERR_INVALID, "ns_matrix_partition: NULL output with nnz > 0");
    if (cap < nnz) return fail_fmt(NS_ERR_CAPACITY, "ns_matrix_partition: cap %llu < nnz %llu",
                                   (unsigned long long)cap, (unsigned long long)nnz);
    // A's nonzero list, ascending, into the context's scratch
    Buf lk, lc, cc;
    st = buf_reserve(lk, nnz * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(lc, nnz * sizeof(u64));
    const u64 chunks = (nnz + kPartChunk - 1) / kPartChunk;
    if (st == NS_OK) st = buf_reserve(cc, (chunks + 1) * sizeof(u64));
    uint64_t got = 0;
    if (st == NS_OK) st = ns_matrix_export(m, (uint64_t*)lk.p, (uint64_t*)lc.p, nnz, &got, stream);
    if (st == NS_OK && got != nnz) st = set_fail(NS_ERR_STATE, "ns_matrix_partition: the matrix changed");
    // one stable compaction per part, the groups back to back
    u64 at = 0;
    for (uint32_t p = 0; p < parts && st == NS_OK; ++p) {
        u64* counts = (u64*)cc.p;
        k_part_count<<<(unsigned)chunks, kPartThreads, 0, s>>>((const u64*)lk.p, nnz, by, parts, p, counts);
        k_part_scan<<<1, 1024, 0, s>>>(counts, chunks, counts + chunks);
        k_part_write<<<(unsigned)chunks, kPartThreads, 0, s>>>((const u64*)lk.p, (const u64*)lc.p, nnz, by, parts,
                                                               p, counts, (u64*)d_keys + at, (u64*)d_counts + at);
        u64 total = 0;
        if (cudaMemcpyAsync(&total, counts + chunks, sizeof(u64), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            st = set_fail(NS_ERR_CUDA, "ns_matrix_partition: group failed");
            break;
        }
        h_offsets[p] = at;
        at += total;
    }
    h_offsets[parts] = at;
    if (st == NS_OK && at != nnz) st = set_fail(NS_ERR_STATE, "ns_matrix_partition: groups do not cover A");
    if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
    buf_free(lk);
    buf_free(lc);
    buf_free(cc);
    return st == NS_OK ? check_launch() : st;
}

ns_status ns_matrix_add_entries(ns_ctx* c, ns_matrix* m, const uint64_t* d_keys, const uint64_t* d_counts,
                                uint64_t n, ns_stream_t stream) {
    if (!c || !m) return set_fail(NS_ERR_INVALID, "ns_matrix_add_entries: NULL argument");
    if (n > 0 && (!d_keys || !d_counts)) return set_fail(NS_ERR_INVALID, "ns_matrix_add_entries: NULL input");
    if (m->ctx != c) return set_fail(NS_ERR_INVALID, "ns_matrix_add_entries: matrix belongs to another context");
    cudaStream_t s = (cudaStream_t)stream;
    CallScope scope(c, s);
    ns_status st = to_hash(m, n, s);
    if (st != NS_OK || n == 0) return st;
    {
        TraceScope ts(&c->tracer, "k_insert_list", s);
        launch_insert_list((const u64*)d_keys, (const u64*)d_counts, n, nullptr, hash_view(m), c->sms, s);
    }
    m->bound += n;
    return check_launch();
}

}  // extern "C"
