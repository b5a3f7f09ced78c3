// ns_nodes.cu -- per-source and per-destination vectors of A, the distinct
// addresses of src and dst together, and address anonymization.
//
// Vectors (Table 2 rows 6 and 8, and their reverses by the Table 2 caption):
// A's sorted nonzero list is taken (exported from a hash matrix, or the sort
// path's own list); runs of equal source give A 1 and |A|_0 1; the (dst,
// count) pairs sorted by dst give 1^T A and 1^T |A|_0.  The distinct
// addresses (section "Graph Analytics": each column's distinct values, the
// common ones once) are the sorted union of the two id lists.
//
// Anonymization (section "Implementation", paragraph "IP Address
// Anonymization"): the distinct addresses of the src and dst columns are
// found with a hash set (the paragraph's hash-table way of `unique`), then
// compacted and sorted; the caller's random keys, one per distinct address,
// are sorted with their positions attached, which yields a uniformly random
// permutation (as the shuffle of 0..N-1 does); every packet's addresses are
// then replaced by their labels, found through a prefix table and a short
// binary search in the sorted distinct addresses (the gather).
#include <algorithm>

#include "ns.h"
#include "ns_api_internal.h"
#include "ns_kernels.h"

using namespace ns;

namespace {

int grid_of(u64 n, int sms) {
    const u64 want = (n + 255) / 256;
    const u64 cap = (u64)sms * 8;
    return (int)std::max<u64>(1, std::min(want, cap));
}

// Vectors from runs: run r starts at pos[r] and ends before pos[r + 1].
// MODE 0: the id is the upper half of a u64 key; MODE 1: the id is a u32 key.
template <int MODE>
__global__ void k_node_vectors(const void* __restrict__ keys, const u64* __restrict__ pos,
                               const u64* __restrict__ psum, const u64* __restrict__ R_ptr, u32* __restrict__ ids,
                               u64* __restrict__ packets, u64* __restrict__ degree, u64 cap) {
    const u64 R = *R_ptr;
    const u64 m = R < cap ? R : cap;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += stride) {
        const u64 p = pos[r];
        if (ids) {
            if constexpr (MODE == 0) ids[r] = (u32)(reinterpret_cast<const u64*>(keys)[p] >> 32);
            else ids[r] = reinterpret_cast<const u32*>(keys)[p];
        }
        if (packets) packets[r] = psum[r + 1] - psum[r];
        if (degree) degree[r] = pos[r + 1] - pos[r];
    }
}

// out[i] = a[i] (i < na), out[na + i] = b[i] (i < nb), widened to u64
__global__ void k_concat_u32(const u32* __restrict__ a, u64 na, const u32* __restrict__ b, u64 nb,
                             u64* __restrict__ out) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride)
        out[i] = i < na ? (u64)a[i] : (u64)b[i - na];
}

// out[r] = (u32) in[r] for r < min(*n_ptr, cap)
__global__ void k_narrow(const u64* __restrict__ in, const u64* __restrict__ n_ptr, u64 cap, u32* __restrict__ out) {
    const u64 n = *n_ptr < cap ? *n_ptr : cap;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (u32)in[i];
}

__global__ void k_iota(u64* __restrict__ out, u64 n) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = i;
}

// order[t] = the position whose random key is the t-th smallest: its label is t
__global__ void k_labels(const u64* __restrict__ order, u64 n, u32* __restrict__ label) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const u64 i = order[t];
        if (i < n) label[i] = (u32)t;
    }
}

// The gather looks an address up in two steps: a table over the top
// kBucketBits bits gives the range of the ascending distinct list that holds
// that prefix (bucket[b] = the first position whose address has prefix >= b),
// and a binary search inside the range finds the address.  Addresses are
// spread over all 32 bits, so a range holds a few entries even with tens of
// millions of distinct addresses, and the 32 MiB table stays in L2.
constexpr int kBucketBits = 22;
// the set tables up to which the gather goes through the set (2^25 slots:
// the first table of any window of more than 2^23 packets)
constexpr u64 kSetLabelMaxSlots = 1ull << 25;

__global__ void k_buckets(const u64* __restrict__ u, u64 N, u64* __restrict__ bucket) {
    const u64 nb = 1ull << kBucketBits;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 b = (u64)blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += stride) {
        // first position with (u >> (32 - kBucketBits)) >= b
        u64 lo = 0, hi = N;
        while (lo < hi) {
            const u64 mid = (lo + hi) >> 1;
            if ((u[mid] >> (32 - kBucketBits)) < b) lo = mid + 1;
            else hi = mid;
        }
        bucket[b] = lo;
    }
}

// u[i] := u[i] << 32 | label[i]: each distinct address carries its label,
// so the lookup that finds it needs no further load
__global__ void k_attach_labels(u64* __restrict__ u, const u32* __restrict__ label, u64 N) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) u[i] = (u[i] << 32) | label[i];
}

// the label of x, whose word is in the ascending list w[0..N) of
// (address << 32 | label) (x is in it)
__device__ __forceinline__ u32 find_label(const u64* __restrict__ w, const u64* __restrict__ bucket, u64 N, u32 x) {
    const u32 b = x >> (32 - kBucketBits);
    u64 lo = bucket[b], hi = bucket[b + 1];
    while (lo < hi) {
        const u64 mid = (lo + hi) >> 1;
        if ((u32)(w[mid] >> 32) < x) lo = mid + 1;
        else hi = mid;
    }
    return (u32)w[lo < N ? lo : N - 1];
}

__global__ void k_relabel(const u32* src, const u32* dst, u64 n, const u64* __restrict__ w,
                          const u64* __restrict__ bucket, u64 N, u32* out_src, u32* out_dst) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const u32 a = src[k], b = dst[k];
        out_src[k] = find_label(w, bucket, N, a);
        out_dst[k] = find_label(w, bucket, N, b);
    }
}

// ---- the distinct addresses of both columns, by hashing ---------------------
//
// A set of addresses in open addressing: a slot holds address + 1 (0 =
// empty); the address 0xFFFFFFFF sets a flag word instead.  Slots only ever
// go from empty to an address, so a plain (possibly cached) load that shows
// the address is final, and one that shows empty is settled by the CAS.
// Skewed traffic repeats a few addresses, whose slots stay in L1/L2; the
// distinct ones are then compacted and sorted, which is far less work than
// sorting both columns.  When the distinct addresses outgrow half the table,
// the kernel stops early and the host retries with a table for every
// address being distinct.
struct SetCounters {
    u64 inserted;  // distinct addresses placed so far
    u64 all_ones;  // address 0xFFFFFFFF seen
    u64 full;      // more than half the slots taken: abandon this table
    u64 out;       // compaction cursor
};

__global__ void k_set_insert(const u32* __restrict__ src, const u32* __restrict__ dst, u64 n, u32* __restrict__ T,
                             u64 mask, SetCounters* sc, DevStats* st) {
    const u32 FULL = 0xFFFFFFFFu;
    const u64 limit = (mask + 1) / 2;
    const u64 total = 2 * n;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 wbase = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    u32 iter = 0;
    for (u64 b = wbase; b < total; b += stride, ++iter) {
        if ((iter & 15) == 0 && ld_volatile(&sc->full)) return;  // whole warps leave together
        const u64 i = b + (threadIdx.x & 31);
        bool inserted = false, ones = false;
        if (i < total) {
            const u32 x = i < n ? src[i] : dst[i - n];
            if (x == 0xFFFFFFFFu) {
                ones = true;
            } else {
                const u32 v = x + 1;
                u64 h = mix32(x) & mask;
                u32 p = 0;
                for (; p < kMaxProbes; ++p) {
                    const u32 cur = T[h];
                    if (cur == v) break;
                    if (cur == 0u) {
                        const u32 old = atomicCAS(&T[h], 0u, v);
                        if (old == 0u) {
                            inserted = true;
                            break;
                        }
                        if (old == v) break;
                    }
                    h = (h + 1) & mask;
                }
                if (p == kMaxProbes) set_error(st, ERR_CAPACITY);
            }
        }
        const u32 ins = __ballot_sync(FULL, inserted);
        if (__any_sync(FULL, ones) && (threadIdx.x & 31) == 0 && !ld_volatile(&sc->all_ones)) sc->all_ones = 1;
        if (ins && (threadIdx.x & 31) == 0) {
            const u64 before = atomicAdd((unsigned long long*)&sc->inserted, (unsigned long long)__popc(ins));
            if (before + __popc(ins) > limit) st_volatile(&sc->full, 1ull);
        }
    }
}

// out[k] = the addresses in the set, in slot order (then sorted)
__global__ void k_set_compact(const u32* __restrict__ T, u64 cap, SetCounters* sc, u32* __restrict__ out) {
    const u32 FULL = 0xFFFFFFFFu;
    const u32 lane = threadIdx.x & 31;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 wbase = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (u64 b = wbase; b < cap; b += stride) {
        const u64 i = b + lane;
        const u32 v = i < cap ? T[i] : 0u;
        const u32 has = __ballot_sync(FULL, v != 0u);
        if (!has) continue;
        u64 base = 0;
        if (lane == 0) base = atomicAdd((unsigned long long*)&sc->out, (unsigned long long)__popc(has));
        base = __shfl_sync(FULL, base, 0);
        if (v != 0u) out[base + __popc(has & ((1u << lane) - 1u))] = v - 1u;
    }
}

// The gather through the address set itself, when its table is the first,
// L2-sized one: TL[h] = label << 32 | (address + 1) for every occupied slot h
// of the set (its label found once, by the search below), 0 elsewhere.  A
// packet's address then finds its label by the same probe sequence that
// inserted it: usually one line of TL, instead of the prefix table and a
// binary search.
__global__ void k_set_labels(const u32* __restrict__ T, u64 cap, const u64* __restrict__ w,
                             const u64* __restrict__ bucket, u64 N, u64* __restrict__ TL) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 h = (u64)blockIdx.x * blockDim.x + threadIdx.x; h < cap; h += stride) {
        const u32 v = T[h];
        TL[h] = v ? ((u64)find_label(w, bucket, N, v - 1u) << 32) | v : 0ull;
    }
}

__device__ __forceinline__ u32 set_label(const u64* __restrict__ TL, u64 mask, u32 x, const u64* __restrict__ w,
                                         const u64* __restrict__ bucket, u64 N) {
    if (x != 0xFFFFFFFFu) {  // (that address has no slot: it sets a flag word)
        const u32 v = x + 1u;
        u64 h = mix32(x) & mask;
        for (u32 p = 0; p < kMaxProbes; ++p) {
            const u64 t = TL[h];
            if ((u32)t == v) return (u32)(t >> 32);
            h = (h + 1) & mask;
        }
    }
    return find_label(w, bucket, N, x);  // every address of the columns has a slot, so only 0xFFFFFFFF gets here
}

__global__ void k_relabel_set(const u32* src, const u32* dst, u64 n, const u64* __restrict__ TL, u64 mask,
                              const u64* __restrict__ w, const u64* __restrict__ bucket, u64 N, u32* out_src,
                              u32* out_dst) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const u32 a = src[k], b = dst[k];
        out_src[k] = set_label(TL, mask, a, w, bucket, N);
        out_dst[k] = set_label(TL, mask, b, w, bucket, N);
    }
}

// Device scratch of one blocking call; freed on every return path.
struct Scratch {
    Buf b[8];
    ~Scratch() {
        for (Buf& x : b) buf_free(x);
    }
};

ns_status read_u64(const u64* d, u64* h, cudaStream_t s) {
    if (cudaMemcpyAsync(h, d, sizeof(u64), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_fail(NS_ERR_CUDA, "device read failed");
    return NS_OK;
}

// Errors the sort and run kernels recorded in the call's statistics record.
ns_status check_errors(const DevStats* d, cudaStream_t s) {
    DevStats h;
    if (cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_fail(NS_ERR_CUDA, "device read failed");
    if (h.err & ERR_TIMEOUT) return set_fail(NS_ERR_TIMEOUT, "a device-side wait gave up (look-back)");
    if (h.err & ERR_CAPACITY) return set_fail(NS_ERR_CAPACITY, "a device-side bound was exceeded");
    return NS_OK;
}

}  // namespace

extern "C" {

ns_status ns_matrix_nodes(ns_ctx* c, const ns_matrix* m, int which, uint32_t* d_ids, uint64_t* d_packets,
                          uint64_t* d_degree, uint64_t cap, uint64_t* h_count, ns_stream_t stream) {
    if (!c || !m || !h_count) return set_fail(NS_ERR_INVALID, "ns_matrix_nodes: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    touch(m, (cudaStream_t)stream);
    if (which < NS_NODES_SRC || which > NS_NODES_ANY) return set_fail(NS_ERR_INVALID, "ns_matrix_nodes: unknown which");
    if (m->ctx != c) return set_fail(NS_ERR_INVALID, "ns_matrix_nodes: matrix belongs to another context");
    *h_count = 0;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t nnz = 0;
    ns_status st = ns_matrix_nnz(m, &nnz, stream);
    if (st != NS_OK) return st;
    if (nnz == 0) return NS_OK;
    if (cap > 0 && !d_ids && !d_packets && !d_degree) return set_fail(NS_ERR_INVALID, "ns_matrix_nodes: no output");
    // buffers: 0 keys, 1 counts, 2 pos, 3 psum, 4 stats + counters, 5 source ids,
    // 6 destination ids, 7 the union's words
    Scratch x;
    st = buf_reserve(x.b[0], nnz * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x.b[1], nnz * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x.b[2], (nnz + 1) * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x.b[3], (nnz + 1) * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x.b[4], sizeof(DevStats) + 8 * sizeof(u64));
    if (st != NS_OK) return st;
    if (cudaMemsetAsync(x.b[4].p, 0, sizeof(DevStats) + 8 * sizeof(u64), s) != cudaSuccess)
        return set_fail(NS_ERR_CUDA, "ns_matrix_nodes: memset failed");
    uint64_t got = 0;
    st = ns_matrix_export(m, (uint64_t*)x.b[0].p, (uint64_t*)x.b[1].p, nnz, &got, stream);
    if (st != NS_OK) return st;
    DevStats* dst_err = (DevStats*)x.b[4].p;
    u64* R = (u64*)((char*)x.b[4].p + sizeof(DevStats));  // R[0] sources, R[1] destinations, R[2] union
    u64* pos = (u64*)x.b[2].p;
    u64* psum = (u64*)x.b[3].p;
    const u64* keys = (const u64*)x.b[0].p;
    const u64* counts = (const u64*)x.b[1].p;
    st = sort_scratch(c, 2 * nnz);
    if (st != NS_OK) return st;
    const int grid = grid_of(nnz, c->sms);
    const bool any = which == NS_NODES_ANY;
    if (any) {
        st = buf_reserve(x.b[5], nnz * sizeof(u32));
        if (st == NS_OK) st = buf_reserve(x.b[6], nnz * sizeof(u32));
        if (st != NS_OK) return st;
    }
    if (which == NS_NODES_SRC || any) {
        // runs of equal source over the source-major list
        launch_runs(RUN_SRC_OF_U64, true, keys, counts, nnz, nullptr, nullptr, pos, psum, R + 0, c->sc, dst_err, s);
        u32* ids = any ? (u32*)x.b[5].p : d_ids;
        k_node_vectors<0><<<grid, 256, 0, s>>>(keys, pos, psum, R + 0, ids, any ? nullptr : (u64*)d_packets,
                                               any ? nullptr : (u64*)d_degree, any ? nnz : cap);
    }
    if (which == NS_NODES_DST || any) {
        // (dst, count) pairs sorted by dst, then runs of equal destination
        st = buf_reserve(c->k32[0], nnz * sizeof(u32));
        if (st == NS_OK) st = buf_reserve(c->k32[1], nnz * sizeof(u32));
        if (st == NS_OK) st = buf_reserve(c->v64[0], nnz * sizeof(u64));
        if (st == NS_OK) st = buf_reserve(c->v64[1], nnz * sizeof(u64));
        if (st != NS_OK) return st;
        u32* ck[2] = {(u32*)c->k32[0].p, (u32*)c->k32[1].p};
        u64* cv[2] = {(u64*)c->v64[0].p, (u64*)c->v64[1].p};
        const int r2 = radix_sort_dst_pairs(keys, counts, nullptr, ck, cv, nnz, c->sc, dst_err, s);
        launch_runs(RUN_U32, true, ck[r2], cv[r2], nnz, nullptr, nullptr, pos, psum, R + 1, c->sc, dst_err, s);
        u32* ids = any ? (u32*)x.b[6].p : d_ids;
        k_node_vectors<1><<<grid, 256, 0, s>>>(ck[r2], pos, psum, R + 1, ids, any ? nullptr : (u64*)d_packets,
                                               any ? nullptr : (u64*)d_degree, any ? nnz : cap);
    }
    if (cudaGetLastError() != cudaSuccess) return set_fail(NS_ERR_CUDA, "ns_matrix_nodes: launch failed");
    u64 count = 0;
    if (!any) {
        st = read_u64(R + (which == NS_NODES_SRC ? 0 : 1), &count, s);
        if (st != NS_OK) return st;
    } else {
        u64 S = 0, D = 0;
        st = read_u64(R + 0, &S, s);
        if (st == NS_OK) st = read_u64(R + 1, &D, s);
        if (st != NS_OK) return st;
        const u64 both = S + D;
        st = buf_reserve(x.b[7], both * sizeof(u64));
        if (st == NS_OK) st = buf_reserve(x.b[2], (both + 1) * sizeof(u64));  // run positions of the union
        if (st == NS_OK) st = buf_reserve(c->k64[0], both * sizeof(u64));
        if (st == NS_OK) st = buf_reserve(c->k64[1], both * sizeof(u64));
        if (st == NS_OK) st = buf_reserve(c->xk, both * sizeof(u64));
        if (st != NS_OK) return st;
        k_concat_u32<<<grid_of(both, c->sms), 256, 0, s>>>((const u32*)x.b[5].p, S, (const u32*)x.b[6].p, D,
                                                            (u64*)x.b[7].p);
        u64* kb[2] = {(u64*)c->k64[0].p, (u64*)c->k64[1].p};
        const int r = radix_sort_lo32((const u64*)x.b[7].p, nullptr, kb, both, c->sc, dst_err, s);
        // the distinct words, ascending, as the run heads' keys
        launch_runs(RUN_U64, false, kb[r], nullptr, both, nullptr, (u64*)c->xk.p, (u64*)x.b[2].p, nullptr, R + 2,
                    c->sc, dst_err, s);
        if (d_ids) k_narrow<<<grid_of(both, c->sms), 256, 0, s>>>((const u64*)c->xk.p, R + 2, cap, d_ids);
        if (cudaGetLastError() != cudaSuccess) return set_fail(NS_ERR_CUDA, "ns_matrix_nodes: launch failed");
        st = read_u64(R + 2, &count, s);
        if (st != NS_OK) return st;
    }
    st = check_errors(dst_err, s);
    if (st != NS_OK) return st;
    *h_count = count;
    if (count > cap)
        return fail_fmt(NS_ERR_CAPACITY, "ns_matrix_nodes: %llu entries, cap %llu (first cap written)",
                        (unsigned long long)count, (unsigned long long)cap);
    return NS_OK;
}

ns_status ns_anonymize(ns_ctx* c, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n, const uint64_t* d_rand,
                       uint64_t rand_count, uint32_t* d_out_src, uint32_t* d_out_dst, uint64_t* h_unique,
                       ns_stream_t stream) {
    if (!c || !h_unique) return set_fail(NS_ERR_INVALID, "ns_anonymize: NULL argument");
    CallScope scope(c, (cudaStream_t)stream);
    *h_unique = 0;
    if (n == 0) return NS_OK;
    if (!d_src || !d_dst || !d_out_src || !d_out_dst) return set_fail(NS_ERR_INVALID, "ns_anonymize: NULL column");
    if (n >= (1ull << 39)) return set_fail(NS_ERR_INVALID, "ns_anonymize: n too large");
    cudaStream_t s = (cudaStream_t)stream;
    const u64 m2 = 2 * n;
    // 0 the address set, 1 stats + set counters, 2 the gather's prefix table,
    // 3 the distinct addresses (unsorted, then sorted ping-pong)
    Scratch x;
    ns_status st = buf_reserve(x.b[1], sizeof(DevStats) + sizeof(SetCounters));
    if (st != NS_OK) return st;
    DevStats* err = (DevStats*)x.b[1].p;
    SetCounters* setc = (SetCounters*)((char*)x.b[1].p + sizeof(DevStats));
    // 1. the distinct addresses of both columns: a hash set sized for up to
    // 2^24 of them first, and for every address being distinct if that
    // overflows; then compaction, and a sort of the distinct ones
    const u64 first = std::min<u64>(m2, 1ull << 24);
    u64 cap = 0;
    SetCounters hs{};
    for (int attempt = 0; attempt < 2; ++attempt) {
        const u64 want = attempt == 0 ? first : m2;
        cap = 1024;
        while (cap < 2 * want) cap <<= 1;
        st = buf_reserve(x.b[0], cap * sizeof(u32));
        if (st != NS_OK) return st;
        if (cudaMemsetAsync(x.b[0].p, 0, cap * sizeof(u32), s) != cudaSuccess ||
            cudaMemsetAsync(x.b[1].p, 0, sizeof(DevStats) + sizeof(SetCounters), s) != cudaSuccess)
            return set_fail(NS_ERR_CUDA, "ns_anonymize: memset failed");
        {
            TraceScope t(&c->tracer, "k_set_insert", s);
            k_set_insert<<<grid_of(m2, c->sms), 256, 0, s>>>(d_src, d_dst, n, (u32*)x.b[0].p, cap - 1, setc, err);
        }
        if (cudaGetLastError() != cudaSuccess) return set_fail(NS_ERR_CUDA, "ns_anonymize: launch failed");
        if (cudaMemcpyAsync(&hs, setc, sizeof hs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return set_fail(NS_ERR_CUDA, "ns_anonymize: device read failed");
        if (!hs.full) break;
        if (attempt == 1) return set_fail(NS_ERR_CAPACITY, "ns_anonymize: address set overflowed");
    }
    st = check_errors(err, s);
    if (st != NS_OK) return st;
    const u64 N = hs.inserted + (hs.all_ones ? 1 : 0);
    *h_unique = N;
    if (!d_rand || rand_count < N)
        return fail_fmt(NS_ERR_CAPACITY, "ns_anonymize: %llu distinct addresses, %llu random keys",
                        (unsigned long long)N, (unsigned long long)rand_count);
    st = buf_reserve(x.b[3], std::max<u64>(N, 1) * sizeof(u32));
    if (st == NS_OK) st = buf_reserve(c->k32[0], std::max<u64>(N, 1) * sizeof(u32));
    if (st == NS_OK) st = buf_reserve(c->k32[1], std::max<u64>(N, 1) * sizeof(u32));
    if (st == NS_OK) st = buf_reserve(c->xk, std::max<u64>(N, 1) * sizeof(u64));
    if (st == NS_OK) st = sort_scratch(c, N);
    if (st != NS_OK) return st;
    {
        TraceScope t(&c->tracer, "k_set_compact", s);
        k_set_compact<<<grid_of(cap, c->sms), 256, 0, s>>>((const u32*)x.b[0].p, cap, setc, (u32*)x.b[3].p);
    }
    if (hs.all_ones) {
        const u32 ones = 0xFFFFFFFFu;
        if (cudaMemcpyAsync((u32*)x.b[3].p + hs.inserted, &ones, sizeof ones, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return set_fail(NS_ERR_CUDA, "ns_anonymize: copy failed");
    }
    u32* kb32[2] = {(u32*)c->k32[0].p, (u32*)c->k32[1].p};
    const int r = radix_sort_u32((const u32*)x.b[3].p, nullptr, kb32, N, c->sc, err, s);
    u64* uniq = (u64*)c->xk.p;
    {
        TraceScope t(&c->tracer, "k_concat_u32", s);
        k_concat_u32<<<grid_of(N, c->sms), 256, 0, s>>>(kb32[r], N, nullptr, 0, uniq);
    }
    if (cudaGetLastError() != cudaSuccess) return set_fail(NS_ERR_CUDA, "ns_anonymize: launch failed");
    // 2. the permutation: positions sorted by their random keys (stable)
    st = buf_reserve(c->psum, (N + 1) * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(c->v64[0], N * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(c->v64[1], N * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(c->k64[0], N * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(c->k64[1], N * sizeof(u64));
    if (st == NS_OK) st = buf_reserve(x.b[2], ((1ull << kBucketBits) + 1) * sizeof(u64));
    if (st == NS_OK) st = sort_scratch(c, N);
    if (st != NS_OK) return st;
    {
        TraceScope t(&c->tracer, "k_iota", s);
        k_iota<<<grid_of(N, c->sms), 256, 0, s>>>((u64*)c->psum.p, N);
    }
    u64* kb[2] = {(u64*)c->k64[0].p, (u64*)c->k64[1].p};
    u64* vb[2] = {(u64*)c->v64[0].p, (u64*)c->v64[1].p};
    const int r2 = radix_sort_pairs64((const u64*)d_rand, (const u64*)c->psum.p, nullptr, kb, vb, N, c->sc, err, s);
    u32* label = (u32*)c->k32[0].p;  // the sorted columns are no longer needed
    {
        TraceScope t(&c->tracer, "k_labels", s);
        k_labels<<<grid_of(N, c->sms), 256, 0, s>>>(vb[r2], N, label);
    }
    // 3. the gather: every address replaced by its label
    u64* bucket = (u64*)x.b[2].p;
    {
        TraceScope t(&c->tracer, "k_buckets", s);
        k_buckets<<<grid_of((1ull << kBucketBits) + 1, c->sms), 256, 0, s>>>(uniq, N, bucket);
    }
    {
        TraceScope t(&c->tracer, "k_attach_labels", s);
        k_attach_labels<<<grid_of(N, c->sms), 256, 0, s>>>(uniq, label, N);
    }
    if (cap <= kSetLabelMaxSlots) {
        // the set's own table, widened to carry the labels (256 MiB at most)
        st = buf_reserve(x.b[4], cap * sizeof(u64));
        if (st != NS_OK) return st;
        u64* TL = (u64*)x.b[4].p;
        {
            TraceScope t(&c->tracer, "k_set_labels", s);
            k_set_labels<<<grid_of(cap, c->sms), 256, 0, s>>>((const u32*)x.b[0].p, cap, uniq, bucket, N, TL);
        }
        TraceScope t(&c->tracer, "k_relabel", s);
        k_relabel_set<<<grid_of(n, c->sms), 256, 0, s>>>(d_src, d_dst, n, TL, cap - 1, uniq, bucket, N, d_out_src,
                                                         d_out_dst);
    } else {
        TraceScope t(&c->tracer, "k_relabel", s);
        k_relabel<<<grid_of(n, c->sms), 256, 0, s>>>(d_src, d_dst, n, uniq, bucket, N, d_out_src, d_out_dst);
    }
    if (cudaGetLastError() != cudaSuccess) return set_fail(NS_ERR_CUDA, "ns_anonymize: launch failed");
    return check_errors(err, s);
}

}  // extern "C"
