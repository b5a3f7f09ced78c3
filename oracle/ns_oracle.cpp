/*
 * ns_oracle.cpp -- plain, slow, obviously correct CPU oracle for the
 * traffic-matrix hot path.  TEST INFRASTRUCTURE ONLY: it is called by the test
 * suite, by the package's smoke check and by the benchmark's CPU-baseline
 * leg, never by the library.  It shares no code with the CUDA path.
 *
 * What it computes (paper, Table 2 and its caption; section "Implementation",
 * paragraph "Graph Analytics"):
 *   A_t(i,j)   = number of packets from source i to destination j    (Table 2 row 3)
 *   valid      = sum_ij A(i,j)                      = 1^T A 1         (row 1)
 *   links      = sum_ij |A(i,j)|_0                  = 1^T |A|_0 1     (row 2)
 *   max link   = max_ij A(i,j)                                        (row 4)
 *   sources    = sum_i |sum_j A(i,j)|_0             = 1^T |A 1|_0     (row 5)
 *   src pkts   = max_i sum_j A(i,j)                 = max(A 1)        (rows 6-7)
 *   fan-out    = max_i sum_j |A(i,j)|_0             = max(|A|_0 1)    (rows 8-9)
 *   and the reverse operations with src and dst exchanged (Table 2 caption):
 *   destinations = 1^T |1^T A|_0, dst pkts = max(1^T A), fan-in = max(1^T |A|_0).
 * Windows are summed: A = sum_t A_t, which is the matrix of the concatenated
 * packet stream.  A maximum over an empty set is 0.
 *
 * Method, in the order the definitions suggest and nothing cleverer:
 *   1. key = (src << 32) | dst for every packet; std::sort the keys;
 *      one linear scan emits each distinct key with its run length.  This is
 *      A's nonzero list, ascending by key (source-major).
 *   2. Scalars of the whole matrix from that list.
 *   3. Rows: runs of equal (key >> 32) in the sorted list.
 *   4. Columns: the (dst, count) pairs std::sort-ed by dst, then runs.
 * Accumulation (A += A_t) merges two sorted nonzero lists, adding the counts
 * of equal keys.
 *
 * The all-cores variants (oracle_build_parallel, oracle_stats_parallel) use
 * the same steps on every host core and nothing else: the packets are cut
 * into one chunk per thread, each chunk's matrix is built by oracle_build,
 * and the chunk matrices are summed pairwise by oracle_accumulate -- the
 * matrix of a concatenated stream is the sum of its pieces' matrices, the
 * summation rule above.  Columns: each thread sorts the (dst, count) pairs of
 * one slice of the nonzero list and sums equal destinations; the per-slice
 * lists are then merged pairwise, adding the sums of equal destinations.
 *
 * Every count is uint64; no floating point is involved.
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <utility>
#include <vector>

namespace {

/* Fields of the statistics record, in this order. */
enum {
    VALID_PACKETS = 0,
    UNIQUE_LINKS,
    UNIQUE_SOURCES,
    UNIQUE_DESTINATIONS,
    MAX_SRC_PACKETS,
    MAX_SRC_FANOUT,
    MAX_DST_PACKETS,
    MAX_DST_FANIN,
    MAX_LINK_PACKETS,
    N_FIELDS
};

}  // namespace

extern "C" {

/* Step 1: A_t's sorted nonzero list from n packets.  keys_out/counts_out must
 * hold n entries; *nnz_out receives the number of distinct links. */
int oracle_build(const uint32_t* src, const uint32_t* dst, uint64_t n, uint64_t* keys_out,
                 uint64_t* counts_out, uint64_t* nnz_out) {
    std::vector<uint64_t> key(n);
    for (uint64_t i = 0; i < n; ++i) key[i] = ((uint64_t)src[i] << 32) | (uint64_t)dst[i];
    std::sort(key.begin(), key.end());
    uint64_t u = 0;
    uint64_t i = 0;
    while (i < n) {
        uint64_t j = i;
        while (j < n && key[j] == key[i]) ++j;
        keys_out[u] = key[i];
        counts_out[u] = j - i;
        ++u;
        i = j;
    }
    *nnz_out = u;
    return 0;
}

/* A += A_t on sorted nonzero lists: a two-way merge adding equal keys.
 * keys_out/counts_out must hold na + nb entries. */
int oracle_accumulate(const uint64_t* ka, const uint64_t* ca, uint64_t na, const uint64_t* kb,
                      const uint64_t* cb, uint64_t nb, uint64_t* keys_out, uint64_t* counts_out,
                      uint64_t* nnz_out) {
    uint64_t i = 0, j = 0, u = 0;
    while (i < na || j < nb) {
        if (j >= nb || (i < na && ka[i] < kb[j])) {
            keys_out[u] = ka[i];
            counts_out[u] = ca[i];
            ++i;
        } else if (i >= na || kb[j] < ka[i]) {
            keys_out[u] = kb[j];
            counts_out[u] = cb[j];
            ++j;
        } else {
            keys_out[u] = ka[i];
            counts_out[u] = ca[i] + cb[j];
            ++i;
            ++j;
        }
        ++u;
    }
    *nnz_out = u;
    return 0;
}

/* Steps 2-4: the statistics record of a matrix given by its sorted nonzero
 * list (keys strictly ascending, counts >= 1).  stats must hold 9 entries. */
int oracle_stats(const uint64_t* keys, const uint64_t* counts, uint64_t nnz, uint64_t* stats) {
    for (int f = 0; f < N_FIELDS; ++f) stats[f] = 0;

    /* whole matrix: 1^T A 1, 1^T |A|_0 1, max(A) */
    for (uint64_t u = 0; u < nnz; ++u) {
        stats[VALID_PACKETS] += counts[u];
        if (counts[u] > stats[MAX_LINK_PACKETS]) stats[MAX_LINK_PACKETS] = counts[u];
    }
    stats[UNIQUE_LINKS] = nnz;

    /* rows: A 1 and |A|_0 1, one run of equal sources at a time */
    uint64_t u = 0;
    while (u < nnz) {
        uint64_t s = keys[u] >> 32;
        uint64_t packets = 0, fanout = 0;
        while (u < nnz && (keys[u] >> 32) == s) {
            packets += counts[u];
            fanout += 1;
            ++u;
        }
        stats[UNIQUE_SOURCES] += 1;
        if (packets > stats[MAX_SRC_PACKETS]) stats[MAX_SRC_PACKETS] = packets;
        if (fanout > stats[MAX_SRC_FANOUT]) stats[MAX_SRC_FANOUT] = fanout;
    }

    /* columns: 1^T A and 1^T |A|_0 after grouping the entries by destination */
    std::vector<std::pair<uint32_t, uint64_t>> col(nnz);
    for (uint64_t v = 0; v < nnz; ++v) col[v] = {(uint32_t)(keys[v] & 0xFFFFFFFFu), counts[v]};
    std::sort(col.begin(), col.end());
    uint64_t v = 0;
    while (v < nnz) {
        uint32_t d = col[v].first;
        uint64_t packets = 0, fanin = 0;
        while (v < nnz && col[v].first == d) {
            packets += col[v].second;
            fanin += 1;
            ++v;
        }
        stats[UNIQUE_DESTINATIONS] += 1;
        if (packets > stats[MAX_DST_PACKETS]) stats[MAX_DST_PACKETS] = packets;
        if (fanin > stats[MAX_DST_FANIN]) stats[MAX_DST_FANIN] = fanin;
    }
    return 0;
}

/* Per-source vectors A 1 and |A|_0 1 (Table 2 rows 6 and 8): the distinct
 * sources ascending with their packet and fan-out counts.  Outputs must hold
 * nnz entries; *ns_out receives the number of sources. */
int oracle_rows(const uint64_t* keys, const uint64_t* counts, uint64_t nnz, uint32_t* src_out,
                uint64_t* packets_out, uint64_t* fanout_out, uint64_t* ns_out) {
    uint64_t u = 0, s_idx = 0;
    while (u < nnz) {
        uint64_t s = keys[u] >> 32;
        uint64_t packets = 0, fanout = 0;
        while (u < nnz && (keys[u] >> 32) == s) {
            packets += counts[u];
            fanout += 1;
            ++u;
        }
        src_out[s_idx] = (uint32_t)s;
        packets_out[s_idx] = packets;
        fanout_out[s_idx] = fanout;
        ++s_idx;
    }
    *ns_out = s_idx;
    return 0;
}

/* Order-independent digest of a nonzero list: sum of mix(key) * count mod
 * 2^64, with mix the SplitMix64 output function.  Lets a large matrix be
 * compared without a full host diff. */
uint64_t oracle_digest(const uint64_t* keys, const uint64_t* counts, uint64_t nnz) {
    uint64_t h = 0;
    for (uint64_t u = 0; u < nnz; ++u) {
        uint64_t z = keys[u] + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        h += z * counts[u];
    }
    return h;
}

/* Columns (the reverse operation of oracle_rows, Table 2 caption): per
 * destination j, ascending by j: packets 1^T A (j) and fan-in 1^T |A|_0 (j).
 * The (dst, count) pairs of the nonzero list are std::sort-ed by dst, then
 * equal destinations are summed in one scan.  Outputs hold nnz entries. */
int oracle_cols(const uint64_t* keys, const uint64_t* counts, uint64_t nnz, uint32_t* dst_out,
                uint64_t* packets_out, uint64_t* fanin_out, uint64_t* nd_out) {
    std::vector<std::pair<uint32_t, uint64_t>> col(nnz);
    for (uint64_t u = 0; u < nnz; ++u) col[u] = {(uint32_t)keys[u], counts[u]};
    std::sort(col.begin(), col.end());
    uint64_t u = 0, d_idx = 0;
    while (u < nnz) {
        const uint32_t d = col[u].first;
        uint64_t packets = 0, fanin = 0;
        while (u < nnz && col[u].first == d) {
            packets += col[u].second;
            fanin += 1;
            ++u;
        }
        dst_out[d_idx] = d;
        packets_out[d_idx] = packets;
        fanin_out[d_idx] = fanin;
        ++d_idx;
    }
    *nd_out = d_idx;
    return 0;
}

/* Globally unique addresses (section "Graph Analytics"): the distinct values
 * of the src and dst columns together -- each column's distinct values with
 * the ones common to both counted once.  From A's nonzero list: every key
 * contributes its source and its destination; std::sort, std::unique.
 * out holds 2 * nnz entries; *n_out receives the count, out the addresses
 * ascending. */
int oracle_unique_addresses(const uint64_t* keys, uint64_t nnz, uint32_t* out, uint64_t* n_out) {
    std::vector<uint32_t> a;
    a.reserve(2 * nnz);
    for (uint64_t u = 0; u < nnz; ++u) {
        a.push_back((uint32_t)(keys[u] >> 32));
        a.push_back((uint32_t)keys[u]);
    }
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    std::copy(a.begin(), a.end(), out);
    *n_out = a.size();
    return 0;
}

/* Address anonymization (section "Implementation", paragraph "IP Address
 * Anonymization"): the N distinct addresses of src and dst get the labels of
 * a random permutation of 0..N-1, and every packet's addresses are replaced
 * by their labels (a gather).
 *   1. u = the distinct values of src and dst, ascending (std::sort, std::unique);
 *   2. the permutation: u[i] is given label t when rnd[i] is the t-th
 *      smallest of rnd[0..N) (ties by i) -- sorting independent random keys
 *      yields a uniformly random permutation, as the shuffle of 0..N-1 does;
 *      rnd is the caller's array of random 64-bit keys (at least N of them);
 *   3. out[k] = label of src[k] (resp. dst[k]), found by binary search in u.
 * Returns -1 (and writes nothing) if rnd_n < N. */
int oracle_anonymize(const uint32_t* src, const uint32_t* dst, uint64_t n, const uint64_t* rnd,
                     uint64_t rnd_n, uint32_t* out_src, uint32_t* out_dst, uint64_t* n_unique) {
    std::vector<uint32_t> u(src, src + n);
    u.insert(u.end(), dst, dst + n);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    const uint64_t N = u.size();
    *n_unique = N;
    if (rnd_n < N) return -1;
    std::vector<uint64_t> order(N);
    for (uint64_t i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return rnd[a] < rnd[b]; });
    std::vector<uint32_t> label(N);
    for (uint64_t t = 0; t < N; ++t) label[order[t]] = (uint32_t)t;
    for (uint64_t k = 0; k < n; ++k) {
        out_src[k] = label[std::lower_bound(u.begin(), u.end(), src[k]) - u.begin()];
        out_dst[k] = label[std::lower_bound(u.begin(), u.end(), dst[k]) - u.begin()];
    }
    return 0;
}

/* ---- all host cores ------------------------------------------------------ */

}  // extern "C"

namespace {

int thread_count(int threads) {
    if (threads > 0) return threads;
    const unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

struct List {
    std::vector<uint64_t> keys, counts;
};

/* Runs f(i) for i in [0, m) on up to m threads and waits for all of them. */
template <typename F>
void run_all(int m, F f) {
    std::vector<std::thread> pool;
    for (int i = 0; i < m; ++i) pool.emplace_back(f, i);
    for (auto& t : pool) t.join();
}

/* Per-destination sums of one part: destination, packets, entries. */
struct ColSum {
    uint32_t dst;
    uint64_t packets, entries;
};

std::vector<ColSum> merge_cols(const std::vector<ColSum>& a, const std::vector<ColSum>& b) {
    std::vector<ColSum> out;
    out.reserve(a.size() + b.size());
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {
        if (j >= b.size() || (i < a.size() && a[i].dst < b[j].dst)) out.push_back(a[i++]);
        else if (i >= a.size() || b[j].dst < a[i].dst) out.push_back(b[j++]);
        else {
            out.push_back({a[i].dst, a[i].packets + b[j].packets, a[i].entries + b[j].entries});
            ++i;
            ++j;
        }
    }
    return out;
}

}  // namespace

extern "C" {

/* oracle_build on all host cores (threads <= 0: std::thread's
 * hardware_concurrency): one chunk of packets per thread through
 * oracle_build, then the chunk matrices summed pairwise by
 * oracle_accumulate until one is left.  Same outputs as oracle_build. */
int oracle_build_parallel(const uint32_t* src, const uint32_t* dst, uint64_t n, uint64_t* keys_out,
                          uint64_t* counts_out, uint64_t* nnz_out, int threads) {
    const int T = thread_count(threads);
    const uint64_t chunks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, n));
    std::vector<List> part(chunks);
    run_all((int)chunks, [&](int c) {
        const uint64_t a = n * (uint64_t)c / chunks, b = n * (uint64_t)(c + 1) / chunks;
        List& L = part[c];
        L.keys.resize(b - a);
        L.counts.resize(b - a);
        uint64_t u = 0;
        oracle_build(src + a, dst + a, b - a, L.keys.data(), L.counts.data(), &u);
        L.keys.resize(u);
        L.counts.resize(u);
        L.keys.shrink_to_fit();
        L.counts.shrink_to_fit();
    });
    while (part.size() > 1) {
        const size_t pairs = part.size() / 2;
        std::vector<List> next(pairs + (part.size() & 1));
        run_all((int)pairs, [&](int i) {
            const List& x = part[2 * i];
            const List& y = part[2 * i + 1];
            List& z = next[i];
            z.keys.resize(x.keys.size() + y.keys.size());
            z.counts.resize(z.keys.size());
            uint64_t u = 0;
            oracle_accumulate(x.keys.data(), x.counts.data(), x.keys.size(), y.keys.data(), y.counts.data(),
                              y.keys.size(), z.keys.data(), z.counts.data(), &u);
            z.keys.resize(u);
            z.counts.resize(u);
        });
        if (part.size() & 1) next.back() = std::move(part.back());
        part.swap(next);
    }
    const List& A = part[0];
    std::copy(A.keys.begin(), A.keys.end(), keys_out);
    std::copy(A.counts.begin(), A.counts.end(), counts_out);
    *nnz_out = A.keys.size();
    return 0;
}

/* oracle_stats on all host cores: the whole-matrix and row quantities by the
 * same linear scans; the columns by per-thread sorts of slices of the (dst,
 * count) pairs, each summed per destination, then merged pairwise. */
int oracle_stats_parallel(const uint64_t* keys, const uint64_t* counts, uint64_t nnz, uint64_t* stats,
                          int threads) {
    for (int f = 0; f < N_FIELDS; ++f) stats[f] = 0;
    for (uint64_t u = 0; u < nnz; ++u) {
        stats[VALID_PACKETS] += counts[u];
        if (counts[u] > stats[MAX_LINK_PACKETS]) stats[MAX_LINK_PACKETS] = counts[u];
    }
    stats[UNIQUE_LINKS] = nnz;
    uint64_t u = 0;
    while (u < nnz) {
        const uint64_t s = keys[u] >> 32;
        uint64_t packets = 0, fanout = 0;
        while (u < nnz && (keys[u] >> 32) == s) {
            packets += counts[u];
            fanout += 1;
            ++u;
        }
        stats[UNIQUE_SOURCES] += 1;
        if (packets > stats[MAX_SRC_PACKETS]) stats[MAX_SRC_PACKETS] = packets;
        if (fanout > stats[MAX_SRC_FANOUT]) stats[MAX_SRC_FANOUT] = fanout;
    }
    const int T = thread_count(threads);
    const uint64_t slices = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, nnz));
    std::vector<std::vector<ColSum>> part(slices);
    run_all((int)slices, [&](int c) {
        const uint64_t a = nnz * (uint64_t)c / slices, b = nnz * (uint64_t)(c + 1) / slices;
        std::vector<std::pair<uint32_t, uint64_t>> col(b - a);
        for (uint64_t v = a; v < b; ++v) col[v - a] = {(uint32_t)(keys[v] & 0xFFFFFFFFu), counts[v]};
        std::sort(col.begin(), col.end());
        std::vector<ColSum>& out = part[c];
        uint64_t v = 0;
        while (v < col.size()) {
            ColSum cs{col[v].first, 0, 0};
            while (v < col.size() && col[v].first == cs.dst) {
                cs.packets += col[v].second;
                cs.entries += 1;
                ++v;
            }
            out.push_back(cs);
        }
    });
    while (part.size() > 1) {
        const size_t pairs = part.size() / 2;
        std::vector<std::vector<ColSum>> next(pairs + (part.size() & 1));
        run_all((int)pairs, [&](int i) { next[i] = merge_cols(part[2 * i], part[2 * i + 1]); });
        if (part.size() & 1) next.back() = std::move(part.back());
        part.swap(next);
    }
    for (const ColSum& cs : part[0]) {
        stats[UNIQUE_DESTINATIONS] += 1;
        if (cs.packets > stats[MAX_DST_PACKETS]) stats[MAX_DST_PACKETS] = cs.packets;
        if (cs.entries > stats[MAX_DST_FANIN]) stats[MAX_DST_FANIN] = cs.entries;
    }
    return 0;
}

/* The thread count the all-cores variants use for threads <= 0. */
int oracle_hardware_threads(void) { return thread_count(0); }

}  // extern "C"
