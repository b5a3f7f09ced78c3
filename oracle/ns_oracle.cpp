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
 * Every count is uint64; no floating point is involved.
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
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

}  // extern "C"
