// ns_kernels.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "ns_common.cuh"

namespace ns {

// key loading modes of the radix sort
enum { LOAD_KEYS = 0, LOAD_PACK = 1, LOAD_DST_OF = 2 };
// run-key modes
// RUN_HI_OF_PACKED: u64 words (key << 32 | value), runs of equal key with
// the low halves as values
enum { RUN_U64 = 0, RUN_SRC_OF_U64 = 1, RUN_U32 = 2, RUN_HI_OF_PACKED = 3 };
// run-statistics modes
enum { RS_LINKS = 0, RS_ROWS = 1, RS_COLS = 2 };

// Input of a sort pass.  n_dev, when set, holds the true element count on the
// device (the host passes an upper bound): kernels read it, so a stage can
// consume a count produced by the previous stage without a host round trip.
struct SortIn {
    const void* keys;
    const u64* vals;
    const u32* src;
    const u32* dst;
    const u64* n_dev;
    bool bulk;  // every input address is 16-byte aligned: stage tiles with bulk copies
    const char* trace_name;  // tracer label of the digit passes (NULL: by key type)
};

// Per-kernel timing (ns_trace.cu): a TraceScope around a launch records an
// event pair on the launch stream when the context's tracer is on and the
// stream is not capturing.
struct Tracer {
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> recs;
};
struct TraceScope {
    TraceScope(Tracer* t, const char* name, cudaStream_t s);
    ~TraceScope();
    Tracer* t;
    const char* name;
    cudaStream_t s;
    cudaEvent_t a;
};
void tracer_destroy(Tracer* t);

// Per-context scratch of the sort path.
struct SortScratch {
    u64* ghist;          // [8][256] digit histograms (wide plan: 4096 bins)
    u64* offs;           // [8][256] bucket starts, then [256] slot cursors of an unstable first pass
                         // (wide plan: 4096 bucket starts, then 1024 cursors)
    u64* status;         // look-back status words
    u64 status_words;
    u32* tile_counters;  // [16]
    u32 tag;             // last look-back tag issued
    int sms;
    Tracer* tr;          // the context's tracer (may be off)
    int tile_shape;      // digit passes over 64-bit keys: 0 = 512 threads x 16 keys,
                         // 1 = 512 x 12, 2 = 256 x 16 (kSortTileShapes)
    int digit_plan;      // 64-bit keys alone: kDigits8 (eight 8-bit passes) or kDigitsWide
                         // (a 10-bit unstable pass, then six 9-bit stable passes)
};
constexpr int kSortTileShapes = 3;
constexpr int kDigits8 = 0, kDigitsWide = 1, kDigitPlans = 2;

// Look-back tags are 16 bits; when they wrap, the status words are cleared
// on the stream so no stale word can carry a live tag.
//
// A CUDA graph fixes each launch's tag at capture, so a replay would find
// the previous replay's words under the very tag it waits for.  While the
// stream is capturing, the words a launch uses are therefore cleared first,
// as a node of the graph (outside a capture nothing is cleared).
inline void clear_status_in_capture(u64* p, u64 words, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (words && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaMemsetAsync(p, 0, words * sizeof(u64), s);
}

inline u32 next_tag(SortScratch& sc, cudaStream_t s) {
    if (sc.tag >= 0xFFFFu) {
        cudaMemsetAsync(sc.status, 0, sc.status_words * sizeof(u64), s);
        sc.tag = 0;
    }
    return ++sc.tag;
}

u64 sort_tiles(u64 n);
// CTAs of kernel fn resident at once on the current GPU (the kernel's shared
// memory attribute is set on first use, per device).
int resident_ctas_of(const void* fn, int threads, size_t smem);
// The sort path's hot-key split (ns_split.cu): A's sorted nonzero list of n
// packets with the heaviest sampled links counted apart from the sort.
u64 split_state_bytes();
void sort_links_split(const u32* src, const u32* dst, u64 n, u64* kb[2], u64* heads, u64* pos, void* state,
                      u64* keys_out, u64* counts_out, SortScratch& sc, DevStats* st, int sms, cudaStream_t s);
cudaError_t split_info(const void* state, u64* hot_keys, u64* cold_packets, cudaStream_t s);
// the column side's hot-destination split (ns_colsplit.cu)
u64 col_split_state_bytes();
void col_split_runs(const u64* words, const u64* nnz, u64 n, u64* kb[2], u64* pos, u64* psum, void* state,
                    u64* runs_out, SortScratch& sc, DevStats* st, int sms, cudaStream_t s);
cudaError_t col_split_info(const void* state, u64* hot, u64* cold, cudaStream_t s);
void launch_diag_wait(int which, u64* status_word, DevStats* st, cudaStream_t s);
void launch_diag_rand3(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed, cudaStream_t s);
// a, b, c: tables of mask + 1 16-byte slots (2 (mask + 1) words); mode 0..2
void launch_diag_claims(u64* a, u64* b, u64* c, u64 mask, u64 threads, u64 seed, int mode, u64* sink,
                        cudaStream_t s);
// look-back status words per tile of a digit pass under a digit plan
int sort_radix(int digit_plan);

// Batched windows: per-window tables carved from one arena (ns_batch.cu).
struct BatchDev {
    const u32* src;
    const u32* dst;
    const u64* win_off;   // [W+1] packet offsets of the windows
    const u64* tile_off;  // [W+1] tile offsets (tiles of T packets per window)
    const u64* tab_off;   // [W] first slot of the window's tables in the arena
    const u64* tab_cap;   // [W] power-of-two table capacity (plus one side slot)
    LinkSlot* links;
    NodeSlot* rows;
    NodeSlot* cols;
    DevStats* wstats;  // [W]
    u64 W;
    u32 T;
};

// hash path (ns_hash.cu)
// `cache`: stage skewed keys in per-CTA shared-memory tables first.
// `snap`: update existing nodes from the claim's snapshot with one CAS (for
// inserts into a large resident matrix; the snapshot launch always does).
void launch_insert_packets(const u32* src, const u32* dst, u64 n, const HashView& M,
                           int sms, bool cache, cudaStream_t s, bool snap = false);
void launch_insert_packets_snapshot(const u32* src, const u32* dst, u64 n, const HashView& M,
                                    u64* out, int sms, bool cache, cudaStream_t s);
// `cache` (default on): stage rows and columns that repeat across the
// inserted links in per-CTA shared-memory tables (pays under skew)
// total_dev (optional): the number of slots to read, on the device (then
// in_cap + 1 is only an upper bound that sizes the grid)
void launch_insert_slots(const LinkSlot* in, u64 in_cap, const HashView& M, int sms,
                         cudaStream_t s, bool cache = true, const u64* total_dev = nullptr);
void launch_insert_list(const u64* keys, const u64* counts, u64 n_bound,
                        const u64* n_dev, const HashView& M, int sms, cudaStream_t s);
void launch_compact_links(const LinkSlot* in, u64 cap, u64* out_keys, u64* out_counts,
                          u64* out_n, u64 out_cap, DevStats* st, int sms, cudaStream_t s);
void launch_stats_out(const DevStats* st, u64* out, cudaStream_t s);
// total_dev (optional): the tile count on the device (total_tiles is then an
// upper bound that sizes the grid)
void launch_batch_insert(const BatchDev& B, u32* tile_counter, u64 total_tiles, int sms, int per_sm,
                         bool cache, cudaStream_t s, const u64* total_dev = nullptr);
void launch_batch_stats_out(const DevStats* wstats, u64 W, u64* out, int sms, cudaStream_t s);

// sort path (ns_sort.cu).  Each radix sort returns the index of kbuf/vbuf
// holding the result.  n is an upper bound when n_dev is given.  Sorts with
// values are stable; keys-only sorts order only the sorted bits.
int radix_sort_packets(const u32* src, const u32* dst, u64* kbuf[2], u64 n,
                       SortScratch& sc, DevStats* st, cudaStream_t s);
// n_dev (<= n) u64 keys from `keys` (which must not be kbuf[0]), all 64 bits.
// trace_name labels the digit passes (NULL: "k_onesweep<u64 key>").
int radix_sort_keys64(const u64* keys, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                      cudaStream_t s, const char* trace_name);
int radix_sort_pairs64(const u64* keys, const u64* vals, const u64* n_dev,
                       u64* kbuf[2], u64* vbuf[2], u64 n, SortScratch& sc,
                       DevStats* st, cudaStream_t s);
// Sorts n_dev (<= n) u64 words by their upper 32 bits (four 8-bit digit
// passes; words with equal upper halves come out in any order, since the
// first pass keeps none); returns the index of the buffer holding the result.
// Keys-only sorts below share this: only the sorted bits are ordered.
int radix_sort_hi32(const u64* packed, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                    cudaStream_t s, const char* trace_name = nullptr);
// n_dev (<= n) uint32 keys (four 8-bit digit passes).
int radix_sort_u32(const u32* keys, const u64* n_dev, u32* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                   cudaStream_t s);
// The same by their lower 32 bits (words holding one uint32 each).
int radix_sort_lo32(const u64* keys, const u64* n_dev, u64* kbuf[2], u64 n, SortScratch& sc, DevStats* st,
                    cudaStream_t s);
int radix_sort_dst_pairs(const u64* link_keys, const u64* counts, const u64* n_dev,
                         u32* kbuf[2], u64* vbuf[2], u64 n, SortScratch& sc,
                         DevStats* st, cudaStream_t s);
// pack_out (RUN_SRC_OF_U64 only, may be NULL): also writes, for every input
// element i, (low half of key i) << 32 | low half of value i.
void launch_runs(int keymode, bool has_v, const void* keys, const u64* vals, u64 n,
                 const u64* n_dev, u64* head_keys, u64* pos, u64* psum,
                 u64* R_out, SortScratch& sc, DevStats* st, cudaStream_t s, u64* pack_out = nullptr);
void launch_run_stats(int mode, const u64* pos, const u64* psum, const u64* R_ptr,
                      u64 bound, u64* counts_out, DevStats* st, int sms, Tracer* tr, cudaStream_t s);

}  // namespace ns
