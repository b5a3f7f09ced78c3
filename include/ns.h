/*
 * ns.h -- C ABI of the network-sensing traffic-matrix library (CUDA, sm_103a).
 *
 * The library turns a stream of anonymized (src, dst) 32-bit address pairs
 * into the hypersparse 2^32 x 2^32 traffic matrix A, where A(i,j) is the
 * number of packets from source i to destination j, and computes the
 * network quantities the paper lists in Table 2 (section "Implementation",
 * paragraph "Graph Analytics"; the reverse quantities follow by exchanging
 * src and dst, Table 2 caption).  The paper's graph is one dataframe with the
 * columns src, dst and n_packets (same paragraph); here the columns are two
 * uint32 arrays in, and A's nonzero list (uint64 key = src << 32 | dst,
 * uint64 count) out.  Windows of packets are summed: A = sum_t A_t.
 *
 * Conventions that hold for every call:
 *  - Pointers named d_* are CUDA device pointers (device memory, or managed
 *    or mapped memory the device can address); h_* are host pointers.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it; only calls documented as blocking synchronize it.
 *  - The caller owns the input buffers and must keep them valid and
 *    unmodified until the stream work completes.  The library owns matrices
 *    and all scratch memory it allocates.
 *  - Device memory: the serving slots' buffers and window matrices come from
 *    the context's memory pool and are allocated, grown and freed in stream
 *    order on the slot's own stream, so that a slot that grows stalls no
 *    other slot.  Every other buffer comes from cudaMalloc and is released
 *    with cudaFree, which waits for the device.  A buffer cannot grow while
 *    its stream is being captured into a CUDA graph: such a call returns
 *    NS_ERR_STATE (run it once before the capture so that every buffer has
 *    its size).
 *  - n == 0 is legal everywhere and gives an empty matrix / zero statistics.
 *    Null pointers with n > 0, unknown enum values and mismatched devices
 *    return NS_ERR_INVALID.  No call aborts, traps or hangs: device-side
 *    bounded waits and probes record an error word that the next blocking
 *    call (ns_network_stats, ns_matrix_nnz, ns_matrix_export, ns_sync)
 *    returns as NS_ERR_CAPACITY or NS_ERR_TIMEOUT.
 *  - ns_last_error() returns a thread-local message for the last non-OK
 *    status on the calling thread.
 *  - A context and its matrices are not thread-safe; use one per host thread
 *    (the serving calls ns_stream_* are the exception and are thread-safe).
 */
#ifndef NS_H
#define NS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ns_stream_t; /* identical to cudaStream_t */
typedef struct ns_ctx ns_ctx;
typedef struct ns_matrix ns_matrix;

typedef enum {
    NS_OK = 0,
    NS_ERR_INVALID = 1,  /* bad argument */
    NS_ERR_OOM = 2,      /* device allocation failed (or admission budget) */
    NS_ERR_CAPACITY = 3, /* a hash probe exceeded its bound */
    NS_ERR_CUDA = 4,     /* a CUDA runtime call failed */
    NS_ERR_TIMEOUT = 5,  /* a device-side wait gave up, or a host wait timed out */
    NS_ERR_BUSY = 6,     /* serving queue full (retry later), or the service is not idle */
    NS_ERR_STATE = 7,    /* call not valid in the object's current state */
    NS_ERR_IO = 8        /* a file could not be opened, read or written */
} ns_status;

/* The nine quantities of Table 2 (matrix notation), all exact uint64:
 *   valid_packets       1^T A 1            (row 1)
 *   unique_links        1^T |A|_0 1        (row 2)
 *   unique_sources      1^T |A 1|_0        (row 5)
 *   unique_destinations 1^T |1^T A|_0      (row 5 reversed)
 *   max_src_packets     max(A 1)           (row 7)
 *   max_src_fanout      max(|A|_0 1)       (row 9)
 *   max_dst_packets     max(1^T A)         (row 7 reversed)
 *   max_dst_fanin       max(1^T |A|_0)     (row 9 reversed)
 *   max_link_packets    max(A)             (row 4)
 * A maximum over an empty matrix is 0. */
typedef struct {
    uint64_t valid_packets;
    uint64_t unique_links;
    uint64_t unique_sources;
    uint64_t unique_destinations;
    uint64_t max_src_packets;
    uint64_t max_src_fanout;
    uint64_t max_dst_packets;
    uint64_t max_dst_fanin;
    uint64_t max_link_packets;
} ns_stats;

/* Aggregation path.  Both give bit-identical results. */
enum {
    NS_PATH_AUTO = 0, /* per window size: ns_path_tune's choice, else sort from 2^24 packets */
    NS_PATH_SORT = 1, /* LSD radix sort of packed keys + run-length encode */
    NS_PATH_HASH = 2  /* open-addressing hash table with atomic counts */
};

/* Per-CTA shared-memory staging of hot links, sources and destinations in
 * the hash path (see ns_config.cta_cache).  For ns_accumulate, AUTO and ON
 * stage, OFF does not (staging pays when sources and destinations repeat,
 * e.g. under Zipf skew, and costs time on nearly distinct RMAT windows). */
enum {
    NS_CACHE_AUTO = 0, /* ns_path_tune's choice for the size, else on from 2^22 packets */
    NS_CACHE_ON = 1,
    NS_CACHE_OFF = 2
};

/* How the sort path orders A's nonzeros by destination (both exact). */
enum {
    NS_COLSORT_AUTO = 0,  /* below 2^32 packets (every count < 2^32): one u64 word
                             (dst << 32 | count) per nonzero, sorted by its upper
                             half; from 2^32 packets: (dst, count) pairs */
    NS_COLSORT_PAIRS = 1  /* always (u32 dst, u64 count) pairs */
};

/* The sort path's hot-key split (see ns_config.sort_split): before the
 * radix sort, the links a sample of the packets shows to be the heaviest
 * (up to 4096) are counted in shared memory during one pass over the
 * packets, and only the other ("cold") packets are sorted; the two are then
 * merged.  Exact either way; it saves sort work under skew. */
enum {
    NS_SPLIT_AUTO = 0, /* ns_path_tune's choice for the size, else on from 2^23 packets */
    NS_SPLIT_ON = 1,   /* from 2^16 packets (smaller windows never split) */
    NS_SPLIT_OFF = 2
};

/* The tile of the sort path's digit passes over 64-bit keys (threads x keys
 * per thread; see ns_config.sort_tile).  Exact either way. */
enum {
    NS_TILE_AUTO = 0,   /* ns_path_tune's choice for the size, else 512 x 16 */
    NS_TILE_512X16 = 1, /* 8192-key tiles, two CTAs per SM */
    NS_TILE_512X12 = 2, /* 6144-key tiles */
    NS_TILE_256X16 = 3  /* 4096-key tiles, four CTAs per SM */
};

/* The digit plan of the sort path's radix sorts of 64-bit keys (the packed
 * packets, or the cold keys of the hot-key split; see ns_config.sort_digits).
 * Exact either way. */
enum {
    NS_DIGITS_AUTO = 0, /* ns_path_tune's choice for the size, else NS_DIGITS_8 */
    NS_DIGITS_8 = 1,    /* eight passes of 8-bit digits (256 buckets) */
    NS_DIGITS_WIDE = 2  /* seven passes: one of 10-bit digits (1024 buckets, the
                           unordered first pass), then six of 9-bit digits (512) */
};

typedef struct {
    int path;                  /* NS_PATH_* used by ns_window_build */
    uint64_t hbm_budget_bytes; /* serving admission and batch arena budget; 0 = 64 GiB */
    int max_slots;             /* serving: windows in flight at once; 0 = 8 */
    const char* tuner_cache;   /* autotuner cache file (JSON); NULL = none */
    int cta_cache;             /* NS_CACHE_* for hash-path packet inserts */
    int column_sort;           /* NS_COLSORT_* for the sort path's per-destination side */
    double hash_load;          /* load bound of the link, source and destination tables the
                                  library sizes (builds, reserves, growth), in [0.05, 0.9];
                                  0 = 0.5.  Lower costs memory and shortens probe chains. */
    int sort_split;            /* NS_SPLIT_* for the sort path */
    int sort_tile;             /* NS_TILE_* for the sort path's digit passes */
    int sort_digits;           /* NS_DIGITS_* for the sort path's digit passes */
} ns_config;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  cfg may be NULL for defaults.
 * *ctx is owned by the caller and released with ns_destroy.  Every call that
 * takes a context, or an object made from one, runs on the context's device
 * and leaves the calling thread's current device as it found it; streams
 * passed in must belong to that device. */
ns_status ns_create(ns_ctx** ctx, const ns_config* cfg, int device);

/* Waits for the device, then frees everything the context owns (matrices,
 * batches, sliders and servers created from it must be freed first); its
 * memory pool gives the memory back once every buffer from it is freed. */
void ns_destroy(ns_ctx* ctx);

/* Blocks until all work the context enqueued on `stream` is done, then
 * returns any device-side error recorded since the last blocking call. */
ns_status ns_sync(ns_ctx* ctx, ns_stream_t stream);

/* ---- matrices ---------------------------------------------------------- */

/* Creates an empty matrix owned by the library (no device memory yet). */
ns_status ns_matrix_create(ns_ctx* ctx, ns_matrix** out);

/* Pre-sizes a matrix for at least `max_links` nonzeros (and as many sources
 * and destinations) so later builds and accumulations never reallocate.
 * Optional: tables also grow on demand.  Enqueued on `stream`. */
ns_status ns_matrix_reserve(ns_matrix* m, uint64_t max_links, ns_stream_t stream);

/* As ns_matrix_reserve, for an empty matrix, with a promise that A will
 * never have more than max_nodes distinct sources nor more than max_nodes
 * distinct destinations (e.g. the size of the address space in use), so the
 * per-source and per-destination tables can be sized by it rather than by
 * the number of links.  If the promise is broken, inserts that find no room
 * are dropped and the next blocking call returns NS_ERR_CAPACITY. */
ns_status ns_matrix_reserve_ex(ns_matrix* m, uint64_t max_links, uint64_t max_nodes, ns_stream_t stream);

/* Makes the matrix empty (A = 0) keeping its memory.  Enqueued on stream. */
ns_status ns_matrix_clear(ns_matrix* m, ns_stream_t stream);

/* Frees the matrix after its pending work completes (memory from the
 * serving pool is released in stream order behind the work of the last
 * stream that used the matrix). */
void ns_matrix_free(ns_matrix* m);

/* Number of nonzeros of A (unique links).  Blocking. */
ns_status ns_matrix_nnz(const ns_matrix* m, uint64_t* h_nnz, ns_stream_t stream);

/* Writes A's nonzero list ascending by key = src << 32 | dst into
 * d_keys[0..nnz) and d_counts[0..nnz) (device uint64 arrays of `cap`
 * entries each) and its length to *h_nnz.  Returns NS_ERR_CAPACITY (and
 * writes nothing) if cap < nnz.  Blocking (it must read nnz). */
ns_status ns_matrix_export(const ns_matrix* m, uint64_t* d_keys, uint64_t* d_counts,
                           uint64_t cap, uint64_t* h_nnz, ns_stream_t stream);

/* Which vectors ns_matrix_nodes exports. */
enum {
    NS_NODES_SRC = 0, /* per source i: id, A 1 (i), |A|_0 1 (i)      (Table 2 rows 6, 8) */
    NS_NODES_DST = 1, /* per destination j: id, 1^T A (j), 1^T |A|_0 (j) (their reverses) */
    NS_NODES_ANY = 2  /* the distinct addresses of src and dst together: ids only */
};

/* Per-entity vectors of A, ascending by address, into device arrays of `cap`
 * entries: d_ids (uint32), d_packets and d_degree (uint64; each may be NULL,
 * and both are ignored for NS_NODES_ANY).  NS_NODES_ANY gives the globally
 * unique addresses of section "Graph Analytics" (each column's distinct
 * values, the ones common to both counted once).  *h_count receives the
 * number of entries (S, D or |src u dst|); if it exceeds cap, the first cap
 * are written and NS_ERR_CAPACITY is returned.  Allocates scratch for the
 * call; blocking. */
ns_status ns_matrix_nodes(ns_ctx* ctx, const ns_matrix* m, int which, uint32_t* d_ids, uint64_t* d_packets,
                          uint64_t* d_degree, uint64_t cap, uint64_t* h_count, ns_stream_t stream);

/* Address anonymization (section "Implementation", paragraph "IP Address
 * Anonymization"): the N distinct addresses of d_src[0..n) and d_dst[0..n)
 * are relabelled by a random permutation of 0..N-1 and every packet's
 * addresses replaced by their labels: d_out_src[k] = label(d_src[k]),
 * d_out_dst[k] = label(d_dst[k]).  The permutation is the one the caller's
 * random keys define -- the address at position i of the ascending distinct
 * list, whose key is d_rand[i], gets label t when d_rand[i] is the t-th
 * smallest of d_rand[0..N) (ties by position) -- so the random draws are an
 * input, and any source of independent keys yields a uniformly random
 * permutation.  rand_count must be at least N (at most 2n); otherwise
 * NS_ERR_CAPACITY, with *h_unique = N and nothing written.  The outputs may
 * be the inputs.  Allocates scratch; blocking. */
ns_status ns_anonymize(ns_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                       const uint64_t* d_rand, uint64_t rand_count, uint32_t* d_out_src, uint32_t* d_out_dst,
                       uint64_t* h_unique, ns_stream_t stream);

/* ---- per-window and sliding-window statistics ---------------------------- */

typedef struct ns_slider ns_slider;

/* A slider over the last `windows` (K >= 1) windows: it keeps their matrices
 * A_t (the time-indexed matrices of the Table 2 caption).  Owned by the
 * caller; released with ns_slider_free. */
ns_status ns_slider_create(ns_ctx* ctx, uint32_t windows, ns_slider** out);
void ns_slider_free(ns_slider* slider);

/* Builds A_t of the next window (as ns_window_build), writes its nine
 * quantities to d_window and those of the sliding sum A_{t-K+1} + ... + A_t
 * (of all windows pushed so far while fewer than K) to d_sliding; each may be
 * NULL.  The sliding sum is re-formed from the K window matrices on every
 * push, so every quantity is exact.  Asynchronous, except when the sliding
 * sum's tables must grow.  Not from the paper: its analyses use one static
 * matrix; the per-window and sliding forms follow from A_t being
 * time-indexed. */
ns_status ns_slider_push(ns_ctx* ctx, ns_slider* slider, const uint32_t* d_src, const uint32_t* d_dst,
                         uint64_t n, ns_stats* d_window, ns_stats* d_sliding, ns_stream_t stream);

/* The slider's current sliding-sum matrix (owned by the slider; valid until
 * the next push or ns_slider_free), e.g. for ns_matrix_export or
 * ns_matrix_nodes. */
ns_status ns_slider_matrix(const ns_slider* slider, const ns_matrix** out);

/* ---- the hot path (paper, Table 2) -------------------------------------- */

/* out := A_t, the traffic matrix of one window of n packets given as two
 * uint32 columns d_src[0..n), d_dst[0..n) (Table 2 row 3: link packets from
 * i to j).  Any previous content of `out` is discarded.  Uses the context's
 * path (sort or hash).  Asynchronous. */
ns_status ns_window_build(ns_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                          ns_matrix* out, ns_stream_t stream);

/* ns_window_build for packets in host memory, with the quantities read
 * back: h_src[0..n) and h_dst[0..n) are copied (on `stream`) into device
 * buffers the context owns and keeps for later calls, out := A_t of those
 * packets, and, if h_stats is not NULL, A_t's nine quantities are written to
 * *h_stats (host memory).  Pinned host columns are copied by DMA at the
 * link's full rate; pageable ones are staged by the driver.  This is the
 * end-to-end form of the hot path (host columns in, statistics out).
 * Blocking: returns once the statistics are on the host (or, with h_stats
 * NULL, once the build is done), with any device-side error as its status.
 * The host columns may be reused as soon as it returns. */
ns_status ns_window_build_host(ns_ctx* ctx, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n,
                               ns_matrix* out, ns_stats* h_stats, ns_stream_t stream);

/* Path tuner: builds A from d_src/d_dst (n > 0 packets, device memory)
 * with the sort path in every combination of hot-key split (without, with;
 * no split below 2^16 packets), digit plan (the two NS_DIGITS_* plans) and
 * digit-pass tile (the three NS_TILE_* shapes) -- only the ones the
 * context's sort_split, sort_digits and sort_tile allow --
 * and the hash path without and with per-CTA caches (only the one the
 * context's cta_cache forces, if it forces one), three times each, and
 * keeps the fastest of the last two timings of each.  The winner becomes
 * the context's NS_PATH_AUTO / NS_CACHE_AUTO choice, and the fastest sort
 * variant its NS_SPLIT_AUTO / NS_DIGITS_AUTO / NS_TILE_AUTO choice (see
 * ns_sort_resolve), for every n' with
 * floor(log2 n') = floor(log2 n); all are stored in the tuner cache file
 * (if the context has one) keyed by GPU name and that power of two, where
 * later contexts on the same GPU find them.  *chosen (NS_PATH_SORT or
 * NS_PATH_HASH), *sort_ms (the faster sort variant) and *hash_ms (the faster
 * hash variant) may each be NULL.  Allocates a temporary matrix; blocking.
 * The paper has no counterpart: its two aggregation paths are this
 * library's own. */
ns_status ns_path_tune(ns_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                       ns_stream_t stream, int* chosen, float* sort_ms, float* hash_ms);

/* What the context's last sort-path build did with the hot-key split:
 * *used = 1 if it split, then *hot_keys = the links counted apart from the
 * sort and *cold_packets = the packets that went through the sort (each
 * pointer may be NULL).  Blocking (reads two counters). */
ns_status ns_sort_split_info(ns_ctx* ctx, int* used, uint64_t* hot_keys, uint64_t* cold_packets,
                             ns_stream_t stream);

/* What the context's last sort-path build did with the column side's
 * hot-destination split (taken with the hot-key split, on windows of fewer
 * than 2^32 packets): *used = 1 if it split, then *hot_destinations = the
 * destinations counted apart from the column sort (their column words
 * never sorted) and *cold_words = the column words that went through the
 * sort (each pointer may be NULL).  Blocking (reads two counters).  No
 * counterpart in the paper. */
ns_status ns_column_split_info(ns_ctx* ctx, int* used, uint64_t* hot_destinations, uint64_t* cold_words,
                               ns_stream_t stream);

/* The path ns_window_build would take for a window of n packets
 * (NS_PATH_SORT or NS_PATH_HASH). */
ns_status ns_path_resolve(const ns_ctx* ctx, uint64_t n, int* path);

/* The variant a sort-path build of n packets would take, from the context's
 * settings, else ns_path_tune's choices for the size, else the size rules:
 * *split = 1 if it takes the hot-key split (else 0), *tile = its NS_TILE_*
 * digit-pass tile (never NS_TILE_AUTO), *digits = its NS_DIGITS_* digit plan
 * (never NS_DIGITS_AUTO).  Each pointer may be NULL.  No device work.  No
 * counterpart in the paper (the tuner's knobs are this library's own). */
ns_status ns_sort_resolve(const ns_ctx* ctx, uint64_t n, int* split, int* tile, int* digits);

/* acc := acc + add (A = sum_t A_t; equal keys add their counts).  `add` is
 * unchanged and may be rebuilt as soon as the stream work completes.
 * acc and add must be distinct.  Asynchronous. */
ns_status ns_accumulate(ns_ctx* ctx, ns_matrix* acc, const ns_matrix* add, ns_stream_t stream);

/* acc := acc + A_t(d_src, d_dst): ns_window_build followed by ns_accumulate
 * fused into one pass, without materializing A_t.  Asynchronous. */
ns_status ns_window_ingest(ns_ctx* ctx, ns_matrix* acc, const uint32_t* d_src,
                           const uint32_t* d_dst, uint64_t n, ns_stream_t stream);

/* ns_window_ingest followed by ns_network_stats_async(acc, d_out) in one
 * kernel launch: the last CTA of the ingest writes the statistics of the
 * updated acc.  This is the per-window call of a streaming pipeline that
 * wants the running quantities after every window.  Asynchronous. */
ns_status ns_window_ingest_stats(ns_ctx* ctx, ns_matrix* acc, const uint32_t* d_src,
                                 const uint32_t* d_dst, uint64_t n, ns_stats* d_out,
                                 ns_stream_t stream);

/* The nine quantities of m into *h_out (host memory).  Blocking: waits for
 * the stream, then reports any device-side error of the matrix. */
ns_status ns_network_stats(ns_ctx* ctx, const ns_matrix* m, ns_stats* h_out, ns_stream_t stream);

/* Same quantities written to d_out (device memory, or mapped pinned host
 * memory) when the stream reaches this point; does not block.  Device-side
 * errors surface on the next blocking call. */
ns_status ns_network_stats_async(ns_ctx* ctx, const ns_matrix* m, ns_stats* d_out,
                                 ns_stream_t stream);

/* ---- batched windows ----------------------------------------------------- */

/* Many independent windows at once: the windows are laid end to end in two
 * uint32 columns, window w being packets [h_offsets[w], h_offsets[w+1]).
 * Each window's nine quantities (Table 2, of that window alone) are written
 * to d_window_stats[w], and, if acc is not NULL, acc := acc + sum_w A_w (the
 * running aggregate).  Persistent segmented launches process all windows:
 * CTAs take fixed-size tiles of packets in window order, each window's tables
 * are carved from one arena, and windows are grouped into chunks that fit it.
 * Results are bit-identical to ns_window_build + ns_network_stats per window
 * and ns_accumulate into acc. */
typedef struct ns_batch ns_batch;

/* Launch parameters the autotuner chooses (ns_batch_tune). */
typedef struct {
    uint32_t tile_packets; /* packets per CTA work item (multiple of 32) */
    uint32_t ctas_per_sm;  /* persistent CTAs per SM */
    double max_load;       /* per-window table load bound, in [0.5, 0.9] */
    uint32_t cta_cache;    /* 1 = stage hot keys in shared memory per tile */
} ns_batch_params;

/* A plan for batches of at most max_windows windows and max_packets packets:
 * allocates the arena (capped by the context's hbm_budget_bytes), the
 * per-window metadata and statistics.  Parameters come from the context's
 * tuner cache when it has an entry for this GPU and batch shape. */
ns_status ns_batch_create(ns_ctx* ctx, uint64_t max_windows, uint64_t max_packets, ns_batch** out);
/* Frees the batch after its pending work completes. */
void ns_batch_free(ns_batch* batch);
ns_status ns_batch_get_params(const ns_batch* batch, ns_batch_params* out);
ns_status ns_batch_set_params(ns_batch* batch, const ns_batch_params* params);

/* Runs one batch (see above).  h_offsets is host memory of windows + 1
 * entries, starting at 0 and non-decreasing; d_window_stats is a device array
 * of `windows` ns_stats.  acc must have room reserved for the batch's links
 * if this call is captured into a CUDA graph (growing it needs a blocking
 * read).  When acc is empty and the batch is in the sort path's range (the
 * path ns_window_build would take for all its packets at once), acc
 * receives the batch's matrix from one sort-path build over the packets
 * d_src/d_dst[0, h_offsets[windows]) -- the same A, as a sorted nonzero
 * list -- instead of every window's table being added to it; that build
 * takes the sort path's scratch, sized on first use (capture a graph around
 * this call only after one uncaptured run of the same size).  Asynchronous;
 * allocates nothing otherwise. */
ns_status ns_batch_run(ns_ctx* ctx, ns_batch* batch, const uint32_t* d_src, const uint32_t* d_dst,
                       const uint64_t* h_offsets, uint64_t windows, ns_stats* d_window_stats,
                       ns_matrix* acc, ns_stream_t stream);

/* ns_batch_run with the window offsets in device memory: d_offsets holds
 * windows + 1 uint64 entries (the same meaning as h_offsets).  The plan --
 * each window's table capacity, tile and table offsets -- is computed on the
 * device, so a CUDA graph captured around this call serves any new layout of
 * the same number of windows written into d_offsets before a replay,
 * without re-capture.  All windows of a run must fit the arena at once (one
 * chunk) and total at most the plan's max_packets; offsets that break this,
 * do not start at 0 or decrease make the run do nothing and set an error
 * flag that ns_batch_sync reports as NS_ERR_CAPACITY.  If acc is given it
 * must have room for max_packets more links (it is grown outside a capture
 * if needed).  Asynchronous; allocates nothing once acc has its room. */
ns_status ns_batch_run_device(ns_ctx* ctx, ns_batch* batch, const uint32_t* d_src, const uint32_t* d_dst,
                              const uint64_t* d_offsets, uint64_t windows, ns_stats* d_window_stats,
                              ns_matrix* acc, ns_stream_t stream);

/* Waits for the stream and returns NS_ERR_CAPACITY if the batch's last
 * ns_batch_run_device refused its offsets (see there), else NS_OK. */
ns_status ns_batch_sync(ns_batch* batch, ns_stream_t stream);

/* Autotuner: times ns_batch_run on this batch for every combination of tile
 * size {1024..16384}, CTAs per SM {4, 8, 16} and load bound {0.5, 0.7},
 * keeps the fastest in the plan, returns it in *chosen (may be NULL) and
 * stores it in the context's tuner cache file keyed by GPU name and batch
 * shape.  d_scratch_stats: `windows` device ns_stats for the trial runs.
 * Blocking. */
ns_status ns_batch_tune(ns_ctx* ctx, ns_batch* batch, const uint32_t* d_src, const uint32_t* d_dst,
                        const uint64_t* h_offsets, uint64_t windows, ns_stats* d_scratch_stats,
                        ns_stream_t stream, ns_batch_params* chosen);

/* ---- streaming service (continuous batching) ---------------------------- */

/* A service that takes windows from host threads while earlier ones are on
 * the GPU.  Each submitted window is admitted, in submission order, as soon
 * as a slot is free and its device memory fits the context's
 * hbm_budget_bytes (counting the resident aggregate and the windows in
 * flight); up to ns_config.max_slots windows build concurrently on their own
 * streams.  Each window's A_t is then added to `acc` -- the device-resident
 * running aggregate A -- on one accumulate stream in submission order, so a
 * window's results are the same whether it ran alone or among others.  For
 * each ticket the service returns A_t's quantities (per_window) and A's
 * quantities right after A_t was added (running), with host timestamps.
 * The server owns `ctx` and `acc` while it runs: do not use them from other
 * threads until ns_server_destroy returns.  The ns_stream_* calls are
 * thread-safe. */
typedef struct ns_server ns_server;

typedef struct {
    double submit_us;   /* steady-clock time of ns_stream_submit */
    double admit_us;    /* window admitted (slot and budget available) */
    double complete_us; /* both statistics records on the host */
    uint64_t window_id; /* as submitted */
} ns_stream_timing;

ns_status ns_server_create(ns_ctx* ctx, ns_matrix* acc, ns_server** out);

/* Sizes every slot's device buffers and tables for windows of up to
 * max_window packets, so that no later window makes a slot grow.  Only while
 * the service is idle (else NS_ERR_BUSY); blocking.  Optional: slots
 * otherwise grow on demand, in stream order on the slot's own stream (the
 * slot is idle then), which stalls no other slot. */
ns_status ns_server_reserve(ns_server* server, uint64_t max_window);

/* Empties the aggregate (A = 0) so that the next window's running
 * quantities start afresh.  Only while the service is idle (else
 * NS_ERR_BUSY); blocking. */
ns_status ns_server_clear(ns_server* server);

/* Finishes every submitted window, then stops the service's threads and
 * frees its slots (acc keeps the aggregate). */
void ns_server_destroy(ns_server* server);

/* Queues one window given as host uint32 columns h_src[0..n), h_dst[0..n);
 * they must stay valid and unchanged until ns_stream_wait for this ticket
 * returns (pinned memory makes the copy asynchronous).  Non-blocking;
 * NS_ERR_BUSY when the queue is full (retry later). */
ns_status ns_stream_submit(ns_server* server, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n,
                           uint64_t window_id, uint64_t* ticket);

/* *done = 1 once the ticket's results are ready. */
ns_status ns_stream_poll(ns_server* server, uint64_t ticket, int* done);

/* Waits up to timeout_us (< 0: no limit) for a ticket and returns its
 * results (any pointer may be NULL) and the window's status; NS_ERR_TIMEOUT
 * if the time ran out (the ticket stays valid).  After a completed wait the
 * ticket is forgotten. */
ns_status ns_stream_wait(ns_server* server, uint64_t ticket, ns_stats* per_window, ns_stats* running,
                         int64_t timeout_us, ns_stream_timing* timing);

/* ---- sharding over several ranks ------------------------------------------ */

/* A traffic matrix split over W ranks (one GPU each), the decomposition of
 * the paper's whole-graph quantities into per-rank parts: every rank
 * aggregates its own packets; entries are exchanged so that rank r holds
 * every entry whose source r owns (its rows of A are then complete: the row
 * quantities are local, and links, packets and sources add up over the
 * ranks); a second exchange by destination owner gives rank r every entry
 * of the destinations it owns (the keys are unique across ranks after the
 * first exchange, so each received entry is one link of its column), whose
 * column quantities are then local too.  The maxima reduce by max.  The
 * exchange itself is the caller's (any transport).  The paper has no
 * counterpart: it analyses one graph on one GPU. */
enum { NS_BY_SRC = 0, NS_BY_DST = 1 };

/* The rank in [0, parts) that owns an address: (addr * 0x9E3779B1 mod 2^32)
 * * parts / 2^32, the same on every rank and in device code.  parts == 0
 * gives 0. */
uint32_t ns_owner(uint32_t addr, uint32_t parts);

/* A's nonzeros grouped by owner: d_keys / d_counts (device, cap entries each)
 * receive the nonzero list reordered so that group p holds the entries whose
 * source (by = NS_BY_SRC) or destination (NS_BY_DST) is owned by rank p,
 * ascending by key within the group; h_offsets (host, parts + 1 entries)
 * receives the groups' starts and the total.  NS_ERR_CAPACITY (nothing
 * written) if cap < nnz.  Allocates scratch; blocking. */
ns_status ns_matrix_partition(ns_ctx* ctx, const ns_matrix* m, int by, uint32_t parts, uint64_t* d_keys,
                              uint64_t* d_counts, uint64_t cap, uint64_t* h_offsets, ns_stream_t stream);

/* m := m + the entries (d_keys[i], d_counts[i]), i < n (device arrays; keys
 * in any order, repeated keys add up, zero counts are skipped): how a rank
 * takes in the entries it received.  Asynchronous. */
ns_status ns_matrix_add_entries(ns_ctx* ctx, ns_matrix* m, const uint64_t* d_keys, const uint64_t* d_counts,
                                uint64_t n, ns_stream_t stream);

/* ---- checkpoint / resume ------------------------------------------------ */

/* Checkpoint file of a matrix: a 128-byte little-endian header (magic
 * "NSMATRIX", format version 1, header size, nnz, the nine quantities of
 * ns_stats, zero padding), then the nnz keys (src << 32 | dst, strictly
 * ascending) and the nnz counts, each as uint64.  It is the paper's
 * three-column frame (src, dst, n_packets; section "Implementation") with
 * its Table 2 quantities, so an accumulated A can be carried across a
 * restart of the process that serves the stream. */
#define NS_CHECKPOINT_VERSION 1

/* Writes matrix m to `path` (replaced atomically: written beside it, then
 * renamed).  Allocates scratch; blocking.  NS_ERR_IO if the file cannot be
 * written. */
ns_status ns_matrix_save(const ns_matrix* m, const char* path, ns_stream_t stream);

/* Replaces the contents of m (a matrix of ctx) with the matrix saved in
 * `path`.  The entries are inserted afresh, so m's quantities are recomputed
 * on the GPU; they must equal the saved ones.  NS_ERR_IO if the file cannot
 * be read, and NS_ERR_INVALID if it is malformed (a bad magic, version or
 * size, keys not strictly ascending, a zero count): m is then unchanged.
 * NS_ERR_INVALID too if the recomputed quantities differ from the saved
 * ones, and any error after the file has been checked (a failed copy,
 * allocation or insert): m is then left empty, never partly loaded.  The
 * copies and the insert run on `stream`.  Allocates scratch; blocking. */
ns_status ns_matrix_load(ns_ctx* ctx, const char* path, ns_matrix* m, ns_stream_t stream);

/* ---- statistics without device allocation ------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need a window's statistics -- for
 * example a process whose GPU memory is already fully claimed by another
 * framework's caching allocator, or a capture loop that must never block in
 * cudaMalloc/cudaFree (both may synchronize the device).
 *
 * Writes the nine quantities of the window d_src[0..n), d_dst[0..n) (the
 * same values ns_window_build + ns_network_stats give) to d_out, a device
 * (or mapped pinned host) ns_stats, when the stream reaches this point.
 * Needs no context and allocates nothing: its hash tables live in one fixed
 * device array of about 3 MiB inside the library, which every GPU that loads
 * the library keeps until the process exits.  n must not exceed
 * NS_STATIC_MAX_PACKETS (larger n returns NS_ERR_INVALID and does nothing).
 * Runs on the calling thread's current device, and `stream` must belong to
 * that device (a stream of another device returns NS_ERR_INVALID).  The
 * first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it;
 * make that first call before any stream capture on that device.  All calls
 * on a device share the one array and each starts by clearing it, so calls
 * whose GPU work overlaps (different streams, no ordering between them) race
 * and give wrong results: order them on one stream.  Asynchronous; within
 * the size limit no device-side error can occur. */
#define NS_STATIC_MAX_PACKETS 32768
ns_status ns_window_stats_static(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                                 ns_stats* d_out, ns_stream_t stream);

/* ---- tracing ----------------------------------------------------------- */

/* Per-kernel timing.  While tracing is on, every kernel the context launches
 * on a stream that is not being captured into a CUDA graph is bracketed by
 * two CUDA events on that stream (a few microseconds of overhead per launch).
 * ns_trace_read waits for the recorded events, writes one entry per kernel
 * name (up to cap entries; *count receives the number of names) and forgets
 * the records. */
typedef struct {
    char name[48];
    uint64_t launches;
    double total_ms;
    double max_ms;
} ns_trace_entry;

ns_status ns_trace_enable(ns_ctx* ctx, int on);
ns_status ns_trace_read(ns_ctx* ctx, ns_trace_entry* out, int cap, int* count);

/* Diagnostic of the device-side wait bounds (no counterpart in the paper):
 * runs one of the library's bounded waits against something nothing will
 * signal -- which = 0: a decoupled look-back on a status word that is never
 * published; which = 1: an mbarrier phase expecting bytes no copy delivers;
 * which = 2: the warp-wide look-back of the run kernels, likewise --
 * and returns NS_ERR_TIMEOUT once the wait gives up (about one second for
 * the look-back, two for the mbarrier, which waits a second time so that no
 * copy can still be in flight).  Blocking; the context stays usable. */
ns_status ns_diag_wait_timeout(int which, ns_stream_t stream);

/* Diagnostic of the hardware ceiling the hash ingest is bound by (no
 * counterpart in the paper): `threads` threads each add 1 at one
 * pseudo-random 8-byte word of each of three tables of table_words words
 * (a power of two) -- the link, row and column updates of one packet, with
 * no hashing or probing.  *best_us receives the fastest of `reps` timed
 * launches (after one warm-up).  Allocates and frees its tables; blocking. */
ns_status ns_diag_random_atomics(uint64_t table_words, uint64_t threads, int reps, double* best_us,
                                 ns_stream_t stream);

/* Diagnostic of the ceiling set by the hash ingest's own access structure
 * (no counterpart in the paper).  Three tables of table_slots 16-byte slots
 * (a power of two >= 1024); `threads` threads each touch one pseudo-random
 * slot of each table:
 *   NS_DIAG_CLAIM       three 128-bit compare-and-swap claims from the empty
 *                       value, issued together (one round trip);
 *   NS_DIAG_CLAIM_ADD   the claims, then -- dependent on them -- an 8-byte
 *                       add on the second and third slots: the two round
 *                       trips an ingested packet takes (link, row and column
 *                       claims; then the row and column updates);
 *   NS_DIAG_CLAIM_STALE every slot holds an old entry: the claim from the
 *                       empty value fails and a second compare-and-swap from
 *                       the value it returned claims the slot, then the
 *                       dependent adds -- what marking slots with an epoch,
 *                       instead of clearing the tables, costs on a slot's
 *                       first touch after a clear.
 * *best_us receives the fastest of `reps` timed launches (after one
 * warm-up).  Allocates (3 x 16 x table_slots bytes) and frees its tables;
 * blocking.  NS_ERR_INVALID for a bad argument. */
enum { NS_DIAG_CLAIM = 0, NS_DIAG_CLAIM_ADD = 1, NS_DIAG_CLAIM_STALE = 2 };
ns_status ns_diag_random_claims(uint64_t table_slots, uint64_t threads, int mode, int reps, double* best_us,
                                ns_stream_t stream);

/* ---- errors ------------------------------------------------------------ */

const char* ns_last_error(void);
const char* ns_status_string(ns_status s);

#ifdef __cplusplus
}
#endif

#endif /* NS_H */
