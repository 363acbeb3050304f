/*
 * embedjoin.h -- C ABI of the GB300-native EmbedJoin hot path.
 *
 * Computes the edit-similarity self-join of Section 1 of Zhang & Zhang,
 * "EmbedJoin: Efficient Edit Similarity Joins via Embeddings" (arXiv 1702.00093):
 *     { (s_i, s_j) : i != j, ED(s_i, s_j) <= K }
 * with the randomised method of Algorithms 1-3: CGK embedding (Alg. 1),
 * bit-sampling LSH with AND/OR amplification (Section 3.2, Thm. 1), bucketing of
 * equal signatures with the length filter of Alg. 3, and Ukkonen-banded
 * verification (Section 3.3). All work runs in hand-written CUDA kernels on one
 * GPU (sm_103a). Output has 100% precision; recall depends on r, m, z, L.
 *
 * Naming: r = CGK embeddings per string, m = LSH functions per embedding,
 * z = sampled positions per function. (Table 1 of the paper calls the number of
 * functions z and the signature length m: the letters are swapped here.)
 *
 * Conventions for every entry point
 *  - Return value: an ej_status (0 = EJ_OK). No exception crosses the ABI.
 *    ej_last_error(ctx) gives a one-line description of the last failure.
 *  - Pointers: every array argument may be device memory or host memory
 *    (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes and stages host arrays through its own device
 *    buffers. Parameter structs and scalar out-pointers (n_pairs, n_out,
 *    info, stats) are always host memory.
 *  - Ownership: the caller owns every input and output array. The context
 *    owns its scratch memory and reuses it across calls; scratch grows on
 *    demand and is released by ej_destroy.
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *    Kernels are enqueued on it. Entry points that return a count (ej_plan,
 *    ej_lsh_candidates, ej_verify, ej_join) synchronise that stream before
 *    returning, so the count and the output are valid on return. ej_embed and
 *    ej_sign are asynchronous when all their arrays are device memory.
 *  - One context must not be used by two host threads at once.
 *  - Strings: a packed byte buffer plus n+1 int64 offsets (offsets[0] = 0,
 *    non-decreasing); string i is bytes[offsets[i] .. offsets[i+1]).
 *    n < 2^31, every string shorter than 2^31 bytes, and every byte must be
 *    one of params->alphabet (else EJ_ERR_INVALID_ARG).
 *  - Pairs: uint64 (i << 32) | j with 0 <= i < j < n in input order; every
 *    list of pairs this library returns is sorted ascending and unique.
 */
#ifndef EMBEDJOIN_H
#define EMBEDJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ej_ctx ej_ctx;

typedef enum {
    EJ_OK = 0,
    EJ_ERR_INVALID_ARG = 1,  /* bad parameter, offsets or symbol outside the alphabet */
    EJ_ERR_OOM = 2,          /* device or host allocation failed */
    EJ_ERR_CAPACITY = 3,     /* output larger than the given capacity; the needed
                                count is written to the count out-pointer */
    EJ_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    EJ_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    EJ_ERR_UNSUPPORTED = 6,  /* valid request outside what the kernels support
                                (e.g. a band wider than the verifier's limit) */
    EJ_ERR_TOO_LARGE = 7     /* the request needs more scratch than the fixed
                                array of ej_verify_noalloc holds */
} ej_status;

/* Size of the fixed device scratch array used by ej_verify_noalloc. */
#define EJ_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* Method parameters (Table 1; Alg. 2 and Alg. 3 inputs). */
typedef struct {
    uint32_t r;              /* CGK embeddings per string, 1..255 */
    uint32_t m;              /* LSH functions per embedding, 1..65535 */
    uint32_t z;              /* sampled positions per function, >= 1, with
                                (alphabet_size+1)^z < 2^64 (exact 64-bit keys) */
    uint32_t L;              /* truncation (Section 4.1): positions are drawn from
                                [0, L); 0 => out_len */
    uint32_t out_len;        /* embedding length; 0 => 3N, N = longest string
                                (Alg. 1). Must be >= L. */
    int32_t K;               /* edit distance threshold, inclusive, >= 0 */
    uint64_t seed;           /* seeds the random strings R^l and the positions */
    const uint8_t *alphabet; /* host pointer: alphabet_size distinct raw bytes; the
                                index of a byte here is its symbol code */
    uint32_t alphabet_size;  /* 1..255; the padding symbol (bottom) gets code
                                alphabet_size */
} ej_params;

typedef struct {
    const uint8_t *bytes;    /* packed string bytes (device or host) */
    const int64_t *offsets;  /* n+1 offsets (device or host) */
    int64_t n;               /* number of strings */
} ej_strings;

/* Sizes derived from the strings and parameters (filled by ej_plan). */
typedef struct {
    int64_t n;               /* strings */
    int64_t max_len;         /* N, the longest string */
    int64_t total_bytes;     /* offsets[n] */
    uint32_t out_len;        /* effective embedding length */
    uint32_t L;              /* effective sampling range */
    uint32_t planes;         /* bit planes per embedded symbol: ceil(log2(alphabet_size)), >= 1 */
    uint32_t blocks32;       /* ceil(n / 32): string blocks of the embedding layout */
    uint64_t embedding_bytes;/* bytes of the ej_embed output */
    uint64_t walk_end_count; /* r * n int32 entries of walk_end */
    uint64_t key_count;      /* r * m * n uint64 entries of ej_sign output */
} ej_plan_info;

/* Counters of one join (filled by ej_join when stats != NULL). */
typedef struct {
    int64_t n_raw_pairs;     /* bucket pairs passing the length filter, before dedup */
    int64_t n_candidates;    /* unique candidate pairs (verified) */
    int64_t n_out;           /* output pairs */
    int64_t max_bucket;      /* largest bucket (run of equal keys in one table) */
    /* stage times in ms from CUDA events on `stream` (only with ej_set_timing(ctx, 1)) */
    float ms_prepare;        /* validation, packing, random tables, positions */
    float ms_embed_sign;     /* CGK walks and signature keys */
    float ms_candidates;     /* sort, bucket windows, pair sort, dedup */
    float ms_verify;         /* the verification kernel alone */
    float ms_total;          /* the whole call */
    uint64_t band_cells;     /* sum over candidates of the Ukkonen band size
                                |{(a,b): a<|x|, b<|y|, |a-b|<=K}| (work of the
                                verification, counted algorithmically) */
    uint64_t verify_word_columns; /* 64-bit words of the band the verifier runs
                                times the columns it actually advanced (early
                                exit included): the persistent verifier runs the
                                diagonals a cost-K alignment can use given the
                                pair's length difference d, K_lo + K_hi + 1 <= K + 1
                                (K_lo = floor((K-d)/2), K_hi = floor((K+d)/2)),
                                ceil((K_lo + K_hi + 1)/64) words; the others run
                                Ukkonen's 2K+1 diagonals, ceil((2K+1)/64) words */
    int64_t kernel_launches; /* CUDA kernels this call launched */
    /* finer stage times (ms, only with ej_set_timing(ctx, 1)): the part of
       ms_prepare spent validating and packing the strings, and ms_candidates
       split into the bucket stage (signature sets, or sorted tables, and the
       emission of raw pairs) and the deduplication with the candidate order */
    float ms_pack;
    float ms_buckets;
    float ms_dedup;
    float ms_reserved;       /* 0 */
} ej_join_stats;

/* Create a context bound to CUDA device `device`. *ctx is NULL on failure. */
int ej_create(ej_ctx **ctx, int device);

/* Release the context and all its scratch memory. NULL is ignored. */
void ej_destroy(ej_ctx *ctx);

/* Static description of a status code; never NULL. */
const char *ej_status_string(int status);

/* Description of the last error on this context ("" if none). Valid until the
 * next call on the context. */
const char *ej_last_error(ej_ctx *ctx);

/* Turn per-stage CUDA-event timing of ej_join on (1) or off (0). */
int ej_set_timing(ej_ctx *ctx, int enable);

/*
 * Verifier tiling (the autotuner's knob). lanes_per_pair selects the kernel:
 *   1: one lane per pair, diagonal window of V = 1..8 words (64V >= 2K+1);
 *   2: two lanes per pair (forward and backward halves meeting at the middle
 *      column), block-aligned window of V = 2..12 words (64(V-1) >= 2K+1);
 *   4, 8, 16, 32: that many lanes per pair, V = 1..4 words each (64GV >= 2K+1).
 * warps_per_block 0 = automatic (at most 4 for lanes_per_pair <= 2). All zero
 * restores the automatic choice. A configuration that cannot cover the band of
 * a later call falls back to the automatic choice. Results never depend on it.
 */
int ej_set_verify_config(ej_ctx *ctx, int lanes_per_pair, int words_per_lane, int warps_per_block);

/*
 * Failure detection (the paper has no counterpart): the persistent verifier
 * (ej_schedule.mode 1, and the merged launch of a batch) bounds the passes of
 * each warp's work loop, so that a kernel that could not finish its queue
 * stops instead of running on. When the bound runs out the kernel records it
 * and returns, and the call reports EJ_ERR_TIMEOUT; the context stays usable.
 * passes: loop passes per warp (one pass advances the warp's pairs by 64
 * columns); 0 restores the default of 2^24, far above what any valid input
 * needs. A small value is a test hook that makes the bound run out on
 * ordinary input. Calls made after this one use it; a graph-captured batch
 * keeps the value it was created with. Errors: EJ_ERR_INVALID_ARG for
 * passes < 0.
 */
int ej_set_loop_bound(ej_ctx *ctx, int64_t passes);

/*
 * Measurement helper (the paper has no counterpart): the throughput of the
 * GPU's 32-bit integer instructions, the roofline denominator of the verifier,
 * whose inner step is 32-bit logic, adds with carry and shifts. Every thread of
 * a full-occupancy grid runs independent chains (iters passes of 64
 * instructions) of lop3.b32 and add.u32 alternating (mix 0), lop3.b32 only
 * (mix 1) or add.u32 only (mix 2); the best of three timed launches (CUDA
 * events) gives *ops_per_s, instructions per second over the whole GPU, and
 * *ms its duration. Allocates 4 bytes and a stream of its own.
 * Errors: EJ_ERR_INVALID_ARG (mix outside 0..2, iters <= 0, NULL ops_per_s),
 * EJ_ERR_CUDA.
 */
int ej_measure_int_peak(int device, int32_t mix, int32_t iters, double *ops_per_s, double *ms);

/*
 * Similarity search against a resident index (EmbedJoin's structure kept on the
 * device; the paper has no serving counterpart). ej_index_create packs the
 * strings, builds the walk tables and sampled positions of `params` (r, m, z, L,
 * seed, alphabet; K is not used; L must be > 0 so that queries of any length are
 * walked over the same sampling range) and groups every string's r*m signatures
 * into per-table buckets. Synchronises `stream`. The index keeps its own device
 * memory (packed strings, tables, buckets: about 1.4 GB for 10^6 strings with
 * r = m = 7) until ej_index_destroy.
 *
 * ej_index_search finds, for every query q (host strings) with threshold K[q],
 * the index strings s that share a signature with q in some table, pass
 * ||q| - |s|| <= K[q] and have ED(q, s) <= K[q] (the join's candidate rule and
 * test, from the query's side). Output: (q << 32 | s) ascending, q = query
 * position, s = index position. Synchronous (one search batch; stream unused).
 * Errors: EJ_ERR_INVALID_ARG (a query byte outside the alphabet, bad offsets,
 * K < 0, device query buffers), EJ_ERR_CAPACITY (*n_out = needed).
 */
typedef struct ej_index ej_index;
int ej_index_create(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, ej_index **index,
                    void *stream);
int64_t ej_index_size(const ej_index *index);
int ej_index_search(ej_ctx *ctx, ej_index *index, const ej_strings *queries, const int32_t *K, uint64_t *out,
                    int64_t capacity, int64_t *n_out, void *stream);
void ej_index_destroy(ej_index *index);

/*
 * Serving loop over an index with continuous batching. A worker thread keeps up
 * to `inflight` search batches on the GPU, each on its own stream with its own
 * scratch; whenever one finishes it delivers its results and the requests that
 * arrived meanwhile form the next batch (up to max_batch queries and
 * max_batch_bytes query bytes), so batches overlap on the device. Every slot's
 * scratch is sized for a full batch at creation (if that fits hbm_budget) and
 * at least doubles when a batch needs more. A batch whose scratch would have to
 * grow is admitted only if the growth fits the free device memory minus
 * hbm_reserve and the server's total stays within hbm_budget (0 = no budget):
 * otherwise it waits while other batches are in flight; with none in flight it
 * is cut to fewer queries, and a single query that still does not fit finishes
 * with status EJ_ERR_OOM. Results are the same as ej_index_search for the same
 * query and K, whatever else is in flight.
 *   ej_server_submit copies the query and returns a request id >= 0, or
 *     -EJ_ERR_INVALID_ARG (byte outside the alphabet, K < 0).
 *   ej_server_poll returns up to `max` finished requests (waiting up to wait_us
 *     for the first); `matches` (ascending index positions) stays valid until
 *     ej_server_release(id). latency_ms = submit to results; queue_ms = submit to
 *     the launch of its batch.
 *   ej_server_get_stats: latency percentiles over the requests finished since the
 *     start or the last ej_server_reset_stats, batches, mean batch size,
 *     queries/s over that span, capacity retries, deferred admissions.
 */
typedef struct ej_server ej_server;
typedef struct {
    int32_t max_batch;          /* queries per batch (0 = 256) */
    int32_t inflight;           /* batches on the GPU at once (0 = 4) */
    int64_t max_batch_bytes;    /* query bytes per batch (0 = 8 MiB) */
    uint64_t hbm_reserve;       /* device memory left free (0 = 1 GiB) */
    uint64_t hbm_budget;        /* cap on the server's scratch (0 = none) */
} ej_server_config;
typedef struct {
    int64_t id;
    int32_t status;
    int32_t n_matches;
    const uint32_t *matches;
    double latency_ms;
    double queue_ms;
} ej_search_result;
typedef struct {
    int64_t completed, batches, retries, deferred;
    double mean_batch, p50_ms, p99_ms, mean_ms, queries_per_s;
    uint64_t device_bytes;
} ej_server_stats;
int ej_server_create(ej_index *index, const ej_server_config *config, ej_server **server);
int64_t ej_server_submit(ej_server *server, const uint8_t *query, int32_t len, int32_t K);
int ej_server_poll(ej_server *server, ej_search_result *out, int32_t max, int32_t *n, int32_t wait_us);
int ej_server_release(ej_server *server, int64_t id);
int ej_server_get_stats(ej_server *server, ej_server_stats *stats);
int ej_server_reset_stats(ej_server *server);
void ej_server_destroy(ej_server *server);

/*
 * Batched joins as one CUDA graph (a performance form of ej_join; the paper has
 * no counterpart). ej_batch_create plans the strings once (validate, pack),
 * runs every parameter set once eagerly to size all buffers (the raw-pair
 * capacity gets a margin of 1/8), optionally autotunes each join's back half on
 * its own data (EJ_BATCH_AUTOTUNE: the verifier choice of the autotuner, see
 * ej_set_autotune; an entry of the context's table for the join's length class
 * and K is used as it is),
 * and captures the whole device path of all joins into one graph: validate and
 * pack once, then per parameter set, on its own stream so that the joins
 * overlap, the walk and signatures, buckets, pairs, dedup and verification.
 * Work that several parameter sets share is done once. A set whose (r, m, z)
 * another set with the same seed and L covers takes its signatures from that
 * set's walks (the key of fewer samples is the wider key modulo
 * (|alphabet|+1)^z). Sets with the same seed, L, r and m take their raw pairs
 * from the buckets of the one with the smallest z (ej_schedule.buckets). The
 * sets on the persistent verifier are verified by one merged launch, a pair
 * that several sets list once, at the largest of their K (ej_schedule.chain).
 * Every set still gets exactly ej_join's candidates and output.
 * ej_batch_run replays the graph on `stream` without any host synchronisation;
 * the run itself sorts every join's output (up to 8192 pairs) and stages the
 * counters in pinned host memory. ej_batch_result(i) waits for the run and
 * returns join i's pairs (sorted, the same as ej_join with params[i]) and its
 * counters (no stage timings; kernel_launches counts the kernels of the result
 * call itself: a sort of a larger output). A device `out` is written in stream
 * order on `stream`; a host `out` is complete on return.
 *
 * The strings must be in device memory; the graph reads them at the addresses
 * given here, so their contents may be rewritten between runs (by the caller,
 * on the same stream) as long as n stays, offsets[n] does not grow and the
 * longest string does not grow (nor change, when out_len and L are 0).
 * ej_batch_result reports a violation (EJ_ERR_INVALID_ARG) or raw pairs beyond
 * the capacity (EJ_ERR_CAPACITY); re-create the batch then. All parameter sets
 * share one alphabet; injected test tables are not supported. The stream must
 * not be the legacy default stream (it is captured). The batch keeps its own
 * scratch per parameter set and must be destroyed before its context.
 */
typedef struct ej_batch ej_batch;
#define EJ_BATCH_AUTOTUNE 1
/* EJ_BATCH_EAGER: no graph; every ej_batch_run issues the same device work on
 * its stream (for tools that cannot follow graph launches, e.g. per-kernel
 * profilers). ej_batch_create then also runs the batch once. */
#define EJ_BATCH_EAGER 2
int ej_batch_create(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, int32_t n_params,
                    int32_t flags, ej_batch **batch, void *stream);
int ej_batch_run(ej_batch *batch, void *stream);
int ej_batch_result(ej_batch *batch, int32_t index, uint64_t *out, int64_t capacity, int64_t *n_out,
                    ej_join_stats *stats, void *stream);
/* Kernel launches one ej_batch_run makes (kernel nodes of the graph). */
int64_t ej_batch_kernel_count(const ej_batch *batch);
/* Device time (ms, CUDA events on its stream) of the merged verifier launch in
 * the last run of an EJ_BATCH_EAGER batch (see ej_schedule.chain); waits for it.
 * EJ_ERR_INVALID_ARG if the batch is a graph, has no merged launch or has not run. */
int ej_batch_verify_ms(ej_batch *batch, float *ms);
void ej_batch_destroy(ej_batch *batch);

/*
 * Schedule of ej_join's back half (a performance choice: the output never
 * depends on it; the paper has no counterpart).
 *   mode: 1: persistent verifier where the band fits two lanes per pair (up to
 *     12 words per lane): a fixed grid whose warps pull candidate pairs from a
 *     device work queue and refill a pair slot as soon as its pair is decided;
 *     otherwise the grid-strided verifier. 2: always the grid-strided verifier
 *     (one pass over the pairs; a warp's slots start together and the warp ends
 *     with its slowest pair). 3: the shared-string verifier: the candidates are
 *     grouped by their longer string x into warp tasks of up to 16 pairs, and
 *     the warp keeps one ring of x's match masks per direction for all of them
 *     (built cooperatively, once per task), instead of one per lane (two lanes
 *     per pair, up to 12 words per lane). 0 (default): 1 when the strings' mean
 *     length is at least 2048 (long pairs, where refilling pays); else 3 for
 *     alphabets of more than 4 symbols (whose per-lane rings leave the
 *     grid-strided verifier one or two warps per SM) and 2 for the rest.
 *   chain (batches): how the verifiers of a batch's joins share the GPU: the
 *     persistent ones merged, chained or overlapping, the grid-strided ones
 *     chained unless chain is 1 (the other stages always overlap); see the
 *     field.
 *   slots_per_warp: 0 = 16, else 1..16 pair slots per warp.
 *   warps_per_subpartition: 1..16: at most that many working warps per SM
 *     sub-partition (4 per SM); slots beyond the batch refill from the queue.
 *     0 (default): from the pair count, 1 while one warp's slots would take
 *     fewer than 8 pairs each (more warps only start every pair at once, and a
 *     launch ends with its slowest pairs), 2 below 32, else 4.
 *   order: the order in which candidates enter the verifier. 4: by length
 *     class, longest first (the shorter string's length in 256 classes), so
 *     that the pairs a warp takes have similar lengths and the longest start
 *     first; 5: by the pair's longer string (the one whose match masks the
 *     verifier builds) and, with mode 3 (which always uses it), by the class of
 *     the length difference; 3: by the pair's first string
 *     (a counting sort: the pairs a warp
 *     takes share their first string, so they read the same memory and, through
 *     the length filter, have similar lengths); 1: by decreasing number of tables
 *     in which the two strings collided; 2: hash-table order. 0 (default): 4
 *     with the persistent verifier, 3 with the grid-strided one, 5 with the
 *     shared-string one (whose candidates are grouped by a sort, not a hash
 *     table). In a batch's union launch (chain 0 / 4) the joins' candidates
 *     keep hash order and the union is ordered by the shorter string's length
 *     class, then by the number of joins that list the pair (1: that number
 *     first).
 *   buckets: 0 (default) or 1: equal signatures are grouped by hashing (per
 *     table an open-addressing set whose slots head lists of records); a
 *     record pairs with the later records of its list, so a bucket of b strings
 *     costs b*(b-1)/2 length checks. In a batch, 0 also shares buckets: joins
 *     with the same seed, L, r and m (up to 4) take their pairs from the
 *     buckets of the one with the smallest z, whose signatures are the coarsest
 *     (a signature of z samples is one of more samples modulo (|alphabet|+1)^z),
 *     each partner checked against the join's own signature and K; 1 keeps
 *     every join's own buckets. Tables of up to 21845 records are bucketed in
 *     shared memory, one block per table, which pays for small buckets only;
 *     a batch moves a join whose sizing pass finds a bucket of more than 256
 *     records to the buckets in global memory, and one with a bucket of more
 *     than 4096 records to the sorted tables (2), unshared.
 *     2: the tables are sorted by (signature, length) and each record pairs
 *     with the window after it (the ej_lsh_candidates path). It is much
 *     cheaper when a few signatures collect thousands of strings, e.g. short
 *     strings whose walks end early and whose samples are mostly the bottom
 *     symbol.
 */
typedef struct {
    int32_t mode;
    int32_t slots_per_warp;
    int32_t warps_per_subpartition;
    int32_t order;
    int32_t buckets;
    int32_t chain;   /* batches: joins on the grid-strided verifier are verified one after
                        another unless chain is 1. Joins that use the persistent verifier:
                        4: one merged launch over the union of their candidates: every
                        distinct pair once, at the largest K of the joins that list it, in
                        the widest of their bands; its distance (exact up to that K) decides
                        it for each of them (joins whose signatures nest, e.g. the prefix
                        keys of a batch, share most candidates); pairs listed by more joins
                        enter the queue first; 3: one merged launch over the joins'
                        candidates in turn, largest K first, each pair with its own join's
                        K (the queue runs from one join's pairs into the next, so no join
                        waits for another's last pairs); 2: one launch per join, one after
                        another; 1: one launch per join, free to overlap (two persistent
                        grids sharing the SMs were measured up to 10x slower at times);
                        0 (default): when the wider band adds at most half the
                        word-columns of the joins' own bands (candidate counts of the
                        sizing pass), 4 while the joins' candidates come to fewer than
                        32 per pair slot of one warp per SM sub-partition (the launch is
                        then set by its longest pairs), else 3; otherwise 2 */
} ej_schedule;

/* NULL restores the defaults. Errors: EJ_ERR_INVALID_ARG for values outside
 * the ranges above. */
int ej_set_schedule(ej_ctx *ctx, const ej_schedule *schedule);

/*
 * Autotuner (a performance choice; the output never depends on it). With
 * ej_set_autotune(ctx, 1), ej_join looks up its (length class, K) in the
 * context's table, where the length class is floor(log2(mean string length));
 * on a miss it tunes on the call's own strings and candidates before the join:
 *  - the fused walk's walks (strings) per block: 256, 512 or 1024;
 *  - the verifier and its tiling: the persistent verifier with 16 or 8 pair
 *    slots per warp and one or two working warps per SM sub-partition, the
 *    shared-string verifier, the grid-strided two-lane verifier in
 *    first-string or length-class order, one lane per pair with the band in
 *    registers (bands of up to 8 words), and four lanes per pair (up to 4 words
 *    each); every choice is timed twice (CUDA events) after a warm-up run, on
 *    the join's own candidates, and the fastest is kept in the table.
 * Later joins of the same class and K use the entry without tuning. A batch
 * created with EJ_BATCH_AUTOTUNE tunes each join's back half the same way (or
 * uses the context's entry) and records it in the table. ej_autotune_table
 * copies up to `max` entries, *n = the table's size. ej_set_autotune(ctx, 0)
 * stops using the table; ej_set_autotune(ctx, -1) also clears it.
 */
typedef struct {
    int32_t length_class;    /* floor(log2(mean string length)) */
    int32_t K;
    int32_t walk_threads;    /* walks (strings) per block of the fused walk (0: not tuned) */
    int32_t lanes_per_pair;  /* verifier tiling as for ej_set_verify_config (0 = automatic) */
    int32_t words_per_lane;
    int32_t configs_tried;
    ej_schedule schedule;    /* mode, slots_per_warp, warps_per_subpartition, order chosen */
    float walk_ms;           /* the chosen walk on the tuning join (0: not tuned) */
    float back_ms;           /* the chosen back half: buckets, pairs, dedup, verification */
} ej_tune_entry;
int ej_set_autotune(ej_ctx *ctx, int enable);
int ej_autotune_table(ej_ctx *ctx, ej_tune_entry *out, int32_t max, int32_t *n);

/*
 * Validate the strings against the parameters and report the derived sizes
 * (N, out_len = 3N or params->out_len, L, the embedding layout). Checks
 * offsets (start at 0, non-decreasing), lengths (< 2^31), symbols (all in the
 * alphabet) and parameters (Section 4 constraints listed on ej_params).
 * Synchronises `stream`.
 */
int ej_plan(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, ej_plan_info *info,
            void *stream);

/*
 * CGK embedding (Algorithm 1) of every string, r times.
 * Walk of string x under embedding l: i = 0; for step j = 0 .. out_len-1:
 * if i < |x| emit x[i] and advance i by pi_j^l(x[i]), else emit bottom.
 * pi_j^l(sigma) is the top bit of splitmix64(splitmix64(seed) ^ (1<<56 | l<<48 |
 * j<<8 | sigma)) with sigma the raw byte (the library's reading of the random
 * string R^l of Alg. 1; splitmix64 as published by Steele, Lea and Flood 2014).
 *
 * emb (device or host, info.embedding_bytes bytes), bit-sliced layout:
 *   uint32 word emb[((l * blocks32 + B) * out_len + j) * planes + k]
 *   bit t of that word = bit k of the code of t^l_{32B+t}[j] (0 for strings
 *   >= n and for steps at or after walk_end).
 * walk_end (int32, r*n, [l][i]): the first step whose output is bottom
 *   (out_len if the walk does not finish; 0 for an empty string).
 */
int ej_embed(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, void *emb,
             int32_t *walk_end, void *stream);

/*
 * Bit-sampling LSH signatures (Theorem 1 with AND amplification, Section 3.2):
 * for table t = l*m + f and string i,
 *   keys[t * n + i] = sum_{q<z} c_q * (alphabet_size+1)^q
 * where c_q is the code of t^l_i[P[l][f][q]] (alphabet_size if that step is at
 * or after walk_end) and P[l][f][q] = mulhi64(splitmix64(splitmix64(seed) ^
 * (2<<56 | l<<48 | f<<32 | q)), L) -- positions drawn with replacement from
 * [0, L). emb/walk_end are ej_embed's outputs for the same strings and params.
 */
int ej_sign(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, const void *emb,
            const int32_t *walk_end, uint64_t *keys, void *stream);

/*
 * ej_embed followed by ej_sign without materialising the embedding: the same
 * keys (bit-identical), computed by walking each string once per embedding and
 * reading only the m*z sampled steps (the "only compute the sampled bits"
 * remark of Section 4). keys: [r*m][n] uint64 as for ej_sign. This is the path
 * ej_join uses.
 */
int ej_embed_sign(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, uint64_t *keys,
                  void *stream);

/*
 * Candidate pairs (Algorithm 3, filtering stage): all i < j such that some
 * table t has keys[t*n+i] == keys[t*n+j] and ||s_i| - |s_j|| <= K (the
 * length filter of Alg. 3), deduplicated (Alg. 3 removes duplicate pairs).
 * keys is ej_sign's output. Writes up to `capacity` pairs to `pairs`; on
 * overflow returns EJ_ERR_CAPACITY with the needed count in *n_pairs.
 * If stats_max_bucket != NULL it receives the largest bucket size.
 */
int ej_lsh_candidates(ej_ctx *ctx, const ej_strings *strings, const ej_params *params,
                      const uint64_t *keys, uint64_t *pairs, int64_t capacity, int64_t *n_pairs,
                      int64_t *stats_max_bucket, void *stream);

/*
 * Verification (Section 3.3; last loop of Alg. 3): keeps the pairs with
 * ED(s_i, s_j) <= params->K (only K and the alphabet of params are used).
 * Pairs need not be sorted or unique; i and j must be < n. Output keeps the
 * input order; `out` must hold n_pairs entries. Exact: the result equals a full
 * Ukkonen band DP. Supports K up to 4095.
 */
int ej_verify(ej_ctx *ctx, const ej_strings *strings, const ej_params *params,
              const uint64_t *pairs, int64_t n_pairs, uint64_t *out, int64_t *n_out, void *stream);

/*
 * ej_verify without any memory allocation (the paper has no counterpart; this
 * is a deployment variant of the verification step).
 *
 * For callers that cannot let a library allocate: processes whose device memory
 * is reserved up front by another allocator, and services that must not call
 * cudaMalloc/cudaFree on their request path (those calls can synchronise the
 * device). No context is needed; the call never allocates. Its scratch is one
 * file-scope device array of EJ_NOALLOC_SCRATCH_BYTES (64 MiB). A GPU holds it
 * from when the array's module is loaded on it until the process exits: with
 * lazy module loading (the CUDA default) that is the first call on that
 * device, with eager loading (CUDA_MODULE_LOADING=EAGER) the library load.
 *  - strings->bytes, strings->offsets, pairs and out must be device memory;
 *    params supplies K and the alphabet only; out holds n_pairs entries.
 *  - Output and result are those of ej_verify (passing pairs in input order,
 *    count in *n_out); the call synchronises `stream` before returning.
 *  - Scratch needed: about 16 bytes per string, the packed codes (total bytes x
 *    2/8 for alphabets of at most 4 symbols, else x 1) and 9 bytes per pair;
 *    beyond EJ_NOALLOC_SCRATCH_BYTES the call returns EJ_ERR_TOO_LARGE (checked
 *    before any scratch is written, also for counts whose byte size would
 *    overflow).
 *  - All calls share the array and it keeps the previous call's contents (the
 *    call clears what must start at zero). Calls whose GPU work overlaps, on
 *    different streams or host threads, race on it: serialise them.
 *  - The first call on a device looks the array's address up
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 */
int ej_verify_noalloc(const ej_strings *strings, const ej_params *params, const uint64_t *pairs,
                      int64_t n_pairs, uint64_t *out, int64_t *n_out, void *stream);

/*
 * The whole method (Algorithm 3 with Algorithm 2's preprocessing):
 * embed -> sign -> candidates -> verify. Writes up to `capacity` output pairs
 * (sorted ascending); on overflow returns EJ_ERR_CAPACITY with the needed count
 * in *n_out. n < 2 gives 0 pairs. stats may be NULL.
 */
int ej_join(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, uint64_t *out,
            int64_t capacity, int64_t *n_out, ej_join_stats *stats, void *stream);

/*
 * EmbedJoin+ (Section 5, Algorithms 4 and 5): the join for strings whose
 * alignments start with a long run of insertions (a shift), which plain
 * EmbedJoin's walks do not absorb. Every string s_i is embedded S times, as
 * its suffixes s_i[(k-1)*delta ..] for k = 1 .. S, S = ceil(K/delta) (at least
 * 1), each with the same random strings and sampled positions as ej_join
 * (out_len and L those of the whole strings). A match is a pair of substrings
 * (x, k_x), (y, k_y) of two different strings x, y with ||x| - |y|| <= K whose
 * signatures agree in one table; a pair (x, y) is a candidate when some
 * substring pair of it matches in at least T tables (Section 5 uses T = 2 when
 * S > 1, else 1, with which EmbedJoin+ is EmbedJoin). Candidates with
 * ED <= K are the output, sorted ascending as for ej_join.
 * stats: n_raw_pairs = matches (substring pairs, once per table), n_candidates,
 * n_out, max_bucket (records of one signature in one table, a record being one
 * substring), band_cells and verify_word_columns of the verification; stage
 * times as ej_join's when timing is on (ms_candidates covers the buckets, the
 * match counting and the dedup). Synchronises `stream`.
 * Errors: EJ_ERR_INVALID_ARG (delta <= 0, T < 1, and those of ej_join),
 * EJ_ERR_UNSUPPORTED (n * S * r * m records beyond 2^32), EJ_ERR_CAPACITY
 * (*n_out = needed).
 */
int ej_join_plus(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, int32_t delta, int32_t T,
                 uint64_t *out, int64_t capacity, int64_t *n_out, ej_join_stats *stats, void *stream);

/*
 * Fidelity options of Section 4 (the paper's own choices where this library
 * defaults to others).
 *
 * ej_set_key_hash: bucket keys by the paper's two-level hashing instead of the
 * exact key: the signature's z symbols as a vector u with entries 1..|alphabet|
 * (|alphabet|+1 for the padding symbol), a random vector v in [0, P)^z per
 * function (v[l][f][q] = mulhi64(splitmix64(splitmix64(seed) ^ (3<<56 | l<<48 |
 * f<<32 | q)), P)), key = <u, v> mod P. Equal signatures share a bucket as
 * before; different ones also share it with probability 1/P (extra candidates,
 * removed by the verification). Applies to ej_sign, ej_embed_sign, ej_join,
 * ej_join_plus and ej_join_grouped on this context; ej_batch_create rejects it
 * (EJ_ERR_UNSUPPORTED). P = 0 restores the exact keys; otherwise P must be a
 * prime in [2, 2^32) (EJ_ERR_INVALID_ARG), e.g. 1000003.
 *
 * ej_join_grouped: EmbedJoin with grouping instead of one embedding length for
 * all strings (Section 4.1): with N' = ceil(N/K) K, the strings fall into the
 * groups g = 1 .. N'/K - 1 (at least one) of lengths ((g-1)K, (g+1)K] (the
 * first group also holds the empty strings), so every pair within K in length
 * shares a group; each group is joined on its own (out_len = 3 N of the group,
 * the caller's r, m, z, L, K and seed) and the outputs are united (sorted,
 * unique, as for ej_join). stats: candidates, raw pairs and band work summed
 * over the groups (a pair in two groups counts twice), n_out of the union.
 * Needs K >= 1 (EJ_ERR_INVALID_ARG); other errors as for ej_join.
 */
int ej_set_key_hash(ej_ctx *ctx, uint64_t P);
int ej_join_grouped(ej_ctx *ctx, const ej_strings *strings, const ej_params *params, uint64_t *out,
                    int64_t capacity, int64_t *n_out, ej_join_stats *stats, void *stream);

/*
 * Test hook for the running example of Section 4 (Tables 2-4): replace the
 * random bits and positions with explicit tables (host pointers, copied).
 *   pi: [r][steps][alphabet_size] bytes in {0,1}, code-indexed; steps at or
 *       beyond `steps` read 0.
 *   positions: [r][m][z] uint32, each < L.
 * Either pointer may be NULL to keep the random source for that part.
 * ej_set_test_tables(ctx, NULL, 0, 0, 0, NULL, 0, 0) restores both.
 */
int ej_set_test_tables(ej_ctx *ctx, const uint8_t *pi, uint32_t r, uint32_t steps,
                       uint32_t alphabet_size, const uint32_t *positions, uint32_t m, uint32_t z);

#ifdef __cplusplus
}
#endif
#endif /* EMBEDJOIN_H */
