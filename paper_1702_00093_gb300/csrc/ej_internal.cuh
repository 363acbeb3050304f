// Internal declarations of the EmbedJoin CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/embedjoin.h"

namespace ej {

constexpr unsigned FULL = 0xffffffffu;

// SplitMix64 output function (Steele, Lea, Flood 2014): the counter-based
// source of the random strings R^l (Alg. 1) and of the sampled positions
// (Thm. 1). Written for the device here; the CPU oracle has its own copy.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t walk_counter(uint32_t l, uint64_t j, uint32_t sigma) {
    return (1ull << 56) | ((uint64_t)l << 48) | (j << 8) | (uint64_t)sigma;
}

__host__ __device__ __forceinline__ uint64_t position_counter(uint32_t l, uint32_t f, uint32_t q) {
    return (2ull << 56) | ((uint64_t)l << 48) | ((uint64_t)f << 32) | (uint64_t)q;
}

// Bit planes needed for symbol codes 0..alpha-1.
inline uint32_t planes_for(uint32_t alpha) {
    uint32_t b = 1;
    while ((1u << b) < alpha) b++;
    return b;
}

// u32 words per step of the code-indexed random-bit table.
inline uint32_t table_words_for(uint32_t planes) { return planes <= 5 ? 1u : (1u << (planes - 5)); }

// ---------------------------------------------------------------------------
// Packed symbol codes
// ---------------------------------------------------------------------------
// Every string is re-encoded once as dense codes (index in the alphabet) of
// B = 2 (alphabets of at most 4 symbols) or 8 bits, little-endian inside 128-bit chunks; each string starts
// on its own chunk (16-byte aligned), chunk offsets in pofs[n+1].

inline int packed_bits_for(uint32_t alpha) { return alpha <= 4 ? 2 : 8; }

__host__ __device__ __forceinline__ int64_t chunks_for(int64_t len, int B) {
    return (len * B + 127) / 128;
}

// Sequential reader of one string's packed codes with a two-chunk prefetch:
// the next 16-byte chunk is requested 128/B symbols before it is needed.
template <int B>
struct SymReader {
    const uint4 *p;
    const uint4 *end;
    uint4 cur, nxt;
    int left;

    __device__ __forceinline__ void init(const uint4 *base, int64_t nchunks) {
        p = base;
        end = base + nchunks;
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        cur = (p < end) ? *p : zero;
        p += (p < end);
        nxt = (p < end) ? *p : zero;
        p += (p < end);
        left = 128 / B;
    }
    __device__ __forceinline__ uint32_t code() const { return cur.x & ((1u << B) - 1u); }
    __device__ __forceinline__ void advance() {
        cur.x = __funnelshift_r(cur.x, cur.y, B);
        cur.y = __funnelshift_r(cur.y, cur.z, B);
        cur.z = __funnelshift_r(cur.z, cur.w, B);
        cur.w >>= B;
        if (--left == 0) {
            cur = nxt;
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            nxt = (p < end) ? *p : zero;
            p += (p < end);
            left = 128 / B;
        }
    }
};

// Number of kernels launched by this library (all threads); a launcher adds
// the kernels it enqueued.
void note_launches(int k);
int64_t launches_so_far();

// Device-side error bits.
enum : uint32_t {
    DERR_OFFSETS = 1u,     // offsets not starting at 0 / decreasing / too long
    DERR_SYMBOL = 2u,      // byte outside the alphabet
    DERR_PAIR = 4u,        // pair index out of range
    DERR_TIMEOUT = 8u,     // bounded wait gave up
    DERR_GUARD = 16u,      // a persistent loop exceeded its work bound and stopped
};

// ---------------------------------------------------------------------------
// Kernel launchers (each returns cudaGetLastError() of its launch)
// ---------------------------------------------------------------------------

// Validation + lengths: lens[i] = offsets[i+1]-offsets[i]; err |= DERR_*;
// stats[0] = max length (int64 via unsigned max), stats[1] = total bytes.
cudaError_t launch_validate(const uint8_t *bytes, const int64_t *offsets, int64_t n, int64_t total_cap,
                            const uint8_t *code_map, int32_t *lens, uint32_t *err,
                            unsigned long long *max_len, cudaStream_t s);

// Random-bit table [r][out_len][words]: bit c of row (l, j) = pi_j^l(alphabet[c]).
cudaError_t launch_bit_table(uint64_t seed, uint32_t r, uint32_t out_len, const uint8_t *alphabet_dev,
                             uint32_t alpha, uint32_t words, const uint8_t *pi_inject,
                             uint32_t inject_steps, uint32_t *table, cudaStream_t s);

// Positions [r][m][z] in [0, L).
cudaError_t launch_positions(uint64_t seed, uint32_t r, uint32_t m, uint32_t z, uint32_t L,
                             const uint32_t *pos_inject, uint32_t *pos, cudaStream_t s);

// Chunk counts per string (u32) from lengths.
cudaError_t launch_chunk_counts(const int32_t *lens, int64_t n, int B, uint32_t *counts, cudaStream_t s);
// Pack bytes -> codes; bytes outside the alphabet set DERR_SYMBOL (code 0 is stored).
// total: bytes in the array (every validated string lies inside [0, total)).
cudaError_t launch_pack(const uint8_t *bytes, const int64_t *offsets, const int32_t *lens, int64_t n, int64_t total,
                        const uint8_t *code_map, int B, const uint64_t *pofs, uint4 *packed,
                        uint32_t *err, cudaStream_t s);

cudaError_t launch_embed(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                         uint32_t r, const uint32_t *table, int B, uint32_t out_len, uint32_t planes,
                         uint32_t *emb, int32_t *walk_end, cudaStream_t s);

cudaError_t launch_sign(const uint32_t *emb, const int32_t *walk_end, int64_t n, uint32_t r,
                        uint32_t m, uint32_t z, uint32_t out_len, uint32_t planes, uint32_t alpha,
                        const uint32_t *pos, uint64_t *keys, cudaStream_t s);

// Fused embed + sign (arrival form of Alg. 1 restricted to the sampled steps).
// Per-symbol step bitmaps [r][alpha][LW]: bit b of word w = pi_{32w+b}(alphabet[c])
// for steps < L, 1 for steps >= L (sentinel); LW = L/32 + 2.
cudaError_t launch_symbol_table(uint64_t seed, uint32_t r, uint32_t L, const uint8_t *alphabet_dev,
                                uint32_t alpha, const uint8_t *pi_inject, uint32_t inject_steps,
                                uint32_t *tsym, cudaStream_t s);
size_t symbol_table_words(uint32_t r, uint32_t alpha, uint32_t L);
// Sampled steps of every embedding sorted by step: spos/stag [r][m*z], tag = f<<16 | q.
cudaError_t launch_sort_samples(const uint32_t *pos, uint32_t r, uint32_t m, uint32_t z, uint32_t *spos,
                                uint32_t *stag, cudaStream_t s);
// Shared memory the fused kernel needs (0 if it does not fit: use embed + sign).
// Shared memory of the fused walk with tpb walks per block (0 = the default 512);
// 0 if it does not fit.
size_t embed_sign_smem(uint32_t alpha, uint32_t L, uint32_t m, uint32_t z, int tpb = 0);
// next[l][c][a] = next1_c(a) + 1 (16-bit) when embed_sign_uses_table(alpha, L).
bool embed_sign_uses_table(uint32_t alpha, uint32_t L);
size_t next_table_elems(uint32_t r, uint32_t alpha, uint32_t L);
cudaError_t launch_next_table(const uint32_t *tsym, uint32_t r, uint32_t alpha, uint32_t L, uint16_t *next,
                              cudaStream_t s);
// Optional extra outputs of the fused walk: the keys of the first z[e] <= z
// samples of every function (the same walks and tables), keys[e] [r][m][n].
constexpr int MAX_PREFIX_KEYS = 3;
struct PrefixKeys {
    int32_t n;
    uint32_t z[MAX_PREFIX_KEYS];
    uint64_t *keys[MAX_PREFIX_KEYS];
};
cudaError_t launch_embed_sign(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                              uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t alpha, int B,
                              const uint32_t *tsym, const uint16_t *next, const uint32_t *spos,
                              const uint32_t *stag, uint64_t *keys, cudaStream_t s,
                              const PrefixKeys *prefix = nullptr, int tpb = 0);
// Keys [r][m][n] of (r, m, z) from keys [r_src][m_src][n] of a set with the same
// seed and L and r_src >= r, m_src >= m, z_src >= z: dst = src mod modulus
// ((alpha+1)^z; 0 = plain copy when z = z_src).
cudaError_t launch_derive_keys(const uint64_t *src, uint32_t m_src, int64_t n, uint32_t r, uint32_t m,
                               uint64_t modulus, uint64_t *dst, cudaStream_t s);

// The two-level hash <u, v> mod P of Section 4 in place of exact keys [r*m][n].
cudaError_t launch_keys_modp(uint64_t *keys, int64_t n, uint32_t r, uint32_t m, uint32_t z, uint32_t alpha,
                             uint64_t seed, uint64_t P, cudaStream_t s);
// Grouping (Section 4.1): strings idx[0..gn) gathered at offsets goff, and
// group-local output pairs mapped back to the set's ids.
cudaError_t launch_gather_strings(const uint8_t *bytes, const int64_t *offsets, const int32_t *idx, int64_t gn,
                                  const int64_t *goff, uint8_t *out, cudaStream_t s);
cudaError_t launch_remap_pairs(const uint64_t *pairs, int64_t cnt, const int32_t *idx, uint64_t *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Scan and sort primitives (ej_sort.cu)
// ---------------------------------------------------------------------------

// Exclusive prefix sums of n values into out (uint64), total into *total_dev
// (device pointer, may be null). Input types: u8, u32, u64.
size_t scan_temp_bytes(int64_t n);
cudaError_t exclusive_scan_u8(const uint8_t *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                              void *temp, cudaStream_t s);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                               void *temp, cudaStream_t s);

// Stable LSD radix sort of `nseg` independent segments of `seg_len` records
// each (segment k occupies [k*seg_len, (k+1)*seg_len)), by 8-bit digits at the
// given bit shifts (least significant first). vals may be null.
// keys/vals hold the input; the result ends in (keys, vals) or (keys_alt,
// vals_alt): the function returns which through *in_alt.
struct RadixTemp {
    uint32_t *counts;   // nseg * 256 * tiles_per_seg
    uint64_t *offsets;  // same size
    void *scan_temp;
};
size_t radix_counts_len(int64_t seg_len, int64_t nseg);
// len_dev (nseg == 1 only, may be null): a device count; only the first
// min(*len_dev, seg_len) records are sorted (the rest of both buffers is left
// as it is).
cudaError_t radix_sort_segmented(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                                 int64_t seg_len, int64_t nseg, const int *shifts, int npasses,
                                 RadixTemp tmp, bool *in_alt, cudaStream_t s,
                                 const unsigned long long *len_dev = nullptr);

// One block per table: stable sort of (key, id) records whose key has kb bits and
// whose ids need idb bits (idb + kb <= 64, n <= table_sort_max()); records start
// in perm order (perm may be null). Output keys and ids per table.
int table_sort_max();
cudaError_t launch_table_sort(const uint64_t *src, const uint32_t *perm, int64_t n, int64_t T, int idb, int kb,
                              uint64_t *out_keys, uint32_t *out_ids, cudaStream_t s);

// Candidates: gather keys into length order, per-table bucket windows.
cudaError_t launch_len_order_gather(const uint64_t *keys, const uint32_t *perm, int64_t n, int64_t T,
                                    uint64_t *rec_keys, uint32_t *rec_ids, cudaStream_t s);
cudaError_t launch_iota_u32(uint32_t *v, int64_t n, cudaStream_t s);
cudaError_t launch_len_keys(const int32_t *lens, int64_t n, uint64_t *k, cudaStream_t s);
cudaError_t launch_bucket_count(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens,
                                int64_t n, int64_t T, int32_t K, uint32_t *counts,
                                unsigned long long *max_bucket, cudaStream_t s);
cudaError_t launch_bucket_emit(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens,
                               int64_t n, int64_t T, int32_t K, const uint64_t *offs,
                               uint64_t *pairs, cudaStream_t s);
cudaError_t launch_unique_flags(const uint64_t *sorted, int64_t n, uint8_t *flags, cudaStream_t s);
cudaError_t launch_compact_u64(const uint64_t *in, const uint8_t *flags, const uint64_t *offs,
                               int64_t n, uint64_t *out, cudaStream_t s);

// Pipeline kernels (ej_pipeline.cu). counters: [0] raw pairs, [1] largest
// bucket, [2] candidates, [3] output pairs, [4..5] verifier work.
cudaError_t launch_emit_append(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens, int64_t n,
                               int64_t T, int32_t K, uint64_t *raw, uint64_t cap, unsigned long long *counters,
                               cudaStream_t s);
// EmbedJoin+ (ej_plus.cu): the suffix set of every string (record q = i*S + k)
// and the candidate pairs from the sorted record-pair matches.
cudaError_t launch_suffix_lengths(const int32_t *lens, int64_t n, int32_t S, int32_t delta, uint32_t *sub_len,
                                  int32_t *whole_len, cudaStream_t s);
cudaError_t launch_suffix_copy(const uint8_t *bytes, const int64_t *offsets, int64_t n, int32_t S, int32_t delta,
                               const uint64_t *sub_off, uint8_t *out, cudaStream_t s);
cudaError_t launch_plus_runs(const uint64_t *sorted, int64_t nraw, int32_t S, int32_t T, uint64_t *out,
                             uint64_t cap, unsigned long long *count, unsigned long long *same, cudaStream_t s);
// Buckets by hashing (ej_join): per-table signature sets of H slots
// (bucket_slots_per_table(n)); slot_keys filled with ~0, heads with 0xFF bytes.
uint64_t bucket_slots_per_table(int64_t n);
// Pairs of several joins from the record lists of the coarsest one's buckets
// (joins with the same seed, L, r, m; see bucket_emit_shared_kernel).
constexpr int MAX_SHARED_BUCKETS = 4;
struct SharedEmit {
    int32_t njoins;
    const uint64_t *keys[MAX_SHARED_BUCKETS];        // each join's signatures [T][n]
    int32_t K[MAX_SHARED_BUCKETS];
    uint64_t *raw[MAX_SHARED_BUCKETS];
    uint64_t cap[MAX_SHARED_BUCKETS];
    unsigned long long *counters[MAX_SHARED_BUCKETS];   // [0] raw pairs, [1] largest bucket
};
cudaError_t launch_bucket_emit_shared(const int32_t *lens, int64_t n, int64_t T, const uint32_t *next,
                                      const SharedEmit &se, cudaStream_t s);
// The same pairs with each table's buckets built in shared memory by one block
// (bucket_table_smem(n) > 0: n below 2^16 - 2 and the slots fit); se.keys[0]
// are the bucket signatures. No global bucket state.
size_t bucket_table_smem(int64_t n);
cudaError_t launch_bucket_table(const int32_t *lens, int64_t n, int64_t T, const SharedEmit &se, cudaStream_t s);
cudaError_t launch_bucket_insert(const uint64_t *keys, int64_t n, int64_t T, uint64_t H, uint64_t *slot_keys,
                                 uint32_t *heads, uint32_t *next, uint32_t *err, cudaStream_t s);
cudaError_t launch_bucket_emit(const int32_t *lens, int64_t n, int64_t T, int32_t K, const uint32_t *next,
                               uint64_t *raw, uint64_t cap, unsigned long long *counters, cudaStream_t s);
cudaError_t launch_dedup(const uint64_t *raw, uint64_t cap, uint64_t *table, uint64_t hsize, uint64_t *cand,
                         unsigned long long *counters, cudaStream_t s);
// Dedup that also orders the candidates, highest bin first: by collision count
// (lens null) or by length class (the shorter string's length scaled by
// max_len to 256 classes). hcount (hsize uint32) and bins (count_bins() uint64)
// start at zero.
int count_bins();
// Dedup by sorting, for the shared-string verifier: raw[0 .. counters[0]) (the
// rest of cap is not read) is sorted by (longer string, class of the length
// difference, other string) with the LSD radix sort (alt: cap entries), the
// distinct pairs written in that order to *cand_out (raw or alt, the other
// holding the sorted keys) and counted in counters[2]; per group g = x * nclass
// + class: bins[g] (nb + 1 uint32, cleared here) its count, ends[g] its end
// offset (nb uint64), gstart (nb uint64) scratch. temp: dedup_grouped_temp_bytes.
size_t dedup_grouped_temp_bytes(uint64_t cap);
cudaError_t launch_dedup_grouped(uint64_t *raw, uint64_t *alt, uint64_t cap, int64_t n, const int32_t *lens,
                                 uint32_t nclass, uint32_t width, unsigned long long *counters, void *temp,
                                 uint32_t *bins, uint64_t *ends, uint64_t *gstart, uint64_t **cand_out,
                                 cudaStream_t s);
struct VerifySeg;
// Union of the candidate lists of a merged launch's joins (segs[0 .. nseg)):
// every distinct pair once in upairs, with the mask of the joins that list it
// in umask, ordered by the number of joins (more first), then by the length
// class of the shorter string (longer first), or (length_major) by length class
// first. table/tmask: hsize slots (a power of two >= 2 x the pairs, cleared
// here); bins: count_bins() entries; *ucount = the number of distinct pairs
// (device).
cudaError_t launch_union_candidates(const VerifySeg *segs, int nseg, uint64_t *table, uint32_t *tmask, uint64_t hsize,
                                    unsigned long long *bins, uint64_t *upairs, uint32_t *umask,
                                    unsigned long long *ucount, const int32_t *lens, int64_t max_len,
                                    bool length_major, cudaStream_t s);
cudaError_t launch_dedup_ordered(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                 unsigned long long *bins, uint64_t *cand, unsigned long long *counters,
                                 const int32_t *lens, int64_t max_len, cudaStream_t s);
// Strings validated and packed into a context's buffers (valid until the next
// call that plans strings on that context), for the index and the server.
struct PackedSet {
    const uint4 *packed;
    const uint64_t *pofs;
    const int32_t *lens;
    int64_t n, max_len, total;
    int B;
    const uint8_t *code_map;       // raw byte -> code (255 = not in the alphabet), 256 entries
    const uint8_t *alphabet_dev;   // the alphabet's bytes
};
int ctx_pack(ej_ctx *ctx, const ej_strings *S, const ej_params *p, PackedSet *out, void *stream);
int ctx_device(const ej_ctx *ctx);
int ctx_fail(ej_ctx *ctx, int code, const char *msg);
int ctx_check_params(ej_ctx *ctx, const ej_params *p);

// Records of every table sorted by signature, ties by (length, id), for the
// packed set `set`: rk[T][n] signatures, rid[T][n] ids, in the context's scratch.
int ctx_sorted_records(ej_ctx *ctx, const PackedSet &set, const ej_params *p, const uint64_t *keys,
                       const uint64_t **rk, const uint32_t **rid, cudaStream_t s);

// Search against a resident index: per table, records sorted by signature then
// length (rec = len << 32 | id) and a hashed set mapping each signature to its
// run [x, y) of records.
cudaError_t launch_index_runs(const uint64_t *rk, const uint32_t *rid, const int32_t *lens, int64_t n, int64_t T,
                              uint64_t H, uint64_t *slot_keys, uint2 *runs, uint64_t *rec, uint32_t *err,
                              cudaStream_t s);
cudaError_t launch_index_probe(const uint64_t *qkeys, int64_t Q, int64_t T, const int32_t *qlens, const int32_t *qK,
                               const uint64_t *slot_keys, const uint2 *runs, uint64_t H, const uint64_t *rec,
                               int64_t n, uint64_t *raw, uint64_t cap, unsigned long long *counters, cudaStream_t s);
cudaError_t launch_dedup_classes(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                 const uint8_t *cls, int nc, unsigned long long *bins, uint64_t *cand,
                                 unsigned long long *counters, cudaStream_t s);
// Dedup ordered by the pair's first string (counting sort over n bins): bins
// (n + 1 uint32) and hcount start at zero; starts holds n + 2 uint64.
// With longer_lens, the bins are the pairs' longer strings; after the call
// starts[x] is the end of bin x.
cudaError_t launch_dedup_by_first(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                  int64_t n, uint32_t *bins, uint64_t *starts, void *scan_tmp, uint64_t *cand,
                                  unsigned long long *counters, cudaStream_t s,
                                  const int32_t *longer_lens = nullptr);
// Shared-string verifier (ej_verify_sx.cu): warp tasks of up to 16 candidates
// that share their longer string and length-difference class, from the bins of
// launch_dedup_by_first with longer_lens (nb = n * nclass bins; tcount nb+1
// uint32, tstart nb+1 uint64, tasks up to candidates/16 + nb entries;
// *ntasks_dev = their number), and the verifier.
// sx_band(K): the verifier's window W1 and the class width and count that keep
// a task's band within it: a task's length differences lie in one class of
// width D, so its band (the diagonals a cost-K alignment of any of its pairs
// can use) spans at most K + (D - 1)/2 + 1 diagonals; D uses the rows that
// ceil((K + 1) / 64) words leave (at least 7, else one more word).
struct SxBand {
    int W1;
    uint32_t width, nclass;
};
SxBand sx_band(int32_t K);
size_t sx_smem_bytes(int W1, uint32_t alpha);
cudaError_t launch_sx_tasks(const uint32_t *bins, const uint64_t *ends, int64_t n, uint32_t *tcount, uint64_t *tstart,
                            unsigned long long *ntasks_dev, void *scan_tmp, uint64_t *tasks, cudaStream_t s);
int small_sort_max();
cudaError_t launch_small_sort(uint64_t *a, const unsigned long long *count_dev, uint64_t n_cap, cudaStream_t s);

// ---------------------------------------------------------------------------
// Verification (ej_verify.cu)
// ---------------------------------------------------------------------------

// Where the verifier puts its results. Either flags[p] = pass for every pair
// (input order), or, when app != nullptr, every passing pair is appended to
// app[0 .. app_cap) with *app_count counting them (order unspecified).
// np_dev (optional) holds the number of pairs on the device; the host-side
// np is then only an upper bound used to size the grid.
// One join's share of a merged persistent-verifier launch: its candidates
// (count on the device, at most cap), its threshold and its outputs.
struct VerifySeg {
    const uint64_t *pairs;
    const unsigned long long *np_dev;
    uint64_t cap;
    int32_t K;
    uint64_t *app;
    unsigned long long *app_count;
    uint64_t app_cap;
    unsigned long long *work;   // [0] band cells, [1] word columns (at this join's band)
    uint32_t *err;
};
constexpr int MAX_VERIFY_SEGS = 8;

struct VerifyOut {
    uint8_t *flags;
    uint64_t *app;
    unsigned long long *app_count;
    uint64_t app_cap;
    const unsigned long long *np_dev;
    uint32_t *err;
    unsigned long long *work;
    unsigned long long *queue;   // work-queue head of the persistent verifier (zeroed before the launch)
    unsigned int *sm_tickets;    // per-SM working-warp tickets (SM_TICKETS entries, zeroed before the launch)
    // Search (query x index) pairs (a << 32 | b): when packed_b is set, b indexes
    // this second string set instead of the first (the persistent and grouped
    // verifiers); thr[a], when set, is the pair's threshold (the query's K, at
    // most the band's K), else K.
    const uint4 *packed_b;
    const uint64_t *pofs_b;
    const int32_t *lens_b;
    int64_t n_b;
    const int32_t *thr;
    const unsigned long long *pairs_off_dev;   // when set, the pairs start this many entries in (device value)
    // Merged launch (persistent verifier, self-joins): when segs is set, the
    // queue runs over the nseg joins' candidates one join after another, each
    // pair decided with its join's K (at most the band's) and written to its
    // join's outputs; pairs, np, app*, work and err above are not used.
    const VerifySeg *segs;
    int32_t nseg;
    // Persistent verifier: loop passes per warp before it gives up and sets
    // DERR_TIMEOUT (0 = the default bound, 2^24).
    int64_t max_passes;
    // Merged launch over the union of the joins' candidates: when umask is set
    // (with segs), the queue runs over upairs[0 .. min(*unp_dev, ucap)), pair q
    // listed by the joins whose bits are set in umask[q]; it is verified once at
    // the largest of their K and written to each of them whose K its distance
    // meets (band cells counted per join, word columns to the largest K's join).
    const uint64_t *upairs;
    const uint32_t *umask;
    const unsigned long long *unp_dev;
    uint64_t ucap;
};

constexpr int SM_TICKETS = 1024;

struct VerifyConfig {
    int G;          // lanes per pair
    int V;          // 64-bit words per lane
    int warps;      // warps per block
};

// Picks a configuration for threshold K (band 2K+1 bits) and alphabet size.
VerifyConfig verify_pick(int32_t K, uint32_t alpha, int64_t max_len);
// Shared memory per block of a configuration.
size_t verify_smem_bytes(VerifyConfig c, uint32_t alpha, int64_t max_len, int32_t K);

cudaError_t launch_verify(VerifyConfig c, const uint4 *packed, const uint64_t *pofs, int B,
                          const int32_t *lens, int64_t n, uint32_t alpha,
                          const uint64_t *pairs, int64_t np, int32_t K, int64_t max_len,
                          VerifyOut vo, cudaStream_t s);

// Persistent verifier (two lanes per pair, W1 = 2..12 words per lane, pairs
// pulled from vo.queue). spw_force > 0 fixes the pair slots per warp (1..16);
// wps > 0 caps the working warps at wps per SM sub-partition (slots refill).
// Words per lane the persistent verifier needs for threshold K: its band has at
// most K + 1 diagonals (the length difference narrows Ukkonen's 2K + 1), so
// 1 + ceil(K / 64), at least 2.
inline int pq_words(int32_t K) {
    const int w = 1 + (K + 63) / 64;
    return w < 2 ? 2 : w;
}
size_t pq_smem_bytes(int W1, uint32_t alpha, int threads);
int pq_threads_for(int W1, uint32_t alpha);   // 0 if no block size fits
// lean: the variant for launches set by their longest pairs (few pairs per
// slot): chunks in which every running pair has all its columns skip the
// per-column guard (a second copy of the column loop)
cudaError_t launch_verify_pq(int W1, int threads, int spw_force, int wps, const uint4 *packed, const uint64_t *pofs, int B,
                             const int32_t *lens, int64_t n, uint32_t alpha, const uint64_t *pairs, int64_t np,
                             int32_t K, VerifyOut vo, cudaStream_t s, bool lean = false);
// Shared-string verifier (W1 = 2..12): the pairs of tasks[0 .. *ntasks_dev)
// (at most ntasks_cap), each task up to 16 pairs sharing their longer string.
cudaError_t launch_verify_sx(int W1, const uint4 *packed, const uint64_t *pofs, int B, const int32_t *lens, int64_t n,
                             uint32_t alpha, const uint64_t *pairs, const uint64_t *tasks,
                             const unsigned long long *ntasks_dev, int64_t ntasks_cap, int32_t K, VerifyOut vo,
                             cudaStream_t s);

}  // namespace ej
