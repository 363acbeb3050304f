// C ABI of the EmbedJoin hot path: argument checks, the context's scratch
// arena, host/device pointer staging and the stage orchestration of ej_join.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <map>
#include <vector>

#include "ej_internal.cuh"

using namespace ej;

#include <atomic>
namespace ej {
static std::atomic<int64_t> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ej

namespace {

enum BufId {
    B_BYTES, B_OFFSETS, B_LENS, B_DERR, B_CODEMAP, B_ALPHABET, B_TABLE, B_POS, B_PI, B_POSINJ,
    B_EMB, B_WALK, B_KEYS, B_PAIRS_IN, B_OUT_STAGE,
    B_LKEYS, B_LKEYS_ALT, B_PERM, B_PERM_ALT, B_RK, B_RK_ALT, B_RID, B_RID_ALT,
    B_COUNTS, B_OFFS, B_RAW, B_RAW_ALT, B_FLAGS, B_FLAG_OFFS, B_CAND,
    B_RS_COUNTS, B_RS_OFFS, B_SCAN_TMP, B_SCAN_TMP2, B_COUNTERS,
    B_PACKED, B_CHUNK_CNT, B_POFS, B_SCAN_TMP3, B_TSYM, B_SPOS, B_STAG,
    B_HASH, B_APP, B_JCOUNT, B_NEXT, B_HCOUNT, B_BINS, B_TICKETS, B_BKEYS, B_BHEADS, B_BNEXT, B_FBINS, B_FSTARTS,
    B_FSCAN,
    B_PLUS_SUBLEN, B_PLUS_WHOLE, B_PLUS_SUBOFF, B_PLUS_BYTES, B_PLUS_SCAN, B_PLUS_CAND,
    B_SX_TCOUNT, B_SX_TSTART, B_SX_TASKS, B_SX_SCAN,
    B_GROUP_IDX, B_GROUP_OFF, B_GROUP_BYTES, B_GROUP_OUT,
    B_DG_TEMP, B_GSTART,
    B_NUM
};

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

struct Staged {
    const uint8_t *bytes = nullptr;
    const int64_t *offsets = nullptr;
    int64_t n = 0;
    int64_t total = 0;
};

}  // namespace

struct ej_ctx {
    int device = 0;
    std::string err;
    bool timing = false;
    Buf bufs[B_NUM];
    // test tables
    std::vector<uint8_t> pi;
    uint32_t pi_r = 0, pi_steps = 0, pi_alpha = 0;
    std::vector<uint32_t> posinj;
    uint32_t pos_m = 0, pos_z = 0, pos_r = 0;
    // pinned host counters
    int64_t *h_cnt = nullptr;
    cudaEvent_t ev[9] = {};   // ej_join stage timing: [0] start .. [5] end, [6]/[7] pack, [8] after buckets
    // raw-pair capacity remembered from the previous join (grows on overflow)
    uint64_t raw_cap_hint = 0;
    // verifier tiling override (0 = automatic)
    int vG = 0, vV = 0, vWarps = 0;
    ej_schedule sched{0, 0, 0, 0, 0, 0};   // ej_join's back-half schedule (ej_set_schedule)
    int64_t loop_bound = 0;   // persistent verifier: loop passes per warp (ej_set_loop_bound; 0 = default)
    bool no_smem_buckets = false;   // a batch join with huge buckets: hashed buckets in global memory
    ej_ctx *plus_sub = nullptr;     // ej_join_plus: the context of the suffix set
    ej_ctx *group_sub = nullptr;    // ej_join_grouped: the context of one length group
    uint64_t key_P = 0;             // ej_set_key_hash: 0 = exact keys, else <u, v> mod key_P
    int walk_tpb = 0;               // walks (strings) per block of the fused walk (0: 1024 for at most 4 symbols, else 512)
    bool autotune = false;          // ej_set_autotune: joins consult / fill tune_table
    std::map<uint64_t, ej_tune_entry> tune_table;   // (length class << 32 | K) -> choice
    // cached alphabet
    uint8_t alpha_cache[256];
    uint32_t alpha_cache_n = 0;
};

namespace {

int fail(ej_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(expr)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? EJ_ERR_OOM : EJ_ERR_CUDA,       \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

#define CKS(expr)                     \
    do {                              \
        int s_ = (expr);              \
        if (s_ != EJ_OK) return s_;   \
    } while (0)

int ensure(ej_ctx *ctx, BufId id, size_t bytes, void **out) {
    Buf &b = ctx->bufs[id];
    if (bytes == 0) bytes = 16;
    if (b.cap < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        size_t cap = bytes + bytes / 8 + 256;
        cudaError_t e = cudaMalloc(&b.p, cap);
        if (e != cudaSuccess) {
            b.p = nullptr;
            cudaGetLastError();
            return fail(ctx, EJ_ERR_OOM, "cudaMalloc(%zu) failed: %s", cap, cudaGetErrorString(e));
        }
        b.cap = cap;
    }
    *out = b.p;
    return EJ_OK;
}

template <typename T>
int ensure_t(ej_ctx *ctx, BufId id, size_t count, T **out) {
    void *p = nullptr;
    int s = ensure(ctx, id, count * sizeof(T), &p);
    *out = (T *)p;
    return s;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Input array -> device pointer (copies host arrays into a context buffer).
int stage_in(ej_ctx *ctx, BufId id, const void *p, size_t bytes, const void **dev, cudaStream_t s) {
    if (bytes == 0 || is_device_ptr(p)) {
        *dev = p;
        return EJ_OK;
    }
    void *d = nullptr;
    CKS(ensure(ctx, id, bytes, &d));
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
    *dev = d;
    return EJ_OK;
}

int check_params(ej_ctx *ctx, const ej_params *p, bool need_lsh) {
    if (!p) return fail(ctx, EJ_ERR_INVALID_ARG, "params is NULL");
    if (p->K < 0) return fail(ctx, EJ_ERR_INVALID_ARG, "K must be >= 0 (got %d)", p->K);
    if (p->alphabet_size < 1 || p->alphabet_size > 255 || !p->alphabet)
        return fail(ctx, EJ_ERR_INVALID_ARG, "alphabet_size must be 1..255 with a non-NULL alphabet");
    bool seen[256] = {false};
    for (uint32_t c = 0; c < p->alphabet_size; c++) {
        if (seen[p->alphabet[c]]) return fail(ctx, EJ_ERR_INVALID_ARG, "alphabet byte %u repeated", p->alphabet[c]);
        seen[p->alphabet[c]] = true;
    }
    if (!need_lsh) return EJ_OK;
    if (p->r < 1 || p->r > 255) return fail(ctx, EJ_ERR_INVALID_ARG, "r must be 1..255 (got %u)", p->r);
    if (p->m < 1 || p->m > 65535) return fail(ctx, EJ_ERR_INVALID_ARG, "m must be 1..65535 (got %u)", p->m);
    if ((uint64_t)p->r * p->m > 65535)
        return fail(ctx, EJ_ERR_INVALID_ARG, "r*m must be <= 65535 (got %llu)", (unsigned long long)p->r * p->m);
    if (p->z < 1) return fail(ctx, EJ_ERR_INVALID_ARG, "z must be >= 1");
    // (alpha+1)^z < 2^64
    unsigned __int128 v = 1;
    for (uint32_t q = 0; q < p->z; q++) {
        v *= (unsigned __int128)(p->alphabet_size + 1);
        if (v > (unsigned __int128)UINT64_MAX)
            return fail(ctx, EJ_ERR_INVALID_ARG, "(alphabet_size+1)^z must be < 2^64 (z=%u too large)", p->z);
    }
    return EJ_OK;
}

// Upload the alphabet and the raw-byte -> code map (cached per context).
int upload_alphabet(ej_ctx *ctx, const ej_params *p, cudaStream_t s) {
    uint8_t *d_map = nullptr, *d_alpha = nullptr;
    CKS(ensure_t(ctx, B_CODEMAP, 256, &d_map));
    CKS(ensure_t(ctx, B_ALPHABET, 256, &d_alpha));
    if (ctx->alpha_cache_n == p->alphabet_size && !memcmp(ctx->alpha_cache, p->alphabet, p->alphabet_size))
        return EJ_OK;
    uint8_t *h = (uint8_t *)ctx->h_cnt + 256;  // pinned scratch beyond the counters
    memset(h, 255, 256);
    for (uint32_t c = 0; c < p->alphabet_size; c++) h[p->alphabet[c]] = (uint8_t)c;
    memcpy(h + 256, p->alphabet, p->alphabet_size);
    CK(cudaMemcpyAsync(d_map, h, 256, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_alpha, h + 256, p->alphabet_size, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    memcpy(ctx->alpha_cache, p->alphabet, p->alphabet_size);
    ctx->alpha_cache_n = p->alphabet_size;
    return EJ_OK;
}

struct Plan {
    Staged st;
    int32_t *lens = nullptr;
    const uint4 *packed = nullptr;   // B-bit codes, one chunk run per string
    const uint64_t *pofs = nullptr;  // chunk offset of each string (n+1)
    int B = 2;
    int64_t max_len = 0;
    uint32_t out_len = 0, L = 0, planes = 1;
    int64_t nb32 = 0;
};

int derive_lsh(ej_ctx *ctx, const ej_params *p, Plan *pl);

// Stage strings, validate, compute lengths and derived sizes (synchronises s).
int make_plan(ej_ctx *ctx, const ej_strings *S, const ej_params *p, bool need_lsh, Plan *pl, cudaStream_t s) {
    if (!S) return fail(ctx, EJ_ERR_INVALID_ARG, "strings is NULL");
    CKS(check_params(ctx, p, need_lsh));
    if (S->n < 0 || S->n >= (1ll << 31)) return fail(ctx, EJ_ERR_INVALID_ARG, "n must be in [0, 2^31) (got %lld)", (long long)S->n);
    if (S->n > 0 && (!S->offsets || !S->bytes)) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL bytes/offsets");
    const int64_t n = S->n;
    pl->st.n = n;
    CKS(upload_alphabet(ctx, p, s));
    // offsets
    const void *d_off = nullptr;
    int64_t total = 0;
    if (n > 0) {
        CKS(stage_in(ctx, B_OFFSETS, S->offsets, (size_t)(n + 1) * sizeof(int64_t), &d_off, s));
        CK(cudaMemcpyAsync(ctx->h_cnt, (const int64_t *)d_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        total = ctx->h_cnt[0];
        if (total < 0) return fail(ctx, EJ_ERR_INVALID_ARG, "offsets[n] = %lld < 0", (long long)total);
    }
    pl->st.offsets = (const int64_t *)d_off;
    pl->st.total = total;
    const void *d_bytes = S->bytes;
    if (total > 0) CKS(stage_in(ctx, B_BYTES, S->bytes, (size_t)total, &d_bytes, s));
    pl->st.bytes = (const uint8_t *)d_bytes;
    uint32_t *derr = nullptr;
    CKS(ensure_t(ctx, B_DERR, 8, &derr));
    CK(cudaMemsetAsync(derr, 0, 4 * sizeof(uint32_t), s));
    CKS(ensure_t(ctx, B_LENS, (size_t)(n > 0 ? n : 1), &pl->lens));
    unsigned long long *dmax = (unsigned long long *)(derr + 2);
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[6], s));
    CK(launch_validate(pl->st.bytes, pl->st.offsets, n, total, (const uint8_t *)ctx->bufs[B_CODEMAP].p, pl->lens,
                       derr, dmax, s));
    // pack into B-bit codes: chunk counts -> offsets -> pack (flags bad symbols)
    pl->B = packed_bits_for(p->alphabet_size);
    uint32_t *ccnt = nullptr;
    uint64_t *pofs = nullptr;
    uint4 *packed = nullptr;
    void *stmp = nullptr;
    CKS(ensure_t(ctx, B_CHUNK_CNT, (size_t)n + 1, &ccnt));
    CKS(ensure_t(ctx, B_POFS, (size_t)n + 2, &pofs));
    CKS(ensure(ctx, B_SCAN_TMP3, scan_temp_bytes(n + 1), &stmp));
    const int64_t chunk_bound = (total * pl->B + 127) / 128 + n + 1;
    CKS(ensure_t(ctx, B_PACKED, (size_t)chunk_bound, &packed));
    CK(launch_chunk_counts(pl->lens, n, pl->B, ccnt, s));
    CK(exclusive_scan_u32(ccnt, pofs, n + 1, nullptr, stmp, s));
    CK(launch_pack(pl->st.bytes, pl->st.offsets, pl->lens, n, total, (const uint8_t *)ctx->bufs[B_CODEMAP].p, pl->B,
                   pofs, packed, derr, s));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[7], s));
    pl->packed = packed;
    pl->pofs = pofs;
    CK(cudaMemcpyAsync(ctx->h_cnt, derr, 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t e = (uint32_t)(ctx->h_cnt[0] & 0xffffffffu);
    if (e & DERR_OFFSETS) return fail(ctx, EJ_ERR_INVALID_ARG, "offsets must start at 0 and be non-decreasing, lengths < 2^31");
    if (e & DERR_SYMBOL) return fail(ctx, EJ_ERR_INVALID_ARG, "a string byte is not in the alphabet");
    pl->max_len = (int64_t)((unsigned long long)ctx->h_cnt[1]);
    if (need_lsh) CKS(derive_lsh(ctx, p, pl));
    return EJ_OK;
}

// The parameter-dependent sizes of a plan: out_len (3N unless given), L, planes.
int derive_lsh(ej_ctx *ctx, const ej_params *p, Plan *pl) {
    const int64_t n = pl->st.n;
    {
        uint64_t ol = p->out_len ? p->out_len : (uint64_t)(3 * pl->max_len);
        if (ol == 0) ol = 1;
        if (ol > 0x7fffffffull) return fail(ctx, EJ_ERR_INVALID_ARG, "out_len too large");
        if (ol >= (1ull << 40)) return fail(ctx, EJ_ERR_INVALID_ARG, "out_len too large for the step counter");
        pl->out_len = (uint32_t)ol;
        pl->L = p->L ? p->L : pl->out_len;
        if (pl->L > pl->out_len) return fail(ctx, EJ_ERR_INVALID_ARG, "L (%u) must be <= out_len (%u)", pl->L, pl->out_len);
        pl->planes = planes_for(p->alphabet_size);
        pl->nb32 = (n + 31) / 32;
        if (ctx->pi.size() && (ctx->pi_r != p->r || ctx->pi_alpha != p->alphabet_size))
            return fail(ctx, EJ_ERR_INVALID_ARG, "injected pi table does not match r/alphabet_size");
        if (ctx->posinj.size() && (ctx->pos_r != p->r || ctx->pos_m != p->m || ctx->pos_z != p->z))
            return fail(ctx, EJ_ERR_INVALID_ARG, "injected positions do not match r/m/z");
        for (uint32_t v : ctx->posinj)
            if (v >= pl->L) return fail(ctx, EJ_ERR_INVALID_ARG, "injected position %u >= L", v);
    }
    return EJ_OK;
}

// The device work of make_plan for an existing plan (validate -> chunk counts
// -> scan -> pack), with the plan's sizes as bounds; no host synchronisation.
int plan_device(ej_ctx *ctx, const Plan &pl, cudaStream_t s) {
    const int64_t n = pl.st.n;
    uint32_t *derr = (uint32_t *)ctx->bufs[B_DERR].p;
    CK(cudaMemsetAsync(derr, 0, 4 * sizeof(uint32_t), s));
    unsigned long long *dmax = (unsigned long long *)(derr + 2);
    CK(launch_validate(pl.st.bytes, pl.st.offsets, n, pl.st.total, (const uint8_t *)ctx->bufs[B_CODEMAP].p, pl.lens,
                       derr, dmax, s));
    uint32_t *ccnt = (uint32_t *)ctx->bufs[B_CHUNK_CNT].p;
    CK(launch_chunk_counts(pl.lens, n, pl.B, ccnt, s));
    CK(exclusive_scan_u32(ccnt, (uint64_t *)pl.pofs, n + 1, nullptr, ctx->bufs[B_SCAN_TMP3].p, s));
    CK(launch_pack(pl.st.bytes, pl.st.offsets, pl.lens, n, pl.st.total, (const uint8_t *)ctx->bufs[B_CODEMAP].p, pl.B,
                   pl.pofs, (uint4 *)pl.packed, derr, s));
    return EJ_OK;
}

uint64_t emb_bytes(const Plan &pl, uint32_t r) {
    return (uint64_t)r * pl.nb32 * pl.out_len * pl.planes * sizeof(uint32_t);
}

// Random-bit table and positions into context buffers.
int make_tables(ej_ctx *ctx, const ej_params *p, const Plan &pl, uint32_t **table, uint32_t **pos, cudaStream_t s) {
    const uint32_t words = table_words_for(pl.planes);
    CKS(ensure_t(ctx, B_TABLE, (size_t)p->r * pl.out_len * words, table));
    CKS(ensure_t(ctx, B_POS, (size_t)p->r * p->m * p->z, pos));
    const uint8_t *pi_dev = nullptr;
    if (ctx->pi.size()) {
        uint8_t *d = nullptr;
        CKS(ensure_t(ctx, B_PI, ctx->pi.size(), &d));
        CK(cudaMemcpyAsync(d, ctx->pi.data(), ctx->pi.size(), cudaMemcpyHostToDevice, s));
        pi_dev = d;
    }
    const uint32_t *pos_dev = nullptr;
    if (ctx->posinj.size()) {
        uint32_t *d = nullptr;
        CKS(ensure_t(ctx, B_POSINJ, ctx->posinj.size(), &d));
        CK(cudaMemcpyAsync(d, ctx->posinj.data(), ctx->posinj.size() * 4, cudaMemcpyHostToDevice, s));
        pos_dev = d;
    }
    CK(launch_bit_table(p->seed, p->r, pl.out_len, (const uint8_t *)ctx->bufs[B_ALPHABET].p, p->alphabet_size,
                        words, pi_dev, ctx->pi_steps, *table, s));
    CK(launch_positions(p->seed, p->r, p->m, p->z, pl.L, pos_dev, *pos, s));
    if (pi_dev || pos_dev) CK(cudaStreamSynchronize(s));  // host vectors may change after return
    return EJ_OK;
}

// Keys [r*m][n] for the plan's strings into `keys` (device): the fused walk
// when its tables fit in shared memory, else embed (prefix of length L) + sign.
// phase 1 issues only the tables (bits, positions: parameters only), phase 2
// only the walk over the strings (tables already built), 0 both.
int keys_dev(ej_ctx *ctx, const ej_params *p, const Plan &pl, uint64_t *keys, cudaStream_t s,
             const PrefixKeys *prefix = nullptr, int phase = 0) {
    const int64_t n = pl.st.n;
    if (n == 0) return EJ_OK;
    const bool tables = phase != 2, walk = phase != 1;
    uint32_t *pos = nullptr;
    CKS(ensure_t(ctx, B_POS, (size_t)p->r * p->m * p->z, &pos));
    const uint8_t *pi_dev = nullptr;
    if (ctx->pi.size()) {
        uint8_t *d = nullptr;
        CKS(ensure_t(ctx, B_PI, ctx->pi.size(), &d));
        CK(cudaMemcpyAsync(d, ctx->pi.data(), ctx->pi.size(), cudaMemcpyHostToDevice, s));
        pi_dev = d;
    }
    const uint32_t *pos_inj = nullptr;
    if (ctx->posinj.size()) {
        uint32_t *d = nullptr;
        CKS(ensure_t(ctx, B_POSINJ, ctx->posinj.size(), &d));
        CK(cudaMemcpyAsync(d, ctx->posinj.data(), ctx->posinj.size() * 4, cudaMemcpyHostToDevice, s));
        pos_inj = d;
    }
    if (tables) CK(launch_positions(p->seed, p->r, p->m, p->z, pl.L, pos_inj, pos, s));
    if (embed_sign_smem(p->alphabet_size, pl.L, p->m, p->z, ctx->walk_tpb) > 0 ||
        embed_sign_smem(p->alphabet_size, pl.L, p->m, p->z) > 0) {
        uint32_t *tsym = nullptr, *spos = nullptr, *stag = nullptr;
        CKS(ensure_t(ctx, B_TSYM, symbol_table_words(p->r, p->alphabet_size, pl.L), &tsym));
        CKS(ensure_t(ctx, B_SPOS, (size_t)p->r * p->m * p->z, &spos));
        CKS(ensure_t(ctx, B_STAG, (size_t)p->r * p->m * p->z, &stag));
        if (tables) {
            CK(launch_symbol_table(p->seed, p->r, pl.L, (const uint8_t *)ctx->bufs[B_ALPHABET].p, p->alphabet_size,
                                   pi_dev, ctx->pi_steps, tsym, s));
            CK(launch_sort_samples(pos, p->r, p->m, p->z, spos, stag, s));
        }
        uint16_t *next = nullptr;
        if (embed_sign_uses_table(p->alphabet_size, pl.L)) {
            CKS(ensure_t(ctx, B_NEXT, next_table_elems(p->r, p->alphabet_size, pl.L), &next));
            if (tables) CK(launch_next_table(tsym, p->r, p->alphabet_size, pl.L, next, s));
        }
        if (walk) {
            if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], s));
            CK(launch_embed_sign(pl.packed, pl.pofs, pl.lens, n, p->r, p->m, p->z, pl.L, p->alphabet_size, pl.B,
                                 tsym, next, spos, stag, keys, s, prefix, ctx->walk_tpb));
            if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], s));
        }
        prefix = nullptr;   // written by the walk
    } else {
        // materialise only the prefix [0, L) of every embedding
        Plan pl2 = pl;
        pl2.out_len = pl.L;
        const uint32_t words = table_words_for(pl.planes);
        uint32_t *table = nullptr, *emb = nullptr;
        int32_t *we = nullptr;
        CKS(ensure_t(ctx, B_TABLE, (size_t)p->r * pl2.out_len * words, &table));
        CKS(ensure_t(ctx, B_EMB, (size_t)(emb_bytes(pl2, p->r) / 4), &emb));
        CKS(ensure_t(ctx, B_WALK, (size_t)p->r * n, &we));
        if (tables)
            CK(launch_bit_table(p->seed, p->r, pl2.out_len, (const uint8_t *)ctx->bufs[B_ALPHABET].p,
                                p->alphabet_size, words, pi_dev, ctx->pi_steps, table, s));
        if (walk) {
            if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], s));
            CK(launch_embed(pl.packed, pl.pofs, pl.lens, n, p->r, table, pl.B, pl2.out_len, pl.planes, emb, we, s));
            CK(launch_sign(emb, we, n, p->r, p->m, p->z, pl2.out_len, pl.planes, p->alphabet_size, pos, keys, s));
            if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], s));
        }
    }
    if (prefix && walk) {
        // the unfused path: the prefix keys as the keys modulo (alpha+1)^z
        for (int e = 0; e < prefix->n; e++) {
            uint64_t mod = 1;
            for (uint32_t q = 0; q < prefix->z[e]; q++) mod *= (uint64_t)p->alphabet_size + 1;
            CK(launch_derive_keys(keys, p->m, n, p->r, p->m, prefix->z[e] < p->z ? mod : 0, prefix->keys[e], s));
        }
    }
    if (ctx->key_P && walk)
        CK(launch_keys_modp(keys, n, p->r, p->m, p->z, p->alphabet_size, p->seed, ctx->key_P, s));
    if (pi_dev || pos_inj) CK(cudaStreamSynchronize(s));
    return EJ_OK;
}

int bits_for(uint64_t maxval);

int key_bits(const ej_ctx *ctx, const ej_params *p) {
    if (ctx->key_P) return bits_for(ctx->key_P - 1);   // hashed keys are < P
    unsigned __int128 v = 1;
    for (uint32_t q = 0; q < p->z; q++) v *= (unsigned __int128)(p->alphabet_size + 1);
    uint64_t maxkey = (uint64_t)(v - 1);
    int b = 0;
    while (b < 64 && (maxkey >> b)) b++;
    return b;
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b)) b++;
    return b;
}

// Records (key, id) of every table, sorted by key with ties in (length, id)
// order: the layout both candidate paths start from.
int sorted_records(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *keys,
                   const uint64_t **out_rk, const uint32_t **out_rid, cudaStream_t s) {
    const int64_t n = pl.st.n, T = (int64_t)p->r * p->m;
    const int idb = bits_for((uint64_t)(n > 1 ? n - 1 : 1));
    if (n <= table_sort_max() && idb + key_bits(ctx, p) <= 64 && idb + bits_for((uint64_t)pl.max_len) <= 64) {
        // every table fits one block: length order, then all tables, one block each
        uint64_t *lk = nullptr, *lsorted = nullptr;
        uint32_t *perm = nullptr;
        CKS(ensure_t(ctx, B_LKEYS, (size_t)n, &lk));
        CKS(ensure_t(ctx, B_LKEYS_ALT, (size_t)n, &lsorted));
        CKS(ensure_t(ctx, B_PERM, (size_t)n, &perm));
        CK(launch_len_keys(pl.lens, n, lk, s));
        CK(launch_table_sort(lk, nullptr, n, 1, idb, bits_for((uint64_t)pl.max_len), lsorted, perm, s));
        uint64_t *rk = nullptr;
        uint32_t *rid = nullptr;
        CKS(ensure_t(ctx, B_RK, (size_t)(n * T), &rk));
        CKS(ensure_t(ctx, B_RID, (size_t)(n * T), &rid));
        CK(launch_table_sort(keys, perm, n, T, idb, key_bits(ctx, p), rk, rid, s));
        *out_rk = rk;
        *out_rid = rid;
        return EJ_OK;
    }
    const size_t rs_len = radix_counts_len(n, T);
    uint32_t *rs_counts = nullptr;
    uint64_t *rs_offs = nullptr;
    void *scan_tmp = nullptr;
    CKS(ensure_t(ctx, B_RS_COUNTS, rs_len, &rs_counts));
    CKS(ensure_t(ctx, B_RS_OFFS, rs_len, &rs_offs));
    CKS(ensure(ctx, B_SCAN_TMP, scan_temp_bytes((int64_t)rs_len), &scan_tmp));
    RadixTemp rt{rs_counts, rs_offs, scan_tmp};
    // 1. length order (stable by id)
    uint64_t *lk = nullptr, *lk2 = nullptr;
    uint32_t *perm = nullptr, *perm2 = nullptr;
    CKS(ensure_t(ctx, B_LKEYS, (size_t)n, &lk));
    CKS(ensure_t(ctx, B_LKEYS_ALT, (size_t)n, &lk2));
    CKS(ensure_t(ctx, B_PERM, (size_t)n, &perm));
    CKS(ensure_t(ctx, B_PERM_ALT, (size_t)n, &perm2));
    CK(launch_len_keys(pl.lens, n, lk, s));
    CK(launch_iota_u32(perm, n, s));
    int shifts[16];
    int np = 0;
    for (int b = 0; b < bits_for((uint64_t)pl.max_len); b += 8) shifts[np++] = b;
    bool alt = false;
    CK(radix_sort_segmented(lk, perm, lk2, perm2, n, 1, shifts, np, rt, &alt, s));
    const uint32_t *order = alt ? perm2 : perm;
    // 2. gather into (key, id) records per table, length order
    uint64_t *rk = nullptr, *rk2 = nullptr;
    uint32_t *rid = nullptr, *rid2 = nullptr;
    CKS(ensure_t(ctx, B_RK, (size_t)(n * T), &rk));
    CKS(ensure_t(ctx, B_RK_ALT, (size_t)(n * T), &rk2));
    CKS(ensure_t(ctx, B_RID, (size_t)(n * T), &rid));
    CKS(ensure_t(ctx, B_RID_ALT, (size_t)(n * T), &rid2));
    CK(launch_len_order_gather(keys, order, n, T, rk, rid, s));
    // 3. stable sort by key within each table
    np = 0;
    for (int b = 0; b < key_bits(ctx, p); b += 8) shifts[np++] = b;
    CK(radix_sort_segmented(rk, rid, rk2, rid2, n, T, shifts, np, rt, &alt, s));
    *out_rk = alt ? rk2 : rk;
    *out_rid = alt ? rid2 : rid;
    return EJ_OK;
}

// Candidates from keys [T][n] on the device (sort-based, sorted unique output).
// Result: sorted unique pairs in *cand (context buffer B_CAND), count in *ncand.
int candidates_dev(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *keys, uint64_t **cand,
                   int64_t *ncand, int64_t *nraw, int64_t *maxb, cudaStream_t s) {
    const int64_t n = pl.st.n, T = (int64_t)p->r * p->m;
    *ncand = 0; *nraw = 0; *maxb = 0;
    *cand = nullptr;
    if (n < 2) return EJ_OK;
    const uint64_t *srk = nullptr;
    const uint32_t *srid = nullptr;
    CKS(sorted_records(ctx, pl, p, keys, &srk, &srid, s));
    int shifts[16];
    int np = 0;
    bool alt = false;
    const size_t rs_len = radix_counts_len(n, T);
    uint32_t *rsc = nullptr;
    uint64_t *rso = nullptr;
    void *scan_tmp = nullptr;
    CKS(ensure_t(ctx, B_RS_COUNTS, rs_len, &rsc));
    CKS(ensure_t(ctx, B_RS_OFFS, rs_len, &rso));
    CKS(ensure(ctx, B_SCAN_TMP, scan_temp_bytes((int64_t)rs_len), &scan_tmp));
    RadixTemp rt{rsc, rso, scan_tmp};
    // 4. count partners per record, scan
    uint32_t *counts = nullptr;
    uint64_t *offs = nullptr;
    CKS(ensure_t(ctx, B_COUNTS, (size_t)(n * T), &counts));
    CKS(ensure_t(ctx, B_OFFS, (size_t)(n * T) + 1, &offs));
    uint64_t *dcnt = nullptr;
    CKS(ensure_t(ctx, B_COUNTERS, 8, &dcnt));
    CK(cudaMemsetAsync(dcnt, 0, 8 * sizeof(uint64_t), s));
    CK(launch_bucket_count(srk, srid, pl.lens, n, T, p->K, counts, (unsigned long long *)(dcnt + 1), s));
    void *scan_tmp2 = nullptr;
    CKS(ensure(ctx, B_SCAN_TMP2, scan_temp_bytes(n * T), &scan_tmp2));
    CK(exclusive_scan_u32(counts, offs, n * T, dcnt, scan_tmp2, s));
    CK(cudaMemcpyAsync(ctx->h_cnt, dcnt, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t raw = ctx->h_cnt[0];
    *nraw = raw;
    *maxb = ctx->h_cnt[1];
    if (raw == 0) return EJ_OK;
    // 5. emit, sort, unique
    uint64_t *pr = nullptr, *pr2 = nullptr;
    CKS(ensure_t(ctx, B_RAW, (size_t)raw, &pr));
    CKS(ensure_t(ctx, B_RAW_ALT, (size_t)raw, &pr2));
    CK(launch_bucket_emit(srk, srid, pl.lens, n, T, p->K, offs, pr, s));
    const int nb = bits_for((uint64_t)(n - 1));
    np = 0;
    for (int b = 0; b < nb; b += 8) shifts[np++] = b;
    for (int b = 0; b < nb; b += 8) shifts[np++] = 32 + b;
    const size_t rs2 = radix_counts_len(raw, 1);
    uint32_t *c2 = nullptr;
    uint64_t *o2 = nullptr;
    if (rs2 > rs_len) {
        CKS(ensure_t(ctx, B_RS_COUNTS, rs2, &c2));
        CKS(ensure_t(ctx, B_RS_OFFS, rs2, &o2));
        CKS(ensure(ctx, B_SCAN_TMP, scan_temp_bytes((int64_t)rs2), &scan_tmp));
        rt = RadixTemp{c2, o2, scan_tmp};
    }
    CK(radix_sort_segmented(pr, nullptr, pr2, nullptr, raw, 1, shifts, np, rt, &alt, s));
    const uint64_t *sp = alt ? pr2 : pr;
    uint8_t *fl = nullptr;
    uint64_t *fo = nullptr;
    CKS(ensure_t(ctx, B_FLAGS, (size_t)raw, &fl));
    CKS(ensure_t(ctx, B_FLAG_OFFS, (size_t)raw, &fo));
    CK(launch_unique_flags(sp, raw, fl, s));
    CKS(ensure(ctx, B_SCAN_TMP2, scan_temp_bytes(raw), &scan_tmp2));
    CK(exclusive_scan_u8(fl, fo, raw, dcnt + 2, scan_tmp2, s));
    CK(cudaMemcpyAsync(ctx->h_cnt, dcnt + 2, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t nc = ctx->h_cnt[0];
    uint64_t *cd = nullptr;
    CKS(ensure_t(ctx, B_CAND, (size_t)nc, &cd));
    CK(launch_compact_u64(sp, fl, fo, raw, cd, s));
    *cand = cd;
    *ncand = nc;
    return EJ_OK;
}

// Verifier tiling: the automatic choice, or the context's override if it covers the band.
int pick_verify(ej_ctx *ctx, const ej_params *p, const Plan &pl, VerifyConfig *out) {
    VerifyConfig vc = verify_pick(p->K, p->alphabet_size, pl.max_len);
    const int64_t cover = ctx->vG == 2 ? 64ll * (ctx->vV - 1) : 64ll * ctx->vG * ctx->vV;
    if (ctx->vG > 0 && cover >= 2ll * p->K + 1) {
        VerifyConfig o{ctx->vG, ctx->vV, ctx->vWarps > 0 ? ctx->vWarps : 1};
        if (ctx->vWarps <= 0) {
            VerifyConfig one{o.G, o.V, 1};
            const size_t per_warp = verify_smem_bytes(one, p->alphabet_size, pl.max_len, p->K);
            int w = (int)((96 * 1024) / (per_warp ? per_warp : 1));
            const int wmax = o.G <= 2 ? 4 : 8;
            o.warps = w < 1 ? 1 : (w > wmax ? wmax : w);
        }
        if (o.G <= 2 && o.warps > 4) o.warps = 4;
        if (verify_smem_bytes(o, p->alphabet_size, pl.max_len, p->K) <= 200 * 1024) vc = o;
    }
    if (vc.G == 0)
        return fail(ctx, EJ_ERR_UNSUPPORTED, "no verifier configuration for K=%d, alphabet %u, max length %lld",
                    p->K, p->alphabet_size, (long long)pl.max_len);
    *out = vc;
    return EJ_OK;
}

// Verify device pairs; passing pairs (input order) into `out_dev` if it has
// room (capacity), count in *n_out. If out_dev is null only counts.
int verify_dev(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *pairs, int64_t np,
               uint64_t *out_dev, int64_t capacity, int64_t *n_out, cudaStream_t s,
               uint64_t *work_out = nullptr) {
    *n_out = 0;
    if (np == 0) return EJ_OK;
    VerifyConfig vc;
    CKS(pick_verify(ctx, p, pl, &vc));
    uint8_t *fl = nullptr;
    uint64_t *fo = nullptr;
    CKS(ensure_t(ctx, B_FLAGS, (size_t)np, &fl));
    CKS(ensure_t(ctx, B_FLAG_OFFS, (size_t)np, &fo));
    uint32_t *derr = (uint32_t *)ctx->bufs[B_DERR].p;
    uint64_t *dcnt = nullptr;
    CKS(ensure_t(ctx, B_COUNTERS, 8, &dcnt));
    CK(cudaMemsetAsync(derr, 0, 4, s));
    CK(cudaMemsetAsync(dcnt + 4, 0, 2 * sizeof(uint64_t), s));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[3], s));
    VerifyOut vo{fl, nullptr, nullptr, 0, nullptr, derr, (unsigned long long *)(dcnt + 4), nullptr, nullptr};
    CK(launch_verify(vc, pl.packed, pl.pofs, pl.B, pl.lens, pl.st.n, p->alphabet_size, pairs, np, p->K,
                     pl.max_len, vo, s));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[4], s));
    void *tmp = nullptr;
    CKS(ensure(ctx, B_SCAN_TMP2, scan_temp_bytes(np), &tmp));
    CK(exclusive_scan_u8(fl, fo, np, dcnt + 3, tmp, s));
    CK(cudaMemcpyAsync(ctx->h_cnt, dcnt + 3, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_cnt + 1, derr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_cnt + 2, dcnt + 4, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (work_out) {
        work_out[0] = (uint64_t)ctx->h_cnt[2];
        work_out[1] = (uint64_t)ctx->h_cnt[3];
    }
    if ((uint32_t)ctx->h_cnt[1] & DERR_PAIR) return fail(ctx, EJ_ERR_INVALID_ARG, "pair index >= n");
    const int64_t cnt = ctx->h_cnt[0];
    *n_out = cnt;
    if (!out_dev) return EJ_OK;
    if (cnt > capacity) return fail(ctx, EJ_ERR_CAPACITY, "output needs %lld pairs, capacity %lld", (long long)cnt, (long long)capacity);
    CK(launch_compact_u64(pairs, fl, fo, np, out_dev, s));
    return EJ_OK;
}

// ej_join's back half without host round trips between stages: bucket the
// signatures, emit the pairs of every bucket, a device hash set keeps the first
// copy of each pair, the verifier reads the candidate count from the device and
// appends passing pairs, and only the output is sorted. The host reads the
// counters once, after the verifier; if the raw pairs outgrew the capacity it
// enlarges it and reruns from the emit step (the buckets are kept).
// back_buckets + back_attempt issue device work only (no host synchronisation,
// no allocation once the buffers have their size), so they can be captured.
struct BackState {
    bool hashed = false;
    bool table_smem = false;           // hashed, each table's buckets built in shared memory
    const uint64_t *keys = nullptr;    // the signatures (table_smem)
    const uint64_t *srk = nullptr;
    const uint32_t *srid = nullptr;
    uint32_t *bnext = nullptr;
    VerifyConfig vc{0, 0, 0};
    bool any_order = false;            // the candidates feed a batch's union launch, which orders them itself
};

// Largest bucket (records of one signature in one table) that a batch join
// keeps in shared memory; its sizing pass moves joins with larger ones to the
// hashed buckets in global memory.
constexpr unsigned SMEM_BUCKET_MAX = 256;
// Largest bucket above which a batch join (schedule buckets 0) takes the sorted
// tables with length windows instead of hashed buckets.
constexpr unsigned SORTED_BUCKET_MIN = 4096;

int back_buckets(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *keys, BackState *bs,
                 cudaStream_t s) {
    const int64_t n = pl.st.n, T = (int64_t)p->r * p->m;
    uint32_t *derr = nullptr;
    CKS(ensure_t(ctx, B_DERR, 8, &derr));
    CK(cudaMemsetAsync(derr, 0, 4, s));
    bs->hashed = ctx->sched.buckets != 2 && n * T < (int64_t)0xFFFFFFFFll;
    bs->table_smem = bs->hashed && bucket_table_smem(n) > 0 && !ctx->no_smem_buckets;
    bs->keys = keys;
    if (bs->table_smem) {
        // built by the emitting kernel, one block per table
    } else if (bs->hashed) {
        // buckets by hashing: no sort of the r*m tables
        const uint64_t H = bucket_slots_per_table(n);
        uint64_t *bkeys = nullptr;
        uint32_t *bheads = nullptr;
        CKS(ensure_t(ctx, B_BKEYS, (size_t)(H * T), &bkeys));
        CKS(ensure_t(ctx, B_BHEADS, (size_t)(H * T), &bheads));
        CKS(ensure_t(ctx, B_BNEXT, (size_t)(n * T), &bs->bnext));
        CK(cudaMemsetAsync(bkeys, 0xFF, H * T * sizeof(uint64_t), s));
        CK(cudaMemsetAsync(bheads, 0xFF, H * T * sizeof(uint32_t), s));
        CK(launch_bucket_insert(keys, n, T, H, bkeys, bheads, bs->bnext, derr, s));
    } else {
        CKS(sorted_records(ctx, pl, p, keys, &bs->srk, &bs->srid, s));
    }
    CKS(pick_verify(ctx, p, pl, &bs->vc));
    return EJ_OK;
}

uint64_t raw_cap_start(ej_ctx *ctx, int64_t n) {
    return ctx->raw_cap_hint ? ctx->raw_cap_hint : (uint64_t)(n * 4 > 65536 ? n * 4 : 65536);
}

// Threads per block of the persistent verifier this join uses, 0 for the
// grid-strided one. Mode 0 picks the persistent verifier for long strings only
// (mean length >= 2048): on short, mostly rejected pairs its per-pair refill
// costs more than it saves (measured 2x slower on the protein-like shape).
int pq_choice(const ej_ctx *ctx, const Plan &pl, const ej_params *p, const VerifyConfig &vc) {
    const bool long_pairs = pl.st.n > 0 && pl.st.total / pl.st.n >= 2048;
    const bool want_pq = ctx->sched.mode == 1 || (ctx->sched.mode == 0 && long_pairs);
    return (vc.G == 2 && want_pq) ? pq_threads_for(pq_words(p->K), p->alphabet_size) : 0;
}

// The shared-string verifier (mode 3; mode 0 for short strings over more than
// four symbols, where the per-lane match-mask rings of the grid-strided
// verifier leave one or two warps per SM): two lanes per pair, the band within
// 12 words per lane, the warp's shared area within the block's budget.
bool sx_choice(const ej_ctx *ctx, const Plan &pl, const ej_params *p, const VerifyConfig &vc) {
    const int W1 = sx_band(p->K).W1;
    if (vc.G != 2 || W1 > 12 || sx_smem_bytes(W1, p->alphabet_size) > 220 * 1024) return false;
    const bool long_pairs = pl.st.n > 0 && pl.st.total / pl.st.n >= 2048;
    return ctx->sched.mode == 3 || (ctx->sched.mode == 0 && !long_pairs && p->alphabet_size > 4);
}

// verify_after / verify_done (optional): the verifier launch waits for the
// first event and records the second (a batch chains its joins' verifiers, so
// that persistent verifiers never run concurrently). defer (optional): no
// verifier launch; *defer describes this join's share of a merged launch.
int back_attempt(ej_ctx *ctx, const Plan &pl, const ej_params *p, const BackState &bs, uint64_t cap,
                 cudaStream_t s, cudaEvent_t verify_after = nullptr, cudaEvent_t verify_done = nullptr,
                 VerifySeg *defer = nullptr, bool emitted = false) {
    const int64_t n = pl.st.n, T = (int64_t)p->r * p->m;
    unsigned long long *cnt = nullptr;
    CKS(ensure_t(ctx, B_JCOUNT, 8, &cnt));
    uint32_t *derr = (uint32_t *)ctx->bufs[B_DERR].p;
    uint64_t hsize = 1;
    while (hsize < 2 * cap) hsize <<= 1;
    uint64_t *raw = nullptr, *cand = nullptr, *table = nullptr, *app = nullptr;
    CKS(ensure_t(ctx, B_RAW, (size_t)cap, &raw));
    CKS(ensure_t(ctx, B_CAND, (size_t)cap, &cand));
    CKS(ensure_t(ctx, B_APP, (size_t)cap, &app));
    // the verifier and the candidate order it takes
    const bool sx = !defer && sx_choice(ctx, pl, p, bs.vc);
    const int pq_threads = sx ? 0 : pq_choice(ctx, pl, p, bs.vc);
    // the shared-string verifier needs its pairs grouped by their longer string
    const int order = sx ? 5 : bs.any_order ? 2 : ctx->sched.order != 0 ? ctx->sched.order : (pq_threads > 0 ? 4 : 3);
    // emitted: the raw pairs and counters [0], [1] are already written (shared
    // buckets of a batch)
    CK(cudaMemsetAsync(emitted ? cnt + 2 : cnt, 0, (emitted ? 6 : 8) * sizeof(unsigned long long), s));
    if (!sx) {   // the shared-string verifier's candidates are deduplicated by sorting
        CKS(ensure_t(ctx, B_HASH, (size_t)hsize, &table));
        CK(cudaMemsetAsync(table, 0xFF, hsize * sizeof(uint64_t), s));
    }
    if (emitted) {
    } else if (bs.table_smem) {
        SharedEmit se{};
        se.njoins = 1;
        se.keys[0] = bs.keys;
        se.K[0] = p->K;
        se.raw[0] = raw;
        se.cap[0] = cap;
        se.counters[0] = cnt;
        CK(launch_bucket_table(pl.lens, n, T, se, s));
    } else if (bs.hashed)
        CK(launch_bucket_emit(pl.lens, n, T, p->K, bs.bnext, raw, cap, cnt, s));
    else
        CK(launch_emit_append(bs.srk, bs.srid, pl.lens, n, T, p->K, raw, cap, cnt, s));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[8], s));
    // queue order: 0 follows the verifier (persistent: length classes; grid-
    // strided: by first string), measured best for each on the long-DNA and the
    // protein-like / text-like shapes
    uint32_t *fbins = nullptr;
    uint64_t *fstarts = nullptr;
    // the shared-string verifier's window and length-difference classes
    const SxBand sb = sx ? sx_band(p->K) : SxBand{0, 1u, 1u};
    const int64_t nb = n * (int64_t)sb.nclass;   // the shared-string verifier's candidate groups
    if (sx) {
        // the shared-string verifier's tasks: the distinct pairs sorted by their
        // longer string and the class of their length difference
        void *dgt = nullptr;
        uint64_t *gstart = nullptr, *sorted_cand = nullptr;
        CKS(ensure_t(ctx, B_FBINS, (size_t)nb + 1, &fbins));
        CKS(ensure_t(ctx, B_FSTARTS, (size_t)nb + 2, &fstarts));
        CKS(ensure_t(ctx, B_GSTART, (size_t)nb + 1, &gstart));
        CKS(ensure(ctx, B_DG_TEMP, dedup_grouped_temp_bytes(cap), &dgt));
        CK(launch_dedup_grouped(raw, cand, cap, n, pl.lens, sb.nclass, sb.width, cnt, dgt, fbins, fstarts, gstart,
                                &sorted_cand, s));
        cand = sorted_cand;
    } else if (order == 3 || order == 5) {
        // candidates ordered by their first string (a warp's pairs share it), or
        // by their longer string
        uint32_t *hcount = nullptr;
        void *fscan = nullptr;
        CKS(ensure_t(ctx, B_HCOUNT, (size_t)hsize, &hcount));
        CKS(ensure_t(ctx, B_FBINS, (size_t)n + 1, &fbins));
        CKS(ensure_t(ctx, B_FSTARTS, (size_t)n + 2, &fstarts));
        CKS(ensure(ctx, B_FSCAN, scan_temp_bytes(n + 1), &fscan));
        CK(cudaMemsetAsync(hcount, 0, hsize * sizeof(uint32_t), s));
        CK(cudaMemsetAsync(fbins, 0, (size_t)(n + 1) * sizeof(uint32_t), s));
        CK(launch_dedup_by_first(raw, cap, table, hcount, hsize, n, fbins, fstarts, fscan, cand, cnt, s,
                                 order == 5 ? pl.lens : nullptr));
    } else if (order != 2) {
        // candidates handed to the verifier longest first (order 4: length classes,
        // so that the pairs a warp takes have similar lengths) or most-collided
        // first (order 1: similar pairs, which run longest)
        uint32_t *hcount = nullptr;
        unsigned long long *bins = nullptr;
        CKS(ensure_t(ctx, B_HCOUNT, (size_t)hsize, &hcount));
        CKS(ensure_t(ctx, B_BINS, (size_t)count_bins(), &bins));
        CK(cudaMemsetAsync(hcount, 0, hsize * sizeof(uint32_t), s));
        CK(cudaMemsetAsync(bins, 0, count_bins() * sizeof(unsigned long long), s));
        CK(launch_dedup_ordered(raw, cap, table, hcount, hsize, bins, cand, cnt, order == 4 ? pl.lens : nullptr,
                                pl.max_len, s));
    } else {
        CK(launch_dedup(raw, cap, table, hsize, cand, cnt, s));
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[3], s));
    if (defer) {
        *defer = VerifySeg{cand, cnt + 2, cap, p->K, app, cnt + 3, cap, cnt + 4, derr};
        return EJ_OK;
    }
    unsigned int *tickets = nullptr;
    CKS(ensure_t(ctx, B_TICKETS, (size_t)SM_TICKETS, &tickets));
    CK(cudaMemsetAsync(tickets, 0, SM_TICKETS * sizeof(unsigned int), s));
    VerifyOut vo{nullptr, app, cnt + 3, cap, cnt + 2, derr, cnt + 4, cnt + 6, tickets};
    vo.max_passes = ctx->loop_bound;
    const VerifyConfig &vc = bs.vc;
    if (sx) {
        // warp tasks of up to 16 candidates sharing their longer string and the
        // class of their length difference
        const int64_t tcap = (int64_t)(cap / 16) + nb + 1;
        uint32_t *tcount = nullptr;
        uint64_t *tstart = nullptr, *tasks = nullptr;
        void *tscan = nullptr;
        CKS(ensure_t(ctx, B_SX_TCOUNT, (size_t)nb + 1, &tcount));
        CKS(ensure_t(ctx, B_SX_TSTART, (size_t)nb + 1, &tstart));
        CKS(ensure_t(ctx, B_SX_TASKS, (size_t)tcap, &tasks));
        CKS(ensure(ctx, B_SX_SCAN, scan_temp_bytes(nb + 1), &tscan));
        CK(launch_sx_tasks(fbins, fstarts, nb, tcount, tstart, cnt + 7, tscan, tasks, s));
        if (verify_after) CK(cudaStreamWaitEvent(s, verify_after, 0));
        CK(launch_verify_sx(sb.W1, pl.packed, pl.pofs, pl.B, pl.lens, n, p->alphabet_size, cand, tasks, cnt + 7,
                            tcap, p->K, vo, s));
    } else {
    if (verify_after) CK(cudaStreamWaitEvent(s, verify_after, 0));
    if (pq_threads > 0)
        // defaults: 16 slots per warp (they refill from the queue); working warps
        // per SM sub-partition from the pair count (the kernel's automatic rule)
        CK(launch_verify_pq(pq_words(p->K), pq_threads, ctx->sched.slots_per_warp ? ctx->sched.slots_per_warp : 16,
                            ctx->sched.warps_per_subpartition,
                            pl.packed, pl.pofs, pl.B, pl.lens, n, p->alphabet_size, cand, (int64_t)cap, p->K, vo,
                            s));
    else
        CK(launch_verify(vc, pl.packed, pl.pofs, pl.B, pl.lens, n, p->alphabet_size, cand, (int64_t)cap, p->K,
                         pl.max_len, vo, s));
    }
    if (verify_done) CK(cudaEventRecord(verify_done, s));
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[4], s));
    return EJ_OK;
}

// This join's share of a merged verifier launch: the buffers back_attempt
// with capacity cap uses (already sized; nothing is launched).
int back_segment(ej_ctx *ctx, const ej_params *p, uint64_t cap, VerifySeg *seg) {
    unsigned long long *cnt = nullptr;
    uint64_t *cand = nullptr, *app = nullptr;
    CKS(ensure_t(ctx, B_JCOUNT, 8, &cnt));
    CKS(ensure_t(ctx, B_CAND, (size_t)cap, &cand));
    CKS(ensure_t(ctx, B_APP, (size_t)cap, &app));
    *seg = VerifySeg{cand, cnt + 2, cap, p->K, app, cnt + 3, cap, cnt + 4, (uint32_t *)ctx->bufs[B_DERR].p};
    return EJ_OK;
}

// Counters of the last attempt: [0] raw, [1] max bucket, [2] candidates,
// [3] output, [4] band cells, [5] word columns, [6] device error bits.
int back_read(ej_ctx *ctx, unsigned long long hc[8], cudaStream_t s) {
    CK(cudaMemcpyAsync(ctx->h_cnt, ctx->bufs[B_JCOUNT].p, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_cnt + 6, ctx->bufs[B_DERR].p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memcpy(hc, ctx->h_cnt, 8 * sizeof(unsigned long long));
    hc[6] &= 0xffffffffull;
    if ((uint32_t)hc[6] & DERR_PAIR) return fail(ctx, EJ_ERR_INVALID_ARG, "internal: pair index out of range");
    if ((uint32_t)hc[6] & DERR_TIMEOUT)
        return fail(ctx, EJ_ERR_TIMEOUT, "the persistent verifier gave up after its bound of loop passes per warp");
    if ((uint32_t)hc[6] & DERR_GUARD) return fail(ctx, EJ_ERR_CUDA, "internal: a work bound was exceeded");
    return EJ_OK;
}

// Sort the appended output pairs and copy them to `out`.
int back_finish(ej_ctx *ctx, const Plan &pl, const ej_params *p, const unsigned long long hc[8], uint64_t *out,
                int64_t capacity, int64_t *n_out, ej_join_stats *stats, cudaStream_t s) {
    const int64_t n = pl.st.n, T = (int64_t)p->r * p->m;
    const int64_t cntout = (int64_t)hc[3];
    if (stats) {
        stats->n_raw_pairs = (int64_t)hc[0];
        stats->max_bucket = (int64_t)hc[1];
        stats->n_candidates = (int64_t)hc[2];
        stats->n_out = cntout;
        stats->band_cells = hc[4];
        stats->verify_word_columns = hc[5];
    }
    *n_out = cntout;
    if (cntout > capacity)
        return fail(ctx, EJ_ERR_CAPACITY, "output needs %lld pairs, capacity %lld", (long long)cntout, (long long)capacity);
    if (cntout == 0) return EJ_OK;
    uint64_t *app = (uint64_t *)ctx->bufs[B_APP].p, *raw = (uint64_t *)ctx->bufs[B_RAW].p;
    unsigned long long *cnt = (unsigned long long *)ctx->bufs[B_JCOUNT].p;
    const uint64_t *sorted = app;
    if (cntout <= small_sort_max()) {
        CK(launch_small_sort(app, cnt + 3, (uint64_t)cntout, s));
    } else {
        const int nb = bits_for((uint64_t)(n - 1));
        int shifts[16], np = 0;
        for (int b = 0; b < nb; b += 8) shifts[np++] = b;
        for (int b = 0; b < nb; b += 8) shifts[np++] = 32 + b;
        const size_t rs2 = radix_counts_len(cntout, 1);
        uint32_t *c2 = nullptr;
        uint64_t *o2 = nullptr;
        void *st2 = nullptr;
        CKS(ensure_t(ctx, B_RS_COUNTS, rs2 > radix_counts_len(n, T) ? rs2 : radix_counts_len(n, T), &c2));
        CKS(ensure_t(ctx, B_RS_OFFS, rs2 > radix_counts_len(n, T) ? rs2 : radix_counts_len(n, T), &o2));
        CKS(ensure(ctx, B_SCAN_TMP, scan_temp_bytes((int64_t)rs2), &st2));
        RadixTemp rt{c2, o2, st2};
        bool alt = false;
        CK(radix_sort_segmented(app, nullptr, raw, nullptr, cntout, 1, shifts, np, rt, &alt, s));
        sorted = alt ? raw : app;
    }
    CK(cudaMemcpyAsync(out, sorted, (size_t)cntout * sizeof(uint64_t), cudaMemcpyDefault, s));
    return EJ_OK;
}

int join_back(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *keys, uint64_t *out,
              int64_t capacity, int64_t *n_out, ej_join_stats *stats, cudaStream_t s) {
    BackState bs;
    CKS(back_buckets(ctx, pl, p, keys, &bs, s));
    uint64_t cap = raw_cap_start(ctx, pl.st.n);
    unsigned long long hc[8];
    for (int attempt = 0;; attempt++) {
        CKS(back_attempt(ctx, pl, p, bs, cap, s));
        CKS(back_read(ctx, hc, s));
        if (hc[0] <= cap) break;
        if (attempt > 0) return fail(ctx, EJ_ERR_CUDA, "raw pair count changed between attempts");
        cap = hc[0] + hc[0] / 4 + 1024;
    }
    ctx->raw_cap_hint = cap;
    return back_finish(ctx, pl, p, hc, out, capacity, n_out, stats, s);
}

// ---------------------------------------------------------------------------
// Autotuner: per (length class, K), the walk's block size and the verifier's
// kind and tiling, timed on the join's own strings and candidates
// ---------------------------------------------------------------------------

struct TuneCand {
    ej_schedule sc;   // mode, slots_per_warp, warps_per_subpartition, order (buckets, chain kept)
    int G, V;         // verifier tiling (0 = automatic)
};

std::vector<TuneCand> tune_candidates(const ej_params *p) {
    const int W = (2 * p->K + 1 + 63) / 64;
    std::vector<TuneCand> c = {
        {{1, 16, 1, 0, 0, 0}, 0, 0}, {{1, 16, 2, 0, 0, 0}, 0, 0}, {{1, 16, 4, 0, 0, 0}, 0, 0},
        {{1, 8, 1, 0, 0, 0}, 0, 0},
        {{3, 0, 0, 0, 0, 0}, 0, 0},  {{2, 0, 0, 3, 0, 0}, 0, 0},  {{2, 0, 0, 4, 0, 0}, 0, 0},
    };
    if (W <= 8) c.push_back({{2, 0, 0, 3, 0, 0}, 1, W});
    if ((W + 3) / 4 <= 4) c.push_back({{2, 0, 0, 3, 0, 0}, 4, (W + 3) / 4});
    return c;
}

uint64_t tune_key(const Plan &pl, const ej_params *p) {
    const int64_t mean = pl.st.n > 0 ? pl.st.total / pl.st.n : 0;
    int cls = 0;
    while (cls < 62 && (mean >> (cls + 1)) > 0) cls++;
    return ((uint64_t)(uint32_t)cls << 32) | (uint32_t)p->K;
}

void apply_tune(ej_ctx *ctx, const ej_tune_entry &e) {
    ctx->sched.mode = e.schedule.mode;
    ctx->sched.slots_per_warp = e.schedule.slots_per_warp;
    ctx->sched.warps_per_subpartition = e.schedule.warps_per_subpartition;
    ctx->sched.order = e.schedule.order;
    ctx->vG = e.lanes_per_pair;
    ctx->vV = e.words_per_lane;
    if (e.walk_threads) ctx->walk_tpb = e.walk_threads;
}

// Times the back half (buckets .. verification, raw capacity cap) under every
// candidate and leaves the fastest in *best (the context's own settings are
// restored). Candidates that fail to launch are skipped.
int tune_back(ej_ctx *ctx, const Plan &pl, const ej_params *p, const uint64_t *keys, uint64_t cap, cudaStream_t s,
              ej_tune_entry *best) {
    const ej_schedule sc0 = ctx->sched;
    const int vG0 = ctx->vG, vV0 = ctx->vV;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int tried = 0;
    for (const TuneCand &c : tune_candidates(p)) {
        ctx->sched = sc0;
        ctx->sched.mode = c.sc.mode;
        ctx->sched.slots_per_warp = c.sc.slots_per_warp;
        ctx->sched.warps_per_subpartition = c.sc.warps_per_subpartition;
        ctx->sched.order = c.sc.order;
        ctx->vG = c.G;
        ctx->vV = c.V;
        float t = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; rep++) {
            BackState bs;
            ok = cudaEventRecord(e0, s) == cudaSuccess && back_buckets(ctx, pl, p, keys, &bs, s) == EJ_OK &&
                 back_attempt(ctx, pl, p, bs, cap, s) == EJ_OK && cudaEventRecord(e1, s) == cudaSuccess &&
                 cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.f;
            if (ok) cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t += ms;   // the first run warms the choice up
        }
        if (!ok) {
            cudaGetLastError();
            cudaStreamSynchronize(s);
            continue;
        }
        tried++;
        if (t < best_ms) {
            best_ms = t;
            best->schedule = ctx->sched;
            best->lanes_per_pair = c.G;
            best->words_per_lane = c.V;
        }
    }
    ctx->sched = sc0;
    ctx->vG = vG0;
    ctx->vV = vV0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best->back_ms = best_ms / 2.f;
    best->configs_tried += tried;
    return tried ? EJ_OK : fail(ctx, EJ_ERR_CUDA, "no verifier choice ran");
}

// The whole tuning of one join: the walk's block size, then the back half.
int tune_join(ej_ctx *ctx, const Plan &pl, const ej_params *p, uint64_t *keys, cudaStream_t s, ej_tune_entry *out) {
    const uint64_t key = tune_key(pl, p);
    memset(out, 0, sizeof *out);
    out->length_class = (int32_t)(key >> 32);
    out->K = p->K;
    const int tpb0 = ctx->walk_tpb;
    ctx->walk_tpb = 0;
    CKS(keys_dev(ctx, p, pl, keys, s));   // tables and a first walk
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int tpb : {256, 512, 1024}) {
        if (embed_sign_smem(p->alphabet_size, pl.L, p->m, p->z, tpb) == 0) continue;
        ctx->walk_tpb = tpb;
        float t = 0.f;
        for (int rep = 0; rep < 3; rep++) {
            CK(cudaEventRecord(e0, s));
            CKS(keys_dev(ctx, p, pl, keys, s, nullptr, 2));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) t += ms;
        }
        out->configs_tried++;
        if (t < best) {
            best = t;
            out->walk_threads = tpb;
            out->walk_ms = t / 2.f;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->walk_tpb = tpb0;
    // the back half with a raw-pair capacity sized by one ordinary run
    BackState bs;
    CKS(back_buckets(ctx, pl, p, keys, &bs, s));
    uint64_t cap = raw_cap_start(ctx, pl.st.n);
    unsigned long long hc[8];
    for (int attempt = 0;; attempt++) {
        CKS(back_attempt(ctx, pl, p, bs, cap, s));
        CKS(back_read(ctx, hc, s));
        if (hc[0] <= cap) break;
        if (attempt > 0) return fail(ctx, EJ_ERR_CUDA, "raw pair count changed between attempts");
        cap = hc[0] + hc[0] / 4 + 1024;
    }
    ctx->raw_cap_hint = cap;
    return tune_back(ctx, pl, p, keys, cap, s, out);
}

// Output array: device pointer or a staging buffer to copy to host after.
int out_target(ej_ctx *ctx, BufId id, void *user, size_t bytes, void **dev, bool *is_host) {
    if (is_device_ptr(user)) {
        *dev = user;
        *is_host = false;
        return EJ_OK;
    }
    *is_host = true;
    return ensure(ctx, id, bytes, dev);
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

#define CKB(b, expr)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) return fail((b)->ctx, EJ_ERR_CUDA, "%s", cudaGetErrorString(e_)); \
    } while (0)

// One join of a batch: its own context (scratch, counters), parameters and plan.
struct BatchJoin {
    ej_ctx *sub = nullptr;
    ej_params p{};
    std::vector<uint8_t> alphabet;
    Plan pl;
    BackState bs;
    uint64_t cap = 0;
    uint64_t *keys = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t verified = nullptr;   // this join's verifier finished (chains the verifiers)
    cudaEvent_t keyed = nullptr;      // this join's keys are written
    int src = -1;                     // join whose walks give this join's keys (-1: its own)
    uint64_t modulus = 0;             // keys = src keys mod modulus (0: same z)
    bool alias = false;               // same r, m, z as src: read src's keys directly
    bool in_walk = false;             // same r, m, smaller z: written by src's walk kernel
    uint64_t ncand = 0;               // candidates in the eager pass
    int seg = -1;                     // share of the merged verifier launch (-1: none)
    int bucket_owner = -1;            // join whose buckets give this join's pairs (-1: its own)
    std::vector<int> bucket_members;  // owner: the joins (itself first) its buckets serve
    cudaEvent_t emitted = nullptr;    // owner: every member's pairs are written
};

}  // namespace

struct ej_batch {
    ej_ctx *ctx = nullptr;
    Plan pl;
    std::vector<BatchJoin> joins;
    cudaEvent_t fork = nullptr;
    cudaEvent_t start = nullptr;      // the run's start on its stream (the tables wait for it)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernel_nodes = 0;
    bool ran = false;
    // merged persistent verifier: one launch over the joins' candidates in turn
    std::vector<int> merged;           // join indices in launch order (largest K first)
    int mW1 = 0, mK = 0, mthreads = 0;
    VerifySeg *segs_dev = nullptr;
    unsigned long long *mqueue = nullptr;
    unsigned int *mtickets = nullptr;
    // ... over the union of their candidates (chain 4): each distinct pair once
    bool munion = false;
    uint64_t ucap = 0, uhsize = 0;
    uint64_t *utable = nullptr, *upairs = nullptr;
    uint32_t *utmask = nullptr, *umask = nullptr;
    unsigned long long *ubins = nullptr;      // count_bins() + 1: the bins, then the pair count
    cudaEvent_t v0 = nullptr, v1 = nullptr;   // around the merged launch
    bool eager = false;                       // no graph: every run issues the work
    // results staged by the run itself: per join 8 counters + the error word, and
    // the plan's error word and longest string (pinned), complete at `done`
    unsigned long long *h_stat = nullptr;
    cudaEvent_t done = nullptr;
};

namespace {

void batch_free(ej_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->start) cudaEventDestroy(b->start);
    if (b->v0) cudaEventDestroy(b->v0);
    if (b->v1) cudaEventDestroy(b->v1);
    if (b->done) cudaEventDestroy(b->done);
    if (b->h_stat) cudaFreeHost(b->h_stat);
    if (b->segs_dev) cudaFree(b->segs_dev);
    if (b->mqueue) cudaFree(b->mqueue);
    if (b->mtickets) cudaFree(b->mtickets);
    if (b->utable) cudaFree(b->utable);
    if (b->upairs) cudaFree(b->upairs);
    if (b->utmask) cudaFree(b->utmask);
    if (b->umask) cudaFree(b->umask);
    if (b->ubins) cudaFree(b->ubins);
    for (auto &j : b->joins) {
        if (j.done) cudaEventDestroy(j.done);
        if (j.verified) cudaEventDestroy(j.verified);
        if (j.keyed) cudaEventDestroy(j.keyed);
        if (j.emitted) cudaEventDestroy(j.emitted);
        if (j.side) cudaStreamDestroy(j.side);
        if (j.sub) ej_destroy(j.sub);
    }
    delete b;
}

// Keys of one join on stream s: its own walk and signatures, or derived from
// its source join's keys (which must already be written on s's timeline).
int batch_join_keys(std::vector<BatchJoin> &joins, BatchJoin &j, cudaStream_t s, int phase = 0) {
    if (j.src < 0) {
        PrefixKeys pk{};
        for (const BatchJoin &d : joins)
            if (d.in_walk && &joins[(size_t)d.src] == &j) {
                pk.z[pk.n] = d.p.z;
                pk.keys[pk.n] = d.keys;
                pk.n++;
            }
        return keys_dev(j.sub, &j.p, j.pl, j.keys, s, pk.n ? &pk : nullptr, phase);
    }
    if (j.alias || j.in_walk || phase == 1) return EJ_OK;
    ej_ctx *ctx = j.sub;
    const BatchJoin &src = joins[(size_t)j.src];
    CK(launch_derive_keys(src.keys, src.p.m, j.pl.st.n, j.p.r, j.p.m, j.modulus, j.keys, s));
    return EJ_OK;
}

// Join a's walks cover join b's signatures: same seed and sampling range, and
// at least as many embeddings, functions and samples per function.
bool batch_covers(const BatchJoin &a, const BatchJoin &b) {
    return a.p.seed == b.p.seed && a.pl.L == b.pl.L && a.p.r >= b.p.r && a.p.m >= b.p.m && a.p.z >= b.p.z;
}

// Sources: a join walks its strings itself unless another join covers it (and
// is not covered back, or is equal and earlier); it then takes the first such
// self-walking join's keys. Covering is transitive, so one always exists.
void batch_sources(std::vector<BatchJoin> &joins) {
    const size_t n = joins.size();
    std::vector<bool> root(n, true);
    for (size_t i = 0; i < n; i++)
        for (size_t k = 0; k < n && root[i]; k++)
            if (k != i && batch_covers(joins[k], joins[i]) && (!batch_covers(joins[i], joins[k]) || k < i))
                root[i] = false;
    for (size_t i = 0; i < n; i++) {
        BatchJoin &j = joins[i];
        if (root[i]) continue;
        for (size_t k = 0; k < n; k++)
            if (root[k] && batch_covers(joins[k], j)) {
                j.src = (int)k;
                break;
            }
        const BatchJoin &src = joins[(size_t)j.src];
        j.alias = src.p.r == j.p.r && src.p.m == j.p.m && src.p.z == j.p.z;
        int taken = 0;
        for (const BatchJoin &d : joins)
            if (d.in_walk && d.src == j.src) taken++;
        j.in_walk = !j.alias && src.p.r == j.p.r && src.p.m == j.p.m && taken < MAX_PREFIX_KEYS;
        j.modulus = 0;
        if (j.p.z < src.p.z) {
            j.modulus = 1;
            for (uint32_t q = 0; q < j.p.z; q++) j.modulus *= (uint64_t)j.p.alphabet_size + 1;
        }
    }
}

// Merged verification (ej_schedule.chain 0, 3 or 4): the joins that use the
// persistent verifier are verified by one launch at the widest of their bands,
// each pair with its own join's K. Mode 3: the work queue runs over the joins'
// candidates in turn, largest K first, so no launch waits for another launch's
// last pairs. Mode 4: it runs over the union of their candidates, each distinct
// pair once at the largest K of the joins that list it (its distance, exact up
// to that K, decides it for every one of them): joins over the same strings
// whose signatures nest share most of their candidates. Mode 0 merges when the
// wider band adds at most half of the word-columns the joins' own bands would
// run (estimated from the eager pass's candidate counts), as 4 while the
// candidates are few for the slots, else as 3; otherwise, as mode 2, the
// launches are chained.
int batch_plan_merge(ej_batch *b) {
    ej_ctx *ctx = b->ctx;
    const int mode = ctx->sched.chain;
    if (mode == 1 || mode == 2) return EJ_OK;
    std::vector<int> pq;
    for (size_t i = 0; i < b->joins.size(); i++) {
        BatchJoin &j = b->joins[i];
        if (pq_choice(j.sub, j.pl, &j.p, j.bs.vc) > 0) pq.push_back((int)i);
    }
    if (pq.size() < 2) return EJ_OK;
    std::stable_sort(pq.begin(), pq.end(), [&](int x, int y) { return b->joins[(size_t)x].p.K > b->joins[(size_t)y].p.K; });
    if (pq.size() > (size_t)MAX_VERIFY_SEGS) pq.resize(MAX_VERIFY_SEGS);
    int W1 = 0, K = 0;
    double own = 0.0, wide = 0.0;
    for (int i : pq) {
        const BatchJoin &j = b->joins[(size_t)i];
        W1 = std::max(W1, pq_words(j.p.K));
        K = std::max(K, (int)j.p.K);
    }
    for (int i : pq) {
        const BatchJoin &j = b->joins[(size_t)i];
        own += (double)j.ncand * pq_words(j.p.K);
        wide += (double)j.ncand * W1;
    }
    if (mode == 0 && wide > 1.5 * own) return EJ_OK;
    const int threads = pq_threads_for(W1, b->joins[0].p.alphabet_size);
    if (threads == 0 || W1 < pq_words(K)) return EJ_OK;
    CK(cudaMalloc(&b->segs_dev, pq.size() * sizeof(VerifySeg)));
    CK(cudaMalloc(&b->mqueue, sizeof(unsigned long long)));
    CK(cudaMalloc(&b->mtickets, SM_TICKETS * sizeof(unsigned int)));
    b->merged = pq;
    b->mW1 = W1;
    b->mK = K;
    b->mthreads = threads;
    // mode 0: the union while the launch is set by its longest pairs (fewer than
    // 32 pairs per slot of one warp per SM sub-partition, measured faster: 0.63 vs
    // 0.67 ms on long DNA), the joins in turn when its total work sets it (29.6 vs
    // 32.0 ms at 600 pairs per slot)
    double total = 0.0;
    for (int i : pq) total += (double)b->joins[(size_t)i].ncand;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const bool tail_bound = total < 32.0 * (double)(dev_sms > 0 ? dev_sms : 1) * 4 * 16;
    if (mode == 4 || (mode == 0 && tail_bound)) {
        b->munion = true;
        for (int i : pq) b->joins[(size_t)i].bs.any_order = true;   // the union orders the candidates
        for (int i : pq) b->ucap += b->joins[(size_t)i].cap;
        // the union holds at most the joins' capacities together (each of which
        // already has a margin over its candidates): a table of that many slots
        // always has room, and is scanned whole by the union's order pass
        b->uhsize = 1;
        while (b->uhsize < b->ucap + 1) b->uhsize <<= 1;
        CK(cudaMalloc(&b->utable, b->uhsize * sizeof(uint64_t)));
        CK(cudaMalloc(&b->utmask, b->uhsize * sizeof(uint32_t)));
        CK(cudaMalloc(&b->upairs, b->ucap * sizeof(uint64_t)));
        CK(cudaMalloc(&b->umask, b->ucap * sizeof(uint32_t)));
        CK(cudaMalloc(&b->ubins, ((size_t)count_bins() + 1) * sizeof(unsigned long long)));
    }
    for (size_t k = 0; k < pq.size(); k++) b->joins[(size_t)pq[k]].seg = (int)k;
    return EJ_OK;
}

// The merged launch on stream s (after every merged join's candidates).
int batch_merged_verify(ej_batch *b, cudaStream_t s) {
    ej_ctx *ctx = b->ctx;
    CK(cudaMemsetAsync(b->mqueue, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(b->mtickets, 0, SM_TICKETS * sizeof(unsigned int), s));
    uint64_t total_cap = 0;
    for (int i : b->merged) total_cap += b->joins[(size_t)i].cap;
    VerifyOut vo{};
    vo.queue = b->mqueue;
    vo.sm_tickets = b->mtickets;
    vo.segs = b->segs_dev;
    vo.nseg = (int32_t)b->merged.size();
    vo.max_passes = ctx->loop_bound;
    const Plan &pl = b->pl;
    if (b->munion) {
        unsigned long long *ucount = b->ubins + count_bins();
        CK(launch_union_candidates(b->segs_dev, vo.nseg, b->utable, b->utmask, b->uhsize, b->ubins, b->upairs,
                                   b->umask, ucount, pl.lens, pl.max_len, ctx->sched.order != 1, s));
        vo.upairs = b->upairs;
        vo.umask = b->umask;
        vo.unp_dev = ucount;
        vo.ucap = b->ucap;
        total_cap = b->ucap;
    }
    CK(launch_verify_pq(b->mW1, b->mthreads, ctx->sched.slots_per_warp ? ctx->sched.slots_per_warp : 16,
                        ctx->sched.warps_per_subpartition, pl.packed, pl.pofs,
                        pl.B, pl.lens, pl.st.n, b->joins[0].p.alphabet_size, nullptr, (int64_t)total_cap, b->mK, vo, s,
                        b->munion));   // the union launch runs only while its pairs are few
    return EJ_OK;
}

// Shared buckets (ej_schedule.buckets 0): joins with hashed buckets and the
// same seed, L, r and m take their raw pairs from the buckets of the one with
// the fewest samples per function (its signatures are the coarsest), up to
// MAX_SHARED_BUCKETS joins per owner; see bucket_emit_shared_kernel.
int batch_plan_buckets(ej_batch *b) {
    ej_ctx *ctx = b->ctx;
    if (ctx->sched.buckets != 0) return EJ_OK;
    const size_t n = b->joins.size();
    std::vector<bool> used(n, false);
    for (size_t i = 0; i < n; i++) {
        if (used[i] || !b->joins[i].bs.hashed) continue;
        const BatchJoin &a = b->joins[i];
        std::vector<int> group;
        for (size_t k = i; k < n; k++) {
            const BatchJoin &c = b->joins[k];
            if (!used[k] && c.bs.hashed && c.p.seed == a.p.seed && c.pl.L == a.pl.L && c.p.r == a.p.r &&
                c.p.m == a.p.m)
                group.push_back((int)k);
        }
        for (size_t g0 = 0; g0 + 1 < group.size(); g0 += MAX_SHARED_BUCKETS) {
            std::vector<int> chunk(group.begin() + (long)g0,
                                   group.begin() + (long)std::min(group.size(), g0 + MAX_SHARED_BUCKETS));
            if (chunk.size() < 2) break;
            int owner = chunk[0];
            for (int k : chunk)
                if (b->joins[(size_t)k].p.z < b->joins[(size_t)owner].p.z) owner = k;
            BatchJoin &o = b->joins[(size_t)owner];
            o.bucket_members.push_back(owner);
            for (int k : chunk)
                if (k != owner) {
                    o.bucket_members.push_back(k);
                    b->joins[(size_t)k].bucket_owner = owner;
                }
            CK(cudaEventCreateWithFlags(&o.emitted, cudaEventDisableTiming));
        }
        for (int k : group) used[(size_t)k] = true;
    }
    return EJ_OK;
}

// An owner's buckets and its members' raw pairs, on the owner's stream (after
// the owner's keys); the members' keys must be recorded in their `keyed` events.
int batch_shared_emit(ej_batch *b, BatchJoin &o) {
    ej_ctx *ctx = o.sub;
    CKS(back_buckets(o.sub, o.pl, &o.p, o.keys, &o.bs, o.side));
    SharedEmit se{};
    se.njoins = (int32_t)o.bucket_members.size();
    for (size_t k = 0; k < o.bucket_members.size(); k++) {
        BatchJoin &m = b->joins[(size_t)o.bucket_members[k]];
        if (&m != &o) CK(cudaStreamWaitEvent(o.side, m.keyed, 0));
        unsigned long long *cnt = nullptr;
        uint64_t *raw = nullptr;
        CKS(ensure_t(m.sub, B_JCOUNT, 8, &cnt));
        CKS(ensure_t(m.sub, B_RAW, (size_t)m.cap, &raw));
        CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), o.side));
        se.keys[k] = m.keys;
        se.K[k] = m.p.K;
        se.raw[k] = raw;
        se.cap[k] = m.cap;
        se.counters[k] = cnt;
    }
    if (o.bs.table_smem)
        CK(launch_bucket_table(o.pl.lens, o.pl.st.n, (int64_t)o.p.r * o.p.m, se, o.side));
    else
        CK(launch_bucket_emit_shared(o.pl.lens, o.pl.st.n, (int64_t)o.p.r * o.p.m, o.bs.bnext, se, o.side));
    CK(cudaEventRecord(o.emitted, o.side));
    return EJ_OK;
}

// The batch's device work on stream s (captured once into the graph, or issued
// by every run of an eager batch): plan (validate, pack) on s, then every join
// on its own stream, joined back into s at the end.
int batch_issue(ej_batch *b, cudaStream_t s) {
    ej_ctx *ctx = b->ctx;
    int cst = EJ_OK;
    // the walking joins' tables (bits, positions) depend on the parameters only:
    // they are built on the joins' streams while s validates and packs
    if (cudaEventRecord(b->start, s) != cudaSuccess) cst = EJ_ERR_CUDA;
    for (auto &j : b->joins) {
        if (cst != EJ_OK || j.src >= 0) continue;
        if (cudaStreamWaitEvent(j.side, b->start, 0) != cudaSuccess) cst = EJ_ERR_CUDA;
        if (cst == EJ_OK) cst = batch_join_keys(b->joins, j, j.side, 1);
    }
    if (cst == EJ_OK) cst = plan_device(ctx, b->pl, s);
    if (cst == EJ_OK && cudaEventRecord(b->fork, s) != cudaSuccess) cst = EJ_ERR_CUDA;
    // keys: the self-walking joins first, then the derived ones after their source
    for (int pass = 0; pass < 2 && cst == EJ_OK; pass++)
        for (auto &j : b->joins) {
            if (cst != EJ_OK || (pass == 0) != (j.src < 0)) continue;
            cudaEvent_t after = j.src < 0 ? b->fork : b->joins[(size_t)j.src].keyed;
            if (cudaStreamWaitEvent(j.side, after, 0) != cudaSuccess) { cst = EJ_ERR_CUDA; break; }
            cst = batch_join_keys(b->joins, j, j.side, 2);
            if (cst == EJ_OK && cudaEventRecord(j.keyed, j.side) != cudaSuccess) cst = EJ_ERR_CUDA;
        }
    // verifiers run one after another unless chain == 1: two persistent grids
    // sharing the SMs (each capping its working warps per SM) measured from
    // slightly faster to 10x slower from one replay to the next, and two grid-
    // strided ones each fill the GPU; every other stage overlaps
    // shared buckets: each owner inserts and emits its members' pairs
    for (auto &j : b->joins)
        if (cst == EJ_OK && !j.bucket_members.empty()) cst = batch_shared_emit(b, j);
    cudaEvent_t prev_verify = nullptr;
    VerifySeg unused{};
    for (auto &j : b->joins) {
        if (cst != EJ_OK) break;
        const bool shared = j.bucket_owner >= 0 || !j.bucket_members.empty();
        if (j.bucket_owner >= 0 &&
            cudaStreamWaitEvent(j.side, b->joins[(size_t)j.bucket_owner].emitted, 0) != cudaSuccess) {
            cst = EJ_ERR_CUDA;
            break;
        }
        if (!shared) cst = back_buckets(j.sub, j.pl, &j.p, j.keys, &j.bs, j.side);
        if (cst != EJ_OK) break;
        if (j.seg >= 0) {
            // verified by the merged launch below
            cst = back_attempt(j.sub, j.pl, &j.p, j.bs, j.cap, j.side, nullptr, nullptr, &unused, shared);
        } else {
            // every verifier of a batch fills the GPU on its own: they run one
            // after another (chain 1: free to overlap) while the other joins'
            // walks, buckets and dedup overlap them
            const bool heavy = ctx->sched.chain != 1;
            cst = back_attempt(j.sub, j.pl, &j.p, j.bs, j.cap, j.side, heavy ? prev_verify : nullptr,
                               heavy ? j.verified : nullptr, nullptr, shared);
            if (heavy) prev_verify = j.verified;
        }
        if (cst == EJ_OK && cudaEventRecord(j.done, j.side) != cudaSuccess) cst = EJ_ERR_CUDA;
        if (cst == EJ_OK && cudaStreamWaitEvent(s, j.done, 0) != cudaSuccess) cst = EJ_ERR_CUDA;
    }
    if (cst == EJ_OK && !b->merged.empty()) {
        if (prev_verify && cudaStreamWaitEvent(s, prev_verify, 0) != cudaSuccess) cst = EJ_ERR_CUDA;
        // timed in eager batches (under capture a record is only an ordering edge)
        if (cst == EJ_OK && b->eager && cudaEventRecord(b->v0, s) != cudaSuccess) cst = EJ_ERR_CUDA;
        if (cst == EJ_OK) cst = batch_merged_verify(b, s);
        if (cst == EJ_OK && b->eager && cudaEventRecord(b->v1, s) != cudaSuccess) cst = EJ_ERR_CUDA;
    }
    // results: every join's output sorted on the device (up to small_sort_max()
    // pairs; ej_batch_result sorts larger ones) and all counters copied to pinned
    // host memory, so that reading the results waits once
    // (each join on its own stream, after its verifier)
    if (cst == EJ_OK && !b->merged.empty() && cudaEventRecord(b->fork, s) != cudaSuccess) cst = EJ_ERR_CUDA;
    for (size_t k = 0; k < b->joins.size() && cst == EJ_OK; k++) {
        BatchJoin &j = b->joins[k];
        const cudaStream_t js = j.side;
        unsigned long long *cnt = (unsigned long long *)j.sub->bufs[B_JCOUNT].p;
        if ((j.seg >= 0 && cudaStreamWaitEvent(js, b->fork, 0) != cudaSuccess) ||
            launch_small_sort((uint64_t *)j.sub->bufs[B_APP].p, cnt + 3, (uint64_t)small_sort_max(), js) != cudaSuccess ||
            cudaMemcpyAsync(b->h_stat + 16 * k, cnt, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, js) !=
                cudaSuccess ||
            cudaMemcpyAsync(b->h_stat + 16 * k + 8, j.sub->bufs[B_DERR].p, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            js) != cudaSuccess ||
            cudaEventRecord(j.done, js) != cudaSuccess || cudaStreamWaitEvent(s, j.done, 0) != cudaSuccess)
            cst = EJ_ERR_CUDA;
    }
    if (cst == EJ_OK && cudaMemcpyAsync(b->h_stat + 16 * b->joins.size(), ctx->bufs[B_DERR].p, 16,
                                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        cst = EJ_ERR_CUDA;
    return cst;
}

int batch_autotune(ej_ctx *parent, BatchJoin &j, cudaStream_t s, float *best_ms) {
    const uint64_t key = tune_key(j.pl, &j.p);
    auto it = parent->tune_table.find(key);
    if (it == parent->tune_table.end()) {
        ej_tune_entry e;
        memset(&e, 0, sizeof e);
        e.length_class = (int32_t)(key >> 32);
        e.K = j.p.K;
        CKS(tune_back(j.sub, j.pl, &j.p, j.keys, j.cap, s, &e));
        it = parent->tune_table.emplace(key, e).first;
    }
    apply_tune(j.sub, it->second);
    *best_ms = it->second.back_ms;
    return EJ_OK;
}

}  // namespace

namespace ej {

int ctx_pack(ej_ctx *ctx, const ej_strings *S, const ej_params *p, PackedSet *out, void *stream) {
    cudaSetDevice(ctx->device);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, as_stream(stream)));
    out->packed = pl.packed;
    out->pofs = pl.pofs;
    out->lens = pl.lens;
    out->n = pl.st.n;
    out->max_len = pl.max_len;
    out->total = pl.st.total;
    out->B = pl.B;
    out->code_map = (const uint8_t *)ctx->bufs[B_CODEMAP].p;
    out->alphabet_dev = (const uint8_t *)ctx->bufs[B_ALPHABET].p;
    return EJ_OK;
}

int ctx_device(const ej_ctx *ctx) { return ctx->device; }

int ctx_sorted_records(ej_ctx *ctx, const PackedSet &set, const ej_params *p, const uint64_t *keys,
                       const uint64_t **rk, const uint32_t **rid, cudaStream_t s) {
    cudaSetDevice(ctx->device);
    Plan pl;
    pl.st.n = set.n;
    pl.lens = const_cast<int32_t *>(set.lens);
    pl.max_len = set.max_len;
    return sorted_records(ctx, pl, p, keys, rk, rid, s);
}

int ctx_fail(ej_ctx *ctx, int code, const char *msg) { return fail(ctx, code, "%s", msg); }

int ctx_check_params(ej_ctx *ctx, const ej_params *p) { return check_params(ctx, p, true); }

}  // namespace ej

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char *ej_status_string(int status) {
    switch (status) {
        case EJ_OK: return "ok";
        case EJ_ERR_INVALID_ARG: return "invalid argument";
        case EJ_ERR_OOM: return "out of memory";
        case EJ_ERR_CAPACITY: return "output capacity exceeded";
        case EJ_ERR_CUDA: return "CUDA error";
        case EJ_ERR_TIMEOUT: return "device wait timed out";
        case EJ_ERR_UNSUPPORTED: return "unsupported configuration";
        case EJ_ERR_TOO_LARGE: return "request exceeds the fixed scratch of ej_verify_noalloc";
        default: return "unknown status";
    }
}

int ej_create(ej_ctx **out, int device) {
    if (!out) return EJ_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return EJ_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return EJ_ERR_CUDA;
    ej_ctx *c = new (std::nothrow) ej_ctx();
    if (!c) return EJ_ERR_OOM;
    c->device = device;
    if (cudaMallocHost((void **)&c->h_cnt, 4096) != cudaSuccess) {
        delete c;
        return EJ_ERR_OOM;
    }
    for (auto &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            ej_destroy(c);
            return EJ_ERR_CUDA;
        }
    *out = c;
    return EJ_OK;
}

void ej_destroy(ej_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (auto &b : c->bufs)
        if (b.p) cudaFree(b.p);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->plus_sub) ej_destroy(c->plus_sub);
    if (c->group_sub) ej_destroy(c->group_sub);
    delete c;
}

const char *ej_last_error(ej_ctx *c) { return c ? c->err.c_str() : ""; }

int ej_set_timing(ej_ctx *c, int enable) {
    if (!c) return EJ_ERR_INVALID_ARG;
    c->timing = enable != 0;
    return EJ_OK;
}

int ej_set_key_hash(ej_ctx *c, uint64_t P) {
    if (!c) return EJ_ERR_INVALID_ARG;
    if (P != 0 && (P < 2 || P >= (1ull << 32)))
        return fail(c, EJ_ERR_INVALID_ARG, "the hash modulus must be 0 or in [2, 2^32)");
    if (P > 3)
        for (uint64_t d = 2; d * d <= P; d++)
            if (P % d == 0) return fail(c, EJ_ERR_INVALID_ARG, "the hash modulus %llu is not prime", (unsigned long long)P);
    c->key_P = P;
    return EJ_OK;
}

int ej_set_autotune(ej_ctx *c, int enable) {
    if (!c) return EJ_ERR_INVALID_ARG;
    if (enable < 0) c->tune_table.clear();
    c->autotune = enable > 0;
    return EJ_OK;
}

int ej_autotune_table(ej_ctx *c, ej_tune_entry *out, int32_t max, int32_t *n) {
    if (!c || !n || max < 0 || (max > 0 && !out)) return EJ_ERR_INVALID_ARG;
    *n = (int32_t)c->tune_table.size();
    int32_t k = 0;
    for (const auto &kv : c->tune_table) {
        if (k >= max) break;
        out[k++] = kv.second;
    }
    return EJ_OK;
}

int ej_set_loop_bound(ej_ctx *c, int64_t passes) {
    if (!c || passes < 0) return EJ_ERR_INVALID_ARG;
    c->loop_bound = passes;
    return EJ_OK;
}

int ej_set_verify_config(ej_ctx *ctx, int G, int V, int warps) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    if (G == 0 && V == 0) {
        ctx->vG = ctx->vV = ctx->vWarps = 0;
        return EJ_OK;
    }
    const bool okG = G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32;
    const int vmax = G == 1 ? 8 : (G == 2 ? 12 : 4);
    if (!okG || V < (G == 2 ? 2 : 1) || V > vmax || warps < 0 || warps > 8)
        return fail(ctx, EJ_ERR_INVALID_ARG, "verify config G=%d V=%d warps=%d not supported", G, V, warps);
    ctx->vG = G;
    ctx->vV = V;
    ctx->vWarps = warps;
    return EJ_OK;
}

int ej_set_schedule(ej_ctx *ctx, const ej_schedule *sc) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    if (!sc) {
        ctx->sched = ej_schedule{0, 0, 0, 0, 0, 0};
        return EJ_OK;
    }
    if (sc->mode < 0 || sc->mode > 3 || sc->slots_per_warp < 0 || sc->slots_per_warp > 16 ||
        sc->warps_per_subpartition < 0 || sc->warps_per_subpartition > 16 || sc->order < 0 || sc->order > 5 ||
        sc->buckets < 0 || sc->buckets > 2 || sc->chain < 0 || sc->chain > 4)
        return fail(ctx, EJ_ERR_INVALID_ARG,
                    "schedule mode=%d slots_per_warp=%d warps_per_subpartition=%d order=%d buckets=%d not supported",
                    sc->mode, sc->slots_per_warp, sc->warps_per_subpartition, sc->order, sc->buckets);
    ctx->sched = *sc;
    return EJ_OK;
}

int ej_set_test_tables(ej_ctx *ctx, const uint8_t *pi, uint32_t r, uint32_t steps, uint32_t alphabet_size,
                       const uint32_t *positions, uint32_t m, uint32_t z) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    ctx->pi.clear();
    ctx->posinj.clear();
    if (pi) {
        if (r == 0 || steps == 0 || alphabet_size == 0)
            return fail(ctx, EJ_ERR_INVALID_ARG, "pi table needs r, steps, alphabet_size > 0");
        ctx->pi.assign(pi, pi + (size_t)r * steps * alphabet_size);
        ctx->pi_r = r;
        ctx->pi_steps = steps;
        ctx->pi_alpha = alphabet_size;
    }
    if (positions) {
        if (r == 0 || m == 0 || z == 0) return fail(ctx, EJ_ERR_INVALID_ARG, "positions need r, m, z > 0");
        ctx->posinj.assign(positions, positions + (size_t)r * m * z);
        ctx->pos_r = r;
        ctx->pos_m = m;
        ctx->pos_z = z;
    }
    return EJ_OK;
}

int ej_plan(ej_ctx *ctx, const ej_strings *S, const ej_params *p, ej_plan_info *info, void *stream) {
    if (!ctx || !info) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/info");
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    info->n = pl.st.n;
    info->max_len = pl.max_len;
    info->total_bytes = pl.st.total;
    info->out_len = pl.out_len;
    info->L = pl.L;
    info->planes = pl.planes;
    info->blocks32 = (uint32_t)pl.nb32;
    info->embedding_bytes = emb_bytes(pl, p->r);
    info->walk_end_count = (uint64_t)p->r * pl.st.n;
    info->key_count = (uint64_t)p->r * p->m * pl.st.n;
    return EJ_OK;
}

int ej_embed(ej_ctx *ctx, const ej_strings *S, const ej_params *p, void *emb, int32_t *walk_end, void *stream) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    if (pl.st.n == 0) return EJ_OK;
    if (!emb || !walk_end) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL emb/walk_end");
    uint32_t *table = nullptr, *pos = nullptr;
    CKS(make_tables(ctx, p, pl, &table, &pos, s));
    const size_t eb = emb_bytes(pl, p->r), wb = (size_t)p->r * pl.st.n * sizeof(int32_t);
    void *d_emb = nullptr, *d_we = nullptr;
    bool h_emb = false, h_we = false;
    CKS(out_target(ctx, B_EMB, emb, eb, &d_emb, &h_emb));
    CKS(out_target(ctx, B_WALK, walk_end, wb, &d_we, &h_we));
    CK(launch_embed(pl.packed, pl.pofs, pl.lens, pl.st.n, p->r, table, pl.B, pl.out_len, pl.planes,
                    (uint32_t *)d_emb, (int32_t *)d_we, s));
    if (h_emb) CK(cudaMemcpyAsync(emb, d_emb, eb, cudaMemcpyDeviceToHost, s));
    if (h_we) CK(cudaMemcpyAsync(walk_end, d_we, wb, cudaMemcpyDeviceToHost, s));
    if (h_emb || h_we) CK(cudaStreamSynchronize(s));
    return EJ_OK;
}

int ej_sign(ej_ctx *ctx, const ej_strings *S, const ej_params *p, const void *emb, const int32_t *walk_end,
            uint64_t *keys, void *stream) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    if (pl.st.n == 0) return EJ_OK;
    if (!emb || !walk_end || !keys) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL emb/walk_end/keys");
    uint32_t *table = nullptr, *pos = nullptr;
    CKS(make_tables(ctx, p, pl, &table, &pos, s));
    const size_t eb = emb_bytes(pl, p->r), wb = (size_t)p->r * pl.st.n * sizeof(int32_t);
    const void *d_emb = nullptr, *d_we = nullptr;
    CKS(stage_in(ctx, B_EMB, emb, eb, &d_emb, s));
    CKS(stage_in(ctx, B_WALK, walk_end, wb, &d_we, s));
    const size_t kb = (size_t)p->r * p->m * pl.st.n * sizeof(uint64_t);
    void *d_keys = nullptr;
    bool h_keys = false;
    CKS(out_target(ctx, B_KEYS, keys, kb, &d_keys, &h_keys));
    CK(launch_sign((const uint32_t *)d_emb, (const int32_t *)d_we, pl.st.n, p->r, p->m, p->z, pl.out_len,
                   pl.planes, p->alphabet_size, pos, (uint64_t *)d_keys, s));
    if (ctx->key_P)
        CK(launch_keys_modp((uint64_t *)d_keys, pl.st.n, p->r, p->m, p->z, p->alphabet_size, p->seed, ctx->key_P, s));
    if (h_keys) {
        CK(cudaMemcpyAsync(keys, d_keys, kb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return EJ_OK;
}

int ej_embed_sign(ej_ctx *ctx, const ej_strings *S, const ej_params *p, uint64_t *keys, void *stream) {
    if (!ctx) return EJ_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    if (pl.st.n == 0) return EJ_OK;
    if (!keys) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL keys");
    const size_t kb = (size_t)p->r * p->m * pl.st.n * sizeof(uint64_t);
    void *d_keys = nullptr;
    bool h_keys = false;
    CKS(out_target(ctx, B_KEYS, keys, kb, &d_keys, &h_keys));
    CKS(keys_dev(ctx, p, pl, (uint64_t *)d_keys, s));
    if (h_keys) {
        CK(cudaMemcpyAsync(keys, d_keys, kb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return EJ_OK;
}

int ej_lsh_candidates(ej_ctx *ctx, const ej_strings *S, const ej_params *p, const uint64_t *keys,
                      uint64_t *pairs, int64_t capacity, int64_t *n_pairs, int64_t *stats_max_bucket,
                      void *stream) {
    if (!ctx || !n_pairs) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/n_pairs");
    *n_pairs = 0;
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    if (pl.st.n < 2) return EJ_OK;
    if (!keys) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL keys");
    const void *d_keys = nullptr;
    CKS(stage_in(ctx, B_KEYS, keys, (size_t)p->r * p->m * pl.st.n * sizeof(uint64_t), &d_keys, s));
    uint64_t *cand = nullptr;
    int64_t nc = 0, raw = 0, mb = 0;
    CKS(candidates_dev(ctx, pl, p, (const uint64_t *)d_keys, &cand, &nc, &raw, &mb, s));
    *n_pairs = nc;
    if (stats_max_bucket) *stats_max_bucket = mb;
    if (nc > capacity) return fail(ctx, EJ_ERR_CAPACITY, "needs %lld pairs, capacity %lld", (long long)nc, (long long)capacity);
    if (nc == 0) return EJ_OK;
    if (!pairs) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL pairs");
    CK(cudaMemcpyAsync(pairs, cand, (size_t)nc * sizeof(uint64_t), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return EJ_OK;
}

int ej_verify(ej_ctx *ctx, const ej_strings *S, const ej_params *p, const uint64_t *pairs, int64_t n_pairs,
              uint64_t *out, int64_t *n_out, void *stream) {
    if (!ctx || !n_out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/n_out");
    *n_out = 0;
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    if (n_pairs < 0) return fail(ctx, EJ_ERR_INVALID_ARG, "n_pairs < 0");
    Plan pl;
    CKS(make_plan(ctx, S, p, false, &pl, s));
    if (n_pairs == 0) return EJ_OK;
    if (!pairs || !out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL pairs/out");
    const void *d_pairs = nullptr;
    CKS(stage_in(ctx, B_PAIRS_IN, pairs, (size_t)n_pairs * sizeof(uint64_t), &d_pairs, s));
    void *d_out = nullptr;
    bool h_out = false;
    CKS(out_target(ctx, B_OUT_STAGE, out, (size_t)n_pairs * sizeof(uint64_t), &d_out, &h_out));
    int64_t cnt = 0;
    CKS(verify_dev(ctx, pl, p, (const uint64_t *)d_pairs, n_pairs, (uint64_t *)d_out, n_pairs, &cnt, s));
    *n_out = cnt;
    if (h_out && cnt) {
        CK(cudaMemcpyAsync(out, d_out, (size_t)cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return EJ_OK;
}

int ej_join(ej_ctx *ctx, const ej_strings *S, const ej_params *p, uint64_t *out, int64_t capacity,
            int64_t *n_out, ej_join_stats *stats, void *stream) {
    if (!ctx || !n_out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/n_out");
    *n_out = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    const int64_t launches0 = launches_so_far();
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], s));
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    if (pl.st.n < 2) return EJ_OK;
    uint64_t *keys = nullptr;
    CKS(ensure_t(ctx, B_KEYS, (size_t)p->r * p->m * pl.st.n, &keys));
    // autotuner: this call runs with its (length class, K) entry, tuned now if missing
    const ej_schedule sc0 = ctx->sched;
    const int vG0 = ctx->vG, vV0 = ctx->vV, tpb0 = ctx->walk_tpb;
    struct Restore {
        ej_ctx *c; ej_schedule sc; int g, v, t; bool on;
        ~Restore() { if (on) { c->sched = sc; c->vG = g; c->vV = v; c->walk_tpb = t; } }
    } restore{ctx, sc0, vG0, vV0, tpb0, ctx->autotune && !ctx->pi.size() && !ctx->posinj.size()};
    if (restore.on) {
        const uint64_t key = tune_key(pl, p);
        auto it = ctx->tune_table.find(key);
        if (it == ctx->tune_table.end()) {
            ej_tune_entry e;
            CKS(tune_join(ctx, pl, p, keys, s, &e));
            it = ctx->tune_table.emplace(key, e).first;
        }
        apply_tune(ctx, it->second);
        if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], s));
    }
    CKS(keys_dev(ctx, p, pl, keys, s));
    if (!out && capacity > 0) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL out");
    ej_join_stats st_local;
    memset(&st_local, 0, sizeof st_local);
    int64_t cnt = 0;
    const int status = join_back(ctx, pl, p, keys, out, capacity, &cnt, &st_local, s);
    *n_out = cnt;
    if (status != EJ_OK) {
        if (stats) *stats = st_local;
        return status;
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[5], s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        *stats = st_local;
        stats->kernel_launches = launches_so_far() - launches0;
        if (ctx->timing) {
            cudaEventElapsedTime(&stats->ms_prepare, ctx->ev[0], ctx->ev[1]);
            cudaEventElapsedTime(&stats->ms_embed_sign, ctx->ev[1], ctx->ev[2]);
            cudaEventElapsedTime(&stats->ms_candidates, ctx->ev[2], ctx->ev[3]);
            cudaEventElapsedTime(&stats->ms_verify, ctx->ev[3], ctx->ev[4]);
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[5]);
            cudaEventElapsedTime(&stats->ms_pack, ctx->ev[6], ctx->ev[7]);
            cudaEventElapsedTime(&stats->ms_buckets, ctx->ev[2], ctx->ev[8]);
            cudaEventElapsedTime(&stats->ms_dedup, ctx->ev[8], ctx->ev[3]);
        }
    }
    return EJ_OK;
}


// EmbedJoin+ (Section 5, Alg. 4 and 5). The suffixes become the strings of a
// device set of their own (record q = i*S + k), signed by the ordinary fused
// walk with the whole strings' out_len and L; the hashed buckets emit every
// pair of records sharing a bucket once per table, filtered by the whole
// strings' lengths; after a sort of those record pairs (Alg. 5's matches
// (x, y, k_x, k_y)), runs of at least T of them between different strings give
// the candidates, which are verified on the whole strings.
int ej_join_plus(ej_ctx *ctx, const ej_strings *S, const ej_params *p, int32_t delta, int32_t T, uint64_t *out,
                 int64_t capacity, int64_t *n_out, ej_join_stats *stats, void *stream) {
    if (!ctx || !n_out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/n_out");
    *n_out = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    if (delta <= 0 || T < 1) return fail(ctx, EJ_ERR_INVALID_ARG, "delta must be > 0 and T >= 1");
    const int64_t launches0 = launches_so_far();
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], s));
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    const int64_t n = pl.st.n;
    if (n < 2) return EJ_OK;
    if (!out && capacity > 0) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL out");
    const int32_t nsub = p->K > 0 ? (int32_t)(((int64_t)p->K + delta - 1) / delta) : 1;
    const int64_t nq = n * (int64_t)nsub, TT = (int64_t)p->r * p->m;
    if (nq >= (1ll << 31) || nq * TT >= 0xFFFFFFFFll)
        return fail(ctx, EJ_ERR_UNSUPPORTED, "strings x substrings x tables beyond the 32-bit record ids");
    // the suffix set
    uint32_t *sub_len = nullptr;
    int32_t *whole = nullptr;
    uint64_t *sub_off = nullptr;
    void *scan = nullptr;
    CKS(ensure_t(ctx, B_PLUS_SUBLEN, (size_t)nq + 1, &sub_len));
    CKS(ensure_t(ctx, B_PLUS_WHOLE, (size_t)nq, &whole));
    CKS(ensure_t(ctx, B_PLUS_SUBOFF, (size_t)nq + 1, &sub_off));
    CKS(ensure(ctx, B_PLUS_SCAN, scan_temp_bytes(nq + 1), &scan));
    CK(cudaMemsetAsync(sub_len + nq, 0, sizeof(uint32_t), s));
    CK(launch_suffix_lengths(pl.lens, n, nsub, delta, sub_len, whole, s));
    CK(exclusive_scan_u32(sub_len, sub_off, nq + 1, nullptr, scan, s));
    CK(cudaMemcpyAsync(ctx->h_cnt, sub_off + nq, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t sub_total = ctx->h_cnt[0];
    uint8_t *sub_bytes = nullptr;
    CKS(ensure_t(ctx, B_PLUS_BYTES, (size_t)(sub_total > 0 ? sub_total : 1), &sub_bytes));
    CK(launch_suffix_copy(pl.st.bytes, pl.st.offsets, n, nsub, delta, sub_off, sub_bytes, s));
    if (!ctx->plus_sub && ej_create(&ctx->plus_sub, ctx->device) != EJ_OK)
        return fail(ctx, EJ_ERR_OOM, "suffix-set context");
    ej_ctx *sub = ctx->plus_sub;
    sub->sched = ctx->sched;
    ej_strings sset{sub_bytes, (const int64_t *)sub_off, nq};
    ej_params sp = *p;
    sp.out_len = pl.out_len;   // the whole strings' embedding length and sampling range
    sp.L = pl.L;
    Plan spl;
    auto sub_fail = [&](int st) { return fail(ctx, st, "suffix set: %s", sub->err.c_str()); };
    int st = make_plan(sub, &sset, &sp, true, &spl, s);
    if (st != EJ_OK) return sub_fail(st);
    uint64_t *keys = nullptr;
    if ((st = ensure_t(sub, B_KEYS, (size_t)(TT * nq), &keys)) != EJ_OK) return sub_fail(st);
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], s));
    if ((st = keys_dev(sub, &sp, spl, keys, s)) != EJ_OK) return sub_fail(st);
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[2], s));
    // buckets of the suffix records, matches filtered by the whole strings' lengths
    const uint64_t H = bucket_slots_per_table(nq);
    uint64_t *bkeys = nullptr;
    uint32_t *bheads = nullptr, *bnext = nullptr, *derr = nullptr;
    unsigned long long *cnt = nullptr;
    CKS(ensure_t(sub, B_BKEYS, (size_t)(H * TT), &bkeys));
    CKS(ensure_t(sub, B_BHEADS, (size_t)(H * TT), &bheads));
    CKS(ensure_t(sub, B_BNEXT, (size_t)(nq * TT), &bnext));
    CKS(ensure_t(sub, B_DERR, 8, &derr));
    CKS(ensure_t(sub, B_JCOUNT, 8, &cnt));
    CK(cudaMemsetAsync(derr, 0, 4, s));
    CK(cudaMemsetAsync(bkeys, 0xFF, H * TT * sizeof(uint64_t), s));
    CK(cudaMemsetAsync(bheads, 0xFF, H * TT * sizeof(uint32_t), s));
    CK(launch_bucket_insert(keys, nq, TT, H, bkeys, bheads, bnext, derr, s));
    uint64_t cap = (uint64_t)(nq * 4 > 65536 ? nq * 4 : 65536);
    uint64_t *raw = nullptr, *raw2 = nullptr;
    int64_t nraw = 0;
    for (int attempt = 0;; attempt++) {
        CKS(ensure_t(sub, B_RAW, (size_t)cap, &raw));
        CK(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
        CK(launch_bucket_emit(whole, nq, TT, p->K, bnext, raw, cap, cnt, s));
        CK(cudaMemcpyAsync(ctx->h_cnt, cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        nraw = ctx->h_cnt[0];
        if ((uint64_t)nraw <= cap) break;
        if (attempt > 2) return fail(ctx, EJ_ERR_CUDA, "match count changed between attempts");
        cap = (uint64_t)nraw + (uint64_t)nraw / 8 + 1024;
    }
    const int64_t max_bucket = ctx->h_cnt[1];
    // count the matches of every record pair (sorted), keep runs of >= T
    const int nb = bits_for((uint64_t)(nq > 1 ? nq - 1 : 1));
    int shifts[16];
    int np = 0;
    for (int b = 0; b < nb; b += 8) shifts[np++] = b;
    for (int b = 0; b < nb; b += 8) shifts[np++] = 32 + b;
    int64_t ncp = 0;
    uint64_t *cp = nullptr, *cp2 = nullptr;
    const uint64_t *sorted = raw;
    bool alt = false;
    if (nraw > 0) {
        const size_t rs = radix_counts_len(nraw, 1);
        uint32_t *rsc = nullptr;
        uint64_t *rso = nullptr;
        void *stmp = nullptr;
        CKS(ensure_t(sub, B_RAW_ALT, (size_t)nraw, &raw2));
        CKS(ensure_t(sub, B_RS_COUNTS, rs, &rsc));
        CKS(ensure_t(sub, B_RS_OFFS, rs, &rso));
        CKS(ensure(sub, B_SCAN_TMP, scan_temp_bytes((int64_t)rs), &stmp));
        CK(radix_sort_segmented(raw, nullptr, raw2, nullptr, nraw, 1, shifts, np, RadixTemp{rsc, rso, stmp}, &alt, s));
        sorted = alt ? raw2 : raw;
        CKS(ensure_t(sub, B_CAND, (size_t)nraw, &cp));
        CK(launch_plus_runs(sorted, nraw, nsub, T, cp, (uint64_t)nraw, cnt + 2, cnt + 4, s));
        CK(cudaMemcpyAsync(ctx->h_cnt, cnt + 2, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ncp = ctx->h_cnt[0];
        nraw -= ctx->h_cnt[2];   // record pairs of one string's substrings are not matches
    }
    // candidate string pairs: sorted, unique
    int64_t ncand = 0;
    uint64_t *cand = nullptr;
    if (ncp > 0) {
        const int nbs = bits_for((uint64_t)(n - 1));
        np = 0;
        for (int b = 0; b < nbs; b += 8) shifts[np++] = b;
        for (int b = 0; b < nbs; b += 8) shifts[np++] = 32 + b;
        const size_t rs = radix_counts_len(ncp, 1);
        uint32_t *rsc = nullptr;
        uint64_t *rso = nullptr;
        void *stmp = nullptr;
        CKS(ensure_t(sub, B_APP, (size_t)ncp, &cp2));
        CKS(ensure_t(sub, B_RS_COUNTS, rs, &rsc));
        CKS(ensure_t(sub, B_RS_OFFS, rs, &rso));
        CKS(ensure(sub, B_SCAN_TMP, scan_temp_bytes((int64_t)rs), &stmp));
        CK(radix_sort_segmented(cp, nullptr, cp2, nullptr, ncp, 1, shifts, np, RadixTemp{rsc, rso, stmp}, &alt, s));
        const uint64_t *sp_ = alt ? cp2 : cp;
        uint8_t *fl = nullptr;
        uint64_t *fo = nullptr;
        void *stmp2 = nullptr;
        CKS(ensure_t(sub, B_FLAGS, (size_t)ncp, &fl));
        CKS(ensure_t(sub, B_FLAG_OFFS, (size_t)ncp, &fo));
        CKS(ensure(sub, B_SCAN_TMP2, scan_temp_bytes(ncp), &stmp2));
        CK(launch_unique_flags(sp_, ncp, fl, s));
        CK(exclusive_scan_u8(fl, fo, ncp, (uint64_t *)(cnt + 3), stmp2, s));
        CK(cudaMemcpyAsync(ctx->h_cnt, cnt + 3, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ncand = ctx->h_cnt[0];
        CKS(ensure_t(ctx, B_PLUS_CAND, (size_t)(ncand > 0 ? ncand : 1), &cand));
        CK(launch_compact_u64(sp_, fl, fo, ncp, cand, s));
    }
    // verification on the whole strings (Section 3.3)
    int64_t cntout = 0;
    uint64_t work[2] = {0, 0};
    CKS(verify_dev(ctx, pl, p, cand, ncand, nullptr, 0, &cntout, s, work));
    *n_out = cntout;
    if (stats) {
        stats->n_raw_pairs = nraw;
        stats->n_candidates = ncand;
        stats->n_out = cntout;
        stats->max_bucket = max_bucket;
        stats->band_cells = work[0];
        stats->verify_word_columns = work[1];
    }
    if (cntout > capacity)
        return fail(ctx, EJ_ERR_CAPACITY, "output needs %lld pairs, capacity %lld", (long long)cntout,
                    (long long)capacity);
    if (cntout > 0) {
        void *d_out = nullptr;
        bool h_out = false;
        CKS(out_target(ctx, B_OUT_STAGE, out, (size_t)cntout * sizeof(uint64_t), &d_out, &h_out));
        CK(launch_compact_u64(cand, (const uint8_t *)ctx->bufs[B_FLAGS].p, (const uint64_t *)ctx->bufs[B_FLAG_OFFS].p,
                              ncand, (uint64_t *)d_out, s));
        if (h_out) CK(cudaMemcpyAsync(out, d_out, (size_t)cntout * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[5], s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        stats->kernel_launches = launches_so_far() - launches0;
        if (ctx->timing) {
            cudaEventElapsedTime(&stats->ms_prepare, ctx->ev[0], ctx->ev[1]);
            cudaEventElapsedTime(&stats->ms_embed_sign, ctx->ev[1], ctx->ev[2]);
            cudaEventElapsedTime(&stats->ms_candidates, ctx->ev[2], ctx->ev[3]);
            cudaEventElapsedTime(&stats->ms_verify, ctx->ev[3], ctx->ev[4]);
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[0], ctx->ev[5]);
        }
    }
    return EJ_OK;
}


// EmbedJoin with grouping (Section 4.1): every length group runs as a join of
// its own (its strings gathered into a buffer of their own, on a private
// context with this context's schedule and key choice), the group-local output
// pairs are mapped back to the set's ids, and the union is sorted and made
// unique. The groups are chosen on the host from the strings' lengths.
int ej_join_grouped(ej_ctx *ctx, const ej_strings *S, const ej_params *p, uint64_t *out, int64_t capacity,
                    int64_t *n_out, ej_join_stats *stats, void *stream) {
    if (!ctx || !n_out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/n_out");
    *n_out = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    if (p && p->K < 1) return fail(ctx, EJ_ERR_INVALID_ARG, "grouping needs K >= 1");
    const int64_t launches0 = launches_so_far();
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    Plan pl;
    CKS(make_plan(ctx, S, p, true, &pl, s));
    const int64_t n = pl.st.n;
    if (n < 2) return EJ_OK;
    if (!out && capacity > 0) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL out");
    std::vector<int32_t> lens((size_t)n);
    CK(cudaMemcpyAsync(lens.data(), pl.lens, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t K = p->K, N = pl.max_len;
    int64_t G = ((N + K - 1) / K) * K / K - 1;
    if (G < 1) G = 1;
    if (!ctx->group_sub && ej_create(&ctx->group_sub, ctx->device) != EJ_OK)
        return fail(ctx, EJ_ERR_OOM, "group context");
    ej_ctx *sub = ctx->group_sub;
    sub->sched = ctx->sched;
    sub->key_P = ctx->key_P;
    sub->vG = ctx->vG;
    sub->vV = ctx->vV;
    sub->vWarps = ctx->vWarps;
    std::vector<int32_t> idx;
    std::vector<int64_t> goff;
    struct DevBuf {   // the union of the groups' outputs, freed on every return
        uint64_t *p = nullptr;
        ~DevBuf() { if (p) cudaFree(p); }
    } allbuf;
    uint64_t *&all = allbuf.p;
    int64_t nall = 0, cap_all = 0, cand_total = 0, raw_total = 0, maxb = 0;
    uint64_t cells = 0, wcols = 0;
    for (int64_t g = 1; g <= G; g++) {
        idx.clear();
        goff.assign(1, 0);
        for (int64_t i = 0; i < n; i++) {
            const int64_t len = lens[(size_t)i];
            if ((g == 1 && len == 0) || (len > (g - 1) * K && len <= (g + 1) * K)) {
                idx.push_back((int32_t)i);
                goff.push_back(goff.back() + len);
            }
        }
        const int64_t gn = (int64_t)idx.size();
        if (gn < 2) continue;
        int32_t *d_idx = nullptr;
        int64_t *d_goff = nullptr;
        uint8_t *d_gbytes = nullptr;
        CKS(ensure_t(ctx, B_GROUP_IDX, (size_t)gn, &d_idx));
        CKS(ensure_t(ctx, B_GROUP_OFF, (size_t)gn + 1, &d_goff));
        CKS(ensure_t(ctx, B_GROUP_BYTES, (size_t)(goff.back() > 0 ? goff.back() : 1), &d_gbytes));
        CK(cudaMemcpyAsync(d_idx, idx.data(), (size_t)gn * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_goff, goff.data(), (size_t)(gn + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        CK(launch_gather_strings(pl.st.bytes, pl.st.offsets, d_idx, gn, d_goff, d_gbytes, s));
        ej_strings gs{d_gbytes, d_goff, gn};
        ej_params gp = *p;
        gp.out_len = 0;   // the group's own 3N
        ej_join_stats gst;
        int64_t gcount = 0;
        uint64_t *gout = nullptr;
        int64_t gcap = 1 << 16;
        int st = EJ_OK;
        for (;;) {
            CKS(ensure_t(ctx, B_GROUP_OUT, (size_t)gcap, &gout));
            st = ej_join(sub, &gs, &gp, gout, gcap, &gcount, &gst, s);
            if (st != EJ_ERR_CAPACITY) break;
            gcap = gcount;
        }
        if (st != EJ_OK) return fail(ctx, st, "group %lld: %s", (long long)g, sub->err.c_str());
        cand_total += gst.n_candidates;
        raw_total += gst.n_raw_pairs;
        maxb = std::max<int64_t>(maxb, gst.max_bucket);
        cells += gst.band_cells;
        wcols += gst.verify_word_columns;
        if (gcount == 0) continue;
        if (nall + gcount > cap_all) {
            // grow the union buffer (keeping what it holds)
            const int64_t nc = 2 * (nall + gcount) + 1024;
            uint64_t *nb = nullptr;
            if (cudaMalloc(&nb, (size_t)nc * sizeof(uint64_t)) != cudaSuccess)
                return fail(ctx, EJ_ERR_OOM, "grouped output");
            if (nall) CK(cudaMemcpyAsync(nb, all, (size_t)nall * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            CK(cudaStreamSynchronize(s));
            if (all) cudaFree(all);
            all = nb;
            cap_all = nc;
        }
        CK(launch_remap_pairs(gout, gcount, d_idx, all + nall, s));
        nall += gcount;
    }
    // the union: sorted, unique
    int64_t cnt = 0;
    int st = EJ_OK;
    if (nall > 0) {
        uint64_t *alt = nullptr;
        CKS(ensure_t(ctx, B_RAW_ALT, (size_t)nall, &alt));
        const int nb = bits_for((uint64_t)(n - 1));
        int shifts[16], np = 0;
        for (int b = 0; b < nb; b += 8) shifts[np++] = b;
        for (int b = 0; b < nb; b += 8) shifts[np++] = 32 + b;
        const size_t rs = radix_counts_len(nall, 1);
        uint32_t *rsc = nullptr;
        uint64_t *rso = nullptr, *fo = nullptr, *dcnt = nullptr;
        void *stmp = nullptr, *stmp2 = nullptr;
        uint8_t *fl = nullptr;
        CKS(ensure_t(ctx, B_RS_COUNTS, rs, &rsc));
        CKS(ensure_t(ctx, B_RS_OFFS, rs, &rso));
        CKS(ensure(ctx, B_SCAN_TMP, scan_temp_bytes((int64_t)rs), &stmp));
        bool alt_out = false;
        CK(radix_sort_segmented(all, nullptr, alt, nullptr, nall, 1, shifts, np, RadixTemp{rsc, rso, stmp}, &alt_out, s));
        const uint64_t *sorted = alt_out ? alt : all;
        CKS(ensure_t(ctx, B_FLAGS, (size_t)nall, &fl));
        CKS(ensure_t(ctx, B_FLAG_OFFS, (size_t)nall, &fo));
        CKS(ensure(ctx, B_SCAN_TMP2, scan_temp_bytes(nall), &stmp2));
        CKS(ensure_t(ctx, B_COUNTERS, 8, &dcnt));
        CK(launch_unique_flags(sorted, nall, fl, s));
        CK(exclusive_scan_u8(fl, fo, nall, dcnt, stmp2, s));
        CK(cudaMemcpyAsync(ctx->h_cnt, dcnt, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        cnt = ctx->h_cnt[0];
        if (cnt > capacity) {
            st = fail(ctx, EJ_ERR_CAPACITY, "output needs %lld pairs, capacity %lld", (long long)cnt,
                      (long long)capacity);
        } else {
            void *d_out = nullptr;
            bool h_out = false;
            st = out_target(ctx, B_OUT_STAGE, out, (size_t)cnt * sizeof(uint64_t), &d_out, &h_out);
            if (st == EJ_OK) {
                CK(launch_compact_u64(sorted, fl, fo, nall, (uint64_t *)d_out, s));
                if (h_out) CK(cudaMemcpyAsync(out, d_out, (size_t)cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
            }
        }
    }
    *n_out = cnt;
    if (stats) {
        stats->n_raw_pairs = raw_total;
        stats->n_candidates = cand_total;
        stats->n_out = cnt;
        stats->max_bucket = maxb;
        stats->band_cells = cells;
        stats->verify_word_columns = wcols;
        stats->kernel_launches = launches_so_far() - launches0;
    }
    return st;
}


int ej_batch_create(ej_ctx *ctx, const ej_strings *S, const ej_params *params, int32_t n_params, int32_t flags,
                    ej_batch **out, void *stream) {
    if (!ctx || !out) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL ctx/out");
    *out = nullptr;
    if (!S || !params || n_params < 1 || n_params > 64)
        return fail(ctx, EJ_ERR_INVALID_ARG, "a batch needs strings and 1..64 parameter sets");
    if ((flags & ~(EJ_BATCH_AUTOTUNE | EJ_BATCH_EAGER)) != 0)
        return fail(ctx, EJ_ERR_INVALID_ARG, "unknown batch flags %d", flags);
    if (S->n < 2 || !is_device_ptr(S->bytes) || !is_device_ptr(S->offsets))
        return fail(ctx, EJ_ERR_INVALID_ARG, "a batch needs n >= 2 strings in device memory");
    if (ctx->pi.size() || ctx->posinj.size())
        return fail(ctx, EJ_ERR_INVALID_ARG, "injected test tables are not supported in a batch");
    if (ctx->key_P)
        return fail(ctx, EJ_ERR_UNSUPPORTED, "hashed bucket keys (ej_set_key_hash) are not supported in a batch");
    for (int32_t i = 1; i < n_params; i++)
        if (params[i].alphabet_size != params[0].alphabet_size ||
            memcmp(params[i].alphabet, params[0].alphabet, params[0].alphabet_size) != 0)
            return fail(ctx, EJ_ERR_INVALID_ARG, "all parameter sets of a batch share one alphabet");
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    ej_batch *b = new (std::nothrow) ej_batch();
    if (!b) return EJ_ERR_OOM;
    b->ctx = ctx;
    const bool timing_was = ctx->timing;
    ctx->timing = false;
    auto bail = [&](int st) { ctx->timing = timing_was; batch_free(b); return st; };
    int st = make_plan(ctx, S, &params[0], true, &b->pl, s);
    if (st != EJ_OK) return bail(st);
    b->joins.resize((size_t)n_params);
    for (int32_t i = 0; i < n_params; i++) {
        BatchJoin &j = b->joins[(size_t)i];
        j.p = params[i];
        j.alphabet.assign(params[i].alphabet, params[i].alphabet + params[i].alphabet_size);
        j.p.alphabet = j.alphabet.data();
        if ((st = check_params(ctx, &j.p, true)) != EJ_OK) return bail(st);
        j.pl = b->pl;
        if ((st = derive_lsh(ctx, &j.p, &j.pl)) != EJ_OK) return bail(st);
        if ((st = ej_create(&j.sub, ctx->device)) != EJ_OK) return bail(st);
        j.sub->sched = ctx->sched;
        j.sub->vG = ctx->vG;
        j.sub->vV = ctx->vV;
        j.sub->vWarps = ctx->vWarps;
        j.sub->loop_bound = ctx->loop_bound;
        if (cudaStreamCreateWithFlags(&j.side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&j.verified, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&j.keyed, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(ctx, EJ_ERR_CUDA, "stream/event creation failed"));
        if ((st = upload_alphabet(j.sub, &j.p, s)) != EJ_OK) return bail(st);
    }
    // joins whose signatures another join's walks already cover take their keys
    // from it instead of walking the strings again
    batch_sources(b->joins);
    for (auto &j : b->joins)
        if (!j.alias && (st = ensure_t(j.sub, B_KEYS, (size_t)j.p.r * j.p.m * b->pl.st.n, &j.keys)) != EJ_OK)
            return bail(st);
    for (auto &j : b->joins)
        if (j.alias) j.keys = b->joins[(size_t)j.src].keys;
    // eager pass: keys (sources first), then every join's back half, which sizes
    // every buffer (the raw-pair capacity gets a margin)
    for (auto &j : b->joins)
        if (j.src < 0 && (st = batch_join_keys(b->joins, j, s)) != EJ_OK) return bail(st);
    for (auto &j : b->joins)
        if (j.src >= 0 && (st = batch_join_keys(b->joins, j, s)) != EJ_OK) return bail(st);
    for (auto &j : b->joins) {
        if ((st = back_buckets(j.sub, j.pl, &j.p, j.keys, &j.bs, s)) != EJ_OK) return bail(st);
        uint64_t cap = raw_cap_start(j.sub, b->pl.st.n);
        unsigned long long hc[8];
        for (int attempt = 0;; attempt++) {
            if ((st = back_attempt(j.sub, j.pl, &j.p, j.bs, cap, s)) != EJ_OK) return bail(st);
            if ((st = back_read(j.sub, hc, s)) != EJ_OK) return bail(st);
            if (j.bs.hashed && ctx->sched.buckets == 0 && hc[1] > (unsigned long long)SORTED_BUCKET_MIN) {
                // buckets of thousands of records: a list walks all b(b-1)/2 pairs
                // of a bucket, the sorted tables only the pairs within the length
                // window (measured 2x faster on the protein-like shape)
                j.sub->sched.buckets = 2;
                if ((st = back_buckets(j.sub, j.pl, &j.p, j.keys, &j.bs, s)) != EJ_OK) return bail(st);
                attempt = -1;
                continue;
            }
            if (j.bs.table_smem && hc[1] > (unsigned long long)SMEM_BUCKET_MAX) {
                // a table in one block's shared memory walks a bucket of b records
                // in b(b-1)/2 steps on one SM: huge buckets go to global memory,
                // where every SM takes part
                j.sub->no_smem_buckets = true;
                if ((st = back_buckets(j.sub, j.pl, &j.p, j.keys, &j.bs, s)) != EJ_OK) return bail(st);
                attempt = -1;
                continue;
            }
            if (hc[0] <= cap) break;
            if (attempt > 2) return bail(fail(ctx, EJ_ERR_CUDA, "raw pair count changed between attempts"));
            cap = hc[0] + hc[0] / 4 + 1024;
        }
        j.ncand = hc[2];
        j.cap = cap + cap / 8 + 1024;
        if ((st = back_attempt(j.sub, j.pl, &j.p, j.bs, j.cap, s)) != EJ_OK) return bail(st);
        if (flags & EJ_BATCH_AUTOTUNE) {
            float ms = 0.f;
            if ((st = batch_autotune(ctx, j, s, &ms)) != EJ_OK) return bail(st);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ctx, EJ_ERR_CUDA, "eager pass failed"));
    }
    if ((st = batch_plan_merge(b)) != EJ_OK) return bail(st);
    if ((st = batch_plan_buckets(b)) != EJ_OK) return bail(st);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->v0) != cudaSuccess || cudaEventCreate(&b->v1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(ctx, EJ_ERR_CUDA, "event creation failed"));
    if (cudaMallocHost(&b->h_stat, (16 * b->joins.size() + 2) * sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(ctx, EJ_ERR_OOM, "pinned result staging"));
    memset(b->h_stat, 0, (16 * b->joins.size() + 2) * sizeof(unsigned long long));
    if (!b->merged.empty()) {
        std::vector<VerifySeg> segs_h(b->merged.size());
        for (auto &j : b->joins)
            if (j.seg >= 0 && (st = back_segment(j.sub, &j.p, j.cap, &segs_h[(size_t)j.seg])) != EJ_OK) return bail(st);
        if (cudaMemcpy(b->segs_dev, segs_h.data(), segs_h.size() * sizeof(VerifySeg), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return bail(fail(ctx, EJ_ERR_CUDA, "merged verifier table upload failed"));
    }
    if (flags & EJ_BATCH_EAGER) {
        // no graph: every run issues the same work; one run here checks it and
        // counts its kernels
        b->eager = true;
        const int64_t l0 = launches_so_far();
        if ((st = batch_issue(b, s)) != EJ_OK) return bail(st);
        b->kernel_nodes = launches_so_far() - l0;
        if (cudaEventRecord(b->done, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return bail(fail(ctx, EJ_ERR_CUDA, "eager batch run failed"));
        b->ran = true;
        ctx->timing = timing_was;
        *out = b;
        return EJ_OK;
    }
    // capture: plan (validate, pack) on the caller's stream, then every join on
    // its own stream, joined back at the end
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail(fail(ctx, EJ_ERR_CUDA, "stream capture could not start (the stream must not be the legacy default stream)"));
    const int cst = batch_issue(b, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (cst != EJ_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return bail(cst != EJ_OK ? cst : fail(ctx, EJ_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ce)));
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess)
        return bail(fail(ctx, EJ_ERR_CUDA, "graph instantiation failed"));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernel_nodes++;
    }
    ctx->timing = timing_was;
    *out = b;
    return EJ_OK;
}

int ej_batch_run(ej_batch *b, void *stream) {
    if (!b || (!b->exec && !b->eager)) return EJ_ERR_INVALID_ARG;
    cudaSetDevice(b->ctx->device);
    if (b->eager) {
        const int st = batch_issue(b, as_stream(stream));
        if (st != EJ_OK) return st;
    } else {
        CKB(b, cudaGraphLaunch(b->exec, as_stream(stream)));
    }
    CKB(b, cudaEventRecord(b->done, as_stream(stream)));
    b->ran = true;
    return EJ_OK;
}

int ej_batch_verify_ms(ej_batch *b, float *ms) {
    if (!b || !ms) return EJ_ERR_INVALID_ARG;
    *ms = 0.f;
    if (b->merged.empty() || !b->ran || !b->eager)
        return fail(b->ctx, EJ_ERR_INVALID_ARG, "no merged verifier launch of an eager batch has run");
    cudaSetDevice(b->ctx->device);
    CKB(b, cudaEventSynchronize(b->v1));
    CKB(b, cudaEventElapsedTime(ms, b->v0, b->v1));
    return EJ_OK;
}

int ej_batch_result(ej_batch *b, int32_t i, uint64_t *out, int64_t capacity, int64_t *n_out, ej_join_stats *stats,
                    void *stream) {
    if (!b || !n_out) return EJ_ERR_INVALID_ARG;
    ej_ctx *ctx = b->ctx;
    *n_out = 0;
    if (stats) memset(stats, 0, sizeof *stats);
    if (i < 0 || (size_t)i >= b->joins.size()) return fail(ctx, EJ_ERR_INVALID_ARG, "join index %d out of range", i);
    if (!b->ran) return fail(ctx, EJ_ERR_INVALID_ARG, "ej_batch_run has not been called");
    if (!out && capacity > 0) return fail(ctx, EJ_ERR_INVALID_ARG, "NULL out");
    cudaSetDevice(ctx->device);
    cudaStream_t s = as_stream(stream);
    const int64_t launches0 = launches_so_far();
    // the run staged every counter in pinned memory: one wait for the run
    CKB(b, cudaEventSynchronize(b->done));
    const unsigned long long *plan = b->h_stat + 16 * b->joins.size();
    const uint32_t e = (uint32_t)(plan[0] & 0xffffffffu);
    if (e & DERR_OFFSETS)
        return fail(ctx, EJ_ERR_INVALID_ARG, "offsets invalid or grown beyond the batch's plan (%lld bytes)", (long long)b->pl.st.total);
    if (e & DERR_SYMBOL) return fail(ctx, EJ_ERR_INVALID_ARG, "a string byte is not in the alphabet");
    const int64_t max_len = (int64_t)plan[1];
    BatchJoin &j = b->joins[(size_t)i];
    if (max_len > b->pl.max_len || (!j.p.out_len && !j.p.L && max_len != b->pl.max_len))
        return fail(ctx, EJ_ERR_INVALID_ARG, "the longest string changed (%lld, planned %lld): re-create the batch",
                    (long long)max_len, (long long)b->pl.max_len);
    unsigned long long hc[8];
    memcpy(hc, b->h_stat + 16 * (size_t)i, 6 * sizeof(unsigned long long));
    hc[6] = b->h_stat[16 * (size_t)i + 8] & 0xffffffffull;
    hc[7] = 0;
    if ((uint32_t)hc[6] & DERR_PAIR) return fail(ctx, EJ_ERR_INVALID_ARG, "internal: pair index out of range");
    if ((uint32_t)hc[6] & DERR_TIMEOUT)
        return fail(ctx, EJ_ERR_TIMEOUT, "the persistent verifier gave up after its bound of loop passes per warp");
    if ((uint32_t)hc[6] & DERR_GUARD) return fail(ctx, EJ_ERR_CUDA, "internal: a work bound was exceeded");
    if (hc[0] > j.cap)
        return fail(ctx, EJ_ERR_CAPACITY, "raw pairs (%llu) exceed the batch's capacity (%llu): re-create the batch",
                    hc[0], (unsigned long long)j.cap);
    int64_t cnt = 0;
    int st = EJ_OK;
    if ((int64_t)hc[3] <= small_sort_max()) {
        // sorted by the run: copy only
        cnt = (int64_t)hc[3];
        if (stats) {
            stats->n_raw_pairs = (int64_t)hc[0];
            stats->max_bucket = (int64_t)hc[1];
            stats->n_candidates = (int64_t)hc[2];
            stats->n_out = cnt;
            stats->band_cells = hc[4];
            stats->verify_word_columns = hc[5];
        }
        if (cnt > capacity) {
            *n_out = cnt;
            return fail(ctx, EJ_ERR_CAPACITY, "output needs %lld pairs, capacity %lld", (long long)cnt, (long long)capacity);
        }
        if (cnt) CKB(b, cudaMemcpyAsync(out, j.sub->bufs[B_APP].p, (size_t)cnt * sizeof(uint64_t), cudaMemcpyDefault, s));
    } else {
        st = back_finish(j.sub, j.pl, &j.p, hc, out, capacity, &cnt, stats, s);
    }
    *n_out = cnt;
    if (st != EJ_OK) return fail(ctx, st, "%s", ej_last_error(j.sub));
    // a host `out` is complete on return; a device one is ordered on `stream`
    if (cnt && !is_device_ptr(out)) CKB(b, cudaStreamSynchronize(s));
    if (stats) stats->kernel_launches = launches_so_far() - launches0;   // a sort of a large output
    return EJ_OK;
}

int64_t ej_batch_kernel_count(const ej_batch *b) { return b ? b->kernel_nodes : 0; }

void ej_batch_destroy(ej_batch *b) { batch_free(b); }

}  // extern "C"
