/*
 * CPU ORACLE for the EmbedJoin hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C that restates what the paper computes so that
 * the CUDA path can be checked against it. Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load this library; the product path never
 * does. It shares no code, header or table with the CUDA library.
 *
 * Paper: Zhang & Zhang, "EmbedJoin: Efficient Edit Similarity Joins via
 * Embeddings" (arXiv 1702.00093).
 *
 * Naming: r = CGK embeddings per string, m = LSH functions per embedding,
 * z = sampled positions per function. (The paper's Table 1 calls the number of
 * functions z and the signature length m; the two letters are swapped here.)
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - Random bits (Alg. 1 draws "a random string R"): counter-based,
 *      base  = splitmix64(seed)
 *      pi_j^l(sigma) = top bit of splitmix64(base ^ (1<<56 | l<<48 | j<<8 | sigma))
 *    with sigma the RAW BYTE of the symbol and j the 0-based step.
 *    splitmix64 is the published Steele-Lea-Flood (2014) output function.
 *  - Sampled positions of bit-sampling LSH (Thm. 1), drawn with replacement:
 *      P[l][f][q] = mulhi64(splitmix64(base ^ (2<<56 | l<<48 | f<<32 | q)), L)
 *  - Bucket key (Section 4 uses a two-level hash <u,v> mod P): the injective
 *    mixed-radix number  sum_q c_q * (|S|+1)^q  where c_q is the symbol's index
 *    in the declared alphabet, or |S| for the padding symbol (bottom). Buckets
 *    are therefore exact signature equality.
 *  - Truncation (Section 4.1): positions are drawn from [0, L); the embedding
 *    only needs a prefix of length out_len >= L (the walk is causal).
 *  - Verification (Section 3.3, Ukkonen): a full banded DP over diagonals
 *    -K..K, cells outside the band count as K+1; a pair passes iff the result
 *    is <= K (K inclusive, Section 1).
 *  - Output: pairs (i, j), i < j, in input order, packed as (i<<32)|j, sorted
 *    ascending and unique.
 */
#define _POSIX_C_SOURCE 199309L
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2
#define OR_ERR_CAPACITY 3

/* ------------------------------------------------------------------------ */
/* Random bits (reading of Alg. 1's random string R and Thm. 1's sampling)   */
/* ------------------------------------------------------------------------ */

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014). */
uint64_t or_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* pi_j(sigma) of the l-th embedding: Alg. 1, step 1 (one bit per step and symbol). */
int or_walk_bit(uint64_t seed, uint32_t l, uint64_t j, uint8_t sigma_byte) {
    uint64_t base = or_splitmix64(seed);
    uint64_t ctr = (1ull << 56) | ((uint64_t)l << 48) | (j << 8) | (uint64_t)sigma_byte;
    return (int)(or_splitmix64(base ^ ctr) >> 63);
}

/* q-th sampled coordinate of the f-th bit-sampling function of embedding l
 * (Thm. 1: h_i(b) = b_i with i uniform), uniform in [0, L). */
uint32_t or_position(uint64_t seed, uint32_t l, uint32_t f, uint32_t q, uint32_t L) {
    uint64_t base = or_splitmix64(seed);
    uint64_t ctr = (2ull << 56) | ((uint64_t)l << 48) | ((uint64_t)f << 32) | (uint64_t)q;
    uint64_t h = or_splitmix64(base ^ ctr);
    return (uint32_t)(((unsigned __int128)h * (unsigned __int128)L) >> 64);
}

/* ------------------------------------------------------------------------ */
/* CGK embedding, Algorithm 1                                                */
/* ------------------------------------------------------------------------ */

/*
 * Embed x (len bytes) with the l-th random string.
 *   code_of[256]: index of each raw byte in the alphabet (255 = not in it).
 *   bottom: the code written for the padding symbol (= alphabet size).
 *   pi_inject: optional table pi[j*alpha + c] in {0,1} for j < inject_steps
 *              (code-indexed), used in place of the random bits.
 * Writes out[0..out_len) and returns walk_end = first step whose output is
 * bottom (out_len if the walk never leaves x).
 */
int64_t or_cgk_embed(const uint8_t *x, int64_t len, const uint8_t *code_of, uint32_t alpha,
                     uint64_t seed, uint32_t l, int64_t out_len, const uint8_t *pi_inject,
                     int64_t inject_steps, uint8_t *out) {
    int64_t i = 0;              /* Alg. 1 counts from 1; 0-based here */
    int64_t walk_end = out_len;
    for (int64_t j = 0; j < out_len; j++) {
        if (i < len) {
            uint8_t c = code_of[x[i]];
            out[j] = c;
            int bit;
            if (pi_inject) {
                bit = (j < inject_steps) ? pi_inject[j * alpha + c] : 0;
            } else {
                bit = or_walk_bit(seed, l, (uint64_t)j, x[i]);
            }
            i += bit;
        } else {
            if (walk_end == out_len) walk_end = j;
            out[j] = (uint8_t)alpha; /* bottom, a symbol outside the alphabet */
        }
    }
    return walk_end;
}

/* Preprocessing (Alg. 2, embedding part): every string, every l in [r].
 * emb is [r][n][out_len], walk_end is [r][n]. pi_inject is [r][inject_steps][alpha]. */
int or_embed_all(const uint8_t *data, const int64_t *offsets, int64_t n, const uint8_t *alphabet,
                 uint32_t alpha, uint32_t r, int64_t out_len, uint64_t seed,
                 const uint8_t *pi_inject, int64_t inject_steps, uint8_t *emb, int64_t *walk_end) {
    uint8_t code_of[256];
    memset(code_of, 255, sizeof code_of);
    for (uint32_t c = 0; c < alpha; c++) code_of[alphabet[c]] = (uint8_t)c;
    for (int64_t p = 0; p < offsets[n]; p++)
        if (code_of[data[p]] == 255) return OR_ERR_ARG;
    for (uint32_t l = 0; l < r; l++) {
        const uint8_t *pi = pi_inject ? pi_inject + (int64_t)l * inject_steps * alpha : NULL;
        for (int64_t s = 0; s < n; s++) {
            walk_end[(int64_t)l * n + s] =
                or_cgk_embed(data + offsets[s], offsets[s + 1] - offsets[s], code_of, alpha, seed, l,
                             out_len, pi, inject_steps, emb + ((int64_t)l * n + s) * out_len);
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Bit-sampling LSH with AND amplification (Section 3.2)                     */
/* ------------------------------------------------------------------------ */

/* Hash functions f_f^l, f in [m]: z sampled coordinates each. pos is [r][m][z]. */
void or_positions_all(uint64_t seed, uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t *pos) {
    for (uint32_t l = 0; l < r; l++)
        for (uint32_t f = 0; f < m; f++)
            for (uint32_t q = 0; q < z; q++)
                pos[((uint64_t)l * m + f) * z + q] = or_position(seed, l, f, q, L);
}

/* Signature of one embedded string under one function: the z sampled symbols,
 * encoded as sum_q c_q (alpha+1)^q. Positions at or after walk_end read bottom. */
uint64_t or_signature_key(const uint8_t *t, int64_t walk_end, const uint32_t *pos, uint32_t z,
                          uint32_t alpha) {
    uint64_t key = 0, radix = 1;
    for (uint32_t q = 0; q < z; q++) {
        uint64_t c = ((int64_t)pos[q] < walk_end) ? t[pos[q]] : alpha;
        key += c * radix;
        radix *= (uint64_t)alpha + 1;
    }
    return key;
}

/* The paper's two-level hashing of a signature (Section 4): the z sampled
 * symbols as a vector u with entries 1..|S| (and |S|+1 for the padding symbol),
 * a random vector v in [0, P)^z per function, key = <u, v> mod P.
 *   v[l][f][q] = mulhi64(splitmix64(splitmix64(seed) ^ (3<<56 | l<<48 | f<<32 | q)), P)
 * (a counter-based reading of "a random vector"). Equal signatures get equal
 * keys; different ones collide with probability 1/P over v. */
uint32_t or_hash_coefficient(uint64_t seed, uint32_t l, uint32_t f, uint32_t q, uint64_t P) {
    uint64_t base = or_splitmix64(seed);
    uint64_t ctr = (3ull << 56) | ((uint64_t)l << 48) | ((uint64_t)f << 32) | (uint64_t)q;
    return (uint32_t)(((unsigned __int128)or_splitmix64(base ^ ctr) * (unsigned __int128)P) >> 64);
}

uint64_t or_signature_key_modp(const uint8_t *t, int64_t walk_end, const uint32_t *pos, uint32_t z, uint32_t alpha,
                               uint64_t seed, uint32_t l, uint32_t f, uint64_t P) {
    uint64_t acc = 0;
    for (uint32_t q = 0; q < z; q++) {
        uint64_t u = 1 + (((int64_t)pos[q] < walk_end) ? t[pos[q]] : alpha);
        acc = (acc + u * (uint64_t)or_hash_coefficient(seed, l, f, q, P)) % P;
    }
    return acc;
}

/* Hashed keys of every (table, string): keys[(l*m+f)*n + s] = <u, v> mod P. */
void or_sign_all_modp(const uint8_t *emb, const int64_t *walk_end, int64_t n, uint32_t r, uint32_t m, uint32_t z,
                      int64_t out_len, const uint32_t *pos, uint32_t alpha, uint64_t seed, uint64_t P,
                      uint64_t *keys) {
    for (uint32_t l = 0; l < r; l++)
        for (uint32_t f = 0; f < m; f++)
            for (int64_t s = 0; s < n; s++)
                keys[((int64_t)l * m + f) * n + s] = or_signature_key_modp(
                    emb + ((int64_t)l * n + s) * out_len, walk_end[(int64_t)l * n + s],
                    pos + ((uint64_t)l * m + f) * z, z, alpha, seed, l, f, P);
}

/* keys is [r*m][n]: keys[(l*m+f)*n + s]. */
void or_sign_all(const uint8_t *emb, const int64_t *walk_end, int64_t n, uint32_t r, uint32_t m,
                 uint32_t z, int64_t out_len, const uint32_t *pos, uint32_t alpha, uint64_t *keys) {
    for (uint32_t l = 0; l < r; l++)
        for (uint32_t f = 0; f < m; f++)
            for (int64_t s = 0; s < n; s++)
                keys[((int64_t)l * m + f) * n + s] = or_signature_key(
                    emb + ((int64_t)l * n + s) * out_len, walk_end[(int64_t)l * n + s],
                    pos + ((uint64_t)l * m + f) * z, z, alpha);
}

/* Signatures of strings [s0, s1) straight from the walks (Alg. 1, then the
 * AND signature of Section 3.2 for every function), one string and one
 * embedding at a time, so large sets need no [r][n][out_len] buffer. The walk
 * runs for steps [0, L) only: every sampled position is below L, and a walk
 * that has not finished by step L reads the same symbols there as a longer
 * one. keys is [r*m][s1-s0]; pos is [r][m][z] (or_positions_all). Returns 0
 * or an error code (a byte outside the alphabet). */
int or_keys_range(const uint8_t *data, const int64_t *offsets, int64_t s0, int64_t s1,
                  const uint8_t *alphabet, uint32_t alpha, uint32_t r, uint32_t m, uint32_t z,
                  uint32_t L, uint64_t seed, const uint32_t *pos, uint64_t *keys) {
    uint8_t code_of[256];
    memset(code_of, 255, sizeof code_of);
    for (uint32_t c = 0; c < alpha; c++) code_of[alphabet[c]] = (uint8_t)c;
    for (int64_t p = offsets[s0]; p < offsets[s1]; p++)
        if (code_of[data[p]] == 255) return OR_ERR_ARG;
    uint8_t *t = (uint8_t *)malloc((size_t)(L ? L : 1));
    if (!t) return OR_ERR_OOM;
    const int64_t cnt = s1 - s0;
    for (uint32_t l = 0; l < r; l++)
        for (int64_t s = s0; s < s1; s++) {
            int64_t we = or_cgk_embed(data + offsets[s], offsets[s + 1] - offsets[s], code_of, alpha,
                                      seed, l, (int64_t)L, NULL, 0, t);
            for (uint32_t f = 0; f < m; f++)
                keys[((int64_t)l * m + f) * cnt + (s - s0)] =
                    or_signature_key(t, we, pos + ((uint64_t)l * m + f) * z, z, alpha);
        }
    free(t);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* EmbedJoin candidate generation, Algorithm 3 (sliding window over buckets) */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t *v; int64_t n, cap; } ivec;

static int ivec_push(ivec *a, int32_t x) {
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 4;
        int32_t *nv = (int32_t *)realloc(a->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return OR_ERR_OOM;
        a->v = nv; a->cap = nc;
    }
    a->v[a->n++] = x;
    return OR_OK;
}

/* One hash table D_f^l: open addressing from key to a bucket (list of strings). */
typedef struct { uint64_t *keys; int64_t *slot_bucket; int64_t cap; ivec *buckets; int64_t nb; } table_t;

static ivec *table_bucket(table_t *t, uint64_t key, int create) {
    uint64_t h = or_splitmix64(key) & (uint64_t)(t->cap - 1);
    for (;;) {
        if (t->slot_bucket[h] < 0) {
            if (!create) return NULL;
            t->keys[h] = key;
            t->slot_bucket[h] = t->nb;
            ivec e = {0, 0, 0};
            t->buckets[t->nb++] = e;
            return &t->buckets[t->slot_bucket[h]];
        }
        if (t->keys[h] == key) return &t->buckets[t->slot_bucket[h]];
        h = (h + 1) & (uint64_t)(t->cap - 1);
    }
}

typedef struct { const uint8_t *data; const int64_t *offsets; } sort_ctx_t;
static sort_ctx_t g_sort;

/* Alg. 2 step 1: by length increasingly, then alphabetically (ties by index). */
static int cmp_len_lex(const void *a, const void *b) {
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    int64_t li = g_sort.offsets[i + 1] - g_sort.offsets[i];
    int64_t lj = g_sort.offsets[j + 1] - g_sort.offsets[j];
    if (li != lj) return li < lj ? -1 : 1;
    int c = memcmp(g_sort.data + g_sort.offsets[i], g_sort.data + g_sort.offsets[j], (size_t)li);
    if (c) return c;
    return (i > j) - (i < j);
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/*
 * Candidate pairs of Alg. 3: strings are visited in (length, lexicographic)
 * order; for every table (l, f) the visited string is compared with the
 * strings already stored in its bucket. A stored string s with
 * |s_i| - |s| <= K gives the candidate (s, s_i); otherwise s is removed from
 * the bucket (it can never pair with a later, longer string). Then s_i is
 * stored. Duplicates are removed at the end. keys is [T][n], T = r*m.
 * Writes up to `capacity` sorted unique pairs (i<<32|j, i<j in input order)
 * and returns the number of candidates (or a negative error code).
 */
static int candidates_alg3(const uint8_t *data, const int64_t *offsets, int64_t n,
                           const uint64_t *keys, int64_t T, int32_t K, uint64_t **out_list,
                           int64_t *out_count) {
    *out_list = NULL;
    *out_count = 0;
    if (n < 2 || T <= 0) return OR_OK;
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!order) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) order[i] = (int32_t)i;
    g_sort.data = data; g_sort.offsets = offsets;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_len_lex);

    int64_t cap = 1;
    while (cap < 2 * n) cap <<= 1;
    table_t *tabs = (table_t *)calloc((size_t)T, sizeof(table_t));
    for (int64_t t = 0; t < T; t++) {
        tabs[t].cap = cap;
        tabs[t].keys = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
        tabs[t].slot_bucket = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        tabs[t].buckets = (ivec *)malloc((size_t)n * sizeof(ivec));
        for (int64_t h = 0; h < cap; h++) tabs[t].slot_bucket[h] = -1;
    }
    uint64_t *cand = NULL;
    int64_t nc = 0, ccap = 0;
    int err = OR_OK;
    for (int64_t a = 0; a < n && !err; a++) {
        int32_t si = order[a];
        int64_t li = offsets[si + 1] - offsets[si];
        for (int64_t t = 0; t < T && !err; t++) {
            ivec *B = table_bucket(&tabs[t], keys[t * n + si], 1);
            for (int64_t b = 0; b < B->n;) {
                int32_t s = B->v[b];
                int64_t ls = offsets[s + 1] - offsets[s];
                if (li - ls <= K) {
                    if (nc == ccap) {
                        int64_t nca = ccap ? 2 * ccap : 1024;
                        uint64_t *nv = (uint64_t *)realloc(cand, (size_t)nca * sizeof(uint64_t));
                        if (!nv) { err = OR_ERR_OOM; break; }
                        cand = nv; ccap = nca;
                    }
                    uint64_t lo = (uint64_t)(s < si ? s : si), hi = (uint64_t)(s < si ? si : s);
                    cand[nc++] = (lo << 32) | hi;
                    b++;
                } else {
                    B->v[b] = B->v[--B->n];   /* remove s from D_f^l */
                }
            }
            if (!err) err = ivec_push(B, si);
        }
    }
    int64_t nu = 0;
    if (!err && nc) {
        /* Alg. 3 removes duplicate pairs from C */
        qsort(cand, (size_t)nc, sizeof(uint64_t), cmp_u64);
        for (int64_t k = 0; k < nc; k++)
            if (k == 0 || cand[k] != cand[k - 1]) cand[nu++] = cand[k];
    }
    for (int64_t t = 0; t < T; t++) {
        for (int64_t b = 0; b < tabs[t].nb; b++) free(tabs[t].buckets[b].v);
        free(tabs[t].keys); free(tabs[t].slot_bucket); free(tabs[t].buckets);
    }
    free(tabs); free(order);
    if (err) { free(cand); return err; }
    *out_list = cand;
    *out_count = nu;
    return OR_OK;
}

/* Public form: writes up to `capacity` candidates and returns their number
 * (negative error code on failure). */
int64_t or_candidates_alg3(const uint8_t *data, const int64_t *offsets, int64_t n,
                           const uint64_t *keys, int64_t T, int32_t K, uint64_t *out,
                           int64_t capacity) {
    uint64_t *list;
    int64_t cnt;
    int err = candidates_alg3(data, offsets, n, keys, T, K, &list, &cnt);
    if (err) return -err;
    for (int64_t k = 0; k < cnt && k < capacity && out; k++) out[k] = list[k];
    free(list);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Edit distance (Section 3.3)                                               */
/* ------------------------------------------------------------------------ */

/* Ukkonen's threshold edit distance: fill the 2K+1 diagonals d = j - i in
 * [-K, K]; every cell outside the band is taken as K+1 and values are capped at
 * K+1. Returns min(ED(x, y), K+1). */
int32_t or_ed_banded(const uint8_t *x, int64_t lx, const uint8_t *y, int64_t ly, int32_t K) {
    if (K < 0) return 0;
    int64_t diff = ly - lx;
    if (diff > K || -diff > K) return K + 1;
    int64_t W = 2 * (int64_t)K + 1;
    int32_t cap = K + 1;
    /* row arrays indexed by d + 1 (two sentinels), entry (i, d) is cell (i, j = i + d - K) */
    int32_t *prev = (int32_t *)malloc((size_t)(W + 2) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(W + 2) * sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    for (int64_t d = 0; d < W + 2; d++) prev[d] = cur[d] = cap;
    /* row 0: D(0, j) = j */
    for (int64_t d = 0; d < W; d++) {
        int64_t j = d - K;
        prev[d + 1] = (j >= 0 && j <= ly) ? (int32_t)(j < cap ? j : cap) : cap;
    }
    for (int64_t i = 1; i <= lx; i++) {
        for (int64_t d = 0; d < W; d++) {
            int64_t j = i + d - K;
            int32_t v;
            if (j < 0 || j > ly) {
                v = cap;
            } else if (j == 0) {
                v = (int32_t)(i < cap ? i : cap);            /* D(i, 0) = i */
            } else {
                int32_t diag = prev[d + 1] + (x[i - 1] != y[j - 1]); /* (i-1, j-1): same d */
                int32_t up = prev[d + 2] + 1;                         /* (i-1, j):   d+1   */
                int32_t left = cur[d] + 1;                            /* (i, j-1):   d-1   */
                v = diag < up ? diag : up;
                v = v < left ? v : left;
                if (v > cap) v = cap;
            }
            cur[d + 1] = v;
        }
        int32_t *tmp = prev; prev = cur; cur = tmp;
        cur[0] = cur[W + 1] = cap;
    }
    int32_t res = prev[(ly - lx) + K + 1];
    free(prev); free(cur);
    return res;
}

/* The band DP of or_ed_banded with Ukkonen's cutoff: once every cell of a row's
   band exceeds K, so does every later cell (a cell is never below the minimum of
   the row above: each recurrence term adds 0 or 1 to a cell of that row, or 1 to
   an earlier cell of its own row), so the answer is K + 1. Returns the same
   min(ED, K + 1) as or_ed_banded; used for brute-force truth on larger samples. */
int32_t or_ed_banded_cutoff(const uint8_t *x, int64_t lx, const uint8_t *y, int64_t ly, int32_t K) {
    if (K < 0) return 0;
    int64_t diff = ly - lx;
    if (diff > K || -diff > K) return K + 1;
    int64_t W = 2 * (int64_t)K + 1;
    int32_t cap = K + 1;
    int32_t *prev = (int32_t *)malloc((size_t)(W + 2) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(W + 2) * sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    for (int64_t d = 0; d < W + 2; d++) prev[d] = cur[d] = cap;
    for (int64_t d = 0; d < W; d++) {
        int64_t j = d - K;
        prev[d + 1] = (j >= 0 && j <= ly) ? (int32_t)(j < cap ? j : cap) : cap;
    }
    for (int64_t i = 1; i <= lx; i++) {
        int32_t row_min = cap;
        for (int64_t d = 0; d < W; d++) {
            int64_t j = i + d - K;
            int32_t v;
            if (j < 0 || j > ly) {
                v = cap;
            } else if (j == 0) {
                v = (int32_t)(i < cap ? i : cap);
            } else {
                int32_t diag = prev[d + 1] + (x[i - 1] != y[j - 1]);
                int32_t up = prev[d + 2] + 1;
                int32_t left = cur[d] + 1;
                v = diag < up ? diag : up;
                v = v < left ? v : left;
                if (v > cap) v = cap;
            }
            cur[d + 1] = v;
            if (v < row_min) row_min = v;
        }
        int32_t *tmp = prev; prev = cur; cur = tmp;
        cur[0] = cur[W + 1] = cap;
        if (row_min >= cap) { free(prev); free(cur); return cap; }
    }
    int32_t res = prev[(ly - lx) + K + 1];
    free(prev); free(cur);
    return res;
}

/* Brute-force join (Section 1) with the cutoff DP: every pair i<j with ED <= K,
   written to out (capacity entries at most); returns the count. */
int64_t or_join_bruteforce_cutoff(const uint8_t *data, const int64_t *offsets, int64_t n, int32_t K,
                                  uint64_t *out, int64_t capacity) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            int32_t d = or_ed_banded_cutoff(data + offsets[i], offsets[i + 1] - offsets[i],
                                            data + offsets[j], offsets[j + 1] - offsets[j], K);
            if (d >= 0 && d <= K) {
                if (cnt < capacity && out) out[cnt] = ((uint64_t)i << 32) | (uint64_t)j;
                cnt++;
            }
        }
    return cnt;
}

/* Wagner-Fischer full DP (the definition of edit distance, Section 1). */
int64_t or_ed_full(const uint8_t *x, int64_t lx, const uint8_t *y, int64_t ly) {
    int64_t *prev = (int64_t *)malloc((size_t)(ly + 1) * sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc((size_t)(ly + 1) * sizeof(int64_t));
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    for (int64_t j = 0; j <= ly; j++) prev[j] = j;
    for (int64_t i = 1; i <= lx; i++) {
        cur[0] = i;
        for (int64_t j = 1; j <= ly; j++) {
            int64_t v = prev[j - 1] + (x[i - 1] != y[j - 1]);
            if (prev[j] + 1 < v) v = prev[j] + 1;
            if (cur[j - 1] + 1 < v) v = cur[j - 1] + 1;
            cur[j] = v;
        }
        int64_t *tmp = prev; prev = cur; cur = tmp;
    }
    int64_t res = prev[ly];
    free(prev); free(cur);
    return res;
}

/* Verification loop of Alg. 3: flags[k] = 1 iff ED(pair k) <= K. */
void or_verify(const uint8_t *data, const int64_t *offsets, const uint64_t *pairs, int64_t np,
               int32_t K, uint8_t *flags) {
    for (int64_t k = 0; k < np; k++) {
        int64_t a = (int64_t)(pairs[k] >> 32), b = (int64_t)(pairs[k] & 0xffffffffu);
        int32_t d = or_ed_banded(data + offsets[a], offsets[a + 1] - offsets[a], data + offsets[b],
                                 offsets[b + 1] - offsets[b], K);
        flags[k] = (d >= 0 && d <= K) ? 1 : 0;
    }
}

/* The verification loop with the cutoff DP (same flags as or_verify, faster
 * on pairs far above K): flags[k] = 1 iff ED(pair k) <= K. */
void or_verify_cutoff(const uint8_t *data, const int64_t *offsets, const uint64_t *pairs, int64_t np,
                      int32_t K, uint8_t *flags) {
    for (int64_t k = 0; k < np; k++) {
        int64_t a = (int64_t)(pairs[k] >> 32), b = (int64_t)(pairs[k] & 0xffffffffu);
        int32_t d = or_ed_banded_cutoff(data + offsets[a], offsets[a + 1] - offsets[a],
                                        data + offsets[b], offsets[b + 1] - offsets[b], K);
        flags[k] = (d >= 0 && d <= K) ? 1 : 0;
    }
}

/* Brute-force join by definition (Section 1): every pair i<j with ED <= K. */
int64_t or_join_bruteforce(const uint8_t *data, const int64_t *offsets, int64_t n, int32_t K,
                           uint64_t *out, int64_t capacity) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            int32_t d = or_ed_banded(data + offsets[i], offsets[i + 1] - offsets[i],
                                     data + offsets[j], offsets[j + 1] - offsets[j], K);
            if (d <= K) {
                if (cnt < capacity && out) out[cnt] = ((uint64_t)i << 32) | (uint64_t)j;
                cnt++;
            }
        }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* EmbedJoin end to end (Alg. 3 with Alg. 2)                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t r, m, z;
    uint32_t L;          /* sampling range; 0 => out_len */
    int64_t out_len;     /* embedding length; 0 => 3N */
    int32_t K;
    uint64_t seed;
    const uint8_t *alphabet;
    uint32_t alpha;
    const uint8_t *pi_inject;      /* optional [r][inject_steps][alpha] */
    int64_t inject_steps;
    const uint32_t *pos_inject;    /* optional [r][m][z] */
} or_params;

typedef struct {
    int64_t n_candidates;
    int64_t n_out;
    int64_t out_len;
    uint32_t L;
    double t_embed, t_sign, t_candidates, t_verify;  /* seconds per phase */
} or_stats;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Runs the whole method. out gets up to `capacity` output pairs; cand (optional)
 * gets up to cand_capacity candidate pairs. Returns 0 or an error code. */
int or_join_ext(const uint8_t *data, const int64_t *offsets, int64_t n, const or_params *p, uint64_t key_P,
                uint64_t *out, int64_t capacity, uint64_t *cand, int64_t cand_capacity, or_stats *st);

int or_join(const uint8_t *data, const int64_t *offsets, int64_t n, const or_params *p,
            uint64_t *out, int64_t capacity, uint64_t *cand, int64_t cand_capacity, or_stats *st) {
    return or_join_ext(data, offsets, n, p, 0, out, capacity, cand, cand_capacity, st);
}

/* or_join with the bucket key chosen by key_P: 0 = the exact mixed-radix key,
 * else the two-level hash <u, v> mod key_P of Section 4. */
int or_join_ext(const uint8_t *data, const int64_t *offsets, int64_t n, const or_params *p, uint64_t key_P,
                uint64_t *out, int64_t capacity, uint64_t *cand, int64_t cand_capacity, or_stats *st) {
    memset(st, 0, sizeof *st);
    if (n < 0 || p->r == 0 || p->m == 0 || p->z == 0 || p->K < 0 || p->alpha == 0 || p->alpha > 255)
        return OR_ERR_ARG;
    int64_t N = 0;
    for (int64_t s = 0; s < n; s++)
        if (offsets[s + 1] - offsets[s] > N) N = offsets[s + 1] - offsets[s];
    /* Alg. 1 pads to 3N; a set of empty strings still gets one (bottom) step */
    int64_t out_len = p->out_len ? p->out_len : (N > 0 ? 3 * N : 1);
    uint32_t L = p->L ? p->L : (uint32_t)out_len;
    st->out_len = out_len; st->L = L;
    if (n < 2) return OR_OK;
    if ((int64_t)L > out_len || L == 0) return OR_ERR_ARG;

    double t0 = now_s();
    int64_t T = (int64_t)p->r * p->m;
    uint8_t *emb = (uint8_t *)malloc((size_t)(p->r * n * out_len));
    int64_t *we = (int64_t *)malloc((size_t)(p->r * n) * sizeof(int64_t));
    uint32_t *pos = (uint32_t *)malloc((size_t)T * p->z * sizeof(uint32_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)(T * n) * sizeof(uint64_t));
    if (!emb || !we || !pos || !keys) { free(emb); free(we); free(pos); free(keys); return OR_ERR_OOM; }
    int err = or_embed_all(data, offsets, n, p->alphabet, p->alpha, p->r, out_len, p->seed,
                           p->pi_inject, p->inject_steps, emb, we);
    st->t_embed = now_s();
    if (!err) {
        if (p->pos_inject) memcpy(pos, p->pos_inject, (size_t)T * p->z * sizeof(uint32_t));
        else or_positions_all(p->seed, p->r, p->m, p->z, L, pos);
        if (key_P == 0) {
            or_sign_all(emb, we, n, p->r, p->m, p->z, out_len, pos, p->alpha, keys);
        } else {
            for (uint32_t l = 0; l < p->r; l++)
                for (uint32_t f = 0; f < p->m; f++)
                    for (int64_t s = 0; s < n; s++)
                        keys[((int64_t)l * p->m + f) * n + s] = or_signature_key_modp(
                            emb + ((int64_t)l * n + s) * out_len, we[(int64_t)l * n + s],
                            pos + ((uint64_t)l * p->m + f) * p->z, p->z, p->alpha, p->seed, l, f, key_P);
        }
    }
    free(emb); free(we); free(pos);
    if (err) { free(keys); return err; }
    st->t_sign = now_s();
    uint64_t *cl = NULL;
    int64_t nc = 0;
    err = candidates_alg3(data, offsets, n, keys, T, p->K, &cl, &nc);
    free(keys);
    if (err) return err;
    st->t_candidates = now_s();
    uint8_t *flags = (uint8_t *)malloc((size_t)(nc ? nc : 1));
    if (!flags) { free(cl); return OR_ERR_OOM; }
    or_verify(data, offsets, cl, nc, p->K, flags);
    int64_t no = 0;
    for (int64_t k = 0; k < nc; k++) {
        if (cand && k < cand_capacity) cand[k] = cl[k];
        if (flags[k]) {
            if (out && no < capacity) out[no] = cl[k];
            no++;
        }
    }
    st->n_candidates = nc;
    st->n_out = no;
    st->t_verify = now_s();
    st->t_verify -= st->t_candidates;
    st->t_candidates -= st->t_sign;
    st->t_sign -= st->t_embed;
    st->t_embed -= t0;
    free(cl); free(flags);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* EmbedJoin+ (Algorithms 4 and 5): suffix embeddings and match counting     */
/* ------------------------------------------------------------------------ */

/* A match of Alg. 5: substring k_x of string x and substring k_y of string y
 * share a bucket in one table; x is the string visited first (sorted order). */
typedef struct { int32_t x, y, kx, ky; } or_tuple;

static int cmp_tuple(const void *a, const void *b) {
    const or_tuple *p = (const or_tuple *)a, *q = (const or_tuple *)b;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    if (p->y != q->y) return p->y < q->y ? -1 : 1;
    if (p->kx != q->kx) return p->kx < q->kx ? -1 : 1;
    if (p->ky != q->ky) return p->ky < q->ky ? -1 : 1;
    return 0;
}

/* Number of substrings per string, ceil(K / delta), at least 1 (a threshold of 0
 * still embeds the whole string). */
int32_t or_plus_substrings(int32_t K, int32_t delta) {
    if (delta <= 0) return 0;
    int32_t s = (K + delta - 1) / delta;
    return s < 1 ? 1 : s;
}

/*
 * EmbedJoin+ end to end. Alg. 4: strings sorted by (length, lexicographic);
 * for every embedding l and string s_i, the substrings s_{i,k} = s_i[(k-1)delta
 * .. |s_i|) for k = 1 .. ceil(K/delta) (empty once the start passes the end),
 * each CGK-embedded with the same random string R^l. Alg. 5: strings visited in
 * sorted order; for every table (l, f) and substring k, every stored (s, k') of
 * the bucket of its signature with s != s_i gives the match (s, s_i, k', k) if
 * |s_i| - |s| <= K, else (s, k') is removed; then (s_i, k) is stored. Matches
 * are counted per (x, y, k_x, k_y); a pair with some count >= T is a candidate
 * (once), and candidates with ED <= K are the output.
 * stats: n_candidates = candidate pairs, n_out = output pairs. tuples (optional)
 * gets the number of matches (with repetition). Returns 0 or an error code.
 */
int or_join_plus(const uint8_t *data, const int64_t *offsets, int64_t n, const or_params *p, int32_t delta,
                 int32_t T, uint64_t *out, int64_t capacity, uint64_t *cand, int64_t cand_capacity,
                 or_stats *st, int64_t *tuples) {
    memset(st, 0, sizeof *st);
    if (tuples) *tuples = 0;
    if (n < 0 || p->r == 0 || p->m == 0 || p->z == 0 || p->K < 0 || p->alpha == 0 || p->alpha > 255 ||
        delta <= 0 || T < 1)
        return OR_ERR_ARG;
    const int32_t S = or_plus_substrings(p->K, delta);
    int64_t N = 0;
    for (int64_t s = 0; s < n; s++)
        if (offsets[s + 1] - offsets[s] > N) N = offsets[s + 1] - offsets[s];
    int64_t out_len = p->out_len ? p->out_len : (N > 0 ? 3 * N : 1);
    uint32_t L = p->L ? p->L : (uint32_t)out_len;
    st->out_len = out_len; st->L = L;
    if (n < 2) return OR_OK;
    if ((int64_t)L > out_len || L == 0) return OR_ERR_ARG;
    uint8_t code_of[256];
    memset(code_of, 255, sizeof code_of);
    for (uint32_t c = 0; c < p->alpha; c++) code_of[p->alphabet[c]] = (uint8_t)c;
    for (int64_t q = 0; q < offsets[n]; q++)
        if (code_of[data[q]] == 255) return OR_ERR_ARG;

    /* Alg. 4: hash functions, then the embeddings of every substring */
    const int64_t TT = (int64_t)p->r * p->m;
    uint32_t *pos = (uint32_t *)malloc((size_t)TT * p->z * sizeof(uint32_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)TT * (size_t)n * (size_t)S * sizeof(uint64_t));
    uint8_t *t = (uint8_t *)malloc((size_t)out_len);
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!pos || !keys || !t || !order) { free(pos); free(keys); free(t); free(order); return OR_ERR_OOM; }
    if (p->pos_inject) memcpy(pos, p->pos_inject, (size_t)TT * p->z * sizeof(uint32_t));
    else or_positions_all(p->seed, p->r, p->m, p->z, L, pos);
    for (uint32_t l = 0; l < p->r; l++) {
        const uint8_t *pi = p->pi_inject ? p->pi_inject + (int64_t)l * p->inject_steps * p->alpha : NULL;
        for (int64_t s = 0; s < n; s++)
            for (int32_t k = 0; k < S; k++) {
                const int64_t len = offsets[s + 1] - offsets[s];
                const int64_t start = (int64_t)k * delta < len ? (int64_t)k * delta : len;
                int64_t we = or_cgk_embed(data + offsets[s] + start, len - start, code_of, p->alpha, p->seed, l,
                                          out_len, pi, p->inject_steps, t);
                for (uint32_t f = 0; f < p->m; f++)
                    keys[((int64_t)l * p->m + f) * n * S + s * S + k] =
                        or_signature_key(t, we, pos + ((uint64_t)l * p->m + f) * p->z, p->z, p->alpha);
            }
    }
    free(t);
    free(pos);

    /* Alg. 5: sliding window over the tables in sorted order, collecting matches */
    for (int64_t i = 0; i < n; i++) order[i] = (int32_t)i;
    g_sort.data = data; g_sort.offsets = offsets;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_len_lex);
    int64_t cap = 1;
    while (cap < 2 * n * S) cap <<= 1;
    table_t *tabs = (table_t *)calloc((size_t)TT, sizeof(table_t));
    int err = tabs ? OR_OK : OR_ERR_OOM;
    for (int64_t tb = 0; tb < TT && !err; tb++) {
        tabs[tb].cap = cap;
        tabs[tb].keys = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
        tabs[tb].slot_bucket = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        tabs[tb].buckets = (ivec *)malloc((size_t)(n * S) * sizeof(ivec));
        if (!tabs[tb].keys || !tabs[tb].slot_bucket || !tabs[tb].buckets) { err = OR_ERR_OOM; break; }
        for (int64_t h = 0; h < cap; h++) tabs[tb].slot_bucket[h] = -1;
    }
    or_tuple *C = NULL;
    int64_t nc = 0, ccap = 0;
    for (int64_t a = 0; a < n && !err; a++) {
        const int32_t si = order[a];
        const int64_t li = offsets[si + 1] - offsets[si];
        for (int64_t tb = 0; tb < TT && !err; tb++)
            for (int32_t k = 0; k < S && !err; k++) {
                ivec *B = table_bucket(&tabs[tb], keys[tb * n * S + (int64_t)si * S + k], 1);
                for (int64_t b = 0; b < B->n;) {
                    const int32_t rec = B->v[b];
                    const int32_t s = rec / S, kp = rec % S;
                    if (s == si) { b++; continue; }
                    const int64_t ls = offsets[s + 1] - offsets[s];
                    if (li - ls <= p->K) {
                        if (nc == ccap) {
                            int64_t nca = ccap ? 2 * ccap : 1024;
                            or_tuple *nv = (or_tuple *)realloc(C, (size_t)nca * sizeof(or_tuple));
                            if (!nv) { err = OR_ERR_OOM; break; }
                            C = nv; ccap = nca;
                        }
                        C[nc].x = s; C[nc].y = si; C[nc].kx = kp; C[nc].ky = k;
                        nc++;
                        b++;
                    } else {
                        B->v[b] = B->v[--B->n];   /* remove (s, k') from the table */
                    }
                }
                if (!err) err = ivec_push(B, si * S + k);
            }
    }
    for (int64_t tb = 0; tabs && tb < TT; tb++) {
        if (tabs[tb].buckets)
            for (int64_t b = 0; b < tabs[tb].nb; b++) free(tabs[tb].buckets[b].v);
        free(tabs[tb].keys); free(tabs[tb].slot_bucket); free(tabs[tb].buckets);
    }
    free(tabs); free(order); free(keys);
    if (err) { free(C); return err; }
    if (tuples) *tuples = nc;

    /* count every (x, y, k_x, k_y); a pair with some count >= T is a candidate */
    uint64_t *cl = (uint64_t *)malloc((size_t)(nc ? nc : 1) * sizeof(uint64_t));
    if (!cl) { free(C); return OR_ERR_OOM; }
    int64_t ncand = 0;
    if (nc) qsort(C, (size_t)nc, sizeof(or_tuple), cmp_tuple);
    for (int64_t q = 0; q < nc;) {
        int64_t e = q + 1;
        while (e < nc && cmp_tuple(&C[q], &C[e]) == 0) e++;
        if (e - q >= T) {
            const uint64_t lo = (uint64_t)(C[q].x < C[q].y ? C[q].x : C[q].y);
            const uint64_t hi = (uint64_t)(C[q].x < C[q].y ? C[q].y : C[q].x);
            cl[ncand++] = (lo << 32) | hi;
        }
        q = e;
    }
    free(C);
    int64_t nu = 0;
    if (ncand) {
        qsort(cl, (size_t)ncand, sizeof(uint64_t), cmp_u64);
        for (int64_t q = 0; q < ncand; q++)
            if (q == 0 || cl[q] != cl[q - 1]) cl[nu++] = cl[q];
    }
    /* verification of every candidate pair (Section 3.3) */
    uint8_t *flags = (uint8_t *)malloc((size_t)(nu ? nu : 1));
    if (!flags) { free(cl); return OR_ERR_OOM; }
    or_verify(data, offsets, cl, nu, p->K, flags);
    int64_t no = 0;
    for (int64_t q = 0; q < nu; q++) {
        if (cand && q < cand_capacity) cand[q] = cl[q];
        if (flags[q]) {
            if (out && no < capacity) out[no] = cl[q];
            no++;
        }
    }
    st->n_candidates = nu;
    st->n_out = no;
    free(cl); free(flags);
    return OR_OK;
}


/* ------------------------------------------------------------------------ */
/* Grouping (Section 4.1)                                                    */
/* ------------------------------------------------------------------------ */

/* Number of length groups: N' = ceil(N/K)*K, groups 1 .. N'/K - 1 (at least
 * one); group g (1-based) holds the strings of length in ((g-1)K, (g+1)K], the
 * first also the empty strings. K >= 1. */
int64_t or_group_count(int64_t N, int32_t K) {
    int64_t Np = ((N + K - 1) / K) * K;
    int64_t g = Np / K - 1;
    return g < 1 ? 1 : g;
}

int or_in_group(int64_t len, int64_t g, int32_t K) {
    if (g == 1 && len == 0) return 1;
    return len > (g - 1) * (int64_t)K && len <= (g + 1) * (int64_t)K;
}

/*
 * EmbedJoin with grouping: the strings are split into the length groups above
 * (every string in up to two of them, every pair within K in length in a
 * common one), EmbedJoin runs on each group on its own (its own N and 3N, the
 * caller's r, m, z, L, K and seed) and the outputs are united. out gets the
 * sorted unique union; *n_cand the candidates verified over all groups (with
 * the repeats the redundancy causes). key_P as for or_join_ext.
 */
int or_join_grouped(const uint8_t *data, const int64_t *offsets, int64_t n, const or_params *p, uint64_t key_P,
                    uint64_t *out, int64_t capacity, int64_t *n_out, int64_t *n_cand) {
    *n_out = 0; *n_cand = 0;
    if (p->K < 1) return OR_ERR_ARG;
    int64_t N = 0;
    for (int64_t s = 0; s < n; s++)
        if (offsets[s + 1] - offsets[s] > N) N = offsets[s + 1] - offsets[s];
    const int64_t G = or_group_count(N, p->K);
    int32_t *idx = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t *goff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    uint8_t *gdata = (uint8_t *)malloc((size_t)(offsets[n] ? offsets[n] : 1));
    uint64_t *all = NULL;
    int64_t nall = 0, cap_all = 0;
    int err = (idx && goff && gdata) ? OR_OK : OR_ERR_OOM;
    for (int64_t g = 1; g <= G && !err; g++) {
        int64_t gn = 0;
        goff[0] = 0;
        for (int64_t s = 0; s < n; s++) {
            const int64_t len = offsets[s + 1] - offsets[s];
            if (!or_in_group(len, g, p->K)) continue;
            memcpy(gdata + goff[gn], data + offsets[s], (size_t)len);
            goff[gn + 1] = goff[gn] + len;
            idx[gn++] = (int32_t)s;
        }
        if (gn < 2) continue;
        or_stats st;
        int64_t gcap = 1024;
        uint64_t *gout = NULL;
        for (;;) {
            gout = (uint64_t *)malloc((size_t)gcap * sizeof(uint64_t));
            if (!gout) { err = OR_ERR_OOM; break; }
            err = or_join_ext(gdata, goff, gn, p, key_P, gout, gcap, NULL, 0, &st);
            if (err || st.n_out <= gcap) break;
            gcap = st.n_out;
            free(gout);
        }
        if (err) { free(gout); break; }
        *n_cand += st.n_candidates;
        if (nall + st.n_out > cap_all) {
            int64_t nc = 2 * (nall + st.n_out) + 1024;
            uint64_t *nv = (uint64_t *)realloc(all, (size_t)nc * sizeof(uint64_t));
            if (!nv) { free(gout); err = OR_ERR_OOM; break; }
            all = nv; cap_all = nc;
        }
        /* group-local ids are increasing in the global order */
        for (int64_t q = 0; q < st.n_out; q++)
            all[nall++] = ((uint64_t)idx[gout[q] >> 32] << 32) | (uint64_t)idx[gout[q] & 0xffffffffu];
        free(gout);
    }
    free(idx); free(goff); free(gdata);
    if (err) { free(all); return err; }
    int64_t nu = 0;
    if (nall) {
        qsort(all, (size_t)nall, sizeof(uint64_t), cmp_u64);
        for (int64_t q = 0; q < nall; q++)
            if (q == 0 || all[q] != all[q - 1]) all[nu++] = all[q];
    }
    for (int64_t q = 0; q < nu && q < capacity && out; q++) out[q] = all[q];
    *n_out = nu;
    free(all);
    return OR_OK;
}
