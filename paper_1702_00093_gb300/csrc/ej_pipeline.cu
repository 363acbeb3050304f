// Back half of ej_join without host round trips: buckets (sorted windows, hashed
// record lists in global memory, or per-table sets in shared memory) append their
// pairs, a device hash set removes duplicates (Alg. 3's deduplication) and orders
// the candidates for the verifier, and the verified output is sorted at the end.
// Counts stay on the device; the host reads them once, after verification. The
// resident-index search (its buckets and probe) is here as well.
#include "ej_internal.cuh"

namespace ej {

// Window of record p in its table (records sorted by key, then length): the
// following records with the same key and length <= len_p + K.
__device__ __forceinline__ int64_t pl_window_end(const uint64_t *__restrict__ rk, const uint32_t *__restrict__ rid,
                                                 const int32_t *__restrict__ lens, int64_t p, int64_t n,
                                                 uint64_t key, int64_t limit) {
    auto pred = [&](int64_t q) { return rk[q] == key && (int64_t)lens[rid[q]] <= limit; };
    if (p + 1 >= n || !pred(p + 1)) return p + 1;
    int64_t good = p + 1, step = 1;
    while (true) {
        const int64_t nx = good + step;
        if (nx < n && pred(nx)) {
            good = nx;
            step <<= 1;
        } else {
            break;
        }
    }
    int64_t lo = good, hi = min(good + step, n);
    while (hi - lo > 1) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (pred(mid)) lo = mid; else hi = mid;
    }
    return lo + 1;
}

// counters: [0] raw pairs emitted (may exceed cap), [1] largest bucket
__global__ void emit_append_kernel(const uint64_t *__restrict__ rec_keys, const uint32_t *__restrict__ rec_ids,
                                   const int32_t *__restrict__ lens, int64_t n, int64_t T, int32_t K,
                                   uint64_t *__restrict__ raw, uint64_t cap,
                                   unsigned long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int64_t total = n * T;
    unsigned long long mb = 0;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane runs the same number of iterations so the warp collectives converge
    const int64_t iters = (total + step - 1) / step;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t i = start + it * step;
        int64_t cnt = 0, t = 0, p = 0;
        uint32_t a = 0;
        if (i < total) {
            t = i / n;
            p = i - t * n;
            const uint64_t *rk = rec_keys + t * n;
            const uint32_t *rid = rec_ids + t * n;
            const uint64_t key = rk[p];
            a = rid[p];
            cnt = pl_window_end(rk, rid, lens, p, n, key, (int64_t)lens[a] + K) - p - 1;
            if (cnt > 0 && (p == 0 || rk[p - 1] != key)) {
                int64_t e = p + 1;
                while (e < n && rk[e] == key) e++;   // bucket size (stats only, first record of a run)
                mb = max(mb, (unsigned long long)(e - p));
            }
        }
        // warp-aggregated reservation
        unsigned long long incl = (unsigned long long)cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned long long wtotal = __shfl_sync(FULL, incl, 31);
        unsigned long long base = 0;
        if (wtotal) {
            if (lane == 31) base = atomicAdd(&counters[0], wtotal);
            base = __shfl_sync(FULL, base, 31);
        }
        if (cnt > 0) {
            uint64_t o = base + incl - (unsigned long long)cnt;
            const uint32_t *rid = rec_ids + t * n;
            for (int64_t q = p + 1; q <= p + cnt; q++, o++) {
                if (o < cap) {
                    const uint32_t b = rid[q];
                    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
                    raw[o] = (lo << 32) | hi;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(FULL, mb, o);
        mb = v > mb ? v : mb;
    }
    if (lane == 0 && mb) atomicMax(&counters[1], mb);
}

cudaError_t launch_emit_append(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens, int64_t n,
                               int64_t T, int32_t K, uint64_t *raw, uint64_t cap, unsigned long long *counters,
                               cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0) {
        int64_t g = (total + 255) / 256;
        emit_append_kernel<<<(unsigned)(g > 16384 ? 16384 : g), 256, 0, s>>>(rec_keys, rec_ids, lens, n, T, K, raw,
                                                                               cap, counters);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Buckets by hashing (Alg. 3's per-table grouping of equal signatures, without
// sorting): table t owns the slots [t*H, (t+1)*H) of an open-addressing set of
// signatures; each slot heads a list of the records (t*n + i) that carry its
// signature, linked through next[] in insertion order. A record pairs with the
// records after it in its list, so every unordered pair of a bucket is seen
// exactly once, and the length filter ||s_i| - |s_j|| <= K applies per pair.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t key_hash(uint64_t k) {
    k ^= k >> 31;
    k *= 0x7fb5d329728ea185ull;
    k ^= k >> 27;
    k *= 0x81dadef4bc2dd44dull;
    k ^= k >> 33;
    return k;
}

constexpr uint32_t LIST_END = 0xFFFFFFFFu;

// slot_keys pre-filled with ~0 (never a signature: keys are < 2^64 - 1) and
// heads with LIST_END.
__global__ void bucket_insert_kernel(const uint64_t *__restrict__ keys, int64_t n, int64_t T, uint64_t H,
                                     uint64_t *__restrict__ slot_keys, uint32_t *__restrict__ heads,
                                     uint32_t *__restrict__ next, uint32_t *__restrict__ err) {
    const int64_t total = n * T;
    for (int64_t rec = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rec < total; rec += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = rec / n;
        const uint64_t key = keys[rec];
        uint64_t *sk = slot_keys + t * H;
        uint64_t h = key_hash(key) & (H - 1);
        bool placed = false;
        for (uint64_t probe = 0; probe < H; probe++) {
            const unsigned long long old = atomicCAS((unsigned long long *)&sk[h], ~0ull, key);
            if (old == ~0ull || old == key) {
                next[rec] = atomicExch(&heads[t * H + h], (uint32_t)rec);
                placed = true;
                break;
            }
            h = (h + 1) & (H - 1);
        }
        if (!placed) atomicOr(err, (uint32_t)DERR_GUARD);   // cannot happen with H >= n
    }
}

// Pairs of every record with the later records of its list that pass the
// length filter. counters: [0] raw pairs (may exceed cap), [1] largest bucket.
__global__ void bucket_emit_kernel(const int32_t *__restrict__ lens, int64_t n, int64_t T, int32_t K,
                                   const uint32_t *__restrict__ next, uint64_t *__restrict__ raw, uint64_t cap,
                                   unsigned long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int64_t total = n * T;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (total + step - 1) / step;   // the same on every lane: collectives converge
    unsigned long long mb = 0;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t rec = start + it * step;
        int64_t i = 0, base_t = 0;
        uint32_t q0 = LIST_END;
        unsigned long long cnt = 0, len_list = 0;
        int32_t li = 0;
        if (rec < total) {
            base_t = (rec / n) * n;
            i = rec - base_t;
            li = lens[i];
            q0 = next[rec];
            for (uint32_t q = q0; q != LIST_END; q = next[q]) {
                const int32_t lj = lens[(int64_t)q - base_t];
                const int32_t d = li > lj ? li - lj : lj - li;
                cnt += d <= K ? 1u : 0u;
                len_list++;
            }
            mb = max(mb, len_list + 1);
        }
        unsigned long long incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned long long wtotal = __shfl_sync(FULL, incl, 31);
        unsigned long long base = 0;
        if (wtotal) {
            if (lane == 31) base = atomicAdd(&counters[0], wtotal);
            base = __shfl_sync(FULL, base, 31);
        }
        if (cnt > 0) {
            uint64_t o = base + incl - cnt;
            for (uint32_t q = q0; q != LIST_END; q = next[q]) {
                const int64_t j = (int64_t)q - base_t;
                const int32_t lj = lens[j];
                const int32_t d = li > lj ? li - lj : lj - li;
                if (d <= K) {
                    if (o < cap) {
                        const uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
                        raw[o] = (lo << 32) | hi;
                    }
                    o++;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(FULL, mb, o);
        mb = v > mb ? v : mb;
    }
    if (lane == 0 && mb) atomicMax(&counters[1], mb);
}

uint64_t bucket_slots_per_table(int64_t n) {
    uint64_t H = 1;
    while (H < (uint64_t)n + (uint64_t)n / 2 + 1) H <<= 1;
    return H;
}

cudaError_t launch_bucket_insert(const uint64_t *keys, int64_t n, int64_t T, uint64_t H, uint64_t *slot_keys,
                                 uint32_t *heads, uint32_t *next, uint32_t *err, cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0) {
        const int64_t g = (total + 255) / 256;
        bucket_insert_kernel<<<(unsigned)(g > 32768 ? 32768 : g), 256, 0, s>>>(keys, n, T, H, slot_keys, heads, next,
                                                                               err);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_bucket_emit(const int32_t *lens, int64_t n, int64_t T, int32_t K, const uint32_t *next,
                               uint64_t *raw, uint64_t cap, unsigned long long *counters, cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0) {
        const int64_t g = (total + 255) / 256;
        bucket_emit_kernel<<<(unsigned)(g > 32768 ? 32768 : g), 256, 0, s>>>(lens, n, T, K, next, raw, cap, counters);
        note_launches(1);
    }
    return cudaGetLastError();
}

// Shared buckets of a batch: joins with the same embeddings and functions
// (seed, L, r, m) whose z differ. A signature of z samples is the finer one of
// z' > z samples modulo (|alphabet|+1)^z, so every bucket of the finer joins
// lies inside a bucket of the coarsest one. The records are inserted into the
// coarsest join's buckets only; every record walks the later records of its list
// once and hands each partner to every join whose own signatures and length
// filter it passes. Per join the emitted pairs are exactly those of its own
// buckets (each unordered pair once per table), and counters[1] gets its largest
// bucket. At most MAX_SHARED_BUCKETS joins.
__global__ void bucket_emit_shared_kernel(const int32_t *__restrict__ lens, int64_t n, int64_t T,
                                          const uint32_t *__restrict__ next, SharedEmit se) {
    const int lane = threadIdx.x & 31;
    const int64_t total = n * T;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (total + step - 1) / step;   // the same on every lane: collectives converge
    const int nj = se.njoins;
    unsigned long long mb[MAX_SHARED_BUCKETS];
#pragma unroll
    for (int j = 0; j < MAX_SHARED_BUCKETS; j++) mb[j] = 0;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t rec = start + it * step;
        int64_t i = 0, base_t = 0;
        uint32_t q0 = LIST_END;
        unsigned long long cnt[MAX_SHARED_BUCKETS], same[MAX_SHARED_BUCKETS];
        uint64_t ki[MAX_SHARED_BUCKETS];
#pragma unroll
        for (int j = 0; j < MAX_SHARED_BUCKETS; j++) { cnt[j] = 0; same[j] = 0; ki[j] = 0; }
        int32_t li = 0;
        if (rec < total) {
            base_t = (rec / n) * n;
            i = rec - base_t;
            li = lens[i];
            q0 = next[rec];
            if (q0 != LIST_END) {
#pragma unroll
                for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                    if (j < nj) ki[j] = se.keys[j][rec];
                for (uint32_t q = q0; q != LIST_END; q = next[q]) {
                    const int32_t lq = lens[(int64_t)q - base_t];
                    const int32_t d = li > lq ? li - lq : lq - li;
#pragma unroll
                    for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                        if (j < nj && se.keys[j][q] == ki[j]) {
                            same[j]++;
                            cnt[j] += d <= se.K[j] ? 1u : 0u;
                        }
                }
            }
#pragma unroll
            for (int j = 0; j < MAX_SHARED_BUCKETS; j++) mb[j] = max(mb[j], same[j] + 1);
        }
#pragma unroll
        for (int j = 0; j < MAX_SHARED_BUCKETS; j++) {
            if (j >= nj) break;
            unsigned long long incl = cnt[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned long long wtotal = __shfl_sync(FULL, incl, 31);
            unsigned long long base = 0;
            if (wtotal) {
                if (lane == 31) base = atomicAdd(&se.counters[j][0], wtotal);
                base = __shfl_sync(FULL, base, 31);
            }
            cnt[j] = base + incl - cnt[j];   // this lane's first output slot
        }
        if (q0 != LIST_END) {
            for (uint32_t q = q0; q != LIST_END; q = next[q]) {
                const int64_t jq = (int64_t)q - base_t;
                const int32_t lq = lens[jq];
                const int32_t d = li > lq ? li - lq : lq - li;
                const uint64_t lo = (uint64_t)(i < jq ? i : jq), hi = (uint64_t)(i < jq ? jq : i);
#pragma unroll
                for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                    if (j < nj && d <= se.K[j] && se.keys[j][q] == ki[j]) {
                        if (cnt[j] < se.cap[j]) se.raw[j][cnt[j]] = (lo << 32) | hi;
                        cnt[j]++;
                    }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAX_SHARED_BUCKETS; j++) {
        if (j >= nj) break;
        unsigned long long m = mb[j];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(FULL, m, o);
            m = v > m ? v : m;
        }
        if (lane == 0 && m) atomicMax(&se.counters[j][1], m);
    }
}

cudaError_t launch_bucket_emit_shared(const int32_t *lens, int64_t n, int64_t T, const uint32_t *next,
                                      const SharedEmit &se, cudaStream_t s) {
    const int64_t total = n * T;
    if (se.njoins < 1 || se.njoins > MAX_SHARED_BUCKETS) return cudaErrorInvalidValue;
    if (total > 0) {
        const int64_t g = (total + 255) / 256;
        bucket_emit_shared_kernel<<<(unsigned)(g > 32768 ? 32768 : g), 256, 0, s>>>(lens, n, T, next, se);
        note_launches(1);
    }
    return cudaGetLastError();
}

// Buckets of one table in shared memory (one block per table, n small enough
// for 16-bit record indices and the slots in shared memory). Slot h holds the
// first record of its signature (the owner, low 16 bits) and the head of the
// list of the later ones (high 16 bits); s_next links the list. Built with
// shared-memory atomics; then every listed record pairs with the owner and with
// the records after it in the list, which is every unordered pair of the bucket
// once. The pairs go to each join of `se` whose own signature and K they pass,
// as in bucket_emit_shared_kernel (se.keys[0] are the bucket signatures).
constexpr uint32_t TB_EMPTY = 0xFFFFFFFFu;
constexpr uint16_t TB_NONE = 0xFFFFu;   // end of a list
constexpr uint16_t TB_OWNER = 0xFFFEu;  // s_next of an owner

size_t bucket_table_smem(int64_t n) {
    if (n < 1 || n >= 0xFFFE) return 0;
    const uint64_t H = bucket_slots_per_table(n);
    const size_t bytes = (size_t)H * 5 + (((size_t)n * 2 + 15) & ~(size_t)15);
    return bytes <= 220 * 1024 ? bytes : 0;
}

// 8-bit fingerprint of a signature (1..255; 0 marks a slot whose owner has not
// written it yet): a probe that meets another signature's slot skips the
// comparison of the keys in global memory unless the fingerprints agree.
__device__ __forceinline__ uint8_t tb_fp(uint64_t kh) { return (uint8_t)((kh >> 56) | 1ull); }

__global__ void __launch_bounds__(1024)
bucket_table_kernel(const int32_t *__restrict__ lens, int64_t n, uint32_t H, SharedEmit se) {
    extern __shared__ uint32_t tb_smem[];
    uint32_t *slot = tb_smem;
    uint16_t *nxt = reinterpret_cast<uint16_t *>(tb_smem + H);
    uint8_t *fp = reinterpret_cast<uint8_t *>(nxt) + (((size_t)n * 2 + 15) & ~(size_t)15);   // [H]
    const int64_t t = blockIdx.x;
    const uint64_t *bk = se.keys[0] + t * n;
    const int lane = threadIdx.x & 31;
    const int nj = se.njoins;
    for (uint32_t h = threadIdx.x; h < H; h += blockDim.x) {
        slot[h] = TB_EMPTY;
        fp[h] = 0;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t k = bk[i];
        const uint64_t kh = key_hash(k);
        const uint8_t f = tb_fp(kh);
        nxt[i] = TB_OWNER;   // (kept if no slot were found, which H > n rules out)
        uint32_t h = (uint32_t)(kh & (uint64_t)(H - 1));
        for (uint32_t probe = 0; probe < H; probe++) {
            const uint32_t old = atomicCAS(&slot[h], TB_EMPTY, (uint32_t)i | ((uint32_t)TB_NONE << 16));
            if (old == TB_EMPTY) {
                fp[h] = f;
                break;
            }
            const uint8_t fo = fp[h];
            if ((fo == 0 || fo == f) && bk[old & 0xFFFFu] == k) {
                // a later record of this signature: push it onto the slot's list
                uint32_t cur = old, seen;
                while ((seen = atomicCAS(&slot[h], cur, (cur & 0xFFFFu) | ((uint32_t)i << 16))) != cur) cur = seen;
                nxt[i] = (uint16_t)(cur >> 16);
                break;
            }
            h = (h + 1) & (H - 1);
        }
    }
    __syncthreads();
    const int64_t iters = (n + blockDim.x - 1) / blockDim.x;   // the same on every lane
    unsigned long long mb[MAX_SHARED_BUCKETS];
#pragma unroll
    for (int j = 0; j < MAX_SHARED_BUCKETS; j++) mb[j] = 0;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t i = it * blockDim.x + threadIdx.x;
        uint32_t owner = TB_NONE;
        uint16_t q0 = TB_NONE;
        int32_t li = 0;
        unsigned long long cnt[MAX_SHARED_BUCKETS], same[MAX_SHARED_BUCKETS];
        uint64_t ki[MAX_SHARED_BUCKETS];
#pragma unroll
        for (int j = 0; j < MAX_SHARED_BUCKETS; j++) { cnt[j] = 0; same[j] = 0; ki[j] = 0; }
        if (i < n) {
            if (nxt[i] != TB_OWNER) {
                // a listed record: its owner (re-probe) and the list after it
                const uint64_t k = bk[i];
                const uint64_t kh = key_hash(k);
                const uint8_t f = tb_fp(kh);
                uint32_t h = (uint32_t)(kh & (uint64_t)(H - 1));
                for (uint32_t probe = 0; probe < H; probe++) {
                    const uint32_t v = slot[h];
                    if (v != TB_EMPTY && fp[h] == f && bk[v & 0xFFFFu] == k) {
                        owner = v & 0xFFFFu;
                        break;
                    }
                    h = (h + 1) & (H - 1);
                }
                q0 = owner < (uint32_t)n ? nxt[i] : TB_NONE;
                li = lens[i];
#pragma unroll
                for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                    if (j < nj) ki[j] = se.keys[j][t * n + i];
                // partners: the owner, then the list after i
                for (uint32_t q = owner; q < (uint32_t)n; q = (q == owner) ? q0 : nxt[q]) {
                    const int32_t lq = lens[q];
                    const int32_t d = li > lq ? li - lq : lq - li;
#pragma unroll
                    for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                        if (j < nj && se.keys[j][t * n + q] == ki[j]) {
                            same[j]++;
                            cnt[j] += d <= se.K[j] ? 1u : 0u;
                        }
                }
            }
#pragma unroll
            for (int j = 0; j < MAX_SHARED_BUCKETS; j++) mb[j] = max(mb[j], same[j] + 1);
        }
#pragma unroll
        for (int j = 0; j < MAX_SHARED_BUCKETS; j++) {
            if (j >= nj) break;
            unsigned long long incl = cnt[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned long long wtotal = __shfl_sync(FULL, incl, 31);
            unsigned long long base = 0;
            if (wtotal) {
                if (lane == 31) base = atomicAdd(&se.counters[j][0], wtotal);
                base = __shfl_sync(FULL, base, 31);
            }
            cnt[j] = base + incl - cnt[j];
        }
        if (owner != TB_NONE) {
            for (uint32_t q = owner; q < (uint32_t)n; q = (q == owner) ? q0 : nxt[q]) {
                const int32_t lq = lens[q];
                const int32_t d = li > lq ? li - lq : lq - li;
                const uint64_t lo = (uint64_t)(i < (int64_t)q ? i : (int64_t)q), hi = (uint64_t)(i < (int64_t)q ? (int64_t)q : i);
#pragma unroll
                for (int j = 0; j < MAX_SHARED_BUCKETS; j++)
                    if (j < nj && d <= se.K[j] && se.keys[j][t * n + q] == ki[j]) {
                        if (cnt[j] < se.cap[j]) se.raw[j][cnt[j]] = (lo << 32) | hi;
                        cnt[j]++;
                    }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAX_SHARED_BUCKETS; j++) {
        if (j >= nj) break;
        unsigned long long m = mb[j];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(FULL, m, o);
            m = v > m ? v : m;
        }
        if (lane == 0 && m) atomicMax(&se.counters[j][1], m);
    }
}

cudaError_t launch_bucket_table(const int32_t *lens, int64_t n, int64_t T, const SharedEmit &se, cudaStream_t s) {
    const size_t smem = bucket_table_smem(n);
    if (smem == 0 || se.njoins < 1 || se.njoins > MAX_SHARED_BUCKETS) return cudaErrorInvalidValue;
    if (n * T == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(bucket_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    bucket_table_kernel<<<(unsigned)T, 1024, smem, s>>>(lens, n, (uint32_t)bucket_slots_per_table(n), se);
    note_launches(1);
    return cudaGetLastError();
}

__device__ __forceinline__ uint64_t pair_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Insert raw pairs into an open-addressing set of `hsize` (power of two,
// >= 2 * count) slots pre-filled with ~0; the first copy of every pair is
// appended to cand. counters: [0] raw count (read), [2] candidates (written).
__global__ void dedup_kernel(const uint64_t *__restrict__ raw, uint64_t cap, uint64_t *__restrict__ table,
                             uint64_t hsize, uint64_t *__restrict__ cand, unsigned long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nraw_all = counters[0];
    const int64_t nraw = (int64_t)(nraw_all < cap ? nraw_all : cap);
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (nraw + step - 1) / step;
    const uint64_t EMPTY = ~0ull;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t i = start + it * step;
        bool is_new = false;
        uint64_t key = 0;
        if (i < nraw) {
            key = raw[i];
            uint64_t h = pair_hash(key) & (hsize - 1);
            for (uint64_t probe = 0; probe < hsize; probe++) {
                const unsigned long long old = atomicCAS((unsigned long long *)&table[h], EMPTY, key);
                if (old == EMPTY) {
                    is_new = true;
                    break;
                }
                if (old == key) break;
                h = (h + 1) & (hsize - 1);
            }
        }
        const unsigned mask = __ballot_sync(FULL, is_new);
        unsigned long long base = 0;
        if (mask) {
            if (lane == 0) base = atomicAdd(&counters[2], (unsigned long long)__popc(mask));
            base = __shfl_sync(FULL, base, 0);
        }
        if (is_new) cand[base + __popc(mask & ((1u << lane) - 1u))] = key;
    }
}

cudaError_t launch_dedup(const uint64_t *raw, uint64_t cap, uint64_t *table, uint64_t hsize, uint64_t *cand,
                         unsigned long long *counters, cudaStream_t s) {
    int64_t g = ((int64_t)cap + 255) / 256;
    dedup_kernel<<<(unsigned)(g > 8192 ? 8192 : (g ? g : 1)), 256, 0, s>>>(raw, cap, table, hsize, cand, counters);
    note_launches(1);
    return cudaGetLastError();
}

// Same insertion, without appending: hcount[slot] counts the copies of each
// pair, i.e. the number of (embedding, function) tables in which the two
// strings collided. counters: [0] raw count (read).
__global__ void dedup_count_kernel(const uint64_t *__restrict__ raw, uint64_t cap, uint64_t *__restrict__ table,
                                   uint32_t *__restrict__ hcount, uint64_t hsize,
                                   const unsigned long long *__restrict__ counters) {
    const unsigned long long nraw_all = counters[0];
    const int64_t nraw = (int64_t)(nraw_all < cap ? nraw_all : cap);
    const uint64_t EMPTY = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nraw; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = raw[i];
        uint64_t h = pair_hash(key) & (hsize - 1);
        for (uint64_t probe = 0; probe < hsize; probe++) {
            const unsigned long long old = atomicCAS((unsigned long long *)&table[h], EMPTY, key);
            if (old == EMPTY || old == key) {
                atomicAdd(&hcount[h], 1u);
                break;
            }
            h = (h + 1) & (hsize - 1);
        }
    }
}

constexpr int COUNT_BINS = 256;

// Queue bin of a candidate: its collision count, or (lens set) its length
// class, the shorter string's length scaled to 0..255 (both: higher bins first).
__device__ __forceinline__ uint32_t order_bin(uint64_t key, uint32_t count, const int32_t *__restrict__ lens,
                                              uint32_t len_scale) {
    if (!lens) return count < COUNT_BINS ? count : COUNT_BINS - 1;
    const int32_t a = lens[key >> 32], b = lens[key & 0xFFFFFFFFull];
    const uint32_t sh = (uint32_t)(a < b ? a : b);
    const uint64_t c = ((uint64_t)sh * COUNT_BINS) / ((uint64_t)len_scale + 1);
    return c < COUNT_BINS ? (uint32_t)c : COUNT_BINS - 1;
}

// bins[bin] += 1 over the occupied slots; counters[2] = pairs.
__global__ void count_hist_kernel(const uint64_t *__restrict__ table, const uint32_t *__restrict__ hcount,
                                  uint64_t hsize, const int32_t *__restrict__ lens, uint32_t len_scale,
                                  unsigned long long *__restrict__ bins,
                                  unsigned long long *__restrict__ counters) {
    __shared__ unsigned int sb[COUNT_BINS];
    for (int t = threadIdx.x; t < COUNT_BINS; t += blockDim.x) sb[t] = 0;
    __syncthreads();
    unsigned int mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) {
            atomicAdd(&sb[order_bin(key, hcount[i], lens, len_scale)], 1u);
            mine++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&counters[2], (unsigned long long)mine);
    __syncthreads();
    for (int t = threadIdx.x; t < COUNT_BINS; t += blockDim.x)
        if (sb[t]) atomicAdd(&bins[t], (unsigned long long)sb[t]);
}

// bins -> start offsets, highest bin first (in place); one block of COUNT_BINS
// threads, thread t owning bin COUNT_BINS-1-t (a shared-memory scan).
__global__ void count_scan_kernel(unsigned long long *__restrict__ bins) {
    __shared__ unsigned long long sc[COUNT_BINS];
    const int t = threadIdx.x;
    const unsigned long long own = bins[COUNT_BINS - 1 - t];
    sc[t] = own;
    __syncthreads();
    for (int o = 1; o < COUNT_BINS; o <<= 1) {
        const unsigned long long v = t >= o ? sc[t - o] : 0ull;
        __syncthreads();
        sc[t] += v;
        __syncthreads();
    }
    bins[COUNT_BINS - 1 - t] = sc[t] - own;
}

__global__ void count_scatter_kernel(const uint64_t *__restrict__ table, const uint32_t *__restrict__ hcount,
                                     uint64_t hsize, const int32_t *__restrict__ lens, uint32_t len_scale,
                                     unsigned long long *__restrict__ cursor, uint64_t *__restrict__ cand) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) cand[atomicAdd(&cursor[order_bin(key, hcount[i], lens, len_scale)], 1ull)] = key;
    }
}

// Order by the pair's first string (a counting sort on i of (i << 32 | j)):
// consecutive candidates share their first string, so a warp's pairs read the
// same string and, through the length filter, have similar lengths.
// With lens, the bin is the pair's longer string instead (the first one on a
// tie).
__device__ __forceinline__ uint64_t first_bin(uint64_t key, const int32_t *__restrict__ lens) {
    const uint64_t a = key >> 32, b = key & 0xFFFFFFFFull;
    if (!lens) return a;
    return lens[a] >= lens[b] ? a : b;
}

__global__ void first_hist_kernel(const uint64_t *__restrict__ table, uint64_t hsize, const int32_t *__restrict__ lens,
                                  uint32_t *__restrict__ bins, unsigned long long *__restrict__ counters) {
    unsigned int mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) {
            atomicAdd(&bins[first_bin(key, lens)], 1u);
            mine++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&counters[2], (unsigned long long)mine);
}

__global__ void first_scatter_kernel(const uint64_t *__restrict__ table, uint64_t hsize, const int32_t *__restrict__ lens,
                                     unsigned long long *__restrict__ cursor, uint64_t *__restrict__ cand) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) cand[atomicAdd(&cursor[first_bin(key, lens)], 1ull)] = key;
    }
}

cudaError_t launch_dedup_by_first(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                  int64_t n, uint32_t *bins, uint64_t *starts, void *scan_tmp, uint64_t *cand,
                                  unsigned long long *counters, cudaStream_t s, const int32_t *longer_lens) {
    int64_t g = ((int64_t)cap + 255) / 256;
    dedup_count_kernel<<<(unsigned)(g > 8192 ? 8192 : (g ? g : 1)), 256, 0, s>>>(raw, cap, table, hcount, hsize, counters);
    int64_t gh = ((int64_t)hsize + 255) / 256;
    const unsigned gs = (unsigned)(gh > 2048 ? 2048 : (gh ? gh : 1));
    first_hist_kernel<<<gs, 256, 0, s>>>(table, hsize, longer_lens, bins, counters);
    note_launches(2);
    cudaError_t e = exclusive_scan_u32(bins, starts, n + 1, nullptr, scan_tmp, s);
    if (e != cudaSuccess) return e;
    first_scatter_kernel<<<gs, 256, 0, s>>>(table, hsize, longer_lens, (unsigned long long *)starts, cand);
    note_launches(1);
    return cudaGetLastError();
}

int count_bins() { return COUNT_BINS; }

// ---------------------------------------------------------------------------
// Deduplication by sorting, grouped for the shared-string verifier
// ---------------------------------------------------------------------------
// Raw pair (i << 32 | j) -> key x << (cb + yb) | class << yb | y with x the
// longer string (the first on a tie), y the other and class the length
// difference's class, for the raw pairs a[0 .. min(counters[0], cap)).
__global__ void group_key_kernel(uint64_t *__restrict__ a, uint64_t cap, const unsigned long long *__restrict__ counters,
                                 const int32_t *__restrict__ lens, uint32_t yb, uint32_t cb, uint32_t nclass,
                                 uint32_t width) {
    const unsigned long long nraw_all = counters[0];
    const uint64_t nraw = nraw_all < cap ? nraw_all : cap;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nraw; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = a[e], i = v >> 32, j = v & 0xFFFFFFFFull;
        const int32_t li = lens[i], lj = lens[j];
        const bool i_long = li >= lj;
        const uint64_t x = i_long ? i : j, y = i_long ? j : i;
        uint32_t c = (uint32_t)(i_long ? li - lj : lj - li) / width;
        c = c < nclass ? c : nclass - 1u;
        a[e] = (x << (cb + yb)) | ((uint64_t)c << yb) | y;
    }
}

// flags[e] = 1 for the first key of each run of equal keys among the first
// min(counters[0], cap) (0 past them)
__global__ void group_unique_kernel(const uint64_t *__restrict__ k, uint64_t cap,
                                    const unsigned long long *__restrict__ counters, uint8_t *__restrict__ flags) {
    const unsigned long long nraw_all = counters[0];
    const uint64_t nraw = nraw_all < cap ? nraw_all : cap;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cap; e += (uint64_t)gridDim.x * blockDim.x)
        flags[e] = (e < nraw && (e == 0 || k[e - 1] != k[e])) ? 1 : 0;
}

// The distinct keys back to pairs, in key order, at out[offs[e]]; per group
// g = x * nclass + class (< n * nclass) its count (warp-aggregated: a warp's
// keys are sorted, so its lanes of one group are consecutive) and, at the
// group's first key, its start.
__global__ void group_compact_kernel(const uint64_t *__restrict__ k, const uint8_t *__restrict__ flags,
                                     const uint64_t *__restrict__ offs, uint64_t cap, uint32_t yb, uint32_t cb,
                                     uint32_t nclass, uint64_t *__restrict__ out, uint32_t *__restrict__ bins,
                                     uint64_t *__restrict__ gstart) {
    const uint64_t ymask = (1ull << yb) - 1ull, cmask = (1ull << cb) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t base = e0 - (threadIdx.x & 31); base < cap; base += stride) {   // warp-uniform trip count
        const uint64_t e = base + (threadIdx.x & 31);
        const bool f = e < cap && flags[e];
        uint64_t g = ~0ull;
        if (f) {
            const uint64_t v = k[e];
            const uint64_t x = v >> (cb + yb), y = v & ymask;
            out[offs[e]] = x < y ? (x << 32 | y) : (y << 32 | x);
            g = x * nclass + ((v >> yb) & cmask);
            // the group's first distinct key: the key before it is in another group
            if (e == 0 || (k[e - 1] >> yb) != (v >> yb)) gstart[g] = offs[e];
        }
        const unsigned peers = __match_any_sync(FULL, g);
        if (f && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&bins[g], (unsigned)__popc(peers));
    }
}

// ends[g] = start + count of every group (read by the task builder where count > 0)
__global__ void group_ends_kernel(const uint32_t *__restrict__ bins, const uint64_t *__restrict__ gstart, int64_t nb,
                                  uint64_t *__restrict__ ends) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nb; g += (int64_t)gridDim.x * blockDim.x)
        ends[g] = bins[g] ? gstart[g] + bins[g] : 0ull;
}

size_t dedup_grouped_temp_bytes(uint64_t cap) {
    const size_t counts = radix_counts_len((int64_t)cap, 1);
    const size_t a = counts * 4, b = counts * 8;
    const size_t scan = scan_temp_bytes((int64_t)(counts > cap + 1 ? counts : cap + 1));
    const size_t flags = ((size_t)cap + 15) & ~(size_t)15;
    const size_t offs = ((size_t)cap + 1) * 8;
    return ((a + 15) & ~(size_t)15) + ((b + 15) & ~(size_t)15) + ((scan + 15) & ~(size_t)15) + flags + offs;
}

cudaError_t launch_dedup_grouped(uint64_t *raw, uint64_t *alt, uint64_t cap, int64_t n, const int32_t *lens,
                                 uint32_t nclass, uint32_t width, unsigned long long *counters, void *temp,
                                 uint32_t *bins, uint64_t *ends, uint64_t *gstart, uint64_t **cand_out,
                                 cudaStream_t s) {
    if (nclass < 1 || width < 1 || cap == 0) return cudaErrorInvalidValue;
    uint32_t yb = 1;
    while ((1ll << yb) < n) yb++;
    uint32_t cb = 0;
    while ((1u << cb) < nclass) cb++;
    const uint32_t bits = 2 * yb + cb;
    if (bits > 64) return cudaErrorInvalidValue;
    const int64_t nb = n * (int64_t)nclass;
    // carve the temporary area
    char *t = (char *)temp;
    const size_t counts = radix_counts_len((int64_t)cap, 1);
    RadixTemp rt;
    rt.counts = (uint32_t *)t;
    t += (counts * 4 + 15) & ~(size_t)15;
    rt.offsets = (uint64_t *)t;
    t += (counts * 8 + 15) & ~(size_t)15;
    rt.scan_temp = t;
    t += (scan_temp_bytes((int64_t)(counts > cap + 1 ? counts : cap + 1)) + 15) & ~(size_t)15;
    uint8_t *flags = (uint8_t *)t;
    t += ((size_t)cap + 15) & ~(size_t)15;
    uint64_t *offs = (uint64_t *)t;
    const int64_t g = (int64_t)((cap + 255) / 256);
    const unsigned gs = (unsigned)(g > 152 * 64 ? 152 * 64 : (g ? g : 1));
    group_key_kernel<<<gs, 256, 0, s>>>(raw, cap, counters, lens, yb, cb, nclass, width);
    note_launches(1);
    int shifts[8];
    int np = 0;
    for (uint32_t b = 0; b < bits; b += 8) shifts[np++] = (int)b;
    bool in_alt = false;
    cudaError_t e = radix_sort_segmented(raw, nullptr, alt, nullptr, (int64_t)cap, 1, shifts, np, rt, &in_alt, s,
                                         counters);   // the raw count, read on the device
    if (e != cudaSuccess) return e;
    uint64_t *keys = in_alt ? alt : raw, *out = in_alt ? raw : alt;
    group_unique_kernel<<<gs, 256, 0, s>>>(keys, cap, counters, flags);
    note_launches(1);
    if ((e = exclusive_scan_u8(flags, offs, (int64_t)cap, (uint64_t *)&counters[2], rt.scan_temp, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(bins, 0, (size_t)(nb + 1) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    group_compact_kernel<<<gs, 256, 0, s>>>(keys, flags, offs, cap, yb, cb, nclass, out, bins, gstart);
    const int64_t gg = (nb + 255) / 256;
    group_ends_kernel<<<(unsigned)(gg > 4096 ? 4096 : (gg ? gg : 1)), 256, 0, s>>>(bins, gstart, nb, ends);
    note_launches(2);
    *cand_out = out;
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Union of the candidate lists of a merged verifier launch
// ---------------------------------------------------------------------------

// Every candidate of every join into one pair set; tmask[slot] collects the
// bits of the joins that list the pair.
__global__ void union_insert_kernel(const VerifySeg *__restrict__ segs, int nseg, uint64_t *__restrict__ table,
                                    uint32_t *__restrict__ tmask, uint64_t hsize) {
    const uint64_t EMPTY = ~0ull;
    for (int g = 0; g < nseg; g++) {
        const unsigned long long c = *segs[g].np_dev;
        const int64_t cnt = (int64_t)(c < segs[g].cap ? c : segs[g].cap);
        const uint64_t *pairs = segs[g].pairs;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
            const uint64_t key = pairs[i];
            uint64_t h = pair_hash(key) & (hsize - 1);
            for (uint64_t probe = 0; probe < hsize; probe++) {
                const unsigned long long old = atomicCAS((unsigned long long *)&table[h], EMPTY, key);
                if (old == EMPTY || old == key) {
                    atomicOr(&tmask[h], 1u << g);
                    break;
                }
                h = (h + 1) & (hsize - 1);
            }
        }
    }
}

// Queue bin of a union pair: 32 bins per number of listing joins (more joins
// first: a pair that passed the stricter signatures of several joins is the
// more likely to be similar, and a similar pair runs its full length), then the
// shorter string's length class (longer first); with length_major, the length
// class first and the number of joins within it.
__device__ __forceinline__ uint32_t union_bin(uint64_t key, uint32_t mask, const int32_t *__restrict__ lens,
                                              uint32_t len_scale, bool length_major) {
    const int32_t a = lens[key >> 32], b = lens[key & 0xFFFFFFFFull];
    const uint32_t sh = (uint32_t)(a < b ? a : b);
    const uint64_t c = ((uint64_t)sh * 32) / ((uint64_t)len_scale + 1);
    const uint32_t cls = c < 32 ? (uint32_t)c : 31u;
    const uint32_t j = (uint32_t)__popc(mask);
    const uint32_t jb = (j > 8 ? 8u : j) - 1u;   // mask != 0 for an occupied slot
    return length_major ? cls * 8u + jb : jb * 32u + cls;
}

__global__ void union_hist_kernel(const uint64_t *__restrict__ table, const uint32_t *__restrict__ tmask,
                                  uint64_t hsize, const int32_t *__restrict__ lens, uint32_t len_scale,
                                  bool length_major, unsigned long long *__restrict__ bins,
                                  unsigned long long *__restrict__ ucount) {
    __shared__ unsigned int sb[COUNT_BINS];
    for (int t = threadIdx.x; t < COUNT_BINS; t += blockDim.x) sb[t] = 0;
    __syncthreads();
    unsigned int mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) {
            atomicAdd(&sb[union_bin(key, tmask[i], lens, len_scale, length_major)], 1u);
            mine++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(ucount, (unsigned long long)mine);
    __syncthreads();
    for (int t = threadIdx.x; t < COUNT_BINS; t += blockDim.x)
        if (sb[t]) atomicAdd(&bins[t], (unsigned long long)sb[t]);
}

__global__ void union_scatter_kernel(const uint64_t *__restrict__ table, const uint32_t *__restrict__ tmask,
                                     uint64_t hsize, const int32_t *__restrict__ lens, uint32_t len_scale,
                                     bool length_major, unsigned long long *__restrict__ cursor,
                                     uint64_t *__restrict__ upairs, uint32_t *__restrict__ umask) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) {
            const uint32_t mk = tmask[i];
            const unsigned long long at = atomicAdd(&cursor[union_bin(key, mk, lens, len_scale, length_major)], 1ull);
            upairs[at] = key;
            umask[at] = mk;
        }
    }
}

cudaError_t launch_union_candidates(const VerifySeg *segs, int nseg, uint64_t *table, uint32_t *tmask, uint64_t hsize,
                                    unsigned long long *bins, uint64_t *upairs, uint32_t *umask,
                                    unsigned long long *ucount, const int32_t *lens, int64_t max_len,
                                    bool length_major, cudaStream_t s) {
    if (nseg < 1 || nseg > MAX_VERIFY_SEGS || (hsize & (hsize - 1)) != 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(table, 0xFF, hsize * sizeof(uint64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(tmask, 0, hsize * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bins, 0, COUNT_BINS * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ucount, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    const int64_t gh = ((int64_t)hsize + 255) / 256;
    const unsigned gs = (unsigned)(gh > 2048 ? 2048 : (gh ? gh : 1));
    const uint32_t scale = (uint32_t)(max_len > 0x7fffffff ? 0x7fffffff : max_len);
    union_insert_kernel<<<gs, 256, 0, s>>>(segs, nseg, table, tmask, hsize);
    union_hist_kernel<<<gs, 256, 0, s>>>(table, tmask, hsize, lens, scale, length_major, bins, ucount);
    count_scan_kernel<<<1, COUNT_BINS, 0, s>>>(bins);
    union_scatter_kernel<<<gs, 256, 0, s>>>(table, tmask, hsize, lens, scale, length_major, bins, upairs, umask);
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_dedup_ordered(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                 unsigned long long *bins, uint64_t *cand, unsigned long long *counters,
                                 const int32_t *lens, int64_t max_len, cudaStream_t s) {
    int64_t g = ((int64_t)cap + 255) / 256;
    dedup_count_kernel<<<(unsigned)(g > 8192 ? 8192 : (g ? g : 1)), 256, 0, s>>>(raw, cap, table, hcount, hsize, counters);
    int64_t gh = ((int64_t)hsize + 255) / 256;
    const unsigned gs = (unsigned)(gh > 2048 ? 2048 : (gh ? gh : 1));
    const uint32_t scale = (uint32_t)(max_len > 0x7fffffff ? 0x7fffffff : max_len);
    count_hist_kernel<<<gs, 256, 0, s>>>(table, hcount, hsize, lens, scale, bins, counters);
    count_scan_kernel<<<1, COUNT_BINS, 0, s>>>(bins);
    count_scatter_kernel<<<gs, 256, 0, s>>>(table, hcount, hsize, lens, scale, bins, cand);
    note_launches(4);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Search against a resident index (query x index pairs)
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Index buckets (the per-table grouping of equal signatures of Alg. 3, kept
// resident for search): the records of table t are sorted by signature, ties by
// (length, id), and stored as rec[t*n + p] = (len << 32) | id. A bucket is the
// run [start, end) of one signature; table t's open-addressing set (slots
// [t*H, (t+1)*H)) maps the signature to its run. The length filter
// ||s_q| - |s_i|| <= K is then a sub-run found by binary search, so a probe costs
// O(log bucket) plus what it emits, however large the bucket.
// ---------------------------------------------------------------------------

// Records and run starts: rk/rid are the sorted signatures and ids ([T][n]).
// slot_keys pre-filled with ~0 (never a signature).
__global__ void index_runs_kernel(const uint64_t *__restrict__ rk, const uint32_t *__restrict__ rid,
                                  const int32_t *__restrict__ lens, int64_t n, int64_t T, uint64_t H,
                                  uint64_t *__restrict__ slot_keys, uint2 *__restrict__ runs,
                                  uint64_t *__restrict__ rec, uint32_t *__restrict__ err) {
    const int64_t total = n * T;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g / n, p = g - t * n;
        const uint32_t id = rid[g];
        rec[g] = ((uint64_t)(uint32_t)lens[id] << 32) | id;
        const uint64_t key = rk[g];
        if (p > 0 && rk[g - 1] == key) continue;
        uint64_t *sk = slot_keys + t * H;
        uint64_t h = key_hash(key) & (H - 1);
        bool placed = false;
        for (uint64_t probe = 0; probe < H; probe++) {
            const unsigned long long old = atomicCAS((unsigned long long *)&sk[h], ~0ull, key);
            if (old == ~0ull) {   // each signature starts exactly one run: never found already present
                runs[t * H + h].x = (uint32_t)p;
                placed = true;
                break;
            }
            h = (h + 1) & (H - 1);
        }
        if (!placed) atomicOr(err, (uint32_t)DERR_GUARD);   // cannot happen with H > n
    }
}

// Run ends: the last record of each run finds its signature's slot.
__global__ void index_run_ends_kernel(const uint64_t *__restrict__ rk, int64_t n, int64_t T, uint64_t H,
                                      const uint64_t *__restrict__ slot_keys, uint2 *__restrict__ runs,
                                      uint32_t *__restrict__ err) {
    const int64_t total = n * T;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g / n, p = g - t * n;
        const uint64_t key = rk[g];
        if (p + 1 < n && rk[g + 1] == key) continue;
        const uint64_t *sk = slot_keys + t * H;
        uint64_t h = key_hash(key) & (H - 1);
        bool found = false;
        for (uint64_t probe = 0; probe < H; probe++) {
            const uint64_t v = sk[h];
            if (v == key) {
                runs[t * H + h].y = (uint32_t)(p + 1);
                found = true;
                break;
            }
            if (v == ~0ull) break;
            h = (h + 1) & (H - 1);
        }
        if (!found) atomicOr(err, (uint32_t)DERR_GUARD);
    }
}

cudaError_t launch_index_runs(const uint64_t *rk, const uint32_t *rid, const int32_t *lens, int64_t n, int64_t T,
                              uint64_t H, uint64_t *slot_keys, uint2 *runs, uint64_t *rec, uint32_t *err,
                              cudaStream_t s) {
    const int64_t total = n * T;
    if (total == 0) return cudaSuccess;
    const int64_t g = (total + 255) / 256;
    const unsigned grid = (unsigned)(g > 65536 ? 65536 : g);
    index_runs_kernel<<<grid, 256, 0, s>>>(rk, rid, lens, n, T, H, slot_keys, runs, rec, err);
    index_run_ends_kernel<<<grid, 256, 0, s>>>(rk, n, T, H, slot_keys, runs, err);
    note_launches(2);
    return cudaGetLastError();
}

// First p in [lo, hi) with rec[p] >= v (rec ascending on the run).
__device__ __forceinline__ uint32_t run_lower_bound(const uint64_t *__restrict__ rec, uint32_t lo, uint32_t hi,
                                                    uint64_t v) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(rec + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// For every (table t, query q): the index records that carry q's signature in
// table t and pass |len_q - len_i| <= K_q, as pairs (q << 32 | i). Each lane
// finds its sub-run; the warp then writes the sub-runs one after another,
// 32 consecutive pairs at a time. counters: [0] raw pairs (may exceed cap),
// [1] largest bucket met.
__global__ void index_probe_kernel(const uint64_t *__restrict__ qkeys, int64_t Q, int64_t T,
                                   const int32_t *__restrict__ qlens, const int32_t *__restrict__ qK,
                                   const uint64_t *__restrict__ slot_keys, const uint2 *__restrict__ runs,
                                   uint64_t H, const uint64_t *__restrict__ rec, int64_t n,
                                   uint64_t *__restrict__ raw, uint64_t cap, unsigned long long *__restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const int64_t total = Q * T;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (total + step - 1) / step;   // the same on every lane: collectives converge
    unsigned long long mb = 0;
    for (int64_t it = 0; it < iters; it++) {
        const int64_t idx = start + it * step;
        int64_t q = 0;
        const uint64_t *trec = rec;
        uint32_t lo = 0, cnt = 0;
        if (idx < total) {
            const int64_t t = idx / Q;
            q = idx - t * Q;
            trec = rec + t * n;
            const int64_t lq = qlens[q], kq = qK[q];
            const uint64_t key = qkeys[idx];
            const uint64_t *sk = slot_keys + t * H;
            uint64_t h = key_hash(key) & (H - 1);
            for (uint64_t probe = 0; probe < H; probe++) {
                const uint64_t v = sk[h];
                if (v == key) {
                    const uint2 run = runs[t * H + h];
                    mb = max(mb, (unsigned long long)(run.y - run.x));
                    const int64_t lmin = lq - kq, lmax = lq + kq;   // lengths are < 2^31
                    const uint64_t vlo = lmin > 0 ? (uint64_t)lmin << 32 : 0ull;
                    const uint64_t vhi = (uint64_t)(lmax + 1) << 32;
                    lo = run_lower_bound(trec, run.x, run.y, vlo);
                    cnt = run_lower_bound(trec, lo, run.y, vhi) - lo;
                    break;
                }
                if (v == ~0ull) break;
                h = (h + 1) & (H - 1);
            }
        }
        unsigned long long incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned long long wtotal = __shfl_sync(FULL, incl, 31);
        if (wtotal == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&counters[0], wtotal);
        base = __shfl_sync(FULL, base, 31);
        const unsigned long long mine = base + incl - cnt;
        unsigned todo = __ballot_sync(FULL, cnt > 0);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t c = __shfl_sync(FULL, cnt, l), first = __shfl_sync(FULL, lo, l);
            const unsigned long long ob = __shfl_sync(FULL, mine, l);
            const uint64_t hi_word = (uint64_t)__shfl_sync(FULL, (unsigned long long)q, l) << 32;
            const uint64_t *src = (const uint64_t *)__shfl_sync(FULL, (unsigned long long)trec, l) + first;
            for (uint32_t k = lane; k < c; k += 32)
                if (ob + k < cap) raw[ob + k] = hi_word | (uint32_t)__ldg(src + k);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(FULL, mb, o);
        mb = v > mb ? v : mb;
    }
    if (lane == 0 && mb) atomicMax(&counters[1], mb);
}

cudaError_t launch_index_probe(const uint64_t *qkeys, int64_t Q, int64_t T, const int32_t *qlens, const int32_t *qK,
                               const uint64_t *slot_keys, const uint2 *runs, uint64_t H, const uint64_t *rec,
                               int64_t n, uint64_t *raw, uint64_t cap, unsigned long long *counters, cudaStream_t s) {
    const int64_t total = Q * T;
    if (total > 0) {
        const int64_t g = (total + 255) / 256;
        index_probe_kernel<<<(unsigned)(g > 32768 ? 32768 : g), 256, 0, s>>>(qkeys, Q, T, qlens, qK, slot_keys, runs,
                                                                              H, rec, n, raw, cap, counters);
        note_launches(1);
    }
    return cudaGetLastError();
}

// Dedup of query x index pairs, grouped by the verifier class of the query:
// bins[c] = pairs of class c, bins[nc + c] = their start in cand (classes in
// order), counters[2] = all pairs. bins (3*nc) and hcount start at zero.
__global__ void class_hist_kernel(const uint64_t *__restrict__ table, uint64_t hsize, const uint8_t *__restrict__ cls,
                                  unsigned long long *__restrict__ bins, unsigned long long *__restrict__ counters) {
    unsigned int mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) {
            atomicAdd(&bins[cls[key >> 32]], 1ull);
            mine++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&counters[2], (unsigned long long)mine);
}

__global__ void class_scan_kernel(unsigned long long *__restrict__ bins, int nc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long acc = 0;
        for (int c = 0; c < nc; c++) {
            bins[nc + c] = acc;       // start
            bins[2 * nc + c] = acc;   // cursor
            acc += bins[c];
        }
    }
}

__global__ void class_scatter_kernel(const uint64_t *__restrict__ table, uint64_t hsize,
                                     const uint8_t *__restrict__ cls, unsigned long long *__restrict__ cursor,
                                     uint64_t *__restrict__ cand) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)hsize; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = table[i];
        if (key != ~0ull) cand[atomicAdd(&cursor[cls[key >> 32]], 1ull)] = key;
    }
}

cudaError_t launch_dedup_classes(const uint64_t *raw, uint64_t cap, uint64_t *table, uint32_t *hcount, uint64_t hsize,
                                 const uint8_t *cls, int nc, unsigned long long *bins, uint64_t *cand,
                                 unsigned long long *counters, cudaStream_t s) {
    int64_t g = ((int64_t)cap + 255) / 256;
    dedup_count_kernel<<<(unsigned)(g > 8192 ? 8192 : (g ? g : 1)), 256, 0, s>>>(raw, cap, table, hcount, hsize, counters);
    int64_t gh = ((int64_t)hsize + 255) / 256;
    const unsigned gs = (unsigned)(gh > 2048 ? 2048 : (gh ? gh : 1));
    class_hist_kernel<<<gs, 256, 0, s>>>(table, hsize, cls, bins, counters);
    class_scan_kernel<<<1, 32, 0, s>>>(bins, nc);
    class_scatter_kernel<<<gs, 256, 0, s>>>(table, hsize, cls, bins + 2 * nc, cand);
    note_launches(4);
    return cudaGetLastError();
}

// Sorts up to SMALL_SORT_MAX uint64 keys in one block (bitonic network in
// shared memory); the count comes from the device. The stages whose compared
// elements lie 2j apart with 2j within one warp's segment of the array run back
// to back in that warp (warp syncs only); the others take the whole block.
constexpr int SMALL_SORT_MAX = 8192;

__global__ void __launch_bounds__(1024)
small_sort_kernel(uint64_t *__restrict__ a, const unsigned long long *__restrict__ count_dev, uint64_t n_cap) {
    __shared__ uint64_t s[SMALL_SORT_MAX];
    const unsigned long long c = *count_dev;
    if (c > n_cap) return;   // left for a larger sort
    const int n = (int)c;
    if (n < 2) return;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < n ? a[i] : ~0ull;
    __syncthreads();
    const int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int S = P / nwarp;   // elements of a warp's segment (a power of two)
    if (S < 2) S = 2;
    // compare-exchange of pair t of the stage (k, j): i has bit j clear, ixj = i + j
    auto cx = [&](int t, int k, int j) {
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int ixj = i + j;
        const uint64_t x = s[i], y = s[ixj];
        const bool up = (i & k) == 0;
        if ((x > y) == up) {
            s[i] = y;
            s[ixj] = x;
        }
    };
    for (int k = 2; k <= P; k <<= 1) {
        int j = k >> 1;
        for (; j >= S; j >>= 1) {   // across segments: the whole block
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) cx(t, k, j);
            __syncthreads();
        }
        if (j > 0 && w * S < P) {   // within segments: each warp its own
            const int seg_pairs = S >> 1, base_t = w * seg_pairs;
            for (; j > 0; j >>= 1) {
                for (int t = lane; t < seg_pairs; t += 32) cx(base_t + t, k, j);
                __syncwarp();
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = s[i];
}

int small_sort_max() { return SMALL_SORT_MAX; }

cudaError_t launch_small_sort(uint64_t *a, const unsigned long long *count_dev, uint64_t n_cap, cudaStream_t s) {
    small_sort_kernel<<<1, 1024, 0, s>>>(a, count_dev, n_cap > (uint64_t)SMALL_SORT_MAX ? SMALL_SORT_MAX : n_cap);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ej
