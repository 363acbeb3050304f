// Similarity search against a resident index, and a serving loop on top of it.
//
// The index is EmbedJoin's data structure kept on the device: the strings (packed
// codes), the random walk tables and sampled positions of its parameters, and,
// per (embedding, function) table, the signatures of every string grouped into
// buckets (the table's records sorted by signature, then length, and an
// open-addressing set mapping each signature to its run of records).
// A query q with threshold K_q follows Alg. 3 from the query's side: its own
// walk and signatures with the same tables (Alg. 1, Thm. 1), the index strings
// sharing a signature in any table and passing ||q| - |s|| <= K_q, dedup, and
// the exact test ED(q, s) <= K_q (Section 3.3). The paper has no serving
// counterpart; the join's steps are reused as they are.
//
// A search batch is issued on one stream without any host synchronisation:
// pack the queries, walk and sign, probe the buckets, dedup (grouped by the
// verifier's window class of each query's K), verify each class (its band is
// the class's largest K, each pair is decided with its own query's K), and copy
// the counters and the appended results to pinned host memory. The server keeps
// several such batches in flight on their own streams and forms a new batch
// from the requests waiting whenever a slot is free (continuous batching).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ej_internal.cuh"

using namespace ej;

namespace {

using Clock = std::chrono::steady_clock;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Grows (never shrinks) a device buffer, at least doubling it, so that growth
// (whose cudaFree synchronises the device) stays rare; contents are not kept.
cudaError_t dev_grow(DevBuf &b, size_t bytes, size_t *grown = nullptr) {
    if (bytes == 0) bytes = 16;
    if (b.p && bytes <= b.bytes) return cudaSuccess;
    if (b.p && bytes < 2 * b.bytes) bytes = 2 * b.bytes;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    const cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) {
        b.bytes = bytes;
        if (grown) *grown += bytes;
    }
    return e;
}

void dev_free(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b = DevBuf{};
}

template <class T>
T *P(const DevBuf &b) {
    return (T *)b.p;
}

int words_for(int32_t K) { return (2 * K + 1 + 63) / 64; }

#define SV(expr)                                              \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return e_;                     \
    } while (0)

}  // namespace

// ---------------------------------------------------------------------------
// Index
// ---------------------------------------------------------------------------

struct ej_index {
    int device = 0;
    ej_ctx *own = nullptr;   // private context holding the packed strings
    PackedSet set{};
    ej_params p{};
    std::vector<uint8_t> alphabet;
    uint8_t host_map[256];
    int64_t T = 0;
    uint64_t H = 0;
    bool use_table = false;
    DevBuf pos, tsym, spos, stag, next, skeys, runs, rec, err;
};

namespace {

void index_free(ej_index *x) {
    if (!x) return;
    for (DevBuf *b : {&x->pos, &x->tsym, &x->spos, &x->stag, &x->next, &x->skeys, &x->runs, &x->rec, &x->err})
        dev_free(*b);
    if (x->own) ej_destroy(x->own);
    delete x;
}

// ---------------------------------------------------------------------------
// One search batch in flight
// ---------------------------------------------------------------------------

struct Query {
    const uint8_t *bytes;
    int32_t len;
    int32_t K;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf in, qlens, ccnt, qpofs, scan, qpacked, qkeys, raw, table, hcount, bins, cand, app, cnt, derr, queue, tickets;
    void *h_in = nullptr;
    size_t h_in_bytes = 0;
    unsigned long long *h_out = nullptr;   // counters[8], error word, then the result prefix
    size_t h_out_entries = 0;
    uint64_t cap = 1 << 16;                // raw / candidate / output capacity
    // the batch
    int64_t Q = 0;
    size_t device_bytes = 0;
};

constexpr size_t kOutHead = 16;            // u64 words before the result prefix
constexpr size_t kPrefix = 1 << 16;        // results copied back with the counters

void slot_free(Slot &sl) {
    for (DevBuf *b : {&sl.in, &sl.qlens, &sl.ccnt, &sl.qpofs, &sl.scan, &sl.qpacked, &sl.qkeys, &sl.raw, &sl.table,
                      &sl.hcount, &sl.bins, &sl.cand, &sl.app, &sl.cnt, &sl.derr, &sl.queue, &sl.tickets})
        dev_free(*b);
    if (sl.h_in) cudaFreeHost(sl.h_in);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
    sl = Slot{};
}

cudaError_t slot_init(Slot &sl) {
    SV(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking));
    SV(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    SV(cudaMallocHost((void **)&sl.h_out, (kOutHead + kPrefix) * sizeof(unsigned long long)));
    sl.h_out_entries = kPrefix;
    return cudaSuccess;
}

uint64_t hsize_for(uint64_t cap) {
    uint64_t h = 1;
    while (h < 2 * cap) h <<= 1;
    return h;
}

// Device bytes a batch needs beyond what the slot holds (for admission).
size_t slot_growth(const Slot &sl, const ej_index &x, int64_t Q, int64_t total, uint64_t cap) {
    const int64_t chunk_bound = (total * x.set.B + 127) / 128 + Q + 1;
    const uint64_t hs = hsize_for(cap);
    const size_t need[] = {
        (size_t)total + (size_t)(Q + 1) * 8 + (size_t)Q * 5 + 64, (size_t)Q * 4, (size_t)(Q + 1) * 4,
        (size_t)(Q + 2) * 8, scan_temp_bytes(Q + 1), (size_t)chunk_bound * 16, (size_t)x.T * Q * 8, cap * 8,
        hs * 8, hs * 4, 0, cap * 8, cap * 8};
    const DevBuf *have[] = {&sl.in, &sl.qlens, &sl.ccnt, &sl.qpofs, &sl.scan, &sl.qpacked, &sl.qkeys, &sl.raw,
                            &sl.table, &sl.hcount, &sl.bins, &sl.cand, &sl.app};
    size_t g = 0;
    for (size_t i = 0; i < sizeof(need) / sizeof(need[0]); i++)
        if (need[i] > have[i]->bytes) g += need[i];
    return g;
}

// Sizes the slot's buffers (pinned staging and device scratch) for a batch of Q
// queries with `total` bytes and nc window classes at the slot's capacity.
cudaError_t slot_reserve(Slot &sl, const ej_index &x, int64_t Q, int64_t total, int nc) {
    const size_t in_bytes = (((size_t)total + 7) & ~(size_t)7) + (size_t)(Q + 1) * 8 + (size_t)Q * 5 + 64;
    if (in_bytes > sl.h_in_bytes) {
        const size_t want = std::max(in_bytes, 2 * sl.h_in_bytes);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        sl.h_in = nullptr;
        sl.h_in_bytes = 0;
        SV(cudaMallocHost(&sl.h_in, want));
        sl.h_in_bytes = want;
    }
    const uint64_t cap = sl.cap, hs = hsize_for(cap);
    const int64_t chunk_bound = (total * x.set.B + 127) / 128 + Q + 1;
    size_t grown = 0;
    SV(dev_grow(sl.in, in_bytes, &grown));
    SV(dev_grow(sl.qlens, (size_t)Q * 4, &grown));
    SV(dev_grow(sl.ccnt, (size_t)(Q + 1) * 4, &grown));
    SV(dev_grow(sl.qpofs, (size_t)(Q + 2) * 8, &grown));
    SV(dev_grow(sl.scan, scan_temp_bytes(Q + 1), &grown));
    SV(dev_grow(sl.qpacked, (size_t)chunk_bound * 16, &grown));
    SV(dev_grow(sl.qkeys, (size_t)x.T * Q * 8, &grown));
    SV(dev_grow(sl.raw, cap * 8, &grown));
    SV(dev_grow(sl.table, hs * 8, &grown));
    SV(dev_grow(sl.hcount, hs * 4, &grown));
    SV(dev_grow(sl.bins, (size_t)3 * nc * 8, &grown));
    SV(dev_grow(sl.cand, cap * 8, &grown));
    SV(dev_grow(sl.app, cap * 8, &grown));
    SV(dev_grow(sl.cnt, 8 * 8, &grown));
    SV(dev_grow(sl.derr, 16, &grown));
    SV(dev_grow(sl.queue, (size_t)nc * 8, &grown));
    SV(dev_grow(sl.tickets, (size_t)nc * SM_TICKETS * 4, &grown));
    sl.device_bytes += grown;
    return cudaSuccess;
}

// Issues the whole search of `qs` on the slot's stream (no host synchronisation)
// and records sl.done. Query bytes are copied into pinned staging first.
cudaError_t slot_launch(Slot &sl, const ej_index &x, const std::vector<Query> &qs) {
    const int64_t Q = (int64_t)qs.size();
    sl.Q = Q;
    int64_t total = 0;
    int32_t max_q = 0;
    for (const Query &q : qs) {
        total += q.len;
        max_q = std::max(max_q, q.len);
    }
    // window classes: W1 = words(K) + 1 per query, classes in increasing W1
    std::vector<int> w1s;
    for (const Query &q : qs) w1s.push_back(words_for(q.K) + 1);
    std::vector<int> cls_w1 = w1s;
    std::sort(cls_w1.begin(), cls_w1.end());
    cls_w1.erase(std::unique(cls_w1.begin(), cls_w1.end()), cls_w1.end());
    const int nc = (int)cls_w1.size();
    std::vector<int32_t> kband(nc, 0);
    std::vector<uint8_t> cls(Q);
    for (int64_t i = 0; i < Q; i++) {
        const int c = (int)(std::lower_bound(cls_w1.begin(), cls_w1.end(), w1s[i]) - cls_w1.begin());
        cls[i] = (uint8_t)c;
        kband[c] = std::max(kband[c], qs[i].K);
    }
    // pinned staging: bytes | offsets | K | class
    const size_t off_o = ((size_t)total + 7) & ~(size_t)7;
    const size_t off_k = off_o + (size_t)(Q + 1) * 8;
    const size_t off_c = off_k + (size_t)Q * 4;
    const size_t in_bytes = off_c + (size_t)Q + 64;
    SV(slot_reserve(sl, x, Q, total, nc));
    uint8_t *hb = (uint8_t *)sl.h_in;
    int64_t *ho = (int64_t *)(hb + off_o);
    int32_t *hk = (int32_t *)(hb + off_k);
    uint8_t *hc = hb + off_c;
    int64_t o = 0;
    for (int64_t i = 0; i < Q; i++) {
        ho[i] = o;
        if (qs[i].len) memcpy(hb + o, qs[i].bytes, (size_t)qs[i].len);
        o += qs[i].len;
        hk[i] = qs[i].K;
        hc[i] = cls[i];
    }
    ho[Q] = o;
    const uint64_t cap = sl.cap, hs = hsize_for(cap);
    const cudaStream_t s = sl.s;
    uint8_t *d_in = P<uint8_t>(sl.in);
    const uint8_t *qbytes = d_in;
    const int64_t *qoffs = (const int64_t *)(d_in + off_o);
    const int32_t *qK = (const int32_t *)(d_in + off_k);
    const uint8_t *qcls = d_in + off_c;
    unsigned long long *cnt = P<unsigned long long>(sl.cnt);
    uint32_t *derr = P<uint32_t>(sl.derr);
    unsigned long long *bins = P<unsigned long long>(sl.bins);
    SV(cudaMemcpyAsync(d_in, sl.h_in, in_bytes, cudaMemcpyHostToDevice, s));
    SV(cudaMemsetAsync(cnt, 0, 8 * 8, s));
    SV(cudaMemsetAsync(derr, 0, 16, s));
    SV(cudaMemsetAsync(sl.table.p, 0xFF, hs * 8, s));
    SV(cudaMemsetAsync(sl.hcount.p, 0, hs * 4, s));
    SV(cudaMemsetAsync(bins, 0, (size_t)3 * nc * 8, s));
    SV(cudaMemsetAsync(sl.queue.p, 0, (size_t)nc * 8, s));
    SV(cudaMemsetAsync(sl.tickets.p, 0, (size_t)nc * SM_TICKETS * 4, s));
    // pack, walk and sign the queries with the index's tables
    SV(launch_validate(qbytes, qoffs, Q, total, x.set.code_map, P<int32_t>(sl.qlens), derr,
                       (unsigned long long *)(derr + 2), s));
    SV(launch_chunk_counts(P<int32_t>(sl.qlens), Q, x.set.B, P<uint32_t>(sl.ccnt), s));
    SV(exclusive_scan_u32(P<uint32_t>(sl.ccnt), P<uint64_t>(sl.qpofs), Q + 1, nullptr, sl.scan.p, s));
    SV(launch_pack(qbytes, qoffs, P<int32_t>(sl.qlens), Q, total, x.set.code_map, x.set.B, P<uint64_t>(sl.qpofs),
                   P<uint4>(sl.qpacked), derr, s));
    SV(launch_embed_sign(P<uint4>(sl.qpacked), P<uint64_t>(sl.qpofs), P<int32_t>(sl.qlens), Q, x.p.r, x.p.m, x.p.z,
                         x.p.L, x.p.alphabet_size, x.set.B, P<uint32_t>(x.tsym),
                         x.use_table ? P<uint16_t>(x.next) : nullptr, P<uint32_t>(x.spos), P<uint32_t>(x.stag),
                         P<uint64_t>(sl.qkeys), s));
    // buckets -> pairs -> dedup by class
    SV(launch_index_probe(P<uint64_t>(sl.qkeys), Q, x.T, P<int32_t>(sl.qlens), qK, P<uint64_t>(x.skeys),
                          P<uint2>(x.runs), x.H, P<uint64_t>(x.rec), x.set.n, P<uint64_t>(sl.raw), cap, cnt, s));
    SV(launch_dedup_classes(P<uint64_t>(sl.raw), cap, P<uint64_t>(sl.table), P<uint32_t>(sl.hcount), hs, qcls, nc,
                            bins, P<uint64_t>(sl.cand), cnt, s));
    // verify, one launch per window class
    const uint32_t alpha = x.p.alphabet_size;
    const int64_t max_len = std::max<int64_t>(max_q, x.set.max_len);
    for (int c = 0; c < nc; c++) {
        VerifyOut vo{};
        vo.app = P<uint64_t>(sl.app);
        vo.app_count = cnt + 3;
        vo.app_cap = cap;
        vo.np_dev = bins + c;
        vo.err = derr;
        vo.work = cnt + 4;
        vo.queue = P<unsigned long long>(sl.queue) + c;
        vo.sm_tickets = P<unsigned int>(sl.tickets) + (size_t)c * SM_TICKETS;
        vo.packed_b = x.set.packed;
        vo.pofs_b = x.set.pofs;
        vo.lens_b = x.set.lens;
        vo.n_b = x.set.n;
        vo.thr = qK;
        vo.pairs_off_dev = bins + nc + c;
        const int W1 = pq_words(kband[c]);   // the persistent verifier's narrower band
        const int threads = W1 <= 12 ? pq_threads_for(W1, alpha) : 0;
        if (threads > 0) {
            SV(launch_verify_pq(W1, threads, 16, 1, P<uint4>(sl.qpacked), P<uint64_t>(sl.qpofs), x.set.B,
                                P<int32_t>(sl.qlens), Q, alpha, P<uint64_t>(sl.cand), (int64_t)cap, kband[c], vo, s));
        } else {
            const VerifyConfig vc = verify_pick(kband[c], alpha, max_len);
            if (vc.G < 4) return cudaErrorInvalidValue;   // the grouped verifier reads both string sets
            SV(launch_verify(vc, P<uint4>(sl.qpacked), P<uint64_t>(sl.qpofs), x.set.B, P<int32_t>(sl.qlens), Q, alpha,
                             P<uint64_t>(sl.cand), (int64_t)cap, kband[c], max_len, vo, s));
        }
    }
    // counters, error word and the first results back to the host
    SV(cudaMemcpyAsync(sl.h_out, cnt, 8 * 8, cudaMemcpyDeviceToHost, s));
    SV(cudaMemcpyAsync(sl.h_out + 8, derr, 16, cudaMemcpyDeviceToHost, s));
    const size_t pre = std::min<size_t>(cap, sl.h_out_entries);
    SV(cudaMemcpyAsync(sl.h_out + kOutHead, sl.app.p, pre * 8, cudaMemcpyDeviceToHost, s));
    SV(cudaEventRecord(sl.done, s));
    return cudaSuccess;
}

enum CollectStatus { COLLECT_OK = 0, COLLECT_RETRY = 1, COLLECT_ERROR = 2 };

// After sl.done: the sorted result pairs (q << 32 | index id) of the batch.
CollectStatus slot_collect(Slot &sl, std::vector<uint64_t> *pairs, std::string *why) {
    const unsigned long long *h = sl.h_out;
    const unsigned long long raw = h[0], nout = h[3];
    const uint32_t err = (uint32_t)(h[8] & 0xffffffffull);
    if (err & (DERR_OFFSETS | DERR_SYMBOL)) {
        *why = "a query failed validation";
        return COLLECT_ERROR;
    }
    if (err & DERR_TIMEOUT) {
        *why = "the persistent verifier gave up after its bound of loop passes";
        return COLLECT_ERROR;
    }
    if (err & (DERR_PAIR | DERR_GUARD)) {
        *why = "internal verifier error";
        return COLLECT_ERROR;
    }
    if (raw > sl.cap) {
        sl.cap = raw + raw / 4 + 1024;
        return COLLECT_RETRY;
    }
    pairs->resize(nout);
    const size_t pre = std::min<size_t>(std::min<size_t>(sl.cap, sl.h_out_entries), nout);
    if (pre) memcpy(pairs->data(), h + kOutHead, pre * 8);
    if (nout > pre) {
        if (cudaMemcpy(pairs->data() + pre, P<uint64_t>(sl.app) + pre, (nout - pre) * 8, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            *why = "result copy failed";
            return COLLECT_ERROR;
        }
    }
    std::sort(pairs->begin(), pairs->end());
    return COLLECT_OK;
}

bool valid_query(const ej_index &x, const uint8_t *q, int32_t len) {
    if (len < 0 || (len > 0 && !q)) return false;
    for (int32_t i = 0; i < len; i++)
        if (x.host_map[q[i]] == 255) return false;
    return true;
}

}  // namespace

extern "C" {

int ej_index_create(ej_ctx *ctx, const ej_strings *S, const ej_params *p, ej_index **out, void *stream) {
    if (!ctx || !out) return EJ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!S || !p) return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "NULL strings/params");
    int st = ctx_check_params(ctx, p);
    if (st != EJ_OK) return st;
    if (p->L == 0) return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "an index needs a fixed sampling range L > 0");
    if (S->n < 1) return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "an index needs at least one string");
    const int64_t T = (int64_t)p->r * p->m;
    if (S->n * T >= (int64_t)0xFFFFFFFFll) return ctx_fail(ctx, EJ_ERR_UNSUPPORTED, "index too large (n*r*m >= 2^32)");
    if (embed_sign_smem(p->alphabet_size, p->L, p->m, p->z) == 0)
        return ctx_fail(ctx, EJ_ERR_UNSUPPORTED, "the fused walk tables do not fit shared memory for these parameters");
    ej_index *x = new (std::nothrow) ej_index();
    if (!x) return EJ_ERR_OOM;
    x->device = ctx_device(ctx);
    cudaSetDevice(x->device);
    const cudaStream_t s = (cudaStream_t)stream;
    auto bail = [&](int code, const char *msg) {
        index_free(x);
        return ctx_fail(ctx, code, msg);
    };
    if ((st = ej_create(&x->own, x->device)) != EJ_OK) return bail(st, "context creation failed");
    x->p = *p;
    x->alphabet.assign(p->alphabet, p->alphabet + p->alphabet_size);
    x->p.alphabet = x->alphabet.data();
    memset(x->host_map, 255, sizeof x->host_map);
    for (uint32_t c = 0; c < p->alphabet_size; c++) x->host_map[p->alphabet[c]] = (uint8_t)c;
    if ((st = ctx_pack(x->own, S, &x->p, &x->set, stream)) != EJ_OK) {
        const std::string why = ej_last_error(x->own);
        index_free(x);
        return ctx_fail(ctx, st, why.c_str());
    }
    x->T = T;
    const uint32_t r = p->r, m = p->m, z = p->z, L = p->L, alpha = p->alphabet_size;
    x->use_table = embed_sign_uses_table(alpha, L);
    DevBuf keys;
    bool ok = dev_grow(x->pos, (size_t)r * m * z * 4) == cudaSuccess &&
              dev_grow(x->tsym, symbol_table_words(r, alpha, L) * 4) == cudaSuccess &&
              dev_grow(x->spos, (size_t)r * m * z * 4) == cudaSuccess &&
              dev_grow(x->stag, (size_t)r * m * z * 4) == cudaSuccess &&
              (!x->use_table || dev_grow(x->next, next_table_elems(r, alpha, L) * 2) == cudaSuccess) &&
              dev_grow(keys, (size_t)T * x->set.n * 8) == cudaSuccess;
    x->H = bucket_slots_per_table(x->set.n);
    ok = ok && dev_grow(x->skeys, (size_t)x->H * T * 8) == cudaSuccess &&
         dev_grow(x->runs, (size_t)x->H * T * 8) == cudaSuccess &&
         dev_grow(x->rec, (size_t)x->set.n * T * 8) == cudaSuccess && dev_grow(x->err, 16) == cudaSuccess;
    if (!ok) {
        dev_free(keys);
        return bail(EJ_ERR_OOM, "index allocation failed");
    }
    cudaError_t e = launch_positions(p->seed, r, m, z, L, nullptr, P<uint32_t>(x->pos), s);
    if (e == cudaSuccess)
        e = launch_symbol_table(p->seed, r, L, x->set.alphabet_dev, alpha, nullptr, 0, P<uint32_t>(x->tsym), s);
    if (e == cudaSuccess) e = launch_sort_samples(P<uint32_t>(x->pos), r, m, z, P<uint32_t>(x->spos), P<uint32_t>(x->stag), s);
    if (e == cudaSuccess && x->use_table) e = launch_next_table(P<uint32_t>(x->tsym), r, alpha, L, P<uint16_t>(x->next), s);
    if (e == cudaSuccess)
        e = launch_embed_sign(x->set.packed, x->set.pofs, x->set.lens, x->set.n, r, m, z, L, alpha, x->set.B,
                              P<uint32_t>(x->tsym), x->use_table ? P<uint16_t>(x->next) : nullptr,
                              P<uint32_t>(x->spos), P<uint32_t>(x->stag), P<uint64_t>(keys), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->skeys.p, 0xFF, x->skeys.bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->runs.p, 0, x->runs.bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(x->err.p, 0, 16, s);
    // records sorted by signature, then length, in a scratch context released below
    ej_ctx *scratch = nullptr;
    const uint64_t *rk = nullptr;
    const uint32_t *rid = nullptr;
    if (e == cudaSuccess && ej_create(&scratch, x->device) != EJ_OK) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && ctx_sorted_records(scratch, x->set, &x->p, P<uint64_t>(keys), &rk, &rid, s) != EJ_OK)
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = launch_index_runs(rk, rid, x->set.lens, x->set.n, T, x->H, P<uint64_t>(x->skeys), P<uint2>(x->runs),
                              P<uint64_t>(x->rec), P<uint32_t>(x->err), s);
    uint32_t herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, x->err.p, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (scratch) ej_destroy(scratch);
    dev_free(keys);
    if (e != cudaSuccess) return bail(EJ_ERR_CUDA, cudaGetErrorString(e));
    if (herr) return bail(EJ_ERR_CUDA, "index bucket insertion failed");
    *out = x;
    return EJ_OK;
}

void ej_index_destroy(ej_index *x) { index_free(x); }

int64_t ej_index_size(const ej_index *x) { return x ? x->set.n : 0; }

int ej_index_search(ej_ctx *ctx, ej_index *x, const ej_strings *queries, const int32_t *K, uint64_t *out,
                    int64_t capacity, int64_t *n_out, void *stream) {
    (void)stream;
    if (!ctx || !n_out) return EJ_ERR_INVALID_ARG;
    *n_out = 0;
    if (!x || !queries || (queries->n > 0 && (!K || !queries->offsets || !queries->bytes)) || queries->n < 0)
        return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "NULL index/queries/K");
    if (queries->n == 0) return EJ_OK;
    if (queries->n >= (1ll << 31)) return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "too many queries");
    if (!out && capacity > 0) return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "NULL out");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, queries->bytes) == cudaSuccess && pa.type == cudaMemoryTypeDevice)
        return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "queries are read from host memory");
    cudaGetLastError();
    std::vector<Query> qs((size_t)queries->n);
    for (int64_t i = 0; i < queries->n; i++) {
        const int64_t a = queries->offsets[i], b = queries->offsets[i + 1];
        if (a < 0 || b < a || b - a >= (1ll << 31) || K[i] < 0)
            return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "invalid query offsets or K");
        qs[(size_t)i] = Query{queries->bytes + a, (int32_t)(b - a), K[i]};
        if (!valid_query(*x, qs[(size_t)i].bytes, qs[(size_t)i].len))
            return ctx_fail(ctx, EJ_ERR_INVALID_ARG, "a query byte is not in the index's alphabet");
    }
    cudaSetDevice(x->device);
    Slot sl;
    cudaError_t e = slot_init(sl);
    std::vector<uint64_t> pairs;
    std::string why;
    CollectStatus cs = COLLECT_RETRY;
    for (int attempt = 0; e == cudaSuccess && cs == COLLECT_RETRY && attempt < 4; attempt++) {
        e = slot_launch(sl, *x, qs);
        if (e == cudaSuccess) e = cudaEventSynchronize(sl.done);
        if (e == cudaSuccess) cs = slot_collect(sl, &pairs, &why);
    }
    slot_free(sl);
    if (e != cudaSuccess) return ctx_fail(ctx, EJ_ERR_CUDA, cudaGetErrorString(e));
    if (cs != COLLECT_OK) return ctx_fail(ctx, EJ_ERR_CUDA, cs == COLLECT_RETRY ? "raw pairs kept growing" : why.c_str());
    *n_out = (int64_t)pairs.size();
    if ((int64_t)pairs.size() > capacity) {
        ctx_fail(ctx, EJ_ERR_CAPACITY, "output capacity exceeded");
        return EJ_ERR_CAPACITY;
    }
    if (!pairs.empty()) memcpy(out, pairs.data(), pairs.size() * 8);
    return EJ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Server: continuous batching over search slots
// ---------------------------------------------------------------------------

namespace {

struct Request {
    int64_t id = 0;
    std::vector<uint8_t> q;
    int32_t K = 0;
    Clock::time_point t_submit, t_launch, t_done;
    std::vector<uint32_t> matches;
    int32_t status = EJ_OK;
    bool done = false;
};

struct SlotState {
    Slot sl;
    bool busy = false;
    std::vector<int64_t> batch;   // request ids
};

}  // namespace

struct ej_server {
    ej_index *x = nullptr;
    ej_server_config cfg{};
    std::vector<SlotState> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> pending;
    std::deque<int64_t> completed;
    std::unordered_map<int64_t, Request> reqs;
    std::thread worker;
    std::atomic<bool> stop{false};
    int64_t next_id = 0;
    // statistics
    std::vector<double> lat_ms;
    int64_t batches = 0, batched_queries = 0, retries = 0, deferred = 0;
    size_t device_bytes = 0;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
    std::string last_error;
};

namespace {

void server_loop(ej_server *srv) {
    cudaSetDevice(srv->x->device);
    const ej_index &x = *srv->x;
    while (!srv->stop.load()) {
        bool did = false;
        // completions
        for (SlotState &ss : srv->slots) {
            if (!ss.busy || cudaEventQuery(ss.sl.done) != cudaSuccess) continue;
            std::vector<uint64_t> pairs;
            std::string why;
            const CollectStatus cs = slot_collect(ss.sl, &pairs, &why);
            did = true;
            if (cs == COLLECT_RETRY) {
                std::vector<Query> qs;
                {
                    std::lock_guard<std::mutex> lk(srv->mu);
                    for (int64_t id : ss.batch) {
                        Request &r = srv->reqs[id];
                        qs.push_back(Query{r.q.data(), (int32_t)r.q.size(), r.K});
                    }
                    srv->retries++;
                }
                if (slot_launch(ss.sl, x, qs) == cudaSuccess) continue;
                why = "relaunch failed";
            }
            const Clock::time_point now = Clock::now();
            std::lock_guard<std::mutex> lk(srv->mu);
            size_t k = 0;
            for (size_t qi = 0; qi < ss.batch.size(); qi++) {
                Request &r = srv->reqs[ss.batch[qi]];
                r.matches.clear();
                while (k < pairs.size() && (pairs[k] >> 32) == qi) r.matches.push_back((uint32_t)(pairs[k++] & 0xFFFFFFFFu));
                r.status = (cs == COLLECT_OK) ? EJ_OK : EJ_ERR_CUDA;
                r.t_done = now;
                r.done = true;
                srv->completed.push_back(r.id);
                srv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
                if (!srv->any) {
                    srv->t_first = r.t_submit;
                    srv->any = true;
                }
                srv->t_last = now;
            }
            if (cs == COLLECT_ERROR) srv->last_error = why;
            ss.busy = false;
            ss.batch.clear();
            srv->cv_done.notify_all();
        }
        // new batches on free slots
        for (SlotState &ss : srv->slots) {
            if (ss.busy) continue;
            std::vector<Query> qs;
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                if (srv->pending.empty()) break;
                int64_t bytes = 0;
                while (!srv->pending.empty() && (int64_t)qs.size() < srv->cfg.max_batch) {
                    Request &r = srv->reqs[srv->pending.front()];
                    if (!qs.empty() && bytes + (int64_t)r.q.size() > srv->cfg.max_batch_bytes) break;
                    bytes += (int64_t)r.q.size();
                    ss.batch.push_back(r.id);
                    qs.push_back(Query{r.q.data(), (int32_t)r.q.size(), r.K});
                    srv->pending.pop_front();
                }
            }
            // admission by free HBM: the slot may grow only into free memory and
            // within the budget. While other batches are in flight the batch waits;
            // with nothing in flight it is cut down, and a single query that still
            // does not fit fails with EJ_ERR_OOM rather than waiting forever.
            bool others_busy = false;
            for (const SlotState &o : srv->slots) others_busy = others_busy || o.busy;
            bool fits = false;
            for (;;) {
                int64_t total = 0;
                for (const Query &q : qs) total += q.len;
                const size_t growth = slot_growth(ss.sl, x, (int64_t)qs.size(), total, ss.sl.cap);
                size_t free_b = 0, total_b = 0;
                if (growth) cudaMemGetInfo(&free_b, &total_b);
                fits = growth == 0 || (growth + srv->cfg.hbm_reserve <= free_b &&
                                       (srv->cfg.hbm_budget == 0 ||
                                        srv->device_bytes + growth <= srv->cfg.hbm_budget));
                if (fits || others_busy || qs.size() <= 1) break;
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->pending.push_front(ss.batch.back());
                ss.batch.pop_back();
                qs.pop_back();
            }
            if (!fits && others_busy) {
                std::lock_guard<std::mutex> lk(srv->mu);
                for (auto it = ss.batch.rbegin(); it != ss.batch.rend(); ++it) srv->pending.push_front(*it);
                ss.batch.clear();
                srv->deferred++;
                break;
            }
            if (!fits) {
                std::lock_guard<std::mutex> lk(srv->mu);
                for (int64_t id : ss.batch) {
                    Request &r = srv->reqs[id];
                    r.status = EJ_ERR_OOM;
                    r.done = true;
                    r.t_done = Clock::now();
                    srv->completed.push_back(id);
                }
                srv->last_error = "query does not fit the server's HBM budget";
                ss.batch.clear();
                srv->cv_done.notify_all();
                did = true;
                continue;
            }
            const size_t before = ss.sl.device_bytes;
            const Clock::time_point now = Clock::now();
            const cudaError_t e = slot_launch(ss.sl, x, qs);
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->device_bytes += ss.sl.device_bytes - before;
            if (e != cudaSuccess) {
                for (int64_t id : ss.batch) {
                    Request &r = srv->reqs[id];
                    r.status = EJ_ERR_CUDA;
                    r.done = true;
                    r.t_done = Clock::now();
                    srv->completed.push_back(id);
                }
                srv->last_error = cudaGetErrorString(e);
                ss.batch.clear();
                srv->cv_done.notify_all();
            } else {
                for (int64_t id : ss.batch) srv->reqs[id].t_launch = now;
                ss.busy = true;
                srv->batches++;
                srv->batched_queries += (int64_t)ss.batch.size();
            }
            did = true;
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(srv->mu);
            bool busy = false;
            for (const SlotState &ss : srv->slots) busy = busy || ss.busy;
            if (busy)
                srv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(2),
                                      [&] { return srv->stop.load() || !srv->pending.empty(); });
        }
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int ej_server_create(ej_index *x, const ej_server_config *cfg, ej_server **out) {
    if (!x || !out) return EJ_ERR_INVALID_ARG;
    *out = nullptr;
    ej_server_config c{};
    if (cfg) c = *cfg;
    if (c.max_batch <= 0) c.max_batch = 256;
    if (c.inflight <= 0) c.inflight = 4;
    if (c.max_batch_bytes <= 0) c.max_batch_bytes = 8ll << 20;
    if (c.hbm_reserve == 0) c.hbm_reserve = 1ull << 30;
    if (c.max_batch > 65536 || c.inflight > 64) return EJ_ERR_INVALID_ARG;
    ej_server *srv = new (std::nothrow) ej_server();
    if (!srv) return EJ_ERR_OOM;
    srv->x = x;
    srv->cfg = c;
    cudaSetDevice(x->device);
    srv->slots.resize((size_t)c.inflight);
    // every slot sized up front for a full batch (max_batch queries, max_batch_bytes
    // bytes, up to 32 window classes), so that growth during serving is rare
    // (within the HBM budget, if one is set; beyond it slots grow on demand)
    for (SlotState &ss : srv->slots) {
        cudaError_t e = slot_init(ss.sl);
        // room for 2048 candidate pairs per query of a full batch before a retry
        ss.sl.cap = std::max<uint64_t>(ss.sl.cap, (uint64_t)c.max_batch * 2048);
        const size_t full = slot_growth(ss.sl, *x, c.max_batch, c.max_batch_bytes, ss.sl.cap);
        if (e == cudaSuccess && (c.hbm_budget == 0 || srv->device_bytes + full <= c.hbm_budget))
            e = slot_reserve(ss.sl, *x, c.max_batch, c.max_batch_bytes, 32);
        if (e != cudaSuccess) {
            for (SlotState &t : srv->slots) slot_free(t.sl);
            delete srv;
            return EJ_ERR_CUDA;
        }
        srv->device_bytes += ss.sl.device_bytes;
    }
    srv->worker = std::thread(server_loop, srv);
    *out = srv;
    return EJ_OK;
}

int64_t ej_server_submit(ej_server *srv, const uint8_t *query, int32_t len, int32_t K) {
    if (!srv || K < 0 || !valid_query(*srv->x, query, len)) return -(int64_t)EJ_ERR_INVALID_ARG;
    Request r;
    r.q.assign(query, query + len);
    r.K = K;
    r.t_submit = Clock::now();
    int64_t id;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        id = srv->next_id++;
        r.id = id;
        srv->reqs.emplace(id, std::move(r));
        srv->pending.push_back(id);
    }
    srv->cv_work.notify_one();
    return id;
}

int ej_server_poll(ej_server *srv, ej_search_result *out, int32_t max, int32_t *n, int32_t wait_us) {
    if (!srv || !n || (max > 0 && !out)) return EJ_ERR_INVALID_ARG;
    *n = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->completed.empty() && wait_us > 0)
        srv->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !srv->completed.empty(); });
    while (*n < max && !srv->completed.empty()) {
        Request &r = srv->reqs[srv->completed.front()];
        srv->completed.pop_front();
        ej_search_result &o = out[(*n)++];
        o.id = r.id;
        o.status = r.status;
        o.n_matches = (int32_t)r.matches.size();
        o.matches = r.matches.data();
        o.latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
        o.queue_ms = std::chrono::duration<double, std::milli>(r.t_launch - r.t_submit).count();
    }
    return EJ_OK;
}

int ej_server_release(ej_server *srv, int64_t id) {
    if (!srv) return EJ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end() || !it->second.done) return EJ_ERR_INVALID_ARG;
    srv->reqs.erase(it);
    return EJ_OK;
}

int ej_server_get_stats(ej_server *srv, ej_server_stats *st) {
    if (!srv || !st) return EJ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    memset(st, 0, sizeof *st);
    st->completed = (int64_t)srv->lat_ms.size();
    st->batches = srv->batches;
    st->retries = srv->retries;
    st->deferred = srv->deferred;
    st->mean_batch = srv->batches ? (double)srv->batched_queries / (double)srv->batches : 0.0;
    st->p50_ms = percentile(srv->lat_ms, 0.50);
    st->p99_ms = percentile(srv->lat_ms, 0.99);
    double s = 0.0;
    for (double v : srv->lat_ms) s += v;
    st->mean_ms = srv->lat_ms.empty() ? 0.0 : s / (double)srv->lat_ms.size();
    const double span = srv->any ? std::chrono::duration<double>(srv->t_last - srv->t_first).count() : 0.0;
    st->queries_per_s = span > 0 ? (double)st->completed / span : 0.0;
    st->device_bytes = (uint64_t)srv->device_bytes;
    return EJ_OK;
}

int ej_server_reset_stats(ej_server *srv) {
    if (!srv) return EJ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->lat_ms.clear();
    srv->batches = srv->batched_queries = srv->retries = srv->deferred = 0;
    srv->any = false;
    return EJ_OK;
}

void ej_server_destroy(ej_server *srv) {
    if (!srv) return;
    srv->stop.store(true);
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->x->device);
    for (SlotState &ss : srv->slots) {
        if (ss.busy) cudaEventSynchronize(ss.sl.done);
        slot_free(ss.sl);
    }
    delete srv;
}

}  // extern "C"
