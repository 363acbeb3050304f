// Scan, segmented LSD radix sort and the bucket/pair stages of candidate
// generation (Algorithm 3's hash tables, length filter and deduplication,
// restated as sort + run-length windows).
#include "ej_internal.cuh"

namespace ej {

// ---------------------------------------------------------------------------
// Exclusive scan (three kernels: block reduce, scan of block sums, apply)
// ---------------------------------------------------------------------------

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

size_t scan_temp_bytes(int64_t n) {
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    return (size_t)(nb + 1) * sizeof(uint64_t);
}

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *total, uint64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (SCAN_THREADS / 32) ? s_warp[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SCAN_THREADS / 32) s_warp[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) s_warp[SCAN_THREADS / 32] = wi;
    }
    __syncthreads();
    const uint64_t res = s_warp[warp] + inc - v;
    *total = s_warp[SCAN_THREADS / 32];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_kernel(const T *__restrict__ in, int64_t n, uint64_t *__restrict__ block_sums) {
    __shared__ uint64_t s_warp[SCAN_THREADS / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    uint64_t sum = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int64_t i = base + (int64_t)it * SCAN_THREADS + threadIdx.x;
        if (i < n) sum += (uint64_t)in[i];
    }
    uint64_t tot;
    block_excl_scan(sum, &tot, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of nb block sums in place; total in sums[nb].
__global__ void __launch_bounds__(SCAN_THREADS)
scan_sums_kernel(uint64_t *__restrict__ sums, int64_t nb, uint64_t *__restrict__ total_dev) {
    __shared__ uint64_t s_warp[SCAN_THREADS / 32 + 1];
    uint64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_CHUNK) {
        uint64_t v[SCAN_ITEMS];
        uint64_t local = 0;
#pragma unroll
        for (int it = 0; it < SCAN_ITEMS; it++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + it;
            v[it] = i < nb ? sums[i] : 0;
            local += v[it];
        }
        uint64_t tot;
        uint64_t ex = block_excl_scan(local, &tot, s_warp);
        uint64_t run = carry + ex;
#pragma unroll
        for (int it = 0; it < SCAN_ITEMS; it++) {
            int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + it;
            if (i < nb) sums[i] = run;
            run += v[it];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        sums[nb] = carry;
        if (total_dev) *total_dev = carry;
    }
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_apply_kernel(const T *__restrict__ in, uint64_t *__restrict__ out, int64_t n,
                  const uint64_t *__restrict__ block_offs) {
    __shared__ uint64_t s_warp[SCAN_THREADS / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t local = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int64_t i = base + it;
        v[it] = i < n ? (uint64_t)in[i] : 0;
        local += v[it];
    }
    uint64_t tot;
    uint64_t run = block_offs[blockIdx.x] + block_excl_scan(local, &tot, s_warp);
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; it++) {
        int64_t i = base + it;
        if (i < n) out[i] = run;
        run += v[it];
    }
}

template <typename T>
static cudaError_t exclusive_scan(const T *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                                  void *temp, cudaStream_t s) {
    uint64_t *sums = (uint64_t *)temp;
    const int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb > 0) scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
    scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(sums, nb, total_dev);
    if (nb > 0) scan_apply_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    note_launches(nb > 0 ? 3 : 1);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u8(const uint8_t *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                              void *temp, cudaStream_t s) {
    return exclusive_scan<uint8_t>(in, out, n, total_dev, temp, s);
}
cudaError_t exclusive_scan_u32(const uint32_t *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                               void *temp, cudaStream_t s) {
    return exclusive_scan<uint32_t>(in, out, n, total_dev, temp, s);
}

// ---------------------------------------------------------------------------
// Segmented LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
//
// A tile of 4096 records belongs to one segment. Pass = histogram per tile ->
// one exclusive scan over counts laid out [segment][digit][tile] (so the scan
// result is each tile's absolute output offset per digit, segment bases
// included) -> stable scatter. In the scatter, warp w ranks records
// [w*512, (w+1)*512) of the tile round by round with __match_any_sync and a
// per-warp digit counter; a block-wide prefix over warps then orders the warps.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

size_t radix_counts_len(int64_t seg_len, int64_t nseg) {
    int64_t tps = (seg_len + RS_TILE - 1) / RS_TILE;
    return (size_t)(nseg * 256 * (tps ? tps : 1));
}

__global__ void __launch_bounds__(RS_THREADS)
radix_hist_kernel(const uint64_t *__restrict__ keys, int64_t seg_len, int tps, int shift,
                  uint32_t *__restrict__ counts, const unsigned long long *__restrict__ len_dev) {
    __shared__ uint32_t h[256];
    const int tile = blockIdx.x;
    const int64_t seg = blockIdx.y;
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t seg_base = seg * seg_len, tile_base = (int64_t)tile * RS_TILE;
    int64_t len = seg_len;   // records of the segment that take part
    if (len_dev) len = (int64_t)*len_dev < seg_len ? (int64_t)*len_dev : seg_len;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t e = tile_base + i;
        if (e < len) atomicAdd(&h[(uint32_t)(keys[seg_base + e] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    counts[(seg * 256 + threadIdx.x) * tps + tile] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS)
radix_scatter_kernel(const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                     uint64_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                     int64_t seg_len, int tps, int shift, const uint64_t *__restrict__ offsets,
                     const unsigned long long *__restrict__ len_dev) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint64_t s_off[256];
    const int tile = blockIdx.x;
    const int64_t seg = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t seg_base = seg * seg_len;
    const int64_t sub_base = (int64_t)tile * RS_TILE + (int64_t)warp * (RS_ITEMS * 32);
    int64_t len = seg_len;   // records of the segment that take part
    if (len_dev) len = (int64_t)*len_dev < seg_len ? (int64_t)*len_dev : seg_len;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) wcnt[w][threadIdx.x] = 0;
    s_off[threadIdx.x] = offsets[(seg * 256 + threadIdx.x) * tps + tile];
    __syncthreads();

    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t dig[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        const int64_t e = sub_base + it * 32 + lane;
        const bool ok = e < len;
        k[it] = ok ? keys_in[seg_base + e] : 0ull;
        v[it] = (ok && vals_in) ? vals_in[seg_base + e] : 0u;
        const uint32_t d = ok ? ((uint32_t)(k[it] >> shift) & 0xFFu) : 256u;
        dig[it] = d;
        const unsigned peers = __match_any_sync(FULL, d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && ok) {
            base = wcnt[warp][d];
            wcnt[warp][d] = base + __popc(peers);
        }
        base = __shfl_sync(FULL, base, leader);
        rank[it] = base + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t t = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; it++) {
        const uint32_t d = dig[it];
        if (d < 256u) {
            const uint64_t dst = s_off[d] + wcnt[warp][d] + rank[it];
            keys_out[dst] = k[it];
            if (vals_out) vals_out[dst] = v[it];
        }
    }
}

cudaError_t radix_sort_segmented(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                                 int64_t seg_len, int64_t nseg, const int *shifts, int npasses,
                                 RadixTemp tmp, bool *in_alt, cudaStream_t s, const unsigned long long *len_dev) {
    if (len_dev && nseg != 1) return cudaErrorInvalidValue;
    *in_alt = false;
    if (seg_len == 0 || nseg == 0 || npasses == 0) return cudaGetLastError();
    const int tps = (int)((seg_len + RS_TILE - 1) / RS_TILE);
    const int64_t ncounts = nseg * 256 * tps;
    dim3 grid(tps, (unsigned)nseg);
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < npasses; p++) {
        radix_hist_kernel<<<grid, RS_THREADS, 0, s>>>(ki, seg_len, tps, shifts[p], tmp.counts, len_dev);
        cudaError_t e = exclusive_scan_u32(tmp.counts, tmp.offsets, ncounts, nullptr, tmp.scan_temp, s);
        if (e != cudaSuccess) return e;
        radix_scatter_kernel<<<grid, RS_THREADS, 0, s>>>(ki, vi, ko, vo, seg_len, tps, shifts[p],
                                                         tmp.offsets, len_dev);
        note_launches(2);
        uint64_t *kt = ki; ki = ko; ko = kt;
        uint32_t *vt = vi; vi = vo; vo = vt;
        *in_alt = !*in_alt;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidate generation
// ---------------------------------------------------------------------------

static unsigned grid_for(int64_t total, int64_t cap) {
    int64_t g = (total + 255) / 256;
    return (unsigned)(g < cap ? (g > 0 ? g : 1) : cap);
}

__global__ void iota_kernel(uint32_t *v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}
cudaError_t launch_iota_u32(uint32_t *v, int64_t n, cudaStream_t s) {
    if (n > 0) iota_kernel<<<grid_for(n, 4096), 256, 0, s>>>(v, n);
    if (n > 0) note_launches(1);
    return cudaGetLastError();
}

__global__ void len_keys_kernel(const int32_t *lens, int64_t n, uint64_t *k) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        k[i] = (uint64_t)(uint32_t)lens[i];
}
cudaError_t launch_len_keys(const int32_t *lens, int64_t n, uint64_t *k, cudaStream_t s) {
    if (n > 0) len_keys_kernel<<<grid_for(n, 4096), 256, 0, s>>>(lens, n, k);
    if (n > 0) note_launches(1);
    return cudaGetLastError();
}

// rec_keys[t*n + p] = keys[t*n + perm[p]], rec_ids = perm[p]: every table's
// records start in (length, id) order, so the stable key sort that follows
// leaves each bucket ordered by length (the order Alg. 3 visits strings in).
__global__ void len_order_gather_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ perm,
                                        int64_t n, int64_t T, uint64_t *__restrict__ rk,
                                        uint32_t *__restrict__ rid) {
    const int64_t total = n * T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / n, p = i - t * n;
        const uint32_t id = perm[p];
        rk[i] = keys[t * n + id];
        rid[i] = id;
    }
}
cudaError_t launch_len_order_gather(const uint64_t *keys, const uint32_t *perm, int64_t n, int64_t T,
                                    uint64_t *rec_keys, uint32_t *rec_ids, cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0)
        len_order_gather_kernel<<<grid_for(total, 16384), 256, 0, s>>>(
            keys, perm, n, T, rec_keys, rec_ids);
    if (total > 0) note_launches(1);
    return cudaGetLastError();
}

// Within table t (records sorted by (key, length, id)), the partners of record
// p are the following records with the same key and length <= len_p + K: a
// contiguous window found by galloping then binary search.
__device__ __forceinline__ int64_t window_end(const uint64_t *__restrict__ rk, const uint32_t *__restrict__ rid,
                                              const int32_t *__restrict__ lens, int64_t p, int64_t n,
                                              uint64_t key, int64_t limit) {
    auto pred = [&](int64_t q) { return rk[q] == key && (int64_t)lens[rid[q]] <= limit; };
    if (p + 1 >= n || !pred(p + 1)) return p + 1;
    int64_t good = p + 1, step = 1;
    while (true) {
        int64_t nx = good + step;
        if (nx < n && pred(nx)) {
            good = nx;
            step <<= 1;
        } else {
            break;
        }
    }
    int64_t lo = good, hi = min(good + step, n);
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (pred(mid)) lo = mid; else hi = mid;
    }
    return lo + 1;
}

__device__ __forceinline__ int64_t run_end(const uint64_t *__restrict__ rk, int64_t p, int64_t n, uint64_t key) {
    int64_t good = p, step = 1;
    while (true) {
        int64_t nx = good + step;
        if (nx < n && rk[nx] == key) {
            good = nx;
            step <<= 1;
        } else {
            break;
        }
    }
    int64_t lo = good, hi = min(good + step, n);
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (rk[mid] == key) lo = mid; else hi = mid;
    }
    return lo + 1;
}

__global__ void bucket_count_kernel(const uint64_t *__restrict__ rec_keys, const uint32_t *__restrict__ rec_ids,
                                    const int32_t *__restrict__ lens, int64_t n, int64_t T, int32_t K,
                                    uint32_t *__restrict__ counts, unsigned long long *__restrict__ max_bucket) {
    const int64_t total = n * T;
    unsigned long long mb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / n, p = i - t * n;
        const uint64_t *rk = rec_keys + t * n;
        const uint32_t *rid = rec_ids + t * n;
        const uint64_t key = rk[p];
        const int64_t lim = (int64_t)lens[rid[p]] + K;
        const int64_t e = window_end(rk, rid, lens, p, n, key, lim);
        counts[i] = (uint32_t)(e - p - 1);
        if ((p == 0 || rk[p - 1] != key) && p + 1 < n && rk[p + 1] == key) {
            const int64_t re = run_end(rk, p, n, key);
            mb = max(mb, (unsigned long long)(re - p));
        }
    }
    if (mb) atomicMax(max_bucket, mb);
}
cudaError_t launch_bucket_count(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens,
                                int64_t n, int64_t T, int32_t K, uint32_t *counts,
                                unsigned long long *max_bucket, cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0)
        bucket_count_kernel<<<grid_for(total, 16384), 256, 0, s>>>(
            rec_keys, rec_ids, lens, n, T, K, counts, max_bucket);
    if (total > 0) note_launches(1);
    return cudaGetLastError();
}

__global__ void bucket_emit_kernel(const uint64_t *__restrict__ rec_keys, const uint32_t *__restrict__ rec_ids,
                                   const int32_t *__restrict__ lens, int64_t n, int64_t T, int32_t K,
                                   const uint64_t *__restrict__ offs, uint64_t *__restrict__ pairs) {
    const int64_t total = n * T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / n, p = i - t * n;
        const uint64_t *rk = rec_keys + t * n;
        const uint32_t *rid = rec_ids + t * n;
        const uint64_t key = rk[p];
        const uint32_t a = rid[p];
        const int64_t lim = (int64_t)lens[a] + K;
        const int64_t e = window_end(rk, rid, lens, p, n, key, lim);
        uint64_t o = offs[i];
        for (int64_t q = p + 1; q < e; q++) {
            const uint32_t b = rid[q];
            const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            pairs[o++] = (lo << 32) | hi;
        }
    }
}
cudaError_t launch_bucket_emit(const uint64_t *rec_keys, const uint32_t *rec_ids, const int32_t *lens,
                               int64_t n, int64_t T, int32_t K, const uint64_t *offs,
                               uint64_t *pairs, cudaStream_t s) {
    const int64_t total = n * T;
    if (total > 0)
        bucket_emit_kernel<<<grid_for(total, 16384), 256, 0, s>>>(
            rec_keys, rec_ids, lens, n, T, K, offs, pairs);
    if (total > 0) note_launches(1);
    return cudaGetLastError();
}

__global__ void unique_flags_kernel(const uint64_t *__restrict__ a, int64_t n, uint8_t *__restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || a[i] != a[i - 1]) ? 1 : 0;
}
cudaError_t launch_unique_flags(const uint64_t *sorted, int64_t n, uint8_t *flags, cudaStream_t s) {
    if (n > 0) unique_flags_kernel<<<grid_for(n, 16384), 256, 0, s>>>(sorted, n, flags);
    if (n > 0) note_launches(1);
    return cudaGetLastError();
}

__global__ void compact_kernel(const uint64_t *__restrict__ in, const uint8_t *__restrict__ flags,
                               const uint64_t *__restrict__ offs, int64_t n, uint64_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i]) out[offs[i]] = in[i];
}
cudaError_t launch_compact_u64(const uint64_t *in, const uint8_t *flags, const uint64_t *offs,
                               int64_t n, uint64_t *out, cudaStream_t s) {
    if (n > 0) compact_kernel<<<grid_for(n, 16384), 256, 0, s>>>(in, flags, offs, n, out);
    if (n > 0) note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-table sort inside one block (tables that fit in shared memory)
// ---------------------------------------------------------------------------
//
// Block t sorts the n records of table t: record p = (src[t*n + id] << idb) | id
// with id = perm[p] (or p), i.e. the records start in the order of perm. A
// stable LSD sort on the key bits, one bit per pass: the records sit in
// registers (R per thread, blocked order), each pass counts the zero bits of a
// thread's items, a block-wide exclusive scan gives every item its place, the
// items go through one shared-memory buffer and are read back blocked. Padding
// items (all ones) sort last. Output: key and id arrays of the table.

constexpr int TS_THREADS = 1024;
constexpr int TS_ITEMS = 24;   // up to 24576 records per table

int table_sort_max() { return TS_THREADS * TS_ITEMS; }

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *total, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = s_warp[lane];   // TS_THREADS / 32 == 32 warps
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t res = s_warp[warp] + inc - v;
    *total = s_warp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(TS_THREADS, 1)
table_sort_kernel(const uint64_t *__restrict__ src, const uint32_t *__restrict__ perm, int n, int idb, int kb,
                  uint64_t *__restrict__ out_keys, uint32_t *__restrict__ out_ids) {
    extern __shared__ uint64_t ts_buf[];   // n_pad records
    __shared__ uint32_t s_warp[33];
    const int t = blockIdx.x;
    const uint64_t *sk = src + (size_t)t * n;
    const uint64_t idmask = (idb >= 64) ? ~0ull : ((1ull << idb) - 1ull);
    uint64_t r[TS_ITEMS];
#pragma unroll
    for (int k = 0; k < TS_ITEMS; k++) {
        const int p = threadIdx.x * TS_ITEMS + k;
        if (p < n) {
            const uint32_t id = perm ? perm[p] : (uint32_t)p;
            r[k] = (sk[id] << idb) | id;
        } else {
            r[k] = ~0ull;
        }
    }
    for (int b = idb; b < idb + kb; b++) {
        uint32_t z = 0;
#pragma unroll
        for (int k = 0; k < TS_ITEMS; k++) z += ((r[k] >> b) & 1ull) ? 0u : 1u;
        uint32_t zeros_total;
        const uint32_t zb = block_excl_scan_u32(z, &zeros_total, s_warp);
        const uint32_t before = threadIdx.x * TS_ITEMS;   // items before this thread
        uint32_t zi = zb, oi = zeros_total + (before - zb);
#pragma unroll
        for (int k = 0; k < TS_ITEMS; k++) {
            const bool one = (r[k] >> b) & 1ull;
            const uint32_t dst = one ? oi : zi;
            ts_buf[dst] = r[k];
            oi += one ? 1u : 0u;
            zi += one ? 0u : 1u;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TS_ITEMS; k++) r[k] = ts_buf[threadIdx.x * TS_ITEMS + k];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < TS_ITEMS; k++) {
        const int p = threadIdx.x * TS_ITEMS + k;
        if (p < n) {
            out_keys[(size_t)t * n + p] = r[k] >> idb;
            out_ids[(size_t)t * n + p] = (uint32_t)(r[k] & idmask);
        }
    }
}

cudaError_t launch_table_sort(const uint64_t *src, const uint32_t *perm, int64_t n, int64_t T, int idb, int kb,
                              uint64_t *out_keys, uint32_t *out_ids, cudaStream_t s) {
    if (n > table_sort_max() || idb + kb > 64 || T < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)TS_THREADS * TS_ITEMS * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(table_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    table_sort_kernel<<<(unsigned)T, TS_THREADS, smem, s>>>(src, perm, (int)n, idb, kb, out_keys, out_ids);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ej
