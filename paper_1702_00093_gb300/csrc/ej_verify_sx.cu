// Verifier for pairs grouped by their longer string (Section 3.3, the last loop
// of Algorithm 3): the same exact test ED(x, y) <= K as the two-lane
// block-aligned verifier, with the match masks of x shared by a warp.
//
// The candidates arrive grouped by x, the longer string of each pair, and by
// the class of the length difference d = |x| - |y| (sx_band), in warp tasks of
// up to 16 pairs that all share x and the class. A warp runs its 16 pairs in
// two lanes each (forward half and backward half, as in verify_bd_kernel).
// A path of cost <= K of a pair stays on the diagonals i - j in
// [-floor((K - d)/2), floor((K + d)/2)] (the persistent verifier's band); the
// task's band is the union of its pairs' bands, at most K + 1 + (D - 1)/2
// diagonals for a class of width D. All pairs of a task start together and the
// band window of every pair moves at the same columns (klo + 1 + 64t, klo the
// task band's upper reach), so the windows of all forward halves cover the
// same 64-row words of x, and those of all backward halves the same words of
// reversed x: the warp keeps one ring of match masks per direction in
// shared memory instead of one per lane. For large alphabets that is 16x less
// shared memory per pair, which is what limited the per-lane verifier to one or
// two warps per SM, and each word is built once per task, by the whole warp:
// lane t takes rows t and t + 32, and __match_any_sync gives every symbol's
// mask of the word in two steps.
//
// Early exit every 32 columns is decided by both halves of a pair together
// (the joint bound of the other verifiers), and the task ends when all of its
// pairs are decided.
#include "ej_bitpar.cuh"

namespace ej {

namespace {

constexpr int SX_WARPS = 4;    // warps per block
constexpr int SX_CHECK = 32;   // columns between the joint early-exit tests (a power of two)

// Symbol i (0 <= i < m) of a packed string.
template <int B>
__device__ __forceinline__ uint32_t sym_at(const uint4 *__restrict__ xc, int64_t i) {
    if (B == 8) return reinterpret_cast<const uint8_t *>(xc)[i];
    return (reinterpret_cast<const uint32_t *>(xc)[i >> 4] >> (2 * (uint32_t)(i & 15))) & 3u;
}

// Word k (rows 64k+1 .. 64k+64) of x, or of reversed x, built by the whole warp
// into ring slot `slot` (entry c * RS + slot for symbol c): lane t reads rows t
// and t + 32 (coop_load), and the lanes holding the same symbol find one
// another with __match_any_sync, which is that symbol's mask of the 32 rows
// (coop_store). The loads of several words are issued before any of them is
// stored, so that their latencies overlap.
struct WordSyms {
    uint32_t s0, s1;
};

template <int B>
__device__ __forceinline__ WordSyms coop_load(const uint4 *__restrict__ xc, int64_t m, int64_t k, bool rev, int lane) {
    const int64_t i0 = rev ? m - 1 - 64 * k - lane : 64 * k + lane;
    const int64_t i1 = rev ? i0 - 32 : i0 + 32;
    WordSyms w;
    w.s0 = (i0 >= 0 && i0 < m) ? sym_at<B>(xc, i0) : 0xFFFFu;
    w.s1 = (i1 >= 0 && i1 < m) ? sym_at<B>(xc, i1) : 0xFFFFu;
    return w;
}

__device__ __forceinline__ void coop_store(uint64_t *ring, int RS, int slot, WordSyms w, uint32_t alpha, int lane) {
    const unsigned m0 = __match_any_sync(FULL, w.s0);
    const unsigned m1 = __match_any_sync(FULL, w.s1);
    for (uint32_t c = lane; c < alpha; c += 32) ring[(size_t)c * RS + slot] = 0ull;
    __syncwarp();
    // lanes with the same symbol write the same value
    if (w.s0 < alpha) reinterpret_cast<uint32_t *>(ring + (size_t)w.s0 * RS + slot)[0] = m0;
    if (w.s1 < alpha) reinterpret_cast<uint32_t *>(ring + (size_t)w.s1 * RS + slot)[1] = m1;
    __syncwarp();
}

template <int W1, int B>
__global__ void __launch_bounds__(SX_WARPS * 32, 4)
verify_sx_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                 const int32_t *__restrict__ lens, int64_t n_str, uint32_t alpha,
                 const uint64_t *__restrict__ pairs, const uint64_t *__restrict__ tasks,
                 const unsigned long long *__restrict__ ntasks_dev, int64_t ntasks_cap, int32_t K, int32_t RS,
                 int32_t warp_words, VerifyOut vo) {
    uint32_t *__restrict__ err = vo.err;
    unsigned long long *__restrict__ work = vo.work;
    extern __shared__ uint64_t smem[];
    __shared__ int8_t s_nsum[256];
    __shared__ int8_t s_nmin[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        const uint32_t P = t & 15u, M = t >> 4;
        int run = 0, mn = 1 << 20;
        for (int k = 0; k < 4; k++) {
            run += (int)((P >> k) & 1u) - (int)((M >> k) & 1u);
            mn = run < mn ? run : mn;
        }
        s_nsum[t] = (int8_t)run;
        s_nmin[t] = (int8_t)mn;
    }
    __syncthreads();
    constexpr int R = W1;   // ring slots: the new bottom word takes the dropped top word's slot
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint64_t *wbase = smem + (size_t)wib * warp_words;
    uint64_t *ringF = wbase;                          // words of x
    uint64_t *ringB = wbase + (size_t)alpha * RS;     // words of reversed x
    uint64_t *dump = wbase;                           // after a task's columns: entry e of lane L at e*32+L
    const bool rev = lane & 1;
    const int slot_pair = lane >> 1;
    uint64_t *myring = rev ? ringB : ringF;
    const int64_t cap_t = (int64_t)*ntasks_dev;
    const int64_t ntasks = cap_t < ntasks_cap ? cap_t : ntasks_cap;
    const int64_t nw = (int64_t)gridDim.x * SX_WARPS;

    unsigned long long loc_cells = 0, loc_cols = 0;
    // a task's descriptor and this lane's pair are loaded during the task before
    int64_t t = (int64_t)blockIdx.x * SX_WARPS + wib;
    uint64_t tk_next = 0, pr_next = 0;
    if (t < ntasks) {
        tk_next = tasks[t];
        if (slot_pair < (int)(tk_next & 31u)) pr_next = pairs[(int64_t)(tk_next >> 5) + slot_pair];
    }
    for (; t < ntasks; t += nw) {   // warp-uniform
        const uint64_t tk = tk_next;
        const uint64_t pr = pr_next;
        if (t + nw < ntasks) {
            tk_next = tasks[t + nw];
            if (slot_pair < (int)(tk_next & 31u)) pr_next = pairs[(int64_t)(tk_next >> 5) + slot_pair];
        }
        const int64_t first = (int64_t)(tk >> 5);
        const int cnt = (int)(tk & 31u);
        bool valid = slot_pair < cnt;
        int64_t a = 0, b = 0;
        if (valid) {
            a = (int64_t)(pr >> 32);
            b = (int64_t)(pr & 0xFFFFFFFFull);
            if (a >= n_str || b >= n_str) {
                if (!rev) atomicOr(err, (uint32_t)DERR_PAIR);
                valid = false;
            }
        }
        const int32_t la = valid ? lens[a] : 0, lb = valid ? lens[b] : 0;
        const bool a_long = la >= lb;
        const int64_t xi = a_long ? a : b, yi = a_long ? b : a;
        const int32_t m = a_long ? la : lb, n = a_long ? lb : la;
        // every pair of a task has the same x (its first pair's)
        const int64_t xs = __shfl_sync(FULL, valid ? xi : -1, 0);
        if (valid && xi != xs) {
            if (!rev) atomicOr(err, (uint32_t)DERR_GUARD);
            valid = false;
        }
        bool decided = !valid, pass = false;
        if (valid && m - n > K) decided = true;
        else if (valid && n == 0) { decided = true; pass = m <= K; }
        const int32_t n1 = n / 2;
        const int32_t ncols = decided ? 0 : (rev ? n - n1 : n1);
        const int32_t maxcols = (int32_t)__reduce_max_sync(FULL, (unsigned)ncols);
        // the task's band: the diagonals a cost-K alignment of any of its
        // undecided pairs can use (their length differences lie in one class)
        const unsigned nlo = __reduce_min_sync(FULL, decided ? 0xFFFFFFFFu : (unsigned)n);
        const unsigned nhi = __reduce_max_sync(FULL, decided ? 0u : (unsigned)n);

        uint64_t Pv[W1], Mv[W1];
#pragma unroll
        for (int v = 0; v < W1; v++) { Pv[v] = ~0ull; Mv[v] = 0ull; }
        int32_t T = 0, cols_run = 0;
        int64_t k0 = 0;
        bool rejected = false;
        if (maxcols > 0) {
            const int32_t mx = xs >= 0 ? lens[xs] : 0;
            const uint4 *xc = packed + pofs[xs >= 0 ? xs : 0];
            // the first W1 words of both directions, loaded four words at a time
#pragma unroll
            for (int w0 = 0; w0 < W1; w0 += 2) {
                WordSyms f[2], r[2];
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    if (w0 + d < W1) {
                        f[d] = coop_load<B>(xc, mx, w0 + d, false, lane);
                        r[d] = coop_load<B>(xc, mx, w0 + d, true, lane);
                    }
                }
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    if (w0 + d < W1) {
                        coop_store(ringF, RS, w0 + d, f[d], alpha, lane);
                        coop_store(ringB, RS, w0 + d, r[d], alpha, lane);
                    }
                }
            }
            SymReader<B> yf;
            SymReaderRev<B> yb;
            if (!decided) {
                if (rev) yb.init(packed + pofs[yi], n);
                else yf.init(packed + pofs[yi], chunks_for(n1, B));
            }
            const uint32_t cmax = alpha - 1u;
            int base = 0;              // ring slot of the window's top word (the same for the whole warp)
            int64_t kr = 0;            // window moves of the warp so far
            const int32_t klo = (K - (mx - (int32_t)nhi)) >> 1, khi = (K + (mx - (int32_t)nlo)) >> 1;
            if (klo + khi + 64 > 64 * W1 && lane == 0) atomicOr(err, (uint32_t)DERR_GUARD);   // not by construction
            int32_t next_move = klo + 1 + 64;   // the window moves down before the columns klo + 1 + 64t
            bool done = decided;
            for (int32_t j = 1; j <= maxcols; j++) {
                if ((j & (SX_CHECK - 1)) == 0) {
                    // joint early exit at column j-1 of both halves (j <= n1 <= n - n1)
                    const bool chk = !done && j <= n1;
                    int32_t lb = 0;
                    if (chk) {
                        int32_t run = 0, mn = 0;
#pragma unroll
                        for (int v = 0; v < W1; v++) {
#pragma unroll
                            for (int q = 0; q < 16; q++) {
                                const uint32_t idx = (uint32_t)((Pv[v] >> (4 * q)) & 15u) |
                                                     ((uint32_t)((Mv[v] >> (4 * q)) & 15u) << 4);
                                const int32_t cand = run + s_nmin[idx];
                                mn = cand < mn ? cand : mn;
                                run += s_nsum[idx];
                            }
                        }
                        lb = T + mn;
                    }
                    const int32_t lb_other = __shfl_xor_sync(FULL, lb, 1);
                    if (chk && lb + lb_other > K) {
                        rejected = true;
                        done = true;
                        cols_run = j - 1;
                    }
                    if (__all_sync(FULL, done || j > ncols)) break;
                }
                const bool running = !done && j <= ncols;
                if (j == next_move) {   // warp-uniform
                    next_move += 64;
                    if (running) {
                        // drop the top word into T, shift the window down one word
                        T += __popcll(Pv[0]) - __popcll(Mv[0]);
#pragma unroll
                        for (int v = 0; v + 1 < W1; v++) { Pv[v] = Pv[v + 1]; Mv[v] = Mv[v + 1]; }
                        Pv[W1 - 1] = ~0ull;
                        Mv[W1 - 1] = 0ull;
                        k0++;
                    }
                    kr++;
                    const int freed = base;   // the dropped top word's slot takes the new bottom word
                    base = (base + 1 == R) ? 0 : base + 1;
                    const WordSyms f = coop_load<B>(xc, mx, kr + W1 - 1, false, lane);
                    const WordSyms r = coop_load<B>(xc, mx, kr + W1 - 1, true, lane);
                    coop_store(ringF, RS, freed, f, alpha, lane);
                    coop_store(ringB, RS, freed, r, alpha, lane);
                }
                if (running) {
                    uint32_t c;
                    if (rev) { c = yb.code(); yb.advance(); }
                    else { c = yf.code(); yf.advance(); }
                    c = c < cmax ? c : cmax;   // codes of a validated string are < alpha
                    const uint64_t *row = myring + (size_t)c * RS;
                    uint64_t Eq[W1], A[W1], S[W1];
#pragma unroll
                    for (int v = 0; v < W1; v++) {
                        const int sl = base + v;
                        Eq[v] = row[sl >= R ? sl - R : sl];
                        A[v] = Eq[v] & Pv[v];
                    }
                    add_chain<W1>(S, A, Pv);
                    uint64_t Ph[W1], Mh[W1];
#pragma unroll
                    for (int v = 0; v < W1; v++) {
                        const uint64_t Xh = (S[v] ^ Pv[v]) | Eq[v];
                        Ph[v] = Mv[v] | ~(Xh | Pv[v]);
                        Mh[v] = Pv[v] & Xh;
                    }
#pragma unroll
                    for (int v = W1 - 1; v >= 0; v--) {
                        const uint64_t inP = (v > 0) ? (Ph[v > 0 ? v - 1 : 0] >> 63) : 1ull;
                        const uint64_t inM = (v > 0) ? (Mh[v > 0 ? v - 1 : 0] >> 63) : 0ull;
                        Ph[v] = (Ph[v] << 1) | inP;
                        Mh[v] = (Mh[v] << 1) | inM;
                    }
#pragma unroll
                    for (int v = 0; v < W1; v++) {
                        const uint64_t X = Eq[v] | Mv[v];
                        Pv[v] = Mh[v] | ~(X | Ph[v]);
                        Mv[v] = Ph[v] & X;
                    }
                    T += 1;   // the row above the window: +1 per column
                }
            }
            if (!decided && !rejected) cols_run = ncols;
        }
        // exchange through the warp's shared area (the rings are no longer read)
        __syncwarp();
#pragma unroll
        for (int v = 0; v < W1; v++) {
            dump[(size_t)(2 * v) * 32 + lane] = Pv[v];
            dump[(size_t)(2 * v + 1) * 32 + lane] = Mv[v];
        }
        dump[(size_t)(2 * W1) * 32 + lane] = (uint64_t)(uint32_t)T | ((uint64_t)k0 << 32);
        dump[(size_t)(2 * W1 + 1) * 32 + lane] = rejected ? 1ull : 0ull;
        __syncwarp();
        if (!rev && !decided) {
            const uint64_t *rf = dump + lane, *rb = dump + lane + 1;
            const bool rej_b = rb[(size_t)(2 * W1 + 1) * 32] != 0ull;
            if (rejected || rej_b) {
                pass = false;
            } else {
                const uint64_t tb = rb[(size_t)(2 * W1) * 32];
                const int32_t Tb = (int32_t)(uint32_t)(tb & 0xFFFFFFFFull);
                const int64_t k0b = (int64_t)(tb >> 32);
                const int64_t k0f = k0;
                const int64_t f_hi = min((int64_t)m, 64 * (k0f + W1));
                const int64_t b_hi = min((int64_t)m, 64 * (k0b + W1));
                const int64_t i_lo = max(64 * k0f, (int64_t)m - b_hi);
                const int64_t i_hi = min(f_hi, (int64_t)m - 64 * k0b);
                if (i_lo > i_hi) {
                    pass = false;
                } else {
                    // F(i) = value of row i at column n1 (forward), B(i) = value of
                    // row m-i at column n-n1 (backward); ED = min_i F(i) + B(i)
                    auto prefix = [&](const uint64_t *d, int64_t k0x, int32_t Tx, int64_t row) -> int32_t {
                        int32_t acc = Tx;
                        const int64_t nrows = row - 64 * k0x;
                        for (int v = 0; v < W1; v++) {
                            const int64_t lo = 64ll * v;
                            if (lo >= nrows) break;
                            const uint64_t msk = (nrows - lo >= 64) ? ~0ull : ((1ull << (nrows - lo)) - 1ull);
                            acc += __popcll(d[(size_t)(2 * v) * 32] & msk) - __popcll(d[(size_t)(2 * v + 1) * 32] & msk);
                        }
                        return acc;
                    };
                    int32_t F = prefix(rf, k0f, T, i_lo);
                    int32_t Bv = prefix(rb, k0b, Tb, (int64_t)m - i_lo);
                    int32_t best = F + Bv;
                    for (int64_t i = i_lo; i < i_hi; i++) {
                        const int64_t rf_ = i - 64 * k0f;
                        const int64_t rb_ = (int64_t)m - i - 64 * k0b - 1;
                        const uint64_t fp = rf[(size_t)(2 * (rf_ >> 6)) * 32], fm = rf[(size_t)(2 * (rf_ >> 6) + 1) * 32];
                        const uint64_t bp = rb[(size_t)(2 * (rb_ >> 6)) * 32], bm = rb[(size_t)(2 * (rb_ >> 6) + 1) * 32];
                        F += (int32_t)((fp >> (rf_ & 63)) & 1ull) - (int32_t)((fm >> (rf_ & 63)) & 1ull);
                        Bv -= (int32_t)((bp >> (rb_ & 63)) & 1ull) - (int32_t)((bm >> (rb_ & 63)) & 1ull);
                        best = min(best, F + Bv);
                    }
                    pass = best <= K;
                }
            }
        }
        if (valid && !rev) emit_result(vo, first + slot_pair, pairs, pass);
        if (valid) {
            if (!rev) loc_cells += band_cells(m, n, K);
            const int32_t d = m - n;   // the pair's own band: ((K - d) >> 1) + ((K + d) >> 1) + 1 diagonals
            loc_cols += (unsigned long long)cols_run * (unsigned long long)((((K - d) >> 1) + ((K + d) >> 1) + 64) >> 6);
        }
        __syncwarp();   // the shared area is rebuilt by the next task
    }
    // work counters: one atomic per warp (per-pair atomics on two addresses
    // serialise in the memory system)
    if (work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loc_cells += __shfl_xor_sync(FULL, loc_cells, o);
            loc_cols += __shfl_xor_sync(FULL, loc_cols, o);
        }
        if (lane == 0) {
            if (loc_cells) atomicAdd(&work[0], loc_cells);
            if (loc_cols) atomicAdd(&work[1], loc_cols);
        }
    }
}

// tcount[x] = tasks of string x (up to 16 of its pairs each); tcount[n] = 0.
__global__ void sx_task_counts_kernel(const uint32_t *__restrict__ bins, int64_t n, uint32_t *__restrict__ tcount) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += (int64_t)gridDim.x * blockDim.x)
        tcount[x] = x < n ? (bins[x] + 15u) / 16u : 0u;
}

// The tasks of string x: (first pair << 5) | pairs, over its run of candidates
// [ends[x] - bins[x], ends[x]).
__global__ void sx_tasks_kernel(const uint32_t *__restrict__ bins, const uint64_t *__restrict__ ends, int64_t n,
                                const uint64_t *__restrict__ tstart, uint64_t *__restrict__ tasks) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = bins[x];
        if (!c) continue;
        const uint64_t base = ends[x] - c, t0 = tstart[x];
        for (uint32_t k = 0; 16u * k < c; k++) {
            const uint32_t left = c - 16u * k;
            tasks[t0 + k] = ((base + 16ull * k) << 5) | (uint64_t)(left < 16u ? left : 16u);
        }
    }
}

template <int W1, int B>
cudaError_t launch_sx_t(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n, uint32_t alpha,
                        const uint64_t *pairs, const uint64_t *tasks, const unsigned long long *ntasks_dev,
                        int64_t ntasks_cap, int32_t K, VerifyOut vo, cudaStream_t s) {
    const int RS = (W1 & 1) ? W1 : W1 + 1;   // odd: lanes reading different symbols spread over the banks
    const size_t rings = 2 * (size_t)alpha * RS, dumpw = 32 * (size_t)(2 * W1 + 2);
    const size_t warp_words = rings > dumpw ? rings : dumpw;
    const size_t smem = warp_words * sizeof(uint64_t) * SX_WARPS;
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(verify_sx_kernel<W1, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_sx_kernel<W1, B>, SX_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)sms * per_sm;
    const int64_t need = (ntasks_cap + SX_WARPS - 1) / SX_WARPS;
    if (blocks > need) blocks = need > 0 ? need : 1;
    verify_sx_kernel<W1, B><<<(unsigned)blocks, SX_WARPS * 32, smem, s>>>(
        packed, pofs, lens, n, alpha, pairs, tasks, ntasks_dev, ntasks_cap, K, RS, (int32_t)warp_words, vo);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

SxBand sx_band(int32_t K) {
    const int words = (K + 1 + 63) / 64;   // ceil((K + 1) / 64)
    int W = words, slack = 64 * words - (K + 1);
    if (2 * slack + 1 < 7) {   // classes narrower than 7 would split the strings' pairs too finely
        W += 1;
        slack += 64;
    }
    uint32_t D = 2u * (uint32_t)slack + 1u;
    if (D > (uint32_t)K + 1u) D = (uint32_t)K + 1u;
    return SxBand{W + 1, D, ((uint32_t)K + 1u + D - 1u) / D};
}


size_t sx_smem_bytes(int W1, uint32_t alpha) {
    const size_t RS = (W1 & 1) ? W1 : W1 + 1;
    const size_t rings = 2 * (size_t)alpha * RS, dumpw = 32 * (size_t)(2 * W1 + 2);
    return (rings > dumpw ? rings : dumpw) * sizeof(uint64_t) * SX_WARPS;
}

cudaError_t launch_sx_tasks(const uint32_t *bins, const uint64_t *ends, int64_t n, uint32_t *tcount, uint64_t *tstart,
                            unsigned long long *ntasks_dev, void *scan_tmp, uint64_t *tasks, cudaStream_t s) {
    int64_t g = (n + 256) / 256;
    const unsigned gs = (unsigned)(g > 4096 ? 4096 : (g ? g : 1));
    sx_task_counts_kernel<<<gs, 256, 0, s>>>(bins, n, tcount);
    note_launches(1);
    cudaError_t e = exclusive_scan_u32(tcount, tstart, n + 1, (uint64_t *)ntasks_dev, scan_tmp, s);
    if (e != cudaSuccess) return e;
    sx_tasks_kernel<<<gs, 256, 0, s>>>(bins, ends, n, tstart, tasks);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_verify_sx(int W1, const uint4 *packed, const uint64_t *pofs, int B, const int32_t *lens, int64_t n,
                             uint32_t alpha, const uint64_t *pairs, const uint64_t *tasks,
                             const unsigned long long *ntasks_dev, int64_t ntasks_cap, int32_t K, VerifyOut vo,
                             cudaStream_t s) {
    if (ntasks_cap == 0) return cudaGetLastError();
#define EJ_SX(WW)                                                                                          \
    if (W1 == WW) {                                                                                        \
        if (B == 2) return launch_sx_t<WW, 2>(packed, pofs, lens, n, alpha, pairs, tasks, ntasks_dev, ntasks_cap, K, vo, s); \
        return launch_sx_t<WW, 8>(packed, pofs, lens, n, alpha, pairs, tasks, ntasks_dev, ntasks_cap, K, vo, s);   \
    }
    EJ_SX(2) EJ_SX(3) EJ_SX(4) EJ_SX(5) EJ_SX(6) EJ_SX(7) EJ_SX(8) EJ_SX(9) EJ_SX(10) EJ_SX(11) EJ_SX(12)
#undef EJ_SX
    return cudaErrorInvalidValue;
}

}  // namespace ej
