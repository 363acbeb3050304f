// Persistent verifier: the same exact test ED(x, y) <= K as the banded
// bit-parallel verifiers (Section 3.3, the last loop of Algorithm 3), with the
// pairs pulled from a device work queue so that a lane pair whose pair is done
// takes the next one instead of idling until the slowest pair of its warp ends.
//
// Per pair, two lanes: the forward half computes D(., n1) for n1 = n/2 over a
// block-aligned window of W1 64-row words, the backward half runs the same
// recurrence on the reversed strings for the remaining n - n1 columns, and
// ED(x, y) = min_i D(i, n1) + ED(x[i:], y[n1:]) joins them (the argument and the
// boundary conditions are the ones of the block-aligned two-lane verifier).
//
// Band. With x the longer string (m rows), y the shorter (n columns) and
// d = m - n, a path of cost c through cell (i, j) has c >= |i - j| + |d - (i - j)|
// (the distances to the diagonals of both corners), so a path of cost <= K
// stays on the diagonals i - j in [-K_lo, K_hi], K_lo = floor((K - d) / 2),
// K_hi = floor((K + d) / 2): at most K + 1 diagonals, where Ukkonen's band has
// 2K + 1 (the same argument as his cutoff). Both halves use it (reversing both
// strings keeps d). The window of W1 words covers it when W1 >= 1 + K/64
// rounded up, moving down one word before the columns K_lo + 1 + 64t, t >= 1.
//
// Scheduling. A warp advances its 16 pair slots in chunks of 64 columns. A slot
// starts a new pair at a chunk boundary, its column 1 at chunk position s0 =
// (smove - K_lo) mod 64 (the positions before it idle), so that every window
// move of every pair falls on the same chunk position smove and runs once per
// chunk for the whole warp. A finished slot waits at most one chunk. The number
// of working warps is capped (by default one per SM sub-partition), so that a
// batch larger than the slots keeps every slot busy until the queue runs dry.
//
// Early exit. Once per chunk, at the chunk position of the window moves, each
// half that is still running computes the minimum value m_h of its window
// (including the row above it). A path of cost <= K crosses both halves'
// current columns inside their bands, where the values are exact, so
// m_fwd + m_bwd > K proves ED > K; both lanes of the pair stop.
#include <climits>
#include <type_traits>

#include "ej_bitpar.cuh"

namespace ej {

namespace {

constexpr int64_t kMaxIters = 1ll << 24;   // default bound on loop passes per warp (VerifyOut::max_passes)

// The two words under 64/B symbols of a packed string starting at symbol o
// (any int64; words outside the string read as 0) and the bit offset of symbol
// o in the first: loads only, combined by sym_join when the symbols are needed
// (so that the load's latency passes while the previous word is consumed).
struct SymRaw {
    uint64_t a, b;
    uint32_t sh;
};
template <int B>
__device__ __forceinline__ SymRaw sym_fetch(const uint64_t *__restrict__ y64, int64_t nwords, int64_t o) {
    const int64_t bit = o * B;
    const int64_t w0 = bit >= 0 ? (bit >> 6) : -((-bit + 63) >> 6);
    SymRaw r;
    r.sh = (uint32_t)(bit - 64 * w0);
    r.a = (w0 >= 0 && w0 < nwords) ? y64[w0] : 0ull;
    r.b = (w0 + 1 >= 0 && w0 + 1 < nwords) ? y64[w0 + 1] : 0ull;
    return r;
}
__device__ __forceinline__ uint64_t sym_join(const SymRaw &r) {
    return r.sh ? ((r.a >> r.sh) | (r.b << (64u - r.sh))) : r.a;
}


__device__ __forceinline__ unsigned sm_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Reverses the order of the 64/B symbols of a word.
template <int B>
__device__ __forceinline__ uint64_t sym_reverse(uint64_t u) {
    if (B == 8) {
        const uint32_t lo = (uint32_t)u, hi = (uint32_t)(u >> 32);
        return ((uint64_t)__byte_perm(lo, 0u, 0x0123) << 32) | (uint64_t)__byte_perm(hi, 0u, 0x0123);
    }
    const uint64_t r = __brevll(u);   // B == 2: reverse bits, then swap the two bits of each symbol
    return ((r >> 1) & 0x5555555555555555ull) | ((r & 0x5555555555555555ull) << 1);
}

template <int W1, int B, int TPB, bool LEAN>
__global__ void __launch_bounds__(TPB, 1)
verify_pq_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                 const int32_t *__restrict__ lens, int64_t n_str, uint32_t alpha,
                 const uint64_t *__restrict__ pairs, int64_t np, int32_t K, int32_t nsm, int32_t spw_force,
                 int32_t wps, VerifyOut vo) {
    uint32_t *__restrict__ err = vo.err;
    const VerifySeg *__restrict__ segs = vo.segs;   // merged launch: the joins' candidates in turn
    const int nseg = segs ? vo.nseg : 0;
    const bool uni = segs && vo.umask;              // ... or their union, each pair once
    __shared__ long long s_cum[MAX_VERIFY_SEGS + 1];
    if (segs) {
        if (threadIdx.x == 0) {
            long long acc = 0;
            for (int g = 0; g < nseg; g++) {
                s_cum[g] = acc;
                const long long c = (long long)*segs[g].np_dev;
                acc += c < (long long)segs[g].cap ? c : (long long)segs[g].cap;
            }
            if (uni) {
                const unsigned long long c = *vo.unp_dev;
                acc = (long long)(c < vo.ucap ? c : vo.ucap);
            }
            s_cum[nseg] = acc;
        }
    } else {
        if (vo.np_dev) {
            const int64_t dn = (int64_t)*vo.np_dev;
            np = dn < np ? dn : np;
        }
        if (vo.pairs_off_dev) pairs += *vo.pairs_off_dev;
    }
    // error bits of one pair (its join's word in a merged launch), or of the warp
    auto pair_err = [&](int g, uint32_t bits) { atomicOr(segs ? segs[g].err : err, bits); };
    auto warp_err = [&](uint32_t bits) {
        if (!segs) atomicOr(err, bits);
        else
            for (int g = 0; g < nseg; g++) atomicOr(segs[g].err, bits);
    };
    // union pair q (listed by the joins of mask mk) with edit distance ed (or
    // INT_MAX when above the band's K): to every listing join whose K it meets
    auto emit_union = [&](int64_t q, uint32_t mk, int32_t ed) {
        for (int g = 0; g < nseg; g++) {
            if (!((mk >> g) & 1u) || ed > segs[g].K) continue;
            const unsigned long long idx = atomicAdd(segs[g].app_count, 1ull);
            if (idx < segs[g].app_cap) segs[g].app[idx] = vo.upairs[q];
        }
    };
    // a finished pair's result: to its join's outputs in a merged launch
    auto emit = [&](int g, int64_t q, bool pass) {
        if (!segs) {
            emit_result(vo, q, pairs, pass);
        } else if (pass) {
            const VerifySeg &sg_ = segs[g];
            const unsigned long long idx = atomicAdd(sg_.app_count, 1ull);
            if (idx < sg_.app_cap) sg_.app[idx] = sg_.pairs[q];
        }
    };
    constexpr int R = W1 + 1;
    constexpr int R2 = 2 * R;                // ring slots per symbol: every word is kept twice,
                                             // at slot k mod R and k mod R + R, so that the
                                             // window's W1 words sit at consecutive slots
    constexpr int SPW = 64 / B;              // symbols per 64-bit word
    constexpr uint64_t CMASK = (1ull << B) - 1ull;
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
    if (segs) np = s_cum[nseg];
    constexpr int T_ = TPB;                   // slot stride of the per-thread ring
    uint64_t *ring = smem + threadIdx.x;      // (c*R2 + slot)*T_, reused as a dump area
    const int lane = threadIdx.x & 31;
    const bool rev = lane & 1;
    const int slot = lane >> 1;
    const int32_t smove = K & 63;             // chunk position of every window move
    const uint32_t cmax = alpha - 1u;

    // Slots per warp and working warps. The working warps are chosen per SM
    // (the first ones to take a ticket on their SM), so that they are spread
    // evenly over the SMs whatever order the blocks were placed in; at most
    // 4*wps per SM (wps per sub-partition), fewer when the batch is small.
    const int64_t spw = spw_force > 0 ? (spw_force > 16 ? 16 : spw_force) : 16;
    const int64_t warps_needed = (np + spw - 1) / spw;
    int64_t per_sm = (warps_needed + nsm - 1) / (nsm > 0 ? nsm : 1);
    if (wps <= 0) {
        // automatic: one working warp per sub-partition while the pairs are few
        // (more warps would only start them all at once, and the launch ends
        // with its slowest pairs); 2 or 4 when every slot of one warp per
        // sub-partition would take at least 8 or 32 pairs (the second and third
        // warps then hide the step's fixed latencies)
        const int64_t per_slot = np / ((int64_t)(nsm > 0 ? nsm : 1) * 4 * spw);
        wps = per_slot >= 32 ? 4 : per_slot >= 8 ? 2 : 1;
    }
    if (per_sm > 4ll * wps) per_sm = 4ll * wps;
    unsigned ticket = 0;
    if (lane == 0) ticket = atomicAdd(&vo.sm_tickets[sm_id() & (SM_TICKETS - 1)], 1u);
    ticket = __shfl_sync(FULL, ticket, 0);
    bool exhausted = (slot >= spw) || ((int64_t)ticket >= per_sm);
    if (__all_sync(FULL, exhausted)) return;
    // merged launch: the warp's work counters per join, in shared memory (added
    // to the joins' global counters once, when the warp ends)
    __shared__ unsigned long long s_wk[TPB / 32][MAX_VERIFY_SEGS][2];
    unsigned long long *wk = &s_wk[threadIdx.x >> 5][0][0];
    if (lane < 2 * MAX_VERIFY_SEGS) wk[lane] = 0ull;
    __syncwarp();

    unsigned long long loc_cells = 0, loc_cols = 0;
    bool have = false, rejected = false;
    int64_t p = 0, k0 = 0;
    const uint4 *xc = packed;
    const uint64_t *y64 = reinterpret_cast<const uint64_t *>(packed);
    int64_t ywords = 0;
    int32_t m = 0, n = 0, ncols = 0, Tacc = 0, jbase = 1, next_move = 0, rej_col = 0;
    int32_t wpair = 1;       // words of the pair's band, ceil((K_lo + K_hi + 1) / 64) (work counter)
    // the raw word of y's (or reversed y's) symbols from symbol index sidx on
    auto sym_word = [&](int64_t sidx) -> SymRaw {
        return sym_fetch<B>(y64, ywords, rev ? (int64_t)n - SPW - sidx : sidx);
    };
    SymRaw snext{0ull, 0ull, 0u};   // the next word of the stream, already requested
    int32_t kp = K;          // the pair's threshold (<= K, the band)
    int sg = 0;              // the pair's join (merged launch; of the union: the largest K's)
    uint32_t umk = 0;        // union pair: the mask of the joins that list it
    int32_t budget = 0;      // chunks this pair may still take (ncols/64 + 2 suffice)
    int64_t iters = 0;       // loop passes of this warp (bounded by max_iters)
    const int64_t max_iters = vo.max_passes > 0 ? vo.max_passes : kMaxIters;
    int base = 0;
    uint64_t Pv[W1], Mv[W1];
#pragma unroll
    for (int v = 0; v < W1; v++) { Pv[v] = 0; Mv[v] = 0; }
    // Peq word k (of x or of reversed x) into ring slot `slot` and its twin
    auto build_word = [&](int slot, int64_t k) {
        bd_build<B, R2>(ring, T_, slot, xc, m, k, rev, alpha);
        for (uint32_t c = 0; c < alpha; c++)
            ring[(size_t)(c * R2 + slot + R) * T_] = ring[(size_t)(c * R2 + slot) * T_];
    };

    while (true) {
        if (++iters > max_iters) {
            // every lane counts the same passes, so the whole warp leaves here
            // (no block barrier follows); the call reports EJ_ERR_TIMEOUT
            if (lane == 0) warp_err((uint32_t)DERR_TIMEOUT);
            break;
        }
        // refill free slots (both lanes of a slot agree on `have` and `exhausted`)
        while (true) {
            const bool need = !have && !exhausted;
            const unsigned nb = __ballot_sync(FULL, need && !rev);
            if (nb == 0u) break;
            const int leader = __ffs(nb) - 1;
            unsigned long long qb = 0;
            if (lane == leader) qb = atomicAdd(vo.queue, (unsigned long long)__popc(nb));
            qb = __shfl_sync(FULL, qb, leader);
            if (need) {
                const unsigned fl = (unsigned)(lane & ~1);
                const int64_t idx = (int64_t)qb + __popc(nb & ((1u << fl) - 1u));
                if (idx >= np) {
                    exhausted = true;
                } else {
                    p = idx;
                    const uint64_t *pp = pairs;
                    if (uni) {
                        pp = vo.upairs;
                        umk = vo.umask[idx];
                        sg = -1;
                        for (int g = 0; g < nseg; g++)
                            if (((umk >> g) & 1u) && (sg < 0 || segs[g].K > segs[sg].K)) sg = g;
                        if (sg < 0) sg = 0;   // an empty mask cannot occur; its pair reaches no join
                    } else if (segs) {
                        sg = 0;
                        while (sg + 1 < nseg && idx >= s_cum[sg + 1]) sg++;
                        p = idx - s_cum[sg];
                        pp = segs[sg].pairs;
                    }
                    const uint64_t pr = pp[p];
                    const int64_t a = (int64_t)(pr >> 32), b = (int64_t)(pr & 0xFFFFFFFFull);
                    const bool two = vo.packed_b != nullptr;   // b indexes the second set
                    if (a >= n_str || b >= (two ? vo.n_b : n_str)) {
                        if (!rev) pair_err(sg, (uint32_t)DERR_PAIR);
                    } else {
                        const int32_t la = lens[a], lb = two ? vo.lens_b[b] : lens[b];
                        const uint4 *pa = packed + pofs[a];
                        const uint4 *pb = two ? vo.packed_b + vo.pofs_b[b] : packed + pofs[b];
                        const bool a_long = la >= lb;
                        m = a_long ? la : lb;
                        n = a_long ? lb : la;
                        kp = segs ? segs[sg].K : (vo.thr ? vo.thr[a] : K);
                        if (!rev) {
                            if (uni) {
                                for (int g = 0; g < nseg; g++)
                                    if ((umk >> g) & 1u) atomicAdd(&wk[2 * g], band_cells(m, n, segs[g].K));
                            } else if (segs) {
                                atomicAdd(&wk[2 * sg], band_cells(m, n, kp));
                            } else {
                                loc_cells += band_cells(m, n, kp);
                            }
                        }
                        if (m - n > kp || n == 0) {
                            if (!rev) {
                                if (uni) emit_union(p, umk, n == 0 ? m : INT_MAX);
                                else emit(sg, p, n == 0 && m <= kp);
                            }
                        } else {
                            const int32_t n1 = n / 2;
                            ncols = rev ? n - n1 : n1;
                            xc = a_long ? pa : pb;
                            y64 = reinterpret_cast<const uint64_t *>(a_long ? pb : pa);
                            ywords = 2 * chunks_for(n, B);
                            for (int wi = 0; wi < W1; wi++) build_word(wi, wi);
#pragma unroll
                            for (int v = 0; v < W1; v++) {
                                Pv[v] = ~0ull;
                                Mv[v] = 0ull;
                            }
                            // the pair's band (see the head of this file); m - n <= kp here
                            const int32_t klo = (kp - (m - n)) >> 1, khi = (kp + (m - n)) >> 1;
                            wpair = (klo + khi + 64) >> 6;
                            base = 0;
                            k0 = 0;
                            Tacc = 0;
                            jbase = 1 - ((smove - klo) & 63);   // column 1 at chunk position s0
                            snext = sym_word((int64_t)jbase - 1);
                            next_move = klo + 1 + 64;
                            rejected = false;
                            budget = (ncols >> 6) + 4;
                            have = true;
                        }
                    }
                }
            }
        }
        if (!__any_sync(FULL, have)) break;

        // one chunk: columns jbase .. jbase+63 of every active slot
        int32_t lim = (have && !rejected) ? ncols - jbase : -1;   // steps s <= lim are columns of the pair
        const int32_t slo = 1 - jbase;                             // and steps s >= slo (first chunk)
        // symbols of y (forward) or of reversed y, 64/B per word; the word after
        // the current one is requested one word ahead (snext: requested at the
        // previous chunk's last word, or at the pair's start)
        uint64_t sreg = 0;
        // steps s_begin .. s_end-1; GUARD: only the steps that are columns of the
        // lane's pair (without it every lane advances: lanes without a running
        // pair compute values that nothing reads)
        auto run_cols = [&](int s_begin, int s_end, auto guard) {
            constexpr bool GUARD = decltype(guard)::value;
#pragma unroll 2
            for (int s = s_begin; s < s_end; s++) {
                if ((s & (SPW - 1)) == 0) {
                    const uint64_t v = sym_join(snext);
                    sreg = rev ? sym_reverse<B>(v) : v;
                    snext = sym_word((int64_t)jbase - 1 + s + SPW);
                }
                uint32_t c = (uint32_t)(sreg & CMASK);
                sreg >>= B;
                c = c < cmax ? c : cmax;
                if (!GUARD || (s <= lim && s >= slo)) {
                    const uint64_t *row = ring + ((size_t)c * R2 + base) * T_;   // the window's words
                    uint64_t Eq[W1], A[W1], S[W1];
#pragma unroll
                    for (int v = 0; v < W1; v++) {
                        Eq[v] = row[v * T_];
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
                }
            }
        };
        // LEAN (launches set by their longest pairs): a range of steps runs
        // unguarded when every lane with a running pair has all its columns in
        // it (most chunks of long pairs); with many pairs per slot the second
        // copy of the loop costs more in instruction fetch than the guard
        auto run_range = [&](int a, int b) {
            if constexpr (LEAN) {
                const bool whole = !(have && !rejected) || (slo <= a && lim >= b - 1);
                if (__all_sync(FULL, whole)) {
                    run_cols(a, b, std::false_type{});
                    return;
                }
            }
            run_cols(a, b, std::true_type{});
        };
        run_range(0, smove);
        {
            // window move before column j = jbase + smove, then the joint bound
            const int32_t j = jbase + smove;
            // every pair still running takes part in the joint bound, also before
            // its first window move (short pairs have none)
            const bool active = have && !rejected && j >= 1 && j <= ncols;
            const bool moving = active && j == next_move;
            int32_t lb = 0;
            if (moving) {
                next_move += 64;
                Tacc += __popcll(Pv[0]) - __popcll(Mv[0]);
#pragma unroll
                for (int v = 0; v + 1 < W1; v++) { Pv[v] = Pv[v + 1]; Mv[v] = Mv[v + 1]; }
                Pv[W1 - 1] = ~0ull;
                Mv[W1 - 1] = 0ull;
                k0++;
                base = (base + 1 == R) ? 0 : base + 1;
                {
                    const int sl = base + W1 - 1;
                    build_word(sl >= R ? sl - R : sl, k0 + W1 - 1);
                }
            }
            if (active) {
                // minimum over the window at column j-1; row 64*k0 (value T) takes part
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
                lb = Tacc + (j - 1) + mn;
            }
            const int32_t lb_other = __shfl_xor_sync(FULL, lb, 1);
            if (active && lb + lb_other > kp) {
                rejected = true;
                rej_col = j;
                lim = -1;
            }
        }
        run_range(smove, 64);
        jbase += 64;
        if (have && --budget < 0 && !rejected && jbase <= ncols) {
            // cannot happen for a consistent state: stop this pair and report it
            pair_err(sg, (uint32_t)DERR_GUARD);
            rejected = true;
            rej_col = jbase;
        }

        // finished pairs: both halves done (all columns run, or rejected)
        const bool lane_done = have && (rejected || jbase > ncols);
        // every lane takes part in the shuffle (a short-circuit here would leave
        // the warp's other lanes waiting at a different collective)
        const int partner_done = __shfl_xor_sync(FULL, lane_done ? 1 : 0, 1);
        const bool pair_done = lane_done && partner_done != 0;
        if (__any_sync(FULL, pair_done)) {
            const int32_t T = Tacc + (rejected ? rej_col - 1 : ncols);
            if (pair_done) {
                const unsigned long long cols = (unsigned long long)(rejected ? rej_col - 1 : ncols);
                if (segs) atomicAdd(&wk[2 * sg + 1], cols * (unsigned long long)wpair);
                else loc_cols += cols * (unsigned long long)wpair;
#pragma unroll
                for (int v = 0; v < W1; v++) {
                    ring[(size_t)(2 * v) * T_] = Pv[v];
                    ring[(size_t)(2 * v + 1) * T_] = Mv[v];
                }
                ring[(size_t)(2 * W1) * T_] = (uint64_t)(uint32_t)T | ((uint64_t)k0 << 32);
                ring[(size_t)(2 * W1 + 1) * T_] = rejected ? 1ull : 0ull;
            }
            __syncwarp();
            if (pair_done && !rev) {
                bool pass = false;
                int32_t ed = INT_MAX;                           // the distance when <= kp
                const uint64_t *rb = smem + threadIdx.x + 1;   // backward half's dump
                const bool rej_b = rb[(size_t)(2 * W1 + 1) * T_] != 0ull;
                if (!rejected && !rej_b) {
                    const uint64_t tb = rb[(size_t)(2 * W1) * T_];
                    const int32_t Tb = (int32_t)(uint32_t)(tb & 0xFFFFFFFFull);
                    const int64_t k0b = (int64_t)(tb >> 32);
                    const int64_t k0f = k0;
                    const uint64_t *rf = ring;
                    // forward rows [64 k0f, min(m, 64(k0f+W1))]; backward row i' is row m - i'
                    const int64_t f_hi = min((int64_t)m, 64 * (k0f + W1));
                    const int64_t b_hi = min((int64_t)m, 64 * (k0b + W1));
                    const int64_t i_lo = max(64 * k0f, (int64_t)m - b_hi);
                    const int64_t i_hi = min(f_hi, (int64_t)m - 64 * k0b);
                    if (i_lo <= i_hi) {
                        auto prefix = [&](const uint64_t *dump, int64_t k0x, int32_t Tx, int64_t rowx) -> int32_t {
                            int32_t acc = Tx;
                            const int64_t nrows = rowx - 64 * k0x;
                            for (int v = 0; v < W1; v++) {
                                const int64_t lo = 64ll * v;
                                if (lo >= nrows) break;
                                const uint64_t msk = (nrows - lo >= 64) ? ~0ull : ((1ull << (nrows - lo)) - 1ull);
                                acc += __popcll(dump[(size_t)(2 * v) * T_] & msk) -
                                       __popcll(dump[(size_t)(2 * v + 1) * T_] & msk);
                            }
                            return acc;
                        };
                        int32_t F = prefix(rf, k0f, T, i_lo);
                        int32_t Bv = prefix(rb, k0b, Tb, (int64_t)m - i_lo);
                        int32_t best = F + Bv;
                        for (int64_t i = i_lo; i < i_hi; i++) {
                            const int64_t rf_ = i - 64 * k0f;                 // bit of row i+1 in the forward window
                            const int64_t rb_ = (int64_t)m - i - 64 * k0b - 1; // bit of row m-i in the backward window
                            const uint64_t fp = rf[(size_t)(2 * (rf_ >> 6)) * T_], fm = rf[(size_t)(2 * (rf_ >> 6) + 1) * T_];
                            const uint64_t bp = rb[(size_t)(2 * (rb_ >> 6)) * T_], bm = rb[(size_t)(2 * (rb_ >> 6) + 1) * T_];
                            F += (int32_t)((fp >> (rf_ & 63)) & 1ull) - (int32_t)((fm >> (rf_ & 63)) & 1ull);
                            Bv -= (int32_t)((bp >> (rb_ & 63)) & 1ull) - (int32_t)((bm >> (rb_ & 63)) & 1ull);
                            best = min(best, F + Bv);
                        }
                        pass = best <= kp;
                        if (pass) ed = best;
                    }
                }
                if (uni) emit_union(p, umk, ed);
                else emit(sg, p, pass);
            }
            __syncwarp();
            if (pair_done) have = false;
        }
    }

    if (segs) {
        __syncwarp();
        if (lane < 2 * nseg && wk[lane]) atomicAdd(&segs[lane >> 1].work[lane & 1], wk[lane]);
    }
    if (vo.work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loc_cells += __shfl_xor_sync(FULL, loc_cells, o);
            loc_cols += __shfl_xor_sync(FULL, loc_cols, o);
        }
        if (lane == 0) {
            if (loc_cells) atomicAdd(&vo.work[0], loc_cells);
            if (loc_cols) atomicAdd(&vo.work[1], loc_cols);
        }
    }
}

template <int W1, int B, int TPB, bool LEAN>
cudaError_t launch_pq_tt(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n, uint32_t alpha,
                         const uint64_t *pairs, int64_t np, int32_t K, int spw_force, int wps, VerifyOut vo,
                         cudaStream_t s) {
    constexpr int threads = TPB;
    const size_t smem = pq_smem_bytes(W1, alpha, threads);
    cudaError_t e = cudaFuncSetAttribute(verify_pq_kernel<W1, B, TPB, LEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_pq_kernel<W1, B, TPB, LEAN>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t blocks = (int64_t)sms * per_sm;
    verify_pq_kernel<W1, B, TPB, LEAN><<<(unsigned)blocks, threads, smem, s>>>(packed, pofs, lens, n, alpha, pairs, np, K,
                                                                     sms, spw_force, wps, vo);
    note_launches(1);
    return cudaGetLastError();
}

template <int W1, int B>
cudaError_t launch_pq_t(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n, uint32_t alpha,
                        const uint64_t *pairs, int64_t np, int32_t K, int threads, int spw_force, int wps, VerifyOut vo,
                        bool lean, cudaStream_t s) {
    // the lean variant for 2-bit codes and 128 threads (the long-string shape);
    // the other shapes keep the guarded loop only (build time)
    if (threads == 128 && lean && B == 2)
        return launch_pq_tt<W1, 2, 128, true>(packed, pofs, lens, n, alpha, pairs, np, K, spw_force, wps, vo, s);
    if (threads == 128)
        return launch_pq_tt<W1, B, 128, false>(packed, pofs, lens, n, alpha, pairs, np, K, spw_force, wps, vo, s);
    if (threads == 32)
        return launch_pq_tt<W1, B, 32, false>(packed, pofs, lens, n, alpha, pairs, np, K, spw_force, wps, vo, s);
    return cudaErrorInvalidValue;
}

}  // namespace

size_t pq_smem_bytes(int W1, uint32_t alpha, int threads) {
    const size_t R2 = 2 * ((size_t)W1 + 1);
    const size_t per = alpha * R2 > (size_t)(2 * W1 + 2) ? alpha * R2 : (size_t)(2 * W1 + 2);
    return per * sizeof(uint64_t) * (size_t)threads;
}

int pq_threads_for(int W1, uint32_t alpha) {
    if (pq_smem_bytes(W1, alpha, 128) <= 160 * 1024) return 128;
    return pq_smem_bytes(W1, alpha, 32) <= 220 * 1024 ? 32 : 0;
}

cudaError_t launch_verify_pq(int W1, int threads, int spw_force, int wps, const uint4 *packed, const uint64_t *pofs, int B,
                             const int32_t *lens, int64_t n, uint32_t alpha, const uint64_t *pairs, int64_t np,
                             int32_t K, VerifyOut vo, cudaStream_t s, bool lean) {
    if (np == 0) return cudaGetLastError();
    if (!vo.queue || !vo.sm_tickets || (threads != 128 && threads != 32)) return cudaErrorInvalidValue;
#define EJ_PQ(WW)                                                                                          \
    if (W1 == WW) {                                                                                        \
        if (B == 2) return launch_pq_t<WW, 2>(packed, pofs, lens, n, alpha, pairs, np, K, threads, spw_force, wps, vo, lean, s); \
        return launch_pq_t<WW, 8>(packed, pofs, lens, n, alpha, pairs, np, K, threads, spw_force, wps, vo, lean, s);   \
    }
    EJ_PQ(2) EJ_PQ(3) EJ_PQ(4) EJ_PQ(5) EJ_PQ(6) EJ_PQ(7) EJ_PQ(8) EJ_PQ(9) EJ_PQ(10) EJ_PQ(11) EJ_PQ(12)
#undef EJ_PQ
    return cudaErrorInvalidValue;
}

}  // namespace ej
