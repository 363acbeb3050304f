// Verification of candidate pairs: ED(x, y) <= K (Section 3.3, the last loop of
// Algorithm 3), computed exactly with a banded bit-parallel form of the
// edit-distance DP.
//
// Formulation. Rows i = 1..m follow x (the longer string), columns j = 1..n
// follow y (the shorter). D(i, 0) = i, D(0, j) = j. Only a window of 64*W rows
// is kept per column: after the shift at column j it holds rows
// j-K .. j-K+64W-1 (bit b <-> row j-K+b), which covers Ukkonen's band
// |i - j| <= K because 64W >= 2K+1. The window stores vertical differences
// D(i,j) - D(i-1,j) as two bit-vectors (Pv: +1, Mv: -1) and the column is
// advanced with the bit-vector recurrence for unit-cost edit distance (Myers
// 1999, in the form of Hyyro 2001). Cells the window does not hold are
// replaced by upper bounds that keep every difference in {-1, 0, +1}:
//   - the row above the window gains +1 per column (horizontal shift-in 1),
//   - the row entering at the bottom is one more than the row above it,
//   - virtual rows above row 0 start at D(i, 0) = -i (vertical -1), never match.
// With those boundaries every computed value is >= min(D, K+1) and equals D
// wherever D <= K (an optimal path of cost <= K never leaves the band), so
// "value(m, n) <= K" decides ED <= K exactly. The value of the cell above the
// window, T, is tracked explicitly; D(m, n) = T + sum of the differences of
// rows j-K .. m at the last column.
//
// Early exit: every 64 columns the group computes the minimum value in its
// window; the minimum over the band never decreases from one column to the
// next (D(i, j+1) >= D(i-1, j)), so once it exceeds K the pair is rejected.
//
// Mapping: a group of G lanes verifies one pair; lane g holds V consecutive
// 64-bit words of the window. The carry of the multi-word addition crosses
// lanes through two ballots (generate / propagate bits combined with one
// integer addition), the one-bit shifts cross lanes through shuffles.
// The pattern bit-masks Peq[c] of x live in shared memory, one region per
// group, with K zero bits in front so that window bit b at column j is Peq bit
// j-1+b. All groups of a warp step through columns together (the loop bound is
// the warp maximum), so every warp collective runs with the full mask.
#include "ej_bitpar.cuh"

namespace ej {

constexpr int VERIFY_MAX_THREADS = 256;

template <int G, int V, int B>
__global__ void __launch_bounds__(VERIFY_MAX_THREADS)
verify_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
              const int32_t *__restrict__ lens, int64_t n_str,
              uint32_t alpha, const uint64_t *__restrict__ pairs, int64_t np, int32_t K, int32_t Lw,
              VerifyOut vo) {
    uint32_t *__restrict__ err = vo.err;
    unsigned long long *__restrict__ work = vo.work;
    if (vo.np_dev) {
        const int64_t dn = (int64_t)*vo.np_dev;
        np = dn < np ? dn : np;
    }
    if (vo.pairs_off_dev) pairs += *vo.pairs_off_dev;
    unsigned long long loc_cells = 0, loc_cols = 0;
    constexpr int GPW = 32 / G;
    const int32_t w_min = (2 * K + 1 + 63) / 64;
    extern __shared__ uint64_t smem[];
    __shared__ int8_t s_nsum[256];
    __shared__ int8_t s_nmin[256];

    for (int t = threadIdx.x; t < 256; t += blockDim.x) {
        // nibble table: index = P nibble | M nibble << 4; sum and minimum prefix
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

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / G, gl = lane % G;
    const int warps_per_block = blockDim.x >> 5;
    uint64_t *peq = smem + (size_t)(warp * GPW + g) * alpha * Lw;
    const int64_t warps_total = (int64_t)gridDim.x * warps_per_block;

    for (int64_t wb = (int64_t)blockIdx.x * warps_per_block + warp; wb * GPW < np; wb += warps_total) {
        const int64_t p = wb * GPW + g;
        bool valid = p < np;
        int32_t la = 0, lb = 0, kp = K;
        int64_t a = 0, b = 0;
        const bool two = vo.packed_b != nullptr;   // b indexes the second set
        if (valid) {
            const uint64_t pr = pairs[p];
            a = (int64_t)(pr >> 32);
            b = (int64_t)(pr & 0xFFFFFFFFull);
            if (a >= n_str || b >= (two ? vo.n_b : n_str)) {
                if (gl == 0) atomicOr(err, (uint32_t)DERR_PAIR);
                valid = false;
            } else {
                la = lens[a];
                lb = two ? vo.lens_b[b] : lens[b];
                kp = vo.thr ? vo.thr[a] : K;
            }
        }
        const bool a_long = la >= lb;
        const uint4 *pa = packed + (valid ? pofs[a] : 0);
        const uint4 *pb = valid ? (two ? vo.packed_b + vo.pofs_b[b] : packed + pofs[b]) : packed;
        const uint4 *xc_base = a_long ? pa : pb, *yc_base = a_long ? pb : pa;
        const int32_t mlen = a_long ? la : lb;
        const int32_t nlen = a_long ? lb : la;
        bool decided = !valid;
        bool pass = false;
        if (valid && mlen - nlen > kp) {
            decided = true;
        } else if (valid && nlen == 0) {
            decided = true;
            pass = mlen <= kp;
        }
        int32_t ncols = decided ? 0 : nlen;
        const int32_t mrows = decided ? 0 : mlen;
        int32_t cols_run = ncols;  // columns actually advanced (early exit shortens it)

        // Peq[c]: bit K+i set iff code(x[i]) == c
        const int32_t mmax = __reduce_max_sync(FULL, mrows);
        if (mmax > 0) {
            const uint4 *xc = xc_base;
            const int64_t xch = chunks_for(mrows, B);
            if (B == 2) {
                // whole 64-bit words from the 2-bit codes, no atomics
                for (int w = gl; w < Lw; w += G) {
                    const int64_t k0 = 64ll * w - K;
                    uint64_t lo = 0, hi = 0;
                    if (mrows > 0) sym64_planes(xc, xch, k0, lo, hi);
                    const int64_t t_lo = k0 < 0 ? -k0 : 0;
                    const int64_t t_hi = (int64_t)mrows - k0;  // symbols t < t_hi are inside x
                    uint64_t valid_m = 0ull;
                    if (t_hi > t_lo && t_lo < 64) {
                        const uint64_t upto = t_hi >= 64 ? ~0ull : ((1ull << t_hi) - 1ull);
                        const uint64_t from = ~((1ull << t_lo) - 1ull);
                        valid_m = upto & from;
                    }
                    for (uint32_t c = 0; c < alpha; c++)
                        peq[c * Lw + w] = ((c & 1u) ? lo : ~lo) & ((c & 2u) ? hi : ~hi) & valid_m;
                }
            } else {
                for (int i = gl; i < (int)alpha * Lw; i += G) peq[i] = 0ull;
                __syncwarp();
                for (int64_t ch = gl; ch < xch; ch += G) {
                    const uint4 v = xc[ch];
                    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int t = 0; t < 16; t++) {
                        const int64_t k = ch * 16 + t;
                        const uint32_t c = (wv[t >> 2] >> ((t & 3) * 8)) & 0xFFu;
                        if (k < mrows && c < alpha) {
                            const uint32_t q = (uint32_t)K + (uint32_t)k;
                            atomicOr((unsigned long long *)&peq[c * Lw + (q >> 6)], 1ull << (q & 63u));
                        }
                    }
                }
            }
            __syncwarp();
        }
        SymReader<B> yr;
        yr.init(yc_base, chunks_for(ncols, B));

        // column 0: rows -K..0 have difference -1, rows >= 1 have +1; T = K+1
        uint64_t Pv[V], Mv[V];
#pragma unroll
        for (int v = 0; v < V; v++) {
            const int lo = 64 * (gl * V + v);
            if (K >= lo + 63) {
                Mv[v] = ~0ull; Pv[v] = 0ull;
            } else if (K < lo) {
                Mv[v] = 0ull; Pv[v] = ~0ull;
            } else {
                const int nb = K - lo + 1;
                Mv[v] = (1ull << nb) - 1ull;
                Pv[v] = ~Mv[v];
            }
        }
        int32_t T = K + 1;

        int32_t nmax = __reduce_max_sync(FULL, ncols);
        for (int32_t j = 1; j <= nmax; j++) {
            const bool act = j <= ncols;
            const uint32_t c = yr.code();
            if (act) yr.advance();

            // T := value of the row above the shifted window
            if (gl == 0 && act) T += (int32_t)(Pv[0] & 1ull) - (int32_t)(Mv[0] & 1ull) + 1;

            // shift the window down one row; the new bottom row has difference +1
            uint32_t low = (uint32_t)(Pv[0] & 1ull) | ((uint32_t)(Mv[0] & 1ull) << 1);
            uint32_t nxt = (G > 1) ? __shfl_down_sync(FULL, low, 1, G) : low;
            if (gl == G - 1) nxt = 1u;
            uint64_t nP[V], nM[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const uint64_t upP = (v + 1 < V) ? Pv[v + 1 < V ? v + 1 : v] : (uint64_t)(nxt & 1u);
                const uint64_t upM = (v + 1 < V) ? Mv[v + 1 < V ? v + 1 : v] : (uint64_t)(nxt >> 1);
                nP[v] = (Pv[v] >> 1) | (upP << 63);
                nM[v] = (Mv[v] >> 1) | (upM << 63);
            }

            // match masks of the window rows against y[j-1]
            const bool cval = act && c < alpha;  // a symbol outside the alphabet matches nothing
            const uint64_t *row = peq + (size_t)(cval ? c : 0u) * Lw;
            const uint32_t q0 = (uint32_t)(j - 1) + 64u * (uint32_t)(gl * V);
            const uint32_t sh = q0 & 63u;
            const uint32_t i0 = q0 >> 6;
            uint64_t Eq[V];
            {
                uint64_t w_lo = cval ? row[i0] : 0ull;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const uint64_t w_hi = cval ? row[i0 + v + 1] : 0ull;
                    Eq[v] = funnel64(w_lo, w_hi, sh);
                    w_lo = w_hi;
                }
            }

            // bit-vector step (Myers/Hyyro): Xh = (((Eq & Pv) + Pv) ^ Pv) | Eq
            uint64_t S[V];
            uint32_t cy = 0;
#pragma unroll
            for (int v = 0; v < V; v++) {
                const uint64_t x1 = Eq[v] & nP[v];
                const uint64_t t1 = x1 + nP[v];
                const uint32_t c1 = t1 < x1;
                const uint64_t s1 = t1 + cy;
                const uint32_t c2 = s1 < t1;
                S[v] = s1;
                cy = c1 | c2;
            }
            if (G > 1) {
                bool prop = true;
#pragma unroll
                for (int v = 0; v < V; v++) prop = prop && (S[v] == ~0ull);
                const unsigned gb = __ballot_sync(FULL, cy != 0u);
                const unsigned pb = __ballot_sync(FULL, prop);
                const unsigned sel = (G == 32) ? FULL : ((1u << G) - 1u);
                const unsigned gG = (gb >> (g * G)) & sel;
                const unsigned gP = (pb >> (g * G)) & sel;
                const unsigned A = gG | gP;
                const unsigned carries = (A + gG) ^ A ^ gG;  // carry into each lane
                uint32_t cin = (carries >> gl) & 1u;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const uint64_t s2 = S[v] + cin;
                    cin = cin & (s2 == 0ull ? 1u : 0u);
                    S[v] = s2;
                }
            }
            uint64_t Ph[V], Mh[V], X[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                X[v] = Eq[v] | nM[v];
                const uint64_t Xh = (S[v] ^ nP[v]) | Eq[v];
                Ph[v] = nM[v] | ~(Xh | nP[v]);
                Mh[v] = nP[v] & Xh;
            }
            // shift the horizontal differences down one row; the row above the
            // window contributes +1 (Ph shift-in 1, Mh shift-in 0)
            const uint32_t top = (uint32_t)(Ph[V - 1] >> 63) | ((uint32_t)(Mh[V - 1] >> 63) << 1);
            uint32_t prv = (G > 1) ? __shfl_up_sync(FULL, top, 1, G) : top;
            if (gl == 0) prv = 1u;
#pragma unroll
            for (int v = V - 1; v >= 0; v--) {
                const uint64_t inP = (v > 0) ? (Ph[v > 0 ? v - 1 : 0] >> 63) : (uint64_t)(prv & 1u);
                const uint64_t inM = (v > 0) ? (Mh[v > 0 ? v - 1 : 0] >> 63) : (uint64_t)(prv >> 1);
                Ph[v] = (Ph[v] << 1) | inP;
                Mh[v] = (Mh[v] << 1) | inM;
            }
            if (act) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    Pv[v] = Mh[v] | ~(X[v] | Ph[v]);
                    Mv[v] = Ph[v] & X[v];
                }
            }

            // early exit: minimum of the window exceeds K
            if ((j & 63) == 0 && j < nmax) {
                int32_t run = 0, mn = 1 << 30;
#pragma unroll
                for (int v = 0; v < V; v++) {
#pragma unroll
                    for (int k = 0; k < 16; k++) {
                        const uint32_t idx = (uint32_t)((Pv[v] >> (4 * k)) & 15u) |
                                             ((uint32_t)((Mv[v] >> (4 * k)) & 15u) << 4);
                        const int32_t cand = run + s_nmin[idx];
                        mn = cand < mn ? cand : mn;
                        run += s_nsum[idx];
                    }
                }
                // prefix of run over the group's lanes (in lane order)
                int32_t inc = run;
#pragma unroll
                for (int o = 1; o < G; o <<= 1) {
                    const int32_t t = __shfl_up_sync(FULL, inc, o, G);
                    if (gl >= o) inc += t;
                }
                int32_t gmin = mn + (inc - run);
#pragma unroll
                for (int o = 1; o < G; o <<= 1) {
                    const int32_t t = __shfl_xor_sync(FULL, gmin, o, G);
                    gmin = t < gmin ? t : gmin;
                }
                const int32_t T0 = (G > 1) ? __shfl_sync(FULL, T, 0, G) : T;
                if (act && T0 + gmin > kp) {
                    decided = true;
                    pass = false;
                    ncols = 0;
                    cols_run = j;
                }
                nmax = __reduce_max_sync(FULL, ncols);
            }
        }

        {
            // D(m, n) = T + sum of differences of window bits 0 .. m - n + K
            // (computed by every lane so that the collectives stay converged)
            const int32_t bmax = (mrows - ncols) + K;
            int32_t cnt = 0;
#pragma unroll
            for (int v = 0; v < V; v++) {
                const int lo = 64 * (gl * V + v);
                uint64_t mask;
                if (lo > bmax) mask = 0ull;
                else if (lo + 63 <= bmax) mask = ~0ull;
                else mask = (1ull << (bmax - lo + 1)) - 1ull;
                cnt += __popcll(Pv[v] & mask) - __popcll(Mv[v] & mask);
            }
#pragma unroll
            for (int o = 1; o < G; o <<= 1) cnt += __shfl_xor_sync(FULL, cnt, o, G);
            const int32_t T0 = (G > 1) ? __shfl_sync(FULL, T, 0, G) : T;
            if (!decided) pass = (T0 + cnt) <= kp;
        }
        if (valid && gl == 0) {
            emit_result(vo, p, pairs, pass);
            loc_cells += band_cells(mlen, nlen, kp);
            loc_cols += (unsigned long long)cols_run * (unsigned long long)w_min;
        }
        __syncwarp();
    }
    // work counters: one atomic per warp (per-pair atomics on two addresses
    // serialise in the memory system)
    if (work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loc_cells += __shfl_xor_sync(FULL, loc_cells, o);
            loc_cols += __shfl_xor_sync(FULL, loc_cols, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (loc_cells) atomicAdd(&work[0], loc_cells);
            if (loc_cols) atomicAdd(&work[1], loc_cols);
        }
    }
}


// ---------------------------------------------------------------------------
// One lane per pair: the whole window of W <= 8 words lives in one thread
// ---------------------------------------------------------------------------
//
// Same recurrence and boundaries as verify_kernel, without cross-lane traffic.
// The match masks are not stored for all of x: a ring of R = W+2 words per
// symbol holds Peq words i0 .. i0+W (i0 = (j-1)/64) and one new word is built
// every 64 columns, so shared memory per pair is alpha*(W+2) words instead of
// alpha*|x|/64.

constexpr int VG1_MAX_THREADS = 128;

template <int W, int B>
__global__ void __launch_bounds__(VG1_MAX_THREADS)
verify_g1_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                 const int32_t *__restrict__ lens, int64_t n_str, uint32_t alpha,
                 const uint64_t *__restrict__ pairs, int64_t np, int32_t K,
                 VerifyOut vo) {
    uint32_t *__restrict__ err = vo.err;
    unsigned long long *__restrict__ work = vo.work;
    if (vo.np_dev) {
        const int64_t dn = (int64_t)*vo.np_dev;
        np = dn < np ? dn : np;
    }
    constexpr int R = W + 2;
    unsigned long long loc_cells = 0, loc_cols = 0;
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
    const int T_ = blockDim.x;
    // ring word (c, slot) of this thread: smem[(c * R + slot) * T_ + tid]
    uint64_t *ring = smem + threadIdx.x;
    const int32_t w_min = (2 * K + 1 + 63) / 64;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;

    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
        const uint64_t pr = pairs[p];
        const int64_t a = (int64_t)(pr >> 32), b = (int64_t)(pr & 0xFFFFFFFFull);
        if (a >= n_str || b >= n_str) {
            atomicOr(err, (uint32_t)DERR_PAIR);
            continue;
        }
        const int32_t la = lens[a], lb = lens[b];
        const bool a_long = la >= lb;
        const int64_t xi = a_long ? a : b, yi = a_long ? b : a;
        const int32_t mrows = a_long ? la : lb, ncols = a_long ? lb : la;
        bool pass;
        int32_t cols_run = 0;
        if (mrows - ncols > K) {
            pass = false;
        } else if (ncols == 0) {
            pass = mrows <= K;
        } else {
            const uint4 *xc = packed + pofs[xi];
            const int64_t xch = chunks_for(mrows, B);
            // Peq word wi (bits <-> x symbols 64*wi-K .. +63) into ring slot `slot`
            auto build = [&](int64_t wi, int slot) {
                const int64_t k0 = 64ll * wi - K;
                const int64_t t_lo = k0 < 0 ? -k0 : 0;
                const int64_t t_hi = (int64_t)mrows - k0;
                uint64_t valid_m = 0ull;
                if (t_hi > t_lo && t_lo < 64) {
                    const uint64_t upto = t_hi >= 64 ? ~0ull : ((1ull << t_hi) - 1ull);
                    valid_m = upto & ~((1ull << t_lo) - 1ull);
                }
                if (B == 2) {
                    uint64_t lo = 0, hi = 0;
                    if (valid_m) sym64_planes(xc, xch, k0, lo, hi);
                    for (uint32_t c = 0; c < alpha; c++)
                        ring[(size_t)(c * R + slot) * T_] = ((c & 1u) ? lo : ~lo) & ((c & 2u) ? hi : ~hi) & valid_m;
                } else {
                    for (uint32_t c = 0; c < alpha; c++) ring[(size_t)(c * R + slot) * T_] = 0ull;
                    if (valid_m) {
                        const int64_t ks = k0 + t_lo, ke = k0 + (t_hi < 64 ? t_hi : 64);
                        for (int64_t k = ks; k < ke; k++) {
                            const uint4 v = xc[k >> 4];
                            const uint32_t sel = (uint32_t)(k & 15);
                            const uint32_t wv = (sel < 8) ? ((sel < 4) ? v.x : v.y) : ((sel < 12) ? v.z : v.w);
                            const uint32_t c = (wv >> ((sel & 3u) * 8u)) & 0xFFu;
                            if (c < alpha) ring[(size_t)(c * R + slot) * T_] |= 1ull << (uint32_t)(k - k0);
                        }
                    }
                }
            };
#pragma unroll 1
            for (int wi = 0; wi <= W; wi++) build(wi, wi);
            int base = 0;  // ring slot of word i0

            uint64_t Pv[W], Mv[W];
#pragma unroll
            for (int v = 0; v < W; v++) {
                const int lo = 64 * v;
                if (K >= lo + 63) { Mv[v] = ~0ull; Pv[v] = 0ull; }
                else if (K < lo) { Mv[v] = 0ull; Pv[v] = ~0ull; }
                else { Mv[v] = (1ull << (K - lo + 1)) - 1ull; Pv[v] = ~Mv[v]; }
            }
            int32_t T = K + 1;
            SymReader<B> yr;
            yr.init(packed + pofs[yi], chunks_for(ncols, B));
            bool rejected = false;
            int32_t j = 1;
            for (; j <= ncols; j++) {
                const uint32_t jm = (uint32_t)(j - 1);
                if ((jm & 63u) == 0u && j > 1) {
                    // window start moved to word i0: word wi lives in slot wi mod R, so
                    // word i0+W takes the slot of word i0-2 (R = W+2), no longer read
                    const int64_t i0 = jm >> 6;
                    base = (base + 1 == R) ? 0 : base + 1;
                    int slot = base + W;
                    if (slot >= R) slot -= R;
                    build(i0 + W, slot);
                    // early exit: the minimum of the window exceeds K
                    int32_t run = 0, mn = 1 << 30;
#pragma unroll
                    for (int v = 0; v < W; v++) {
#pragma unroll
                        for (int k = 0; k < 16; k++) {
                            const uint32_t idx = (uint32_t)((Pv[v] >> (4 * k)) & 15u) |
                                                 ((uint32_t)((Mv[v] >> (4 * k)) & 15u) << 4);
                            const int32_t cand = run + s_nmin[idx];
                            mn = cand < mn ? cand : mn;
                            run += s_nsum[idx];
                        }
                    }
                    if (T + mn > K) {
                        rejected = true;
                        break;
                    }
                }
                const uint32_t c = yr.code();
                yr.advance();
                T += (int32_t)(Pv[0] & 1ull) - (int32_t)(Mv[0] & 1ull) + 1;
                uint64_t nP[W], nM[W];
#pragma unroll
                for (int v = 0; v < W; v++) {
                    const uint64_t upP = (v + 1 < W) ? Pv[v + 1 < W ? v + 1 : v] : 1ull;
                    const uint64_t upM = (v + 1 < W) ? Mv[v + 1 < W ? v + 1 : v] : 0ull;
                    nP[v] = (Pv[v] >> 1) | (upP << 63);
                    nM[v] = (Mv[v] >> 1) | (upM << 63);
                }
                uint64_t Eq[W];
                {
                    const uint32_t sh = jm & 63u;
                    const uint64_t *row = ring + (size_t)(c < alpha ? c : 0u) * R * T_;
                    int sl = base;
                    uint64_t w_lo = (c < alpha) ? row[(size_t)sl * T_] : 0ull;
#pragma unroll
                    for (int v = 0; v < W; v++) {
                        sl = (sl + 1 == R) ? 0 : sl + 1;
                        const uint64_t w_hi = (c < alpha) ? row[(size_t)sl * T_] : 0ull;
                        Eq[v] = funnel64(w_lo, w_hi, sh);
                        w_lo = w_hi;
                    }
                }
                uint64_t A[W], S[W];
#pragma unroll
                for (int v = 0; v < W; v++) A[v] = Eq[v] & nP[v];
                add_chain<W>(S, A, nP);
                uint64_t Ph[W], Mh[W];
#pragma unroll
                for (int v = 0; v < W; v++) {
                    const uint64_t Xh = (S[v] ^ nP[v]) | Eq[v];
                    Ph[v] = nM[v] | ~(Xh | nP[v]);
                    Mh[v] = nP[v] & Xh;
                }
#pragma unroll
                for (int v = W - 1; v >= 0; v--) {
                    const uint64_t inP = (v > 0) ? (Ph[v > 0 ? v - 1 : 0] >> 63) : 1ull;
                    const uint64_t inM = (v > 0) ? (Mh[v > 0 ? v - 1 : 0] >> 63) : 0ull;
                    Ph[v] = (Ph[v] << 1) | inP;
                    Mh[v] = (Mh[v] << 1) | inM;
                }
#pragma unroll
                for (int v = 0; v < W; v++) {
                    const uint64_t X = Eq[v] | nM[v];
                    Pv[v] = Mh[v] | ~(X | Ph[v]);
                    Mv[v] = Ph[v] & X;
                }
            }
            cols_run = rejected ? j - 1 : ncols;
            if (rejected) {
                pass = false;
            } else {
                const int32_t bmax = (mrows - ncols) + K;
                int32_t cnt = 0;
#pragma unroll
                for (int v = 0; v < W; v++) {
                    const int lo = 64 * v;
                    uint64_t mask;
                    if (lo > bmax) mask = 0ull;
                    else if (lo + 63 <= bmax) mask = ~0ull;
                    else mask = (1ull << (bmax - lo + 1)) - 1ull;
                    cnt += __popcll(Pv[v] & mask) - __popcll(Mv[v] & mask);
                }
                pass = (T + cnt) <= K;
            }
        }
        emit_result(vo, p, pairs, pass);
        loc_cells += band_cells(mrows, ncols, K);
        loc_cols += (unsigned long long)cols_run * (unsigned long long)w_min;
    }
    // work counters: one atomic per warp (per-pair atomics on two addresses
    // serialise in the memory system)
    if (work) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loc_cells += __shfl_xor_sync(FULL, loc_cells, o);
            loc_cols += __shfl_xor_sync(FULL, loc_cols, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (loc_cells) atomicAdd(&work[0], loc_cells);
            if (loc_cols) atomicAdd(&work[1], loc_cols);
        }
    }
}

template <int W, int B>
static cudaError_t launch_g1(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                             uint32_t alpha, const uint64_t *pairs, int64_t np, int32_t K, int warps,
                             VerifyOut vo, cudaStream_t s) {
    const int threads = warps * 32;
    const size_t smem = (size_t)alpha * (W + 2) * sizeof(uint64_t) * threads;
    cudaError_t e = cudaFuncSetAttribute(verify_g1_kernel<W, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_g1_kernel<W, B>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (np + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    verify_g1_kernel<W, B><<<(unsigned)blocks, threads, smem, s>>>(packed, pofs, lens, n, alpha, pairs, np, K,
                                                                    vo);
    note_launches(1);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Two lanes per pair: forward and backward halves of a block-aligned band
// ---------------------------------------------------------------------------
//
// Block-aligned window. Rows are grouped in fixed 64-row words (word k holds
// rows 64k+1 .. 64k+64). At column j the thread keeps W1 consecutive words
// starting at k0 = max(0, floor((j-K-1)/64)); 64*W1 >= 2K+1+64 rows always
// cover Ukkonen's band [j-K, j+K]. Match masks are then Peq words as they are
// (no per-column funnel) and the window moves by one whole word every 64
// columns: the top word's differences are folded into T, the value of row
// 64*k0 (the row above the window), and a fresh bottom word enters with
// vertical differences +1. Row 64*k0 lies outside the band (64*k0 < j-K), so
// it is replaced by the upper bound "+1 per column" (real when k0 = 0: D(0,j)
// = j), and the same argument as for the diagonal window gives exactness for
// values <= K.
//
// Bidirectional split. With n1 = n/2, ED(x, y) = min_i D(i, n1) + ED(x[i:], y[n1:]).
// Lane 2t computes D(., n1) forward; lane 2t+1 runs the same recurrence on the
// reversed strings for n - n1 columns, which gives ED(x[i:], y[n1:]) for the
// rows of its window. Both halves are exact where their value is <= K and
// >= min(true, K+1) elsewhere; an optimal path of cost <= K crosses column n1
// inside both bands, so "min_i F(i) + B(i) <= K" decides ED <= K exactly. The
// two halves run concurrently, halving the sequential chain of a pair.

constexpr int VBD_THREADS = 128;
constexpr int VBD_CHECK = 32;   // columns between the joint early-exit tests (a power of two)

template <int W1, int B>
__global__ void __launch_bounds__(VBD_THREADS)
verify_bd_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                 const int32_t *__restrict__ lens, int64_t n_str, uint32_t alpha,
                 const uint64_t *__restrict__ pairs, int64_t np, int32_t K,
                 VerifyOut vo) {
    uint32_t *__restrict__ err = vo.err;
    unsigned long long *__restrict__ work = vo.work;
    if (vo.np_dev) {
        const int64_t dn = (int64_t)*vo.np_dev;
        np = dn < np ? dn : np;
    }
    constexpr int R = W1 + 1;
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
    const int T_ = blockDim.x;           // slot stride of the per-thread ring
    uint64_t *ring = smem + threadIdx.x;  // per thread: (c*R + slot)*T_, reused as a dump area
    const int lane = threadIdx.x & 31;
    const bool rev = lane & 1;
    const unsigned pmask = 3u << (lane & ~1);
    const int32_t w_min = (2 * K + 1 + 63) / 64;
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 1);
    const int64_t niter = (np + stride - 1) / stride;   // the same on every lane: the warp ends together
    unsigned long long loc_cells = 0, loc_cols = 0;

    for (int64_t it = 0; it < niter; it++) {
        const int64_t p = it * stride + (int64_t)blockIdx.x * (blockDim.x >> 1) + (threadIdx.x >> 1);
        bool valid = p < np;
        int64_t a = 0, b = 0;
        if (valid) {
            const uint64_t pr = pairs[p];
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
        bool decided = !valid, pass = false;
        if (valid && m - n > K) decided = true;
        else if (valid && n == 0) { decided = true; pass = m <= K; }
        const int32_t n1 = n / 2;
        const int32_t ncols = decided ? 0 : (rev ? n - n1 : n1);

        uint64_t Pv[W1], Mv[W1];
        int32_t T = 0;
        int64_t k0 = 0;
        bool rejected = false;
        int32_t cols_run = 0;
        if (!decided) {
            const uint4 *xc = packed + pofs[xi];
            for (int wi = 0; wi < W1; wi++) bd_build<B, R>(ring, T_, wi, xc, m, wi, rev, alpha);
#pragma unroll
            for (int v = 0; v < W1; v++) { Pv[v] = ~0ull; Mv[v] = 0ull; }
            int base = 0;  // slot of word k0
            uint32_t soff[W1];   // element offset of the slot of word k0+v
#pragma unroll
            for (int v = 0; v < W1; v++) soff[v] = (uint32_t)v * T_;
            SymReader<B> yf;
            SymReaderRev<B> yb;
            if (rev) yb.init(packed + pofs[yi], n);
            else yf.init(packed + pofs[yi], chunks_for(n1, B));
            const uint32_t cmax = alpha - 1u;
            int32_t next_move = K + 1 + 64;   // first column whose window starts one word lower
            int32_t j = 1;
            for (; j <= ncols; j++) {
                if ((j & (VBD_CHECK - 1)) == 0 && j <= n1) {
                    // early exit, decided by both halves together: the minimum of each
                    // half's window at its column j-1 (row 64*k0, value T, included).
                    // A path of cost <= K crosses both columns inside the band, where
                    // the values are exact, so the two minima add up to at most its
                    // cost. Both lanes of the pair reach every such column (j <= n1 <=
                    // n - n1), so they exchange and leave together.
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
                    const int32_t lb = T + mn;
                    const int32_t lb_other = __shfl_xor_sync(pmask, lb, 1);
                    if (lb + lb_other > K) {
                        rejected = true;
                        break;
                    }
                }
                if (j == next_move) {
                    next_move += 64;
                    // drop the top word into T, shift the window down one word
                    T += __popcll(Pv[0]) - __popcll(Mv[0]);
#pragma unroll
                    for (int v = 0; v + 1 < W1; v++) { Pv[v] = Pv[v + 1]; Mv[v] = Mv[v + 1]; }
                    Pv[W1 - 1] = ~0ull;
                    Mv[W1 - 1] = 0ull;
                    k0++;
                    base = (base + 1 == R) ? 0 : base + 1;
#pragma unroll
                    for (int v = 0; v < W1; v++) {
                        const int sl = base + v;
                        soff[v] = (uint32_t)(sl >= R ? sl - R : sl) * T_;
                    }
                    bd_build<B, R>(ring, T_, (int)(soff[W1 - 1] / T_), xc, m, k0 + W1 - 1, rev, alpha);
                }
                uint32_t c;
                if (rev) { c = yb.code(); yb.advance(); }
                else { c = yf.code(); yf.advance(); }
                c = c < cmax ? c : cmax;   // codes of a validated string are < alpha
                const uint64_t *row = ring + (size_t)c * R * T_;
                uint64_t Eq[W1];
#pragma unroll
                for (int v = 0; v < W1; v++) Eq[v] = row[soff[v]];
                uint64_t A[W1], S[W1];
#pragma unroll
                for (int v = 0; v < W1; v++) A[v] = Eq[v] & Pv[v];
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
                T += 1;  // the row above the window: +1 per column
            }
            cols_run = rejected ? j - 1 : ncols;
        }
        // exchange: dump state into this thread's ring area
#pragma unroll
        for (int v = 0; v < W1; v++) {
            ring[(size_t)(2 * v) * T_] = Pv[v];
            ring[(size_t)(2 * v + 1) * T_] = Mv[v];
        }
        ring[(size_t)(2 * W1) * T_] = (uint64_t)(uint32_t)T | ((uint64_t)k0 << 32);
        ring[(size_t)(2 * W1 + 1) * T_] = rejected ? 1ull : 0ull;
        __syncwarp(pmask);
        if (!rev && !decided) {
            const uint64_t *rb = smem + threadIdx.x + 1;  // partner (backward) dump
            const bool rej_b = rb[(size_t)(2 * W1 + 1) * T_] != 0ull;
            if (rejected || rej_b) {
                pass = false;
            } else {
                const uint64_t tb = rb[(size_t)(2 * W1) * T_];
                const int32_t Tb = (int32_t)(uint32_t)(tb & 0xFFFFFFFFull);
                const int64_t k0b = (int64_t)(tb >> 32);
                const int64_t k0f = k0;
                const uint64_t *rf = ring;
                // forward rows: [64 k0f, min(m, 64(k0f+W1))]; backward rows i' -> i = m - i'
                const int64_t f_hi = min((int64_t)m, 64 * (k0f + W1));
                const int64_t b_hi = min((int64_t)m, 64 * (k0b + W1));
                const int64_t i_lo = max(64 * k0f, (int64_t)m - b_hi);
                const int64_t i_hi = min(f_hi, (int64_t)m - 64 * k0b);
                if (i_lo > i_hi) {
                    pass = false;
                } else {
                    // F(i_lo) = T_f + sum of forward differences of rows 64k0f+1 .. i_lo
                    auto prefix = [&](const uint64_t *dump, int64_t k0x, int32_t Tx, int64_t row) -> int32_t {
                        int32_t acc = Tx;
                        const int64_t nrows = row - 64 * k0x;  // rows 64k0x+1 .. row
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
                        // F(i+1) = F(i) + dv_f(row i+1); B(i+1) = B(i) - dv_b(row m-i)
                        const int64_t rf_ = i + 1 - 64 * k0f - 1;          // 0-based bit in forward window
                        const int64_t rb_ = (int64_t)m - i - 64 * k0b - 1;   // 0-based bit in backward window
                        const uint64_t fp = rf[(size_t)(2 * (rf_ >> 6)) * T_], fm = rf[(size_t)(2 * (rf_ >> 6) + 1) * T_];
                        const uint64_t bp = rb[(size_t)(2 * (rb_ >> 6)) * T_], bm = rb[(size_t)(2 * (rb_ >> 6) + 1) * T_];
                        F += (int32_t)((fp >> (rf_ & 63)) & 1ull) - (int32_t)((fm >> (rf_ & 63)) & 1ull);
                        Bv -= (int32_t)((bp >> (rb_ & 63)) & 1ull) - (int32_t)((bm >> (rb_ & 63)) & 1ull);
                        best = min(best, F + Bv);
                    }
                    pass = best <= K;
                }
            }
        }
        if (valid && !rev) emit_result(vo, p, pairs, pass);
        if (valid) {
            if (!rev) loc_cells += band_cells(m, n, K);
            loc_cols += (unsigned long long)cols_run * (unsigned long long)w_min;
        }
        __syncwarp(pmask);
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

template <int W1, int B>
static cudaError_t launch_bd(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                             uint32_t alpha, const uint64_t *pairs, int64_t np, int32_t K, int warps,
                             VerifyOut vo, cudaStream_t s) {
    // blocks of `warps` warps (fewer when the per-thread ring of a large alphabet
    // would not fit shared memory)
    int threads = (warps > 0 ? warps : 4) * 32;
    if (threads > VBD_THREADS) threads = VBD_THREADS;
    const int R = W1 + 1;
    const size_t per_thread = (size_t)(alpha * R > 2 * W1 + 2 ? alpha * R : 2 * W1 + 2) * sizeof(uint64_t);
    while (threads > 32 && per_thread * threads > 200 * 1024) threads >>= 1;
    const size_t smem = per_thread * threads;
    cudaError_t e = cudaFuncSetAttribute(verify_bd_kernel<W1, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_bd_kernel<W1, B>, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t pairs_per_block = threads / 2;
    int64_t blocks = (np + pairs_per_block - 1) / pairs_per_block;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    verify_bd_kernel<W1, B><<<(unsigned)blocks, threads, smem, s>>>(packed, pofs, lens, n, alpha, pairs, np, K,
                                                                     vo);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Configuration
// ---------------------------------------------------------------------------

static int words_needed(int32_t K) { return (2 * K + 1 + 63) / 64; }

static int32_t peq_words(int64_t max_len, int32_t K, int W) {
    return (int32_t)(((max_len + (int64_t)K + 64ll * W) >> 6) + 2);
}

size_t verify_smem_bytes(VerifyConfig c, uint32_t alpha, int64_t max_len, int32_t K) {
    if (c.G == 1) return (size_t)c.warps * 32 * alpha * (c.V + 2) * sizeof(uint64_t);
    if (c.G == 2) {
        const size_t per = (size_t)(alpha * (c.V + 1) > (uint32_t)(2 * c.V + 2) ? alpha * (c.V + 1) : 2 * c.V + 2);
        return (size_t)c.warps * 32 * per * sizeof(uint64_t);
    }
    const int W = c.G * c.V;
    return (size_t)c.warps * (32 / c.G) * alpha * (size_t)peq_words(max_len, K, W) * sizeof(uint64_t);
}

VerifyConfig verify_pick(int32_t K, uint32_t alpha, int64_t max_len) {
    const int W = words_needed(K);
    if (W + 1 <= 12) {
        // forward/backward halves, block-aligned window of W+1 words per lane
        VerifyConfig c{2, W + 1, 4};
        while (c.warps > 1 && verify_smem_bytes(c, alpha, max_len, K) > 100 * 1024) c.warps >>= 1;
        if (verify_smem_bytes(c, alpha, max_len, K) <= 200 * 1024) return c;
    }
    if (W <= 8) {
        // one lane per pair, the window in registers, a Peq ring in shared memory
        VerifyConfig c{1, W, 4};
        while (c.warps > 1 && verify_smem_bytes(c, alpha, max_len, K) > 100 * 1024) c.warps >>= 1;
        if (verify_smem_bytes(c, alpha, max_len, K) <= 200 * 1024) return c;
    }
    // wider bands: G lanes per pair (power of two), V words per lane
    VerifyConfig best{0, 0, 0};
    int best_words = 1 << 30;
    bool best_fit = false;
    for (int V = 4; V >= 1; V--) {
        int G = 4;
        while (G * V < W && G < 32) G <<= 1;
        if (G * V < W) continue;
        VerifyConfig c{G, V, 1};
        const size_t per_warp = verify_smem_bytes(c, alpha, max_len, K);
        if (per_warp > 200 * 1024) continue;
        const bool fit = per_warp <= 28 * 1024;
        const int words = G * V;
        if ((fit && !best_fit) || (fit == best_fit && words < best_words)) {
            best = c;
            best_words = words;
            best_fit = fit;
        }
    }
    if (best.G == 0) return best;
    const size_t per_warp = verify_smem_bytes(best, alpha, max_len, K);
    int warps = (int)((96 * 1024) / (per_warp ? per_warp : 1));
    if (warps > VERIFY_MAX_THREADS / 32) warps = VERIFY_MAX_THREADS / 32;
    if (warps < 1) warps = 1;
    best.warps = warps;
    return best;
}

template <int G, int V, int B>
static cudaError_t launch_gv(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                             uint32_t alpha, const uint64_t *pairs, int64_t np,
                             int32_t K, int64_t max_len, int warps, VerifyOut vo, cudaStream_t s) {
    const int32_t Lw = peq_words(max_len, K, G * V);
    const size_t smem = (size_t)warps * (32 / G) * alpha * Lw * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(verify_kernel<G, V, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, verify_kernel<G, V, B>, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t warp_batches = (np + (32 / G) - 1) / (32 / G);
    int64_t blocks = (warp_batches + warps - 1) / warps;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    verify_kernel<G, V, B><<<(unsigned)blocks, warps * 32, smem, s>>>(packed, pofs, lens, n, alpha,
                                                                     pairs, np, K, Lw, vo);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_verify(VerifyConfig c, const uint4 *packed, const uint64_t *pofs, int B,
                          const int32_t *lens, int64_t n, uint32_t alpha,
                          const uint64_t *pairs, int64_t np, int32_t K, int64_t max_len,
                          VerifyOut vo, cudaStream_t s) {
    if (np == 0) return cudaGetLastError();
#define EJ_V(GG, VV)                                                                                     \
    if (c.G == GG && c.V == VV) {                                                                        \
        if (B == 2)                                                                                      \
            return launch_gv<GG, VV, 2>(packed, pofs, lens, n, alpha, pairs, np, K, max_len, c.warps,    \
                                        vo, s);                                            \
        return launch_gv<GG, VV, 8>(packed, pofs, lens, n, alpha, pairs, np, K, max_len, c.warps, vo, s); \
    }
    if (c.G == 1) {
#define EJ_G1(WW)                                                                                         \
    if (c.V == WW) {                                                                                      \
        if (B == 2)                                                                                       \
            return launch_g1<WW, 2>(packed, pofs, lens, n, alpha, pairs, np, K, c.warps, vo, s); \
        return launch_g1<WW, 8>(packed, pofs, lens, n, alpha, pairs, np, K, c.warps, vo, s);     \
    }
        EJ_G1(1) EJ_G1(2) EJ_G1(3) EJ_G1(4) EJ_G1(5) EJ_G1(6) EJ_G1(7) EJ_G1(8)
#undef EJ_G1
        return cudaErrorInvalidValue;
    }
    if (c.G == 2) {
#define EJ_BD(WW)                                                                                          \
    if (c.V == WW) {                                                                                       \
        if (B == 2)                                                                                        \
            return launch_bd<WW, 2>(packed, pofs, lens, n, alpha, pairs, np, K, c.warps, vo, s); \
        return launch_bd<WW, 8>(packed, pofs, lens, n, alpha, pairs, np, K, c.warps, vo, s);     \
    }
        EJ_BD(2) EJ_BD(3) EJ_BD(4) EJ_BD(5) EJ_BD(6) EJ_BD(7) EJ_BD(8) EJ_BD(9) EJ_BD(10) EJ_BD(11) EJ_BD(12)
#undef EJ_BD
        return cudaErrorInvalidValue;
    }
    EJ_V(4, 1) EJ_V(4, 2) EJ_V(4, 3) EJ_V(4, 4)
    EJ_V(8, 1) EJ_V(8, 2) EJ_V(8, 3) EJ_V(8, 4)
    EJ_V(16, 1) EJ_V(16, 2) EJ_V(16, 3) EJ_V(16, 4)
    EJ_V(32, 1) EJ_V(32, 2) EJ_V(32, 3) EJ_V(32, 4)
#undef EJ_V
    return cudaErrorInvalidValue;
}

}  // namespace ej
