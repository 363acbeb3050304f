// Device helpers shared by the bit-parallel verifiers: packed-symbol access,
// multi-word addition, Ukkonen's band size, Peq words of a 64-row block, and
// the result emission of one verified pair.
#pragma once
#include "ej_internal.cuh"

namespace ej {

__device__ __forceinline__ void emit_result(const VerifyOut &vo, int64_t p, const uint64_t *__restrict__ pairs,
                                            bool pass) {
    if (vo.app) {
        if (pass) {
            const unsigned long long idx = atomicAdd(vo.app_count, 1ull);
            if (idx < vo.app_cap) vo.app[idx] = pairs[p];
        }
    } else {
        vo.flags[p] = pass ? 1 : 0;
    }
}


__device__ __forceinline__ uint64_t funnel64(uint64_t lo, uint64_t hi, uint32_t sh) {
    return sh ? ((lo >> sh) | (hi << (64u - sh))) : lo;
}

// Gathers the even bits of x into the low 16 bits.
__device__ __forceinline__ uint32_t compress_even(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// Symbols k0 .. k0+63 of a 2-bit packed string (nch chunks) as two bit-planes:
// bit t of lo/hi = low/high bit of the code of symbol k0+t (0 outside the string).
__device__ __forceinline__ void sym64_planes(const uint4 *__restrict__ xc, int64_t nch, int64_t k0,
                                             uint64_t &lo, uint64_t &hi) {
    const int64_t c0 = (k0 >= 0) ? (k0 >> 6) : -((-k0 + 63) >> 6);
    const uint32_t o = (uint32_t)(k0 - 64 * c0);  // 0..63 symbols
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    const uint4 A = (c0 >= 0 && c0 < nch) ? xc[c0] : zero;
    const uint4 Bc = (c0 + 1 >= 0 && c0 + 1 < nch) ? xc[c0 + 1] : zero;
    uint32_t t0 = A.x, t1 = A.y, t2 = A.z, t3 = A.w, t4 = Bc.x, t5 = Bc.y, t6 = Bc.z, t7 = Bc.w;
    const uint32_t sh = 2u * o, ws = sh >> 5, bs = sh & 31u;
    if (ws & 2u) { t0 = t2; t1 = t3; t2 = t4; t3 = t5; t4 = t6; t5 = t7; t6 = 0u; t7 = 0u; }
    if (ws & 1u) { t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = 0u; }
    const uint32_t w0 = __funnelshift_r(t0, t1, bs), w1 = __funnelshift_r(t1, t2, bs);
    const uint32_t w2 = __funnelshift_r(t2, t3, bs), w3 = __funnelshift_r(t3, t4, bs);
    lo = (uint64_t)compress_even(w0) | ((uint64_t)compress_even(w1) << 16) |
         ((uint64_t)compress_even(w2) << 32) | ((uint64_t)compress_even(w3) << 48);
    hi = (uint64_t)compress_even(w0 >> 1) | ((uint64_t)compress_even(w1 >> 1) << 16) |
         ((uint64_t)compress_even(w2 >> 1) << 32) | ((uint64_t)compress_even(w3 >> 1) << 48);
}

// S = A + Bv as one (64*W)-bit addition; the carry runs through the hardware
// carry flag inside a single asm block.
template <int W>
__device__ __forceinline__ void add_chain(uint64_t (&S)[W], const uint64_t (&A)[W], const uint64_t (&Bv)[W]);
template <>
__device__ __forceinline__ void add_chain<1>(uint64_t (&S)[1], const uint64_t (&A)[1], const uint64_t (&Bv)[1]) {
    S[0] = A[0] + Bv[0];
}

template <>
__device__ __forceinline__ void add_chain<2>(uint64_t (&S)[2], const uint64_t (&A)[2], const uint64_t (&Bv)[2]) {
    asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
        : "=l"(S[0]), "=l"(S[1])
        : "l"(A[0]), "l"(A[1]), "l"(Bv[0]), "l"(Bv[1]));
}

template <>
__device__ __forceinline__ void add_chain<3>(uint64_t (&S)[3], const uint64_t (&A)[3], const uint64_t (&Bv)[3]) {
    asm("add.cc.u64 %0, %3, %6;\n\taddc.cc.u64 %1, %4, %7;\n\taddc.u64 %2, %5, %8;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]));
}

template <>
__device__ __forceinline__ void add_chain<4>(uint64_t (&S)[4], const uint64_t (&A)[4], const uint64_t (&Bv)[4]) {
    asm("add.cc.u64 %0, %4, %8;\n\taddc.cc.u64 %1, %5, %9;\n\taddc.cc.u64 %2, %6, %10;\n\taddc.u64 %3, %7, %11;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]));
}

template <>
__device__ __forceinline__ void add_chain<5>(uint64_t (&S)[5], const uint64_t (&A)[5], const uint64_t (&Bv)[5]) {
    asm("add.cc.u64 %0, %5, %10;\n\taddc.cc.u64 %1, %6, %11;\n\taddc.cc.u64 %2, %7, %12;\n\taddc.cc.u64 %3, %8, %13;\n\taddc.u64 %4, %9, %14;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]));
}

template <>
__device__ __forceinline__ void add_chain<6>(uint64_t (&S)[6], const uint64_t (&A)[6], const uint64_t (&Bv)[6]) {
    asm("add.cc.u64 %0, %6, %12;\n\taddc.cc.u64 %1, %7, %13;\n\taddc.cc.u64 %2, %8, %14;\n\taddc.cc.u64 %3, %9, %15;\n\taddc.cc.u64 %4, %10, %16;\n\taddc.u64 %5, %11, %17;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]));
}

template <>
__device__ __forceinline__ void add_chain<7>(uint64_t (&S)[7], const uint64_t (&A)[7], const uint64_t (&Bv)[7]) {
    asm("add.cc.u64 %0, %7, %14;\n\taddc.cc.u64 %1, %8, %15;\n\taddc.cc.u64 %2, %9, %16;\n\taddc.cc.u64 %3, %10, %17;\n\taddc.cc.u64 %4, %11, %18;\n\taddc.cc.u64 %5, %12, %19;\n\taddc.u64 %6, %13, %20;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]));
}

template <>
__device__ __forceinline__ void add_chain<8>(uint64_t (&S)[8], const uint64_t (&A)[8], const uint64_t (&Bv)[8]) {
    asm("add.cc.u64 %0, %8, %16;\n\taddc.cc.u64 %1, %9, %17;\n\taddc.cc.u64 %2, %10, %18;\n\taddc.cc.u64 %3, %11, %19;\n\taddc.cc.u64 %4, %12, %20;\n\taddc.cc.u64 %5, %13, %21;\n\taddc.cc.u64 %6, %14, %22;\n\taddc.u64 %7, %15, %23;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6]), "=l"(S[7])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]), "l"(Bv[7]));
}

template <>
__device__ __forceinline__ void add_chain<9>(uint64_t (&S)[9], const uint64_t (&A)[9], const uint64_t (&Bv)[9]) {
    asm("add.cc.u64 %0, %9, %18;\n\taddc.cc.u64 %1, %10, %19;\n\taddc.cc.u64 %2, %11, %20;\n\taddc.cc.u64 %3, %12, %21;\n\taddc.cc.u64 %4, %13, %22;\n\taddc.cc.u64 %5, %14, %23;\n\taddc.cc.u64 %6, %15, %24;\n\taddc.cc.u64 %7, %16, %25;\n\taddc.u64 %8, %17, %26;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6]), "=l"(S[7]), "=l"(S[8])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]), "l"(Bv[7]), "l"(Bv[8]));
}

template <>
__device__ __forceinline__ void add_chain<10>(uint64_t (&S)[10], const uint64_t (&A)[10], const uint64_t (&Bv)[10]) {
    asm("add.cc.u64 %0, %10, %20;\n\taddc.cc.u64 %1, %11, %21;\n\taddc.cc.u64 %2, %12, %22;\n\taddc.cc.u64 %3, %13, %23;\n\taddc.cc.u64 %4, %14, %24;\n\taddc.cc.u64 %5, %15, %25;\n\taddc.cc.u64 %6, %16, %26;\n\taddc.cc.u64 %7, %17, %27;\n\taddc.cc.u64 %8, %18, %28;\n\taddc.u64 %9, %19, %29;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6]), "=l"(S[7]), "=l"(S[8]), "=l"(S[9])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(A[9]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]), "l"(Bv[7]), "l"(Bv[8]), "l"(Bv[9]));
}

template <>
__device__ __forceinline__ void add_chain<11>(uint64_t (&S)[11], const uint64_t (&A)[11], const uint64_t (&Bv)[11]) {
    asm("add.cc.u64 %0, %11, %22;\n\taddc.cc.u64 %1, %12, %23;\n\taddc.cc.u64 %2, %13, %24;\n\taddc.cc.u64 %3, %14, %25;\n\taddc.cc.u64 %4, %15, %26;\n\taddc.cc.u64 %5, %16, %27;\n\taddc.cc.u64 %6, %17, %28;\n\taddc.cc.u64 %7, %18, %29;\n\taddc.cc.u64 %8, %19, %30;\n\taddc.cc.u64 %9, %20, %31;\n\taddc.u64 %10, %21, %32;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6]), "=l"(S[7]), "=l"(S[8]), "=l"(S[9]), "=l"(S[10])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(A[9]), "l"(A[10]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]), "l"(Bv[7]), "l"(Bv[8]), "l"(Bv[9]), "l"(Bv[10]));
}

template <>
__device__ __forceinline__ void add_chain<12>(uint64_t (&S)[12], const uint64_t (&A)[12], const uint64_t (&Bv)[12]) {
    asm("add.cc.u64 %0, %12, %24;\n\taddc.cc.u64 %1, %13, %25;\n\taddc.cc.u64 %2, %14, %26;\n\taddc.cc.u64 %3, %15, %27;\n\taddc.cc.u64 %4, %16, %28;\n\taddc.cc.u64 %5, %17, %29;\n\taddc.cc.u64 %6, %18, %30;\n\taddc.cc.u64 %7, %19, %31;\n\taddc.cc.u64 %8, %20, %32;\n\taddc.cc.u64 %9, %21, %33;\n\taddc.cc.u64 %10, %22, %34;\n\taddc.u64 %11, %23, %35;"
        : "=l"(S[0]), "=l"(S[1]), "=l"(S[2]), "=l"(S[3]), "=l"(S[4]), "=l"(S[5]), "=l"(S[6]), "=l"(S[7]), "=l"(S[8]), "=l"(S[9]), "=l"(S[10]), "=l"(S[11])
        : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(A[9]), "l"(A[10]), "l"(A[11]), "l"(Bv[0]), "l"(Bv[1]), "l"(Bv[2]), "l"(Bv[3]), "l"(Bv[4]), "l"(Bv[5]), "l"(Bv[6]), "l"(Bv[7]), "l"(Bv[8]), "l"(Bv[9]), "l"(Bv[10]), "l"(Bv[11]));
}

// |{(a, b): 0 <= a < lx, 0 <= b < ly, |a - b| <= K}|, Ukkonen's band size.
__device__ __forceinline__ unsigned long long band_cells(int64_t lx, int64_t ly, int64_t K) {
    if (lx <= 0 || ly <= 0) return 0ull;
    const int64_t amax = min(lx - 1, ly - 1 + K);   // rows whose band range is non-empty
    if (amax < 0) return 0ull;
    const int64_t t = min(amax + 1, max((int64_t)0, ly - K));  // rows whose range ends at a+K
    const int64_t s1 = t * (t - 1) / 2 + t * (K + 1) + (amax + 1 - t) * ly;
    const int64_t u = max((int64_t)0, amax - K);
    return (unsigned long long)(s1 - u * (u + 1) / 2);
}

// reversed reader: symbols idx, idx-1, ..., 0 of a packed string
template <int B>
struct SymReaderRev {
    const uint4 *base;
    int64_t ch;   // index of the chunk that `nxt` holds (the one before cur)
    uint4 cur, nxt;
    int left;
    __device__ __forceinline__ void init(const uint4 *b, int64_t len) {
        constexpr int S = 128 / B;
        base = b;
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        if (len <= 0) {
            cur = nxt = zero;
            left = S;
            ch = -1;
            return;
        }
        const int64_t last = len - 1;
        const int64_t c = last / S;
        const int s = (int)(last - c * S);  // position of the last symbol in its chunk
        cur = b[c];
        // shift left so that symbol s occupies the top B bits
        const uint32_t sh = (uint32_t)((S - 1 - s) * B);  // 0 .. 128-B
        uint32_t w0 = cur.x, w1 = cur.y, w2 = cur.z, w3 = cur.w;
        if (sh & 64u) { w3 = w1; w2 = w0; w1 = 0u; w0 = 0u; }
        if (sh & 32u) { w3 = w2; w2 = w1; w1 = w0; w0 = 0u; }
        const uint32_t bs = sh & 31u;
        cur.w = __funnelshift_l(w2, w3, bs);
        cur.z = __funnelshift_l(w1, w2, bs);
        cur.y = __funnelshift_l(w0, w1, bs);
        cur.x = w0 << bs;
        left = s + 1;
        ch = c - 1;
        nxt = (ch >= 0) ? b[ch] : zero;
    }
    __device__ __forceinline__ uint32_t code() const { return cur.w >> (32 - B); }
    __device__ __forceinline__ void advance() {
        cur.w = __funnelshift_l(cur.z, cur.w, B);
        cur.z = __funnelshift_l(cur.y, cur.z, B);
        cur.y = __funnelshift_l(cur.x, cur.y, B);
        cur.x <<= B;
        if (--left == 0) {
            cur = nxt;
            ch--;
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            nxt = (ch >= 0) ? base[ch] : zero;
            left = 128 / B;
        }
    }
};

// Peq word k (rows 64k+1 .. 64k+64) of x, or of reversed x when `rev`, for every
// symbol c < alpha, into ring slot `slot` (stride T_ between slots).
template <int B, int R>
__device__ __forceinline__ void bd_build(uint64_t *ring, int T_, int slot, const uint4 *__restrict__ xc,
                                         int64_t m, int64_t k, bool rev, uint32_t alpha) {
    // forward symbols covered: [k0, k0+64) (reversed: x[m-64-64k .. m-1-64k])
    const int64_t k0 = rev ? (m - 64 - 64 * k) : 64 * k;
    const int64_t t_lo = k0 < 0 ? -k0 : 0;
    const int64_t t_hi = m - k0;
    uint64_t valid_m = 0ull;
    if (t_hi > t_lo && t_lo < 64) {
        const uint64_t upto = t_hi >= 64 ? ~0ull : ((1ull << t_hi) - 1ull);
        valid_m = upto & ~((1ull << t_lo) - 1ull);
    }
    const int64_t xch = chunks_for(m, B);
    if (B == 2) {
        uint64_t lo = 0, hi = 0;
        if (valid_m) sym64_planes(xc, xch, k0, lo, hi);
        if (rev) {
            lo = __brevll(lo);
            hi = __brevll(hi);
            valid_m = __brevll(valid_m);
        }
        for (uint32_t c = 0; c < alpha; c++)
            ring[(size_t)(c * R + slot) * T_] = ((c & 1u) ? lo : ~lo) & ((c & 2u) ? hi : ~hi) & valid_m;
    } else {
        for (uint32_t c = 0; c < alpha; c++) ring[(size_t)(c * R + slot) * T_] = 0ull;
        if (valid_m) {
            // each 16-symbol chunk is read once; every symbol sets its bit with a
            // shared-memory OR that returns nothing, so consecutive symbols (which
            // may hit the same word) do not wait on one another
            const int64_t ks = k0 + t_lo, ke = k0 + (t_hi < 64 ? t_hi : 64);
            for (int64_t ch = ks >> 4; ch <= ((ke - 1) >> 4); ch++) {
                const uint4 v = xc[ch];
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int64_t kk = ch * 16 + q;
                    const uint32_t w = q < 4 ? v.x : q < 8 ? v.y : q < 12 ? v.z : v.w;
                    const uint32_t c = (w >> ((q & 3) * 8)) & 0xFFu;
                    if (kk >= ks && kk < ke && c < alpha) {
                        const uint32_t bit = rev ? (uint32_t)(63 - (kk - k0)) : (uint32_t)(kk - k0);
                        atomicOr(reinterpret_cast<unsigned long long *>(ring + (size_t)(c * R + slot) * T_),
                                 1ull << bit);
                    }
                }
            }
        }
    }
}

}  // namespace ej
