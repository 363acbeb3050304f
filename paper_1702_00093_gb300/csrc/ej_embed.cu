// Validation, random-bit tables, CGK embedding (Algorithm 1) and bit-sampling
// signatures (Theorem 1 with AND amplification, Section 3.2).
#include <utility>

#include "ej_internal.cuh"

namespace ej {

// ---------------------------------------------------------------------------
// Validation: offsets, lengths, symbols
// ---------------------------------------------------------------------------

// total_cap bounds offsets[n]: beyond it every length is reported as 0 (and
// DERR_OFFSETS set), so that buffers sized for total_cap bytes are never overrun.
__global__ void validate_offsets_kernel(const int64_t *__restrict__ offsets, int64_t n, int64_t total_cap,
                                        int32_t *__restrict__ lens, uint32_t *__restrict__ err,
                                        unsigned long long *__restrict__ max_len) {
    unsigned long long local_max = 0;
    uint32_t local_err = 0;
    const bool over = offsets[n] > total_cap;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = offsets[i], b = offsets[i + 1];
        int64_t len = b - a;
        if (over || (i == 0 && a != 0) || a < 0 || b > total_cap || len < 0 || len >= (1ll << 31)) {
            local_err |= DERR_OFFSETS;
            len = 0;
        }
        lens[i] = (int32_t)len;
        local_max = len > (int64_t)local_max ? (unsigned long long)len : local_max;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(FULL, local_max, o);
        local_max = v > local_max ? v : local_max;
        local_err |= __shfl_xor_sync(FULL, local_err, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (local_max) atomicMax(max_len, local_max);
        if (local_err) atomicOr(err, local_err);
    }
}

cudaError_t launch_validate(const uint8_t *bytes, const int64_t *offsets, int64_t n, int64_t total_cap,
                            const uint8_t *code_map, int32_t *lens, uint32_t *err,
                            unsigned long long *max_len, cudaStream_t s) {
    if (n > 0) {
        int grid = (int)((n + 255) / 256);
        if (grid > 4096) grid = 4096;
        validate_offsets_kernel<<<grid, 256, 0, s>>>(offsets, n, total_cap, lens, err, max_len);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pack: bytes -> dense B-bit codes, one 16-byte-aligned run of chunks per string
// ---------------------------------------------------------------------------

__global__ void chunk_counts_kernel(const int32_t *__restrict__ lens, int64_t n, int B,
                                    uint32_t *__restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        counts[i] = (i < n) ? (uint32_t)chunks_for(lens[i], B) : 0u;
}

cudaError_t launch_chunk_counts(const int32_t *lens, int64_t n, int B, uint32_t *counts, cudaStream_t s) {
    int64_t g = (n + 1 + 255) / 256;
    chunk_counts_kernel<<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, s>>>(lens, n, B, counts);
    note_launches(1);
    return cudaGetLastError();
}

// Spreads the 32 bits of v to the even bit positions of a 64-bit word.
__device__ __forceinline__ uint64_t spread_even(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// One warp per string. Each load instruction reads 32 consecutive bytes (lane
// t reads symbol 32g+t). For 2-bit codes two ballots give the low and high bit
// planes of the 32 symbols, which interleave into one 64-bit word; lane u keeps
// the word of group g = gbase+u and the warp stores 32 words (256 bytes) at
// once. 8-bit codes are stored byte for byte. Symbols past the end of a
// string are written as 0 up to its chunk boundary.
// One warp per string. With 2-bit codes a lane turns 16 consecutive bytes into
// one 32-bit half of an output word (symbol s of the word at bits 2s, 2s+1); with
// 8-bit codes 4 bytes into one 32-bit word. The bytes are read as aligned 32-bit
// words (five cover any 16-byte window, two any 4-byte one) where those words lie
// inside the byte array [bytes, bytes + total), else one by one; positions past
// the string's end give code 0.
__device__ __forceinline__ uint32_t pack_code(const uint8_t *s_map, uint32_t byte, bool &bad) {
    const uint32_t c = s_map[byte];
    if (c == 255u) {
        bad = true;
        return 0u;
    }
    return c;
}

__global__ void pack_kernel(const uint8_t *__restrict__ bytes, const int64_t *__restrict__ offsets,
                            const int32_t *__restrict__ lens, int64_t n, int64_t total,
                            const uint8_t *__restrict__ code_map, int B, const uint64_t *__restrict__ pofs,
                            uint4 *__restrict__ packed, uint32_t *__restrict__ err) {
    __shared__ uint8_t s_map[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) s_map[t] = code_map[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uintptr_t base = (uintptr_t)bytes;
    const uintptr_t wlo = (base + 3) & ~(uintptr_t)3;            // whole words inside the array
    const uintptr_t whi = (base + (uintptr_t)total) & ~(uintptr_t)3;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t len = lens[i];
        const uint8_t *x = bytes + offsets[i];
        uint32_t *dst = reinterpret_cast<uint32_t *>(packed + pofs[i]);
        const int64_t nout = 4 * chunks_for(len, B);    // 32-bit output words
        const int per = B == 2 ? 16 : 4;                // bytes per output word
#pragma unroll 2
        for (int64_t h = lane; h < nout; h += 32) {
            const int64_t k0 = (int64_t)per * h;
            const int cnt = len - k0 >= per ? per : (len > k0 ? (int)(len - k0) : 0);
            uint32_t out = 0;
            if (cnt > 0) {
                const uintptr_t pa = (uintptr_t)(x + k0);
                const uintptr_t w0 = pa & ~(uintptr_t)3;
                const uint32_t sh = (uint32_t)(pa & 3u) * 8u;
                if (w0 >= wlo && w0 + (uintptr_t)(per + 4) <= whi) {
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(w0);
                    if (B == 2) {
                        uint32_t W[5];
#pragma unroll
                        for (int q = 0; q < 5; q++) W[q] = __ldg(wp + q);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const uint32_t v = __funnelshift_r(W[q], W[q + 1], sh);
#pragma unroll
                            for (int j = 0; j < 4; j++)
                                if (4 * q + j < cnt) out |= pack_code(s_map, (v >> (8 * j)) & 255u, bad) << (2 * (4 * q + j));
                        }
                    } else {
                        const uint32_t v = __funnelshift_r(__ldg(wp), __ldg(wp + 1), sh);
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (j < cnt) out |= pack_code(s_map, (v >> (8 * j)) & 255u, bad) << (8 * j);
                    }
                } else {
                    for (int j = 0; j < cnt; j++)
                        out |= pack_code(s_map, x[k0 + j], bad) << ((B == 2 ? 2 : 8) * j);
                }
            }
            dst[h] = out;
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, (uint32_t)DERR_SYMBOL);
}

cudaError_t launch_pack(const uint8_t *bytes, const int64_t *offsets, const int32_t *lens, int64_t n, int64_t total,
                        const uint8_t *code_map, int B, const uint64_t *pofs, uint4 *packed,
                        uint32_t *err, cudaStream_t s) {
    if (n > 0) {
        int64_t blocks = (n + 7) / 8;   // 8 warps per block
        pack_kernel<<<(unsigned)(blocks > 8192 ? 8192 : blocks), 256, 0, s>>>(bytes, offsets, lens, n, total, code_map,
                                                                                B, pofs, packed, err);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Random-bit table of Alg. 1 and sampled positions of Thm. 1
// ---------------------------------------------------------------------------

// table[(l * out_len + j) * words + w], bit (c - 32w) = pi_j^l(alphabet[c]).
__global__ void bit_table_kernel(uint64_t base, uint32_t r, uint32_t out_len,
                                 const uint8_t *__restrict__ alphabet, uint32_t alpha, uint32_t words,
                                 const uint8_t *__restrict__ pi, uint32_t inject_steps,
                                 uint32_t *__restrict__ table) {
    const uint64_t total = (uint64_t)r * out_len * words;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(idx % words);
        const uint64_t lj = idx / words;
        const uint32_t j = (uint32_t)(lj % out_len);
        const uint32_t l = (uint32_t)(lj / out_len);
        uint32_t word = 0;
        const uint32_t c_end = min(alpha, 32 * w + 32);
        for (uint32_t c = 32 * w; c < c_end; c++) {
            uint32_t bit;
            if (pi) {
                bit = (j < inject_steps) ? (pi[((uint64_t)l * inject_steps + j) * alpha + c] & 1u) : 0u;
            } else {
                bit = (uint32_t)(mix64(base ^ walk_counter(l, j, alphabet[c])) >> 63);
            }
            word |= bit << (c - 32 * w);
        }
        table[idx] = word;
    }
}

cudaError_t launch_bit_table(uint64_t seed, uint32_t r, uint32_t out_len, const uint8_t *alphabet_dev,
                             uint32_t alpha, uint32_t words, const uint8_t *pi_inject,
                             uint32_t inject_steps, uint32_t *table, cudaStream_t s) {
    const uint64_t total = (uint64_t)r * out_len * words;
    if (total) {
        uint64_t g = (total + 255) / 256;
        int grid = (int)(g > 4096 ? 4096 : g);
        bit_table_kernel<<<grid, 256, 0, s>>>(mix64(seed), r, out_len, alphabet_dev, alpha, words,
                                              pi_inject, inject_steps, table);
        note_launches(1);
    }
    return cudaGetLastError();
}

__global__ void positions_kernel(uint64_t base, uint32_t r, uint32_t m, uint32_t z, uint32_t L,
                                 const uint32_t *__restrict__ inject, uint32_t *__restrict__ pos) {
    const uint64_t total = (uint64_t)r * m * z;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        if (inject) {
            pos[idx] = inject[idx];
        } else {
            const uint32_t q = (uint32_t)(idx % z);
            const uint32_t f = (uint32_t)((idx / z) % m);
            const uint32_t l = (uint32_t)(idx / ((uint64_t)z * m));
            pos[idx] = (uint32_t)__umul64hi(mix64(base ^ position_counter(l, f, q)), (uint64_t)L);
        }
    }
}

cudaError_t launch_positions(uint64_t seed, uint32_t r, uint32_t m, uint32_t z, uint32_t L,
                             const uint32_t *pos_inject, uint32_t *pos, cudaStream_t s) {
    const uint64_t total = (uint64_t)r * m * z;
    if (total) {
        int grid = (int)((total + 255) / 256 > 1024 ? 1024 : (total + 255) / 256);
        positions_kernel<<<grid, 256, 0, s>>>(mix64(seed), r, m, z, L, pos_inject, pos);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CGK embedding (Algorithm 1)
// ---------------------------------------------------------------------------
//
// One lane per (string, embedding) walk; a warp walks 32 consecutive strings
// under the same embedding l in lockstep over the steps j, so the random-bit
// row of step j (staged in shared memory) is read by all lanes at once and
// the emitted symbols of the 32 walks are packed by warp ballots into
// bit-planes: one uint32 per (step, plane) with bit t for lane t. Every 32
// steps the warp stores 32 x PLANES words, contiguous in memory.
// Each lane reads its string's packed codes through a two-chunk prefetch
// (SymReader), so the walk never waits on a load it has just issued.

constexpr int EMBED_WARPS = 4;
constexpr int EMBED_TILE = 2048;  // steps of the random-bit table staged at a time

template <int PLANES, int B>
__global__ void __launch_bounds__(EMBED_WARPS * 32)
embed_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
             const int32_t *__restrict__ lens, int64_t n, const uint32_t *__restrict__ table,
             uint32_t out_len, uint32_t *__restrict__ emb, int32_t *__restrict__ walk_end,
             int64_t nblocks32) {
    constexpr int WS = PLANES <= 5 ? 1 : (1 << (PLANES - 5));
    __shared__ uint32_t s_table[EMBED_TILE * WS];

    const uint32_t l = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t B32 = (int64_t)blockIdx.x * EMBED_WARPS + warp;
    const int64_t s = B32 * 32 + lane;
    const bool valid = (B32 < nblocks32) && (s < n);
    const int32_t len = valid ? lens[s] : 0;
    SymReader<B> rd;
    rd.init(packed + (valid ? pofs[s] : 0), valid ? chunks_for(len, B) : 0);

    int32_t pos = 0;
    int32_t wend = (len == 0) ? 0 : (int32_t)out_len;
    uint32_t acc[PLANES];
#pragma unroll
    for (int k = 0; k < PLANES; k++) acc[k] = 0;

    const uint32_t *tab_l = table + (size_t)l * out_len * WS;
    uint32_t *out_base = emb + ((size_t)l * nblocks32 + (size_t)(B32 < nblocks32 ? B32 : 0)) * out_len * PLANES;

    for (uint32_t j0 = 0; j0 < out_len; j0 += EMBED_TILE) {
        const uint32_t tile = min((uint32_t)EMBED_TILE, out_len - j0);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < tile * WS; t += blockDim.x)
            s_table[t] = tab_l[(size_t)j0 * WS + t];
        __syncthreads();
        if (B32 >= nblocks32) continue;  // warp-uniform
        for (uint32_t jj = 0; jj < tile; jj++) {
            const uint32_t j = j0 + jj;
            const bool active = pos < len;
            const uint32_t code = active ? rd.code() : 0u;
#pragma unroll
            for (int k = 0; k < PLANES; k++) {
                const uint32_t bal = __ballot_sync(FULL, (code >> k) & 1u);
                acc[k] = (lane == (int)(j & 31)) ? bal : acc[k];
            }
            if ((j & 31) == 31 || j == out_len - 1) {  // warp-uniform
                const uint32_t jb = j & ~31u;
                if (jb + lane <= j) {
                    uint32_t *o = out_base + (size_t)(jb + lane) * PLANES;
#pragma unroll
                    for (int k = 0; k < PLANES; k++) o[k] = acc[k];
                }
            }
            const uint32_t w = (WS == 1) ? s_table[jj] : s_table[jj * WS + (code >> 5)];
            const bool bit = active && ((w >> (code & 31)) & 1u);
            if (bit) {
                pos++;
                if (pos == len) wend = (int32_t)(j + 1);
                rd.advance();
            }
        }
    }
    if (valid) walk_end[(size_t)l * n + s] = wend;
}

template <int PLANES, int B>
static void embed_launch(dim3 grid, dim3 block, cudaStream_t s, const uint4 *packed, const uint64_t *pofs,
                         const int32_t *lens, int64_t n, const uint32_t *table, uint32_t out_len,
                         uint32_t *emb, int32_t *walk_end, int64_t nb32) {
    embed_kernel<PLANES, B><<<grid, block, 0, s>>>(packed, pofs, lens, n, table, out_len, emb, walk_end, nb32);
}

cudaError_t launch_embed(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                         uint32_t r, const uint32_t *table, int B, uint32_t out_len, uint32_t planes,
                         uint32_t *emb, int32_t *walk_end, cudaStream_t s) {
    if (n == 0 || out_len == 0) return cudaGetLastError();
    const int64_t nb32 = (n + 31) / 32;
    dim3 grid((unsigned)((nb32 + EMBED_WARPS - 1) / EMBED_WARPS), r);
    dim3 block(EMBED_WARPS * 32);
#define EJ_EMB(P, BB) embed_launch<P, BB>(grid, block, s, packed, pofs, lens, n, table, out_len, emb, walk_end, nb32)
    switch (planes) {
        case 1: EJ_EMB(1, 2); break;
        case 2: EJ_EMB(2, 2); break;
        case 3: EJ_EMB(3, 8); break;
        case 4: EJ_EMB(4, 8); break;
        case 5: EJ_EMB(5, 8); break;
        case 6: EJ_EMB(6, 8); break;
        case 7: EJ_EMB(7, 8); break;
        default: EJ_EMB(8, 8); break;
    }
    note_launches(1);
#undef EJ_EMB
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bit-sampling signatures: key = sum_q c_q (alpha+1)^q
// ---------------------------------------------------------------------------
//
// A warp handles the 32 strings of one embedding block for one table
// t = l*m + f. The sampled step p is the same for all lanes, so each plane word
// is one broadcast load and lane t extracts its own bit.

constexpr int SIGN_WARPS = 4;

template <int PLANES>
__global__ void __launch_bounds__(SIGN_WARPS * 32)
sign_kernel(const uint32_t *__restrict__ emb, const int32_t *__restrict__ walk_end, int64_t n,
            uint32_t m, uint32_t z, uint32_t out_len, uint32_t alpha, const uint32_t *__restrict__ pos,
            uint64_t *__restrict__ keys, int64_t nblocks32) {
    const uint32_t t = blockIdx.y;
    const uint32_t l = t / m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t B = (int64_t)blockIdx.x * SIGN_WARPS + warp;
    if (B >= nblocks32) return;
    const int64_t s = B * 32 + lane;
    const bool valid = s < n;
    const int32_t we = valid ? walk_end[(size_t)l * n + s] : 0;
    const uint32_t *eb = emb + ((size_t)l * nblocks32 + B) * out_len * PLANES;
    const uint32_t *P = pos + (size_t)t * z;
    const uint64_t R = (uint64_t)alpha + 1;
    uint64_t key = 0;
    for (int q = (int)z - 1; q >= 0; q--) {
        const uint32_t p = P[q];
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < PLANES; k++) c |= ((eb[(size_t)p * PLANES + k] >> lane) & 1u) << k;
        if ((int32_t)p >= we) c = alpha;  // bottom
        key = key * R + c;
    }
    if (valid) keys[(size_t)t * n + s] = key;
}

cudaError_t launch_sign(const uint32_t *emb, const int32_t *walk_end, int64_t n, uint32_t r,
                        uint32_t m, uint32_t z, uint32_t out_len, uint32_t planes, uint32_t alpha,
                        const uint32_t *pos, uint64_t *keys, cudaStream_t s) {
    if (n == 0) return cudaGetLastError();
    const int64_t nb32 = (n + 31) / 32;
    dim3 grid((unsigned)((nb32 + SIGN_WARPS - 1) / SIGN_WARPS), r * m);
    dim3 block(SIGN_WARPS * 32);
#define EJ_SIGN(P) sign_kernel<P><<<grid, block, 0, s>>>(emb, walk_end, n, m, z, out_len, alpha, pos, keys, nb32)
    switch (planes) {
        case 1: EJ_SIGN(1); break;
        case 2: EJ_SIGN(2); break;
        case 3: EJ_SIGN(3); break;
        case 4: EJ_SIGN(4); break;
        case 5: EJ_SIGN(5); break;
        case 6: EJ_SIGN(6); break;
        case 7: EJ_SIGN(7); break;
        default: EJ_SIGN(8); break;
    }
    note_launches(1);
#undef EJ_SIGN
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused embed + sign: only the sampled steps of each walk are produced
// ---------------------------------------------------------------------------
//
// Algorithm 1 emits x[i] from the step a_i at which the walk arrives at i up to
// and including the first step j >= a_i with pi_j(x[i]) = 1; so
// a_{i+1} = next1_{x[i]}(a_i) + 1. With one step bitmap per symbol, next1 is a
// find-first-set, one per input character instead of work per step. The m*z
// sampled steps of embedding l (Thm. 1 with AND amplification) are visited in
// step order; a sample at step p < a_{i+1} reads x[i], a sample at or after the
// end of the walk reads bottom. Each sample adds c * (alpha+1)^q to the key of
// its function f, kept in shared memory per thread, so the embedded string is
// never written.

__host__ __device__ __forceinline__ uint32_t sym_words(uint32_t L) { return L / 32 + 2; }

__global__ void symbol_table_kernel(uint64_t base, uint32_t r, uint32_t L, const uint8_t *__restrict__ alphabet,
                                    uint32_t alpha, const uint8_t *__restrict__ pi, uint32_t inject_steps,
                                    uint32_t *__restrict__ tsym) {
    const uint32_t LW = sym_words(L);
    const uint64_t total = (uint64_t)r * alpha * LW;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(idx % LW);
        const uint32_t c = (uint32_t)((idx / LW) % alpha);
        const uint32_t l = (uint32_t)(idx / ((uint64_t)LW * alpha));
        uint32_t word = 0;
        for (uint32_t b = 0; b < 32; b++) {
            const uint32_t j = 32 * w + b;
            uint32_t bit;
            if (j >= L) bit = 1u;  // sentinel: the search never runs past the table
            else if (pi) bit = (j < inject_steps) ? (pi[((uint64_t)l * inject_steps + j) * alpha + c] & 1u) : 0u;
            else bit = (uint32_t)(mix64(base ^ walk_counter(l, j, alphabet[c])) >> 63);
            word |= bit << b;
        }
        tsym[idx] = word;
    }
}

cudaError_t launch_symbol_table(uint64_t seed, uint32_t r, uint32_t L, const uint8_t *alphabet_dev,
                                uint32_t alpha, const uint8_t *pi_inject, uint32_t inject_steps,
                                uint32_t *tsym, cudaStream_t s) {
    const uint64_t total = (uint64_t)r * alpha * sym_words(L);
    uint64_t g = (total + 255) / 256;
    symbol_table_kernel<<<(unsigned)(g > 4096 ? 4096 : (g ? g : 1)), 256, 0, s>>>(
        mix64(seed), r, L, alphabet_dev, alpha, pi_inject, inject_steps, tsym);
    note_launches(1);
    return cudaGetLastError();
}

size_t symbol_table_words(uint32_t r, uint32_t alpha, uint32_t L) { return (size_t)r * alpha * sym_words(L); }

// One block per embedding: rank every sample by (step, index).
__global__ void sort_samples_kernel(const uint32_t *__restrict__ pos, uint32_t m, uint32_t z,
                                    uint32_t *__restrict__ spos, uint32_t *__restrict__ stag) {
    const uint32_t l = blockIdx.x, M = m * z;
    const uint32_t *P = pos + (size_t)l * M;
    for (uint32_t i = threadIdx.x; i < M; i += blockDim.x) {
        const uint32_t pi_ = P[i];
        uint32_t rank = 0;
        for (uint32_t k = 0; k < M; k++) {
            const uint32_t pk = P[k];
            rank += (pk < pi_) || (pk == pi_ && k < i);
        }
        spos[(size_t)l * M + rank] = pi_;
        stag[(size_t)l * M + rank] = ((i / z) << 16) | (i % z);
    }
}

cudaError_t launch_sort_samples(const uint32_t *pos, uint32_t r, uint32_t m, uint32_t z, uint32_t *spos,
                                uint32_t *stag, cudaStream_t s) {
    sort_samples_kernel<<<r, 256, 0, s>>>(pos, m, z, spos, stag);
    note_launches(1);
    return cudaGetLastError();
}

constexpr int ES_THREADS = 512;   // default walks (strings) per block
constexpr size_t ES_TABLE_MAX = 48 * 1024;   // next-step table kept in shared memory up to this size

// Per-embedding stride of the next-step table, even so that every table starts
// on a 4-byte boundary.
// Rows of L + 2 entries: arrival steps a = L and L + 1 (the walk has passed the
// sampling range) map to L + 1, so the walk needs no range check.
__host__ __device__ __forceinline__ uint32_t next_row(uint32_t L) { return L + 2; }

__host__ __device__ __forceinline__ uint64_t next_stride(uint32_t alpha, uint32_t L) {
    return ((uint64_t)alpha * next_row(L) + 1) & ~1ull;
}

// next[l][c][a] = next1_c(a) + 1 for a < L, L + 1 for a in {L, L+1} (16-bit),
// from the step bitmaps.
__global__ void next_table_kernel(const uint32_t *__restrict__ tsym, uint32_t r, uint32_t alpha, uint32_t L,
                                  uint16_t *__restrict__ next) {
    const uint32_t LW = sym_words(L), NR = next_row(L);
    const uint64_t total = (uint64_t)r * alpha * NR;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)(idx % NR);
        const uint64_t lc = idx / NR;   // l * alpha + c
        const uint64_t l = lc / alpha, c = lc % alpha;
        if (a >= L) {
            next[l * next_stride(alpha, L) + c * NR + a] = (uint16_t)(L + 1);
            continue;
        }
        const uint32_t *row = tsym + lc * LW;
        uint32_t wi = a >> 5;
        uint32_t w = row[wi] >> (a & 31u);
        uint32_t base = a;
        while (w == 0u) {               // ends at the sentinel bits (steps >= L)
            wi++;
            w = row[wi];
            base = wi << 5;
        }
        next[l * next_stride(alpha, L) + c * NR + a] = (uint16_t)(base + (uint32_t)__ffs((int)w));
    }
}

cudaError_t launch_next_table(const uint32_t *tsym, uint32_t r, uint32_t alpha, uint32_t L, uint16_t *next,
                              cudaStream_t s) {
    const uint64_t total = (uint64_t)r * alpha * next_row(L);
    uint64_t g = (total + 255) / 256;
    next_table_kernel<<<(unsigned)(g > 4096 ? 4096 : (g ? g : 1)), 256, 0, s>>>(tsym, r, alpha, L, next);
    note_launches(1);
    return cudaGetLastError();
}

size_t next_table_elems(uint32_t r, uint32_t alpha, uint32_t L) { return (size_t)r * next_stride(alpha, L); }

bool embed_sign_uses_table(uint32_t alpha, uint32_t L) {
    return (size_t)alpha * next_row(L) * 2 <= ES_TABLE_MAX && L < 65534u;
}

static size_t es_code_words(uint32_t alpha, uint32_t M) {
    const uint32_t per = alpha <= 4 ? 16u : 4u;   // codes per 32-bit word (2 or 8 bits each)
    return (M + per - 1) / per;
}

size_t embed_sign_smem(uint32_t alpha, uint32_t L, uint32_t m, uint32_t z, int tpb) {
    if (tpb <= 0) tpb = ES_THREADS;
    const size_t M = (size_t)m * z;
    if (M > 16384 || z > 65535 || m > 65535) return 0;
    const size_t table = embed_sign_uses_table(alpha, L) ? (size_t)alpha * next_row(L) * 2 : (size_t)alpha * sym_words(L) * 4;
    const size_t bytes = (size_t)z * 8 + (M + 1) * 4 + M * 4 + ((table + 7) & ~(size_t)7) +
                         es_code_words(alpha, (uint32_t)M) * 4 * (size_t)tpb;
    return bytes <= 200 * 1024 ? bytes : 0;
}

// Codes of one string, 64 bits at a time. Every string starts on a chunk
// boundary and the walk consumes exactly one symbol per loop iteration, so all
// lanes of a warp refill at the same iteration.
template <int B>
struct WordReader {
    const uint4 *p;
    const uint4 *end;
    uint64_t w;          // current symbol in the low B bits
    uint4 cur, nxt;
    int left;
    bool hi_next;        // the upper half of cur is still to be consumed
    __device__ __forceinline__ uint4 fetch() {
        const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
        const uint4 v = (p < end) ? *p : zero;
        p += (p < end);
        return v;
    }
    __device__ __forceinline__ void init(const uint4 *base, int64_t nchunks) {
        p = base;
        end = base + nchunks;
        cur = fetch();
        nxt = fetch();
        w = ((uint64_t)cur.y << 32) | cur.x;
        hi_next = true;
        left = 64 / B;
    }
    __device__ __forceinline__ uint32_t code() const { return (uint32_t)w & ((1u << B) - 1u); }
    __device__ __forceinline__ void advance() {
        w >>= B;
        if (--left == 0) {
            left = 64 / B;
            if (hi_next) {
                w = ((uint64_t)cur.w << 32) | cur.z;
                hi_next = false;
            } else {
                cur = nxt;
                nxt = fetch();
                w = ((uint64_t)cur.y << 32) | cur.x;
                hi_next = true;
            }
        }
    }
};

// TABLE: next steps from the 16-bit table (one shared load per character);
// otherwise a find-first-set over the step bitmaps. CB: bits per stored code.
template <int B, bool TABLE, int CB, int TPB>
__global__ void __launch_bounds__(TPB)
embed_sign_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                  const int32_t *__restrict__ lens, int64_t n, uint32_t m, uint32_t z, uint32_t L,
                  uint32_t alpha, const uint32_t *__restrict__ tsym, const uint16_t *__restrict__ next,
                  const uint32_t *__restrict__ spos, const uint32_t *__restrict__ stag,
                  uint64_t *__restrict__ keys, PrefixKeys pk) {
    constexpr uint32_t PER = 32 / CB;   // codes per word
    extern __shared__ uint64_t es_smem[];
    const uint32_t l = blockIdx.y, M = m * z, LW = sym_words(L);
    uint64_t *s_pow = es_smem;                                 // [z]
    uint32_t *s_pos = (uint32_t *)(s_pow + z);                 // [M+1], sentinel at M
    uint32_t *s_rank = s_pos + M + 1;                          // [M]: step-order index of sample f*z+q
    uint32_t *s_tab = s_rank + M;                              // bitmaps [alpha][LW] or next table
    const uint32_t NR = next_row(L);
    const size_t tab_bytes = TABLE ? (size_t)alpha * NR * 2 : (size_t)alpha * LW * 4;
    uint16_t *s_next = (uint16_t *)s_tab;
    uint32_t *s_code = (uint32_t *)((char *)s_tab + ((tab_bytes + 7) & ~(size_t)7));  // [words][TPB]
    for (uint32_t i = threadIdx.x; i <= M; i += blockDim.x) {
        s_pos[i] = i < M ? spos[(size_t)l * M + i] : 0xFFFFFFFFu;
        if (i < M) {
            const uint32_t tag = stag[(size_t)l * M + i];
            s_rank[(tag >> 16) * z + (tag & 0xFFFFu)] = i;
        }
    }
    if (TABLE) {
        const uint32_t *src = (const uint32_t *)(next + (size_t)l * next_stride(alpha, L));
        uint32_t *dst = (uint32_t *)s_next;
        const uint32_t nw = (alpha * NR + 1) / 2;
        for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    } else {
        for (uint32_t i = threadIdx.x; i < alpha * LW; i += blockDim.x) s_tab[i] = tsym[(size_t)l * alpha * LW + i];
    }
    if (threadIdx.x == 0) {
        uint64_t pw = 1;
        for (uint32_t q = 0; q < z; q++) {
            s_pow[q] = pw;
            pw *= (uint64_t)alpha + 1;
        }
    }
    __syncthreads();

    const int64_t s = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const int32_t len = s < n ? lens[s] : 0;
    uint32_t *my = s_code + threadIdx.x;
    if (TABLE) {
        // 16 characters per block: their codes come from one 32-bit word (B = 2)
        // or one 16-byte chunk (B = 8) read a block ahead; the loop conditions
        // are tested once per block and characters past the end record nothing.
        // Recorded codes enter a shift register from the top (sample j of a word
        // ends at bits CB*j once the word is full).
        constexpr int WPB = B / 2;   // 32-bit words per 16-character block
        const uint32_t *src = reinterpret_cast<const uint32_t *>(packed + (s < n ? pofs[s] : 0));
        const int32_t nblk = (len + 15) / 16;
        uint32_t cur[WPB], nxt[WPB];
#pragma unroll
        for (int w = 0; w < WPB; w++) {
            cur[w] = nblk > 0 ? src[w] : 0u;
            nxt[w] = 0u;
        }
        uint32_t a = 0, k = 0, ps = s_pos[0], acc = 0;
        for (int32_t b = 0; b < nblk && k < M; b++) {
            if (b + 1 < nblk) {
#pragma unroll
                for (int w = 0; w < WPB; w++) nxt[w] = src[(size_t)(b + 1) * WPB + w];
            }
            const int32_t rem = len - 16 * b;
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const uint32_t c = (cur[(t * B) >> 5] >> ((t * B) & 31)) & ((1u << B) - 1u);
                const uint32_t a_next = s_next[c * NR + a];
                const bool live = t < rem;
                const bool hit = live && ps < a_next;   // a sample inside this character's steps
                acc = hit ? ((acc >> CB) | (c << (32 - CB))) : acc;
                k += hit ? 1u : 0u;
                if (hit && k % PER == 0) my[(size_t)(k / PER - 1) * TPB] = acc;
                ps = s_pos[k];
                while (live && ps < a_next) {   // rare: another sample in the same character
                    acc = (acc >> CB) | (c << (32 - CB));
                    k++;
                    if (k % PER == 0) my[(size_t)(k / PER - 1) * TPB] = acc;
                    ps = s_pos[k];
                }
                a = a_next;
            }
#pragma unroll
            for (int w = 0; w < WPB; w++) cur[w] = nxt[w];
        }
        if (k % PER) my[(size_t)(k / PER) * TPB] = acc >> (CB * (PER - k % PER));
        if (s < n) {
            for (uint32_t f = 0; f < m; f++) {
                uint64_t key = 0;
                uint32_t q = 0;
                for (int e = 0; e <= pk.n; e++) {   // the prefix keys (ascending z) on the way
                    const uint32_t qe = e < pk.n ? pk.z[e] : z;
                    for (; q < qe; q++) {
                        const uint32_t rk = s_rank[f * z + q];
                        const uint32_t c = (rk < k)
                                               ? ((my[(size_t)(rk / PER) * TPB] >> ((rk % PER) * CB)) & ((1u << CB) - 1u))
                                               : alpha;
                        key += (uint64_t)c * s_pow[q];
                    }
                    if (e < pk.n) pk.keys[e][((size_t)l * m + f) * n + s] = key;
                }
                keys[((size_t)l * m + f) * n + s] = key;
            }
        }
        return;
    }
    WordReader<B> rd;
    rd.init(packed + (s < n ? pofs[s] : 0), s < n ? chunks_for(len, B) : 0);
    // next step after the current character: first step >= a with pi = 1, plus one
    auto step_after = [&](uint32_t c, uint32_t a) -> uint32_t {
        if (a >= L) return L + 1;   // past every sample
        const uint32_t *row = s_tab + c * LW + (a >> 5);
        const uint32_t sh = a & 31u;
        const uint32_t lo = __funnelshift_r(row[0], row[1], sh);
        if (lo != 0u) return a + (uint32_t)__ffs((int)lo);
        const uint32_t hi = row[1] >> sh;
        if (hi != 0u) return a + 32u + (uint32_t)__ffs((int)hi);
        uint32_t j2 = (a >> 5) + 2;
        uint32_t v = s_tab[c * LW + j2];
        while (v == 0u) v = s_tab[c * LW + (++j2)];
        return (j2 << 5) + (uint32_t)__ffs((int)v);
    };
    // Character-major walk, all lanes one character per iteration. A sample
    // inside the current character's steps [a, a_next) is recorded without a
    // branch (at most one per iteration; a second one in the same character
    // takes a short loop).
    int32_t i = 0;
    uint32_t a = 0;                      // step at which the walk arrived at x[i]
    uint32_t k = 0;                      // next sample (in step order)
    uint32_t ps = s_pos[0];              // its step
    uint32_t acc = 0;
    while (i < len && k < M) {
        const uint32_t c = rd.code();
        const uint32_t a_next = step_after(c, a);
        const bool hit = ps < a_next;
        acc |= hit ? (c << ((k % PER) * CB)) : 0u;
        if (hit && (k % PER == PER - 1)) {
            my[(size_t)(k / PER) * TPB] = acc;
            acc = 0;
        }
        k += hit ? 1u : 0u;
        ps = s_pos[k];
        while (ps < a_next) {            // rare: another sample in the same character
            acc |= c << ((k % PER) * CB);
            if (k % PER == PER - 1) {
                my[(size_t)(k / PER) * TPB] = acc;
                acc = 0;
            }
            ps = s_pos[++k];
        }
        a = a_next;
        i++;
        rd.advance();
    }
    const uint32_t k_end = k;            // samples from k_end on lie after the walk: bottom
    if (k % PER) my[(size_t)(k / PER) * TPB] = acc;
    if (s < n) {
        for (uint32_t f = 0; f < m; f++) {
            uint64_t key = 0;
            uint32_t q = 0;
            for (int e = 0; e <= pk.n; e++) {   // the prefix keys (ascending z) on the way
                const uint32_t qe = e < pk.n ? pk.z[e] : z;
                for (; q < qe; q++) {
                    const uint32_t rk = s_rank[f * z + q];
                    const uint32_t c = (rk < k_end)
                                           ? ((my[(size_t)(rk / PER) * TPB] >> ((rk % PER) * CB)) & ((1u << CB) - 1u))
                                           : alpha;
                    key += (uint64_t)c * s_pow[q];
                }
                if (e < pk.n) pk.keys[e][((size_t)l * m + f) * n + s] = key;
            }
            keys[((size_t)l * m + f) * n + s] = key;
        }
    }
}

// Walk + signatures for alphabets of at most four symbols (2-bit codes), with
// the next-step table extended by sample counts. Entry (a, c) of the block's
// table is e = a' << 16 | 2 cnt(a'), where a' = next1_c(a) + 1 is the arrival
// step of the character after a c that arrived at step a (L + 1 past the
// sampling range) and cnt(x) is the number of sampled steps below x. The c read
// at step a covers the samples cnt(a) .. cnt(a') - 1 (in step order), so with e
// the entry of the current arrival, one character is: the next entry
// e' = T[a'][c] (its row offset is e >> 12, the low half being below 4096), and
// 2 (cnt(a') - cnt(a)) = e' - e in its low five bits: that many bits of copies
// of c enter a 64-bit shift register from below (two funnel shifts). After 16
// characters the block's count e_end - e_start decides: below 16 samples the
// register holds every code of the block and at most one 32-bit record word has
// filled, which is written; otherwise (or in a partial last block) the block is
// walked again one character and one sample at a time. The record holds the
// code of sample k (step order) at bits 30 - 2(k mod 16) of word k / 16.
constexpr int ESD_MAX_M = 2047;   // 2 M < 4096: the count fits the entry's low 12 bits

__host__ __device__ __forceinline__ size_t esd_words(uint32_t M) { return (M + 15) / 16 + 1; }

size_t embed_sign_dna_smem(uint32_t L, uint32_t m, uint32_t z, int tpb) {
    const size_t M = (size_t)m * z;
    if (M == 0 || M > ESD_MAX_M || L + 1 >= 65536u) return 0;
    const size_t bytes = (size_t)next_row(L) * 16 + esd_words((uint32_t)M) * 4 * (size_t)tpb + (size_t)z * 8 + M * 8;
    return bytes <= 220 * 1024 ? bytes : 0;
}

template <int TPB>
__global__ void __launch_bounds__(TPB, 1)
embed_sign_dna_kernel(const uint4 *__restrict__ packed, const uint64_t *__restrict__ pofs,
                      const int32_t *__restrict__ lens, int64_t n, uint32_t m, uint32_t z, uint32_t L,
                      uint32_t alpha, const uint16_t *__restrict__ next, const uint32_t *__restrict__ spos,
                      const uint32_t *__restrict__ stag, uint64_t *__restrict__ keys, PrefixKeys pk) {
    extern __shared__ uint64_t esd_smem[];
    const uint32_t l = blockIdx.y, M = m * z, NR = next_row(L);
    // the table first, at a fixed shared-memory address (its loads take the base
    // as an immediate), then the record, powers, sample steps and ranks
    uint32_t *s_tab = (uint32_t *)esd_smem;                        // [NR][4]
    uint32_t *s_rec = s_tab + (size_t)NR * 4;                      // [esd_words(M)][TPB]
    uint64_t *s_pow = (uint64_t *)(s_rec + esd_words(M) * TPB);    // [z] (8-byte aligned: NR*4 + words*TPB is even)
    uint32_t *s_pos = (uint32_t *)(s_pow + z);                     // [M] sample steps, ascending
    uint32_t *s_rank = s_pos + M;                                  // [M] step-order index of sample f*z+q
    for (uint32_t i = threadIdx.x; i < M; i += TPB) {
        s_pos[i] = spos[(size_t)l * M + i];
        const uint32_t tag = stag[(size_t)l * M + i];
        s_rank[(tag >> 16) * z + (tag & 0xFFFFu)] = i;
    }
    if (threadIdx.x == 0) {
        uint64_t pw = 1;
        for (uint32_t q = 0; q < z; q++) {
            s_pow[q] = pw;
            pw *= (uint64_t)alpha + 1;
        }
    }
    __syncthreads();
    const uint16_t *nx = next + (size_t)l * next_stride(alpha, L);
    for (uint32_t idx = threadIdx.x; idx < NR * 4; idx += TPB) {
        const uint32_t a = idx >> 2, c = idx & 3u;
        const uint32_t an = c < alpha ? (uint32_t)nx[c * NR + a] : L + 1;   // codes >= alpha never occur
        uint32_t lo = 0, hi = M;                                            // cnt(an): samples below an
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pos[mid] < an) lo = mid + 1;
            else hi = mid;
        }
        s_tab[idx] = (an << 16) | (2u * lo);
    }
    __syncthreads();

    const int64_t s = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const int32_t len = s < n ? lens[s] : 0;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(packed + (s < n ? pofs[s] : 0));
    const char *tab = reinterpret_cast<const char *>(s_tab);
    uint32_t *rec = s_rec + threadIdx.x;
    const uint32_t KB = 2u * M;   // record bits when every sample is taken
    uint32_t e = 0, hi = 0, lo = 0, kb = 0;
    // exact walk of one character and its samples, one sample at a time
    auto slow_char = [&](uint32_t c) {
        const uint32_t en = *reinterpret_cast<const uint32_t *>(tab + (e >> 12) + 4u * c);
        for (uint32_t d = (en - e) & 0xFFFFu; d > 0; d -= 2) {
            hi = (hi << 2) | (lo >> 30);
            lo = (lo << 2) | c;
            kb += 2;
            if ((kb & 31u) == 0) rec[(size_t)((kb >> 5) - 1) * TPB] = lo;
        }
        e = en;
    };
    const int32_t nfull = len >> 4, nw = (len + 15) >> 4;   // full blocks; words holding codes
    uint32_t w = nw > 0 ? src[0] : 0u;
    int32_t b = 0;
    for (; b < nfull && kb < KB; b++) {
        const uint32_t wn = b + 1 < nw ? src[b + 1] : 0u;   // the next block's codes, a block ahead
        const uint32_t e0 = e, hi0 = hi, lo0 = lo;
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const uint32_t c4 = (t == 0 ? (w << 2) : (w >> (2 * t - 2))) & 0xCu;   // 4 x code
            const uint32_t en = *reinterpret_cast<const uint32_t *>(tab + (e >> 12) + c4);
            const uint32_t d = en - e;                      // 2 x samples of this character (low bits)
            const uint32_t rep = c4 * 0x15555555u;          // the code in every 2-bit field but the lowest
            hi = __funnelshift_l(lo, hi, d);                // (hi:lo) << d, the top d bits of rep below
            lo = __funnelshift_l(rep, lo, d);
            e = en;
        }
        const uint32_t dk = (e - e0) & 0xFFFFu;
        if (dk < 32) {
            const uint32_t kn = kb + dk;
            if ((kn >> 5) != (kb >> 5))   // record word kn/32 - 1 has filled: its last code kn - ((kn>>5)<<5) bits up
                rec[(size_t)((kn >> 5) - 1) * TPB] = __funnelshift_r(lo, hi, kn & 31u);
            kb = kn;
        } else {
            // 16 or more samples in the block: again, exactly
            e = e0;
            hi = hi0;
            lo = lo0;
#pragma unroll 1
            for (int t = 0; t < 16; t++) slow_char((w >> (2 * t)) & 3u);
        }
        w = wn;
    }
    if (b == nfull && kb < KB) {   // the partial last block
        for (int32_t t = 0; t < (len & 15); t++) slow_char((w >> (2 * t)) & 3u);
    }
    const uint32_t k_end = kb >> 1;   // samples from k_end on lie after the walk: bottom
    if (kb & 31u) rec[(size_t)(kb >> 5) * TPB] = lo << (32u - (kb & 31u));
    if (s < n) {
        for (uint32_t f = 0; f < m; f++) {
            uint64_t key = 0;
            uint32_t q = 0;
            for (int ei = 0; ei <= pk.n; ei++) {   // the prefix keys (ascending z) on the way
                const uint32_t qe = ei < pk.n ? pk.z[ei] : z;
                for (; q < qe; q++) {
                    const uint32_t rk = s_rank[f * z + q];
                    const uint32_t c = (rk < k_end) ? ((rec[(size_t)(rk >> 4) * TPB] >> (30u - 2u * (rk & 15u))) & 3u) : alpha;
                    key += (uint64_t)c * s_pow[q];
                }
                if (ei < pk.n) pk.keys[ei][((size_t)l * m + f) * n + s] = key;
            }
            keys[((size_t)l * m + f) * n + s] = key;
        }
    }
}

template <int TPB>
static void esd_launch_t(size_t smem, cudaStream_t s, const uint4 *packed, const uint64_t *pofs, const int32_t *lens,
                         int64_t n, uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t alpha,
                         const uint16_t *next, const uint32_t *spos, const uint32_t *stag, uint64_t *keys,
                         const PrefixKeys &pk) {
    cudaFuncSetAttribute(embed_sign_dna_kernel<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((unsigned)((n + TPB - 1) / TPB), r);
    embed_sign_dna_kernel<TPB><<<grid, TPB, smem, s>>>(packed, pofs, lens, n, m, z, L, alpha, next, spos, stag, keys, pk);
}

template <int B, bool TABLE, int CB, int TPB>
static void es_launch_t(size_t smem, cudaStream_t s, const uint4 *packed, const uint64_t *pofs, const int32_t *lens,
                        int64_t n, uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t alpha, const uint32_t *tsym,
                        const uint16_t *next, const uint32_t *spos, const uint32_t *stag, uint64_t *keys,
                        const PrefixKeys &pk) {
    cudaFuncSetAttribute(embed_sign_kernel<B, TABLE, CB, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((unsigned)((n + TPB - 1) / TPB), r);
    embed_sign_kernel<B, TABLE, CB, TPB><<<grid, TPB, smem, s>>>(packed, pofs, lens, n, m, z, L, alpha, tsym, next,
                                                                 spos, stag, keys, pk);
}

// The walk with tpb walks (strings) per block: 256, 512 (default) or 1024.
template <int B, bool TABLE, int CB>
static void es_launch(int tpb, size_t smem, cudaStream_t s, const uint4 *packed, const uint64_t *pofs,
                      const int32_t *lens, int64_t n, uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t alpha,
                      const uint32_t *tsym, const uint16_t *next, const uint32_t *spos, const uint32_t *stag,
                      uint64_t *keys, const PrefixKeys &pk) {
    if (tpb == 256)
        es_launch_t<B, TABLE, CB, 256>(smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
    else if (tpb == 1024)
        es_launch_t<B, TABLE, CB, 1024>(smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
    else
        es_launch_t<B, TABLE, CB, 512>(smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
}

cudaError_t launch_embed_sign(const uint4 *packed, const uint64_t *pofs, const int32_t *lens, int64_t n,
                              uint32_t r, uint32_t m, uint32_t z, uint32_t L, uint32_t alpha, int B,
                              const uint32_t *tsym, const uint16_t *next, const uint32_t *spos,
                              const uint32_t *stag, uint64_t *keys, cudaStream_t s, const PrefixKeys *prefix,
                              int tpb) {
    if (n == 0) return cudaGetLastError();
    const int tpb_req = tpb;
    if (tpb != 256 && tpb != 1024) tpb = ES_THREADS;
    PrefixKeys pk{};
    if (prefix) pk = *prefix;
    if (pk.n < 0 || pk.n > MAX_PREFIX_KEYS) return cudaErrorInvalidValue;
    for (int e = 0; e < pk.n; e++)
        if (pk.z[e] < 1 || pk.z[e] > z || !pk.keys[e]) return cudaErrorInvalidValue;
    for (int e = 1; e < pk.n; e++)   // ascending z (the kernel stores them in that order)
        for (int f = e; f > 0 && pk.z[f] < pk.z[f - 1]; f--) {
            std::swap(pk.z[f], pk.z[f - 1]);
            std::swap(pk.keys[f], pk.keys[f - 1]);
        }
    const bool table = embed_sign_uses_table(alpha, L) && next != nullptr;
    if (B == 2 && table) {
        // four symbols or fewer: the walk with sample counts in the table, 1024
        // walks per block (one block per SM holds the table), else 512
        const int t2 = tpb_req == 512 ? 512 : 1024;
        const size_t sm2 = embed_sign_dna_smem(L, m, z, t2);
        if (sm2 > 0) {
            if (t2 == 512) esd_launch_t<512>(sm2, s, packed, pofs, lens, n, r, m, z, L, alpha, next, spos, stag, keys, pk);
            else esd_launch_t<1024>(sm2, s, packed, pofs, lens, n, r, m, z, L, alpha, next, spos, stag, keys, pk);
            note_launches(1);
            return cudaGetLastError();
        }
    }
    size_t smem = embed_sign_smem(alpha, L, m, z, tpb);
    if (smem == 0 && tpb != ES_THREADS) smem = embed_sign_smem(alpha, L, m, z, tpb = ES_THREADS);
    if (smem == 0) return cudaErrorInvalidValue;
    if (B == 2) {
        if (table) es_launch<2, true, 2>(tpb, smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
        else es_launch<2, false, 2>(tpb, smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
    } else {
        if (table) es_launch<8, true, 8>(tpb, smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
        else es_launch<8, false, 8>(tpb, smem, s, packed, pofs, lens, n, r, m, z, L, alpha, tsym, next, spos, stag, keys, pk);
    }
    note_launches(1);
    return cudaGetLastError();
}

// Signatures of a parameter set (r, m, z) from those of a wider one (r_src >= r,
// m_src >= m, z_src >= z, same seed and L). The bits pi_l(sigma) and positions
// P[l][f][q] of Sec. 3 depend on (l, f, q) alone, so embedding l and function f
// sample the same steps in both sets, and the key sum_q c_q (alpha+1)^q of the
// first z samples is the wider key mod (alpha+1)^z.
__global__ void derive_keys_kernel(const uint64_t *__restrict__ src, uint32_t m_src, int64_t n, uint32_t r,
                                   uint32_t m, uint64_t modulus, uint64_t *__restrict__ dst) {
    const int64_t total = (int64_t)r * m * n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g / n, s = g - t * n;
        const int64_t l = t / m, f = t - l * m;
        const uint64_t v = src[(l * m_src + f) * n + s];
        dst[g] = modulus ? v % modulus : v;
    }
}

cudaError_t launch_derive_keys(const uint64_t *src, uint32_t m_src, int64_t n, uint32_t r, uint32_t m,
                               uint64_t modulus, uint64_t *dst, cudaStream_t s) {
    const int64_t total = (int64_t)r * m * n;
    if (total == 0) return cudaGetLastError();
    const int64_t g = (total + 255) / 256;
    derive_keys_kernel<<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, s>>>(src, m_src, n, r, m, modulus, dst);
    note_launches(1);
    return cudaGetLastError();
}

// The two-level hash of Section 4 in place of the exact keys [r*m][n]: the
// exact key sum_q c_q (alpha+1)^q is decoded into the signature's codes c_q,
// and the key becomes <u, v> mod P with u_q = c_q + 1 and v[l][f][q] =
// mulhi64(splitmix64(splitmix64(seed) ^ (3<<56 | l<<48 | f<<32 | q)), P).
__global__ void keys_modp_kernel(uint64_t *__restrict__ keys, int64_t n, uint32_t r, uint32_t m, uint32_t z,
                                 uint32_t alpha, uint64_t seed, uint64_t P) {
    const int64_t total = (int64_t)r * m * n;
    const uint64_t base = mix64(seed), radix = (uint64_t)alpha + 1;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g / n;
        const uint32_t l = (uint32_t)(t / m), f = (uint32_t)(t - (int64_t)l * m);
        uint64_t key = keys[g], acc = 0;
        for (uint32_t q = 0; q < z; q++) {
            const uint64_t c = key % radix;
            key /= radix;
            const uint64_t ctr = (3ull << 56) | ((uint64_t)l << 48) | ((uint64_t)f << 32) | (uint64_t)q;
            const uint64_t v = __umul64hi(mix64(base ^ ctr), P);
            acc = (acc + (c + 1) * v) % P;
        }
        keys[g] = acc;
    }
}

cudaError_t launch_keys_modp(uint64_t *keys, int64_t n, uint32_t r, uint32_t m, uint32_t z, uint32_t alpha,
                             uint64_t seed, uint64_t P, cudaStream_t s) {
    const int64_t total = (int64_t)r * m * n;
    if (total == 0) return cudaGetLastError();
    const int64_t g = (total + 255) / 256;
    keys_modp_kernel<<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, s>>>(keys, n, r, m, z, alpha, seed, P);
    note_launches(1);
    return cudaGetLastError();
}

// Strings idx[0 .. gn) of a set gathered into one buffer (goff: their offsets
// there), one warp per string.
__global__ void gather_strings_kernel(const uint8_t *__restrict__ bytes, const int64_t *__restrict__ offsets,
                                      const int32_t *__restrict__ idx, int64_t gn, const int64_t *__restrict__ goff,
                                      uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < gn; q += warps) {
        const int64_t i = idx[q];
        const int64_t len = goff[q + 1] - goff[q];
        const uint8_t *src = bytes + offsets[i];
        for (int64_t t = lane; t < len; t += 32) out[goff[q] + t] = src[t];
    }
}

// Group-local pairs (a << 32 | b) mapped to the ids idx[a], idx[b] (increasing
// in a group, so the order a < b is kept), appended at out[base ..).
__global__ void remap_pairs_kernel(const uint64_t *__restrict__ pairs, int64_t cnt, const int32_t *__restrict__ idx,
                                   uint64_t *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = pairs[e];
        out[e] = ((uint64_t)(uint32_t)idx[v >> 32] << 32) | (uint64_t)(uint32_t)idx[v & 0xFFFFFFFFull];
    }
}

cudaError_t launch_gather_strings(const uint8_t *bytes, const int64_t *offsets, const int32_t *idx, int64_t gn,
                                  const int64_t *goff, uint8_t *out, cudaStream_t s) {
    if (gn == 0) return cudaGetLastError();
    int64_t g = (gn * 32 + 255) / 256;
    gather_strings_kernel<<<(unsigned)(g > 152 * 32 ? 152 * 32 : g), 256, 0, s>>>(bytes, offsets, idx, gn, goff, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_remap_pairs(const uint64_t *pairs, int64_t cnt, const int32_t *idx, uint64_t *out, cudaStream_t s) {
    if (cnt == 0) return cudaGetLastError();
    int64_t g = (cnt + 255) / 256;
    remap_pairs_kernel<<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, s>>>(pairs, cnt, idx, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ej
