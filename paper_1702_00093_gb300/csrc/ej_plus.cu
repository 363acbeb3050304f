// Device kernels of EmbedJoin+ (Section 5, Algorithms 4 and 5).
//
// Alg. 4 embeds, for every string s_i, the substrings (suffixes)
// s_{i,k} = s_i[(k-1)*delta ..] for k = 1 .. S (S = ceil(K/delta), at least 1).
// Here every suffix becomes a string of its own (record q = i*S + k-1) of a
// device string set, so that the ordinary fused walk signs it, and every record
// carries the length of its whole string for the length filter of Alg. 5.
// The hashed buckets then emit each pair of records that share a bucket in a
// table once per table: a record pair (q_a, q_b) is exactly Alg. 5's match
// (x, y, k_x, k_y). After a sort of the record pairs, a run of equal pairs is
// the count of that tuple over the tables; a pair of different strings with a
// count of at least T becomes a candidate (pairs of two substrings of one
// string share buckets too; they are counted apart and dropped).
#include "ej_internal.cuh"

namespace ej {

namespace {

// sub_len[q] = max(0, |s_i| - (k-1)*delta) (uint32, for the offsets scan) and
// whole_len[q] = |s_i| for record q = i*S + (k-1).
__global__ void suffix_lengths_kernel(const int32_t *__restrict__ lens, int64_t n, int32_t S, int32_t delta,
                                      uint32_t *__restrict__ sub_len, int32_t *__restrict__ whole_len) {
    const int64_t nq = n * (int64_t)S;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / S;
        const int64_t start = (q - i * S) * (int64_t)delta;
        const int32_t len = lens[i];
        sub_len[q] = (uint32_t)(start < len ? len - start : 0);
        whole_len[q] = len;
    }
}

// Bytes of every suffix, one warp per record: out[sub_off[q] ..) =
// bytes[offsets[i] + (k-1)*delta ..), sub_len[q] bytes.
__global__ void suffix_copy_kernel(const uint8_t *__restrict__ bytes, const int64_t *__restrict__ offsets, int64_t n,
                                   int32_t S, int32_t delta, const uint64_t *__restrict__ sub_off,
                                   uint8_t *__restrict__ out) {
    const int64_t nq = n * (int64_t)S;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const int64_t i = q / S;
        const uint64_t dst = sub_off[q], cnt = sub_off[q + 1] - dst;
        const uint8_t *src = bytes + offsets[i] + (q - i * S) * (int64_t)delta;
        for (uint64_t t = lane; t < cnt; t += 32) out[dst + t] = src[t];
    }
}

// Runs of equal record pairs in the sorted raw matches: a run of length >= T
// whose records belong to different strings appends the string pair
// (q_a / S) << 32 | (q_b / S) (each pair of records is one tuple; a string
// pair may come from several tuples, duplicates are removed afterwards).
__global__ void plus_runs_kernel(const uint64_t *__restrict__ sorted, int64_t nraw, int32_t S, int32_t T,
                                 uint64_t *__restrict__ out, unsigned long long cap,
                                 unsigned long long *__restrict__ count, unsigned long long *__restrict__ same) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nraw; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = sorted[e];
        if (e > 0 && sorted[e - 1] == v) continue;   // not the first of its run
        int64_t run = 1;
        while (e + run < nraw && sorted[e + run] == v) run++;   // at most one per table
        const uint64_t a = (v >> 32) / (uint64_t)S, b = (v & 0xFFFFFFFFull) / (uint64_t)S;
        if (a == b) {   // two substrings of one string: not a match of Alg. 5
            atomicAdd(same, (unsigned long long)run);
            continue;
        }
        if (run < T) continue;
        const unsigned long long idx = atomicAdd(count, 1ull);
        if (idx < cap) out[idx] = a < b ? (a << 32 | b) : (b << 32 | a);
    }
}

int grid_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_suffix_lengths(const int32_t *lens, int64_t n, int32_t S, int32_t delta, uint32_t *sub_len,
                                  int32_t *whole_len, cudaStream_t s) {
    if (n * (int64_t)S == 0) return cudaSuccess;
    suffix_lengths_kernel<<<grid_for(n * (int64_t)S, 256), 256, 0, s>>>(lens, n, S, delta, sub_len, whole_len);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_suffix_copy(const uint8_t *bytes, const int64_t *offsets, int64_t n, int32_t S, int32_t delta,
                               const uint64_t *sub_off, uint8_t *out, cudaStream_t s) {
    if (n * (int64_t)S == 0) return cudaSuccess;
    suffix_copy_kernel<<<grid_for(n * (int64_t)S * 32, 256), 256, 0, s>>>(bytes, offsets, n, S, delta, sub_off, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plus_runs(const uint64_t *sorted, int64_t nraw, int32_t S, int32_t T, uint64_t *out,
                             uint64_t cap, unsigned long long *count, unsigned long long *same, cudaStream_t s) {
    if (nraw == 0) return cudaSuccess;
    plus_runs_kernel<<<grid_for(nraw, 256), 256, 0, s>>>(sorted, nraw, S, T, out, (unsigned long long)cap, count,
                                                          same);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ej
