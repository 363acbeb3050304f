// ej_verify_noalloc: verification that allocates no memory at all.
//
// Some callers cannot let a library allocate device memory: processes whose
// device memory is fully reserved up front by another allocator (a framework's
// caching pool or a fixed budget decided at start-up), and latency-sensitive
// services that must not call cudaMalloc/cudaFree on their request path because
// those calls can synchronise the device and stall unrelated work. This entry
// point serves them: it needs no context and all of its scratch lives in one
// fixed, file-scope device array (EJ_NOALLOC_SCRATCH_BYTES), so it never calls
// cudaMalloc, cudaFree or any allocating library routine.
//
// Consequences the caller must know:
//  - every GPU on which the array's module is loaded holds it until the process
//    exits: with lazy module loading (the CUDA default) from the first call on
//    that device, with eager loading from when the library is loaded;
//  - all calls share the array and it keeps the previous call's contents, so two
//    calls whose GPU work overlaps (different streams or host threads) race;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) and should come before any stream capture;
//  - requests whose scratch does not fit return EJ_ERR_TOO_LARGE.
#include <cstring>
#include <mutex>

#include "ej_internal.cuh"

namespace ej {
size_t verify_smem_bytes(VerifyConfig c, uint32_t alpha, int64_t max_len, int32_t K);
}

using namespace ej;

namespace {

constexpr size_t kScratchBytes = EJ_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {nullptr};

size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = (unsigned char *)ptr;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define NA_CK(expr)                                       \
    do {                                                  \
        if ((expr) != cudaSuccess) return EJ_ERR_CUDA;    \
    } while (0)

}  // namespace

extern "C" int ej_verify_noalloc(const ej_strings *S, const ej_params *p, const uint64_t *pairs,
                                 int64_t n_pairs, uint64_t *out, int64_t *n_out, void *stream) {
    if (!n_out) return EJ_ERR_INVALID_ARG;
    *n_out = 0;
    if (!S || !p || n_pairs < 0 || p->K < 0 || p->alphabet_size < 1 || p->alphabet_size > 255 || !p->alphabet)
        return EJ_ERR_INVALID_ARG;
    if (S->n < 0 || S->n >= (1ll << 31)) return EJ_ERR_INVALID_ARG;
    if (n_pairs == 0) return EJ_OK;
    if (S->n == 0 || !on_device(S->bytes) || !on_device(S->offsets) || !on_device(pairs) || !on_device(out))
        return EJ_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = S->n;
    const uint32_t alpha = p->alphabet_size;

    // raw byte -> code map, built on the host stack
    uint8_t map[256];
    memset(map, 255, sizeof map);
    for (uint32_t c = 0; c < alpha; c++) {
        if (map[p->alphabet[c]] != 255) return EJ_ERR_INVALID_ARG;
        map[p->alphabet[c]] = (uint8_t)c;
    }

    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev >= kMaxDevices) return EJ_ERR_UNSUPPORTED;
    unsigned char *base = nullptr;
    NA_CK(scratch_address(dev, &base));

    int64_t total = 0;
    NA_CK(cudaMemcpyAsync(&total, S->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (total < 0) return EJ_ERR_INVALID_ARG;
    // sizes far beyond the array are rejected before any size arithmetic that
    // could wrap: at least 16 bytes per string, 9 per pair, 1/4 per byte
    if (n > (int64_t)(kScratchBytes / 16) || n_pairs > (int64_t)(kScratchBytes / 9) ||
        total > (int64_t)kScratchBytes * 4)
        return EJ_ERR_TOO_LARGE;

    // carve the scratch array
    const int B = packed_bits_for(alpha);
    const int64_t chunk_bound = (total * B + 127) / 128 + n + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += round_up(bytes); return base + o; };
    uint32_t *err = (uint32_t *)take(64);                         // err, max length, counters
    uint8_t *d_map = (uint8_t *)take(256);
    int32_t *lens = (int32_t *)take((size_t)n * 4);
    uint32_t *ccnt = (uint32_t *)take((size_t)(n + 1) * 4);
    uint64_t *pofs = (uint64_t *)take((size_t)(n + 2) * 8);
    void *scan_a = take(scan_temp_bytes(n + 1));
    uint4 *packed = (uint4 *)take((size_t)chunk_bound * 16);
    uint8_t *flags = (uint8_t *)take((size_t)n_pairs);
    uint64_t *foffs = (uint64_t *)take((size_t)n_pairs * 8);
    void *scan_b = take(scan_temp_bytes(n_pairs));
    if (off > kScratchBytes) return EJ_ERR_TOO_LARGE;

    NA_CK(cudaMemsetAsync(err, 0, 64, s));
    NA_CK(cudaMemcpyAsync(d_map, map, 256, cudaMemcpyHostToDevice, s));
    unsigned long long *dmax = (unsigned long long *)(err + 2);
    NA_CK(launch_validate(S->bytes, S->offsets, n, total, d_map, lens, err, dmax, s));
    NA_CK(launch_chunk_counts(lens, n, B, ccnt, s));
    NA_CK(exclusive_scan_u32(ccnt, pofs, n + 1, nullptr, scan_a, s));
    NA_CK(launch_pack(S->bytes, S->offsets, lens, n, total, d_map, B, pofs, packed, err, s));
    uint64_t h[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(h, err, 16, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if ((uint32_t)(h[0] & 0xffffffffu) & (DERR_OFFSETS | DERR_SYMBOL)) return EJ_ERR_INVALID_ARG;
    const int64_t max_len = (int64_t)h[1];

    VerifyConfig vc = verify_pick(p->K, alpha, max_len);
    if (vc.G == 0) return EJ_ERR_UNSUPPORTED;
    uint64_t *count = (uint64_t *)(err + 4);
    VerifyOut vo{flags, nullptr, nullptr, 0, nullptr, err, nullptr, nullptr, nullptr};
    NA_CK(launch_verify(vc, packed, pofs, B, lens, n, alpha, pairs, n_pairs, p->K, max_len, vo, s));
    NA_CK(exclusive_scan_u8(flags, foffs, n_pairs, count, scan_b, s));
    uint64_t hc[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(hc, err, 8, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(hc + 1, count, 8, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if ((uint32_t)(hc[0] & 0xffffffffu) & DERR_PAIR) return EJ_ERR_INVALID_ARG;
    NA_CK(launch_compact_u64(pairs, flags, foffs, n_pairs, out, s));
    NA_CK(cudaStreamSynchronize(s));
    *n_out = (int64_t)hc[1];
    return EJ_OK;
}
