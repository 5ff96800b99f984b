// sivf_build_inverted_file_noalloc: the structured inverted-file build of the
// update step (front = moving centroids, back = invariant ones, ascending ids
// in each part) for callers that cannot allocate device memory.
//
// Some callers own every byte of device memory they run in: inference-engine
// plugins whose enqueue step must not allocate, and services that reserve a
// fixed device-memory budget at start-up and cannot let a request path call
// cudaMalloc (it can fail under that budget and it synchronises the device).
// This entry point takes its scratch from a file-scope static device array
// instead, so it calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array is a fixed SIVF_NOALLOC_SCRATCH_BYTES block held by every GPU
// that loads the library until the process exits. All calls share it and it
// keeps the previous call's contents, so everything that must start at zero is
// cleared on each call, and calls that overlap on the GPU (different streams
// or devices sharing a context) race on it.
//
// Host code cannot use the array's name as a device address: it names a host
// stand-in. The device address is looked up once per device, on the first
// call made with that device current, with cudaGetSymbolAddress; make that
// first call before any stream capture starts.
//
// The centroid offsets and terms live in device memory, so the host cannot
// check them. A first kernel checks coff (coff[0] = 0, non-decreasing,
// coff[k] = n_entries) and records a failure in a flag word of the scratch;
// every later kernel reads the flag and does nothing once it is set, and the
// key kernel checks each term against D. The call waits for its stream at the
// end, reads the flag and returns SIVF_ERR_INVALID_ARG when it is set. Every
// access stays inside the caller's arrays and the scratch whatever their
// contents.
#include <mutex>

#include "sivf_internal.cuh"

namespace {

constexpr size_t kMaxEntries = SIVF_NOALLOC_MAX_ENTRIES;
constexpr size_t kMaxTerms = SIVF_NOALLOC_MAX_TERMS;
constexpr size_t kMaxClusters = SIVF_NOALLOC_MAX_CLUSTERS;

// scratch layout, taken by a bump allocator in this order (256-byte aligned):
// check flag, cluster id, keys, values, keys', values' (4 B x entries each),
// per (term, part) counts (2 x terms x 4 B), list lengths ((terms + 1) x 8 B),
// radix histogram (at most 1 MiB at the limits) and scan partials.
constexpr size_t kScratchBytes = SIVF_NOALLOC_SCRATCH_BYTES;
static_assert(kScratchBytes >= 256 + 5 * 4 * kMaxEntries + 2 * 4 * kMaxTerms + 8 * (kMaxTerms + 1) + (1u << 20),
              "scratch too small for the stated limits");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch for the current device (looked up once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

inline unsigned grid_for(int64_t n, int tpb) {
    int64_t b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;  // every kernel below is grid-stride
    return (unsigned)b;
}

// coff[0] = 0, coff[j] <= coff[j+1], coff[k] = n: otherwise *bad = 1.
__global__ void na_check(int32_t k, int64_t n, const int64_t *coff, int *bad) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    if (g == 0 && (coff[0] != 0 || coff[k] != n)) atomicOr(bad, 1);
    for (int64_t j = g; j < k; j += st)
        if (coff[j] > coff[j + 1]) atomicOr(bad, 1);
}

// Cluster id of every centroid entry: one warp per cluster (grid-stride).
__global__ void na_cluster_of(int32_t k, int64_t n, const int64_t *coff, int32_t *clu, const int *bad) {
    if (*bad) return;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < k; j += nw) {
        const int64_t e1 = min(coff[j + 1], n);
        for (int64_t e = coff[j] + lane; e < e1; e += 32) clu[e] = (int32_t)j;
    }
}

// Sort key term << 1 | lambda of the entry's cluster, with per (term, part)
// counts. A term outside [0, D) sets the flag.
__global__ void na_keys(int64_t n, int32_t D, const int32_t *cterm, const int32_t *clu, const uint8_t *lam,
                        uint32_t *keys, uint32_t *vals, uint32_t *cnt2, int *bad) {
    if (*bad) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = cterm[e];
        if (t < 0 || t >= D) {
            atomicOr(bad, 1);
            keys[e] = 0u;
            vals[e] = (uint32_t)e;
            continue;
        }
        const uint32_t key = ((uint32_t)t << 1) | (uint32_t)(lam[clu[e]] ? 1 : 0);
        keys[e] = key;
        vals[e] = (uint32_t)e;
        atomicAdd(cnt2 + key, 1u);
    }
}

__global__ void na_lens(int32_t D, const uint32_t *cnt2, int64_t *len, int32_t *mf0) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D; t += (int64_t)gridDim.x * blockDim.x) {
        len[t] = (int64_t)cnt2[2 * t] + (int64_t)cnt2[2 * t + 1];
        mf0[t] = (int32_t)cnt2[2 * t];
    }
}

__global__ void na_fill(int64_t n, const uint32_t *order, const int32_t *clu, const float *cval, int32_t *cid,
                        float *u, const int *bad) {
    if (*bad) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = order[q];
        cid[q] = clu[e];
        u[q] = cval[e];
    }
}

}  // namespace

extern "C" sivf_status sivf_build_inverted_file_noalloc(int32_t k, int32_t D, int64_t n_entries, const int64_t *coff,
                                                        const int32_t *cterm, const float *cval, const uint8_t *lam,
                                                        int64_t *if_off, int32_t *if_mf0, int32_t *if_cid,
                                                        float *if_u, void *stream) {
    using namespace sivf;
    if (k < 1 || (size_t)k > kMaxClusters || D < 1 || (size_t)D > kMaxTerms || n_entries < 0 ||
        (size_t)n_entries > kMaxEntries)
        return SIVF_ERR_INVALID_ARG;
    if (!coff || !lam || !if_off || !if_mf0 || (n_entries > 0 && (!cterm || !cval || !if_cid || !if_u)))
        return SIVF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SIVF_ERR_CUDA;

    Workspace ws;
    ws.base = static_cast<char *>(base);
    ws.cap = kScratchBytes;
    const size_t n = (size_t)n_entries;
    int *bad = ws.take<int>(1);
    int32_t *clu = ws.take<int32_t>(n + 1);
    uint32_t *k0 = ws.take<uint32_t>(n + 1), *v0 = ws.take<uint32_t>(n + 1);
    uint32_t *k1 = ws.take<uint32_t>(n + 1), *v1 = ws.take<uint32_t>(n + 1);
    uint32_t *cnt2 = ws.take<uint32_t>(2 * (size_t)D);
    int64_t *len = ws.take<int64_t>((size_t)D + 1);
    int64_t *total = ws.take<int64_t>(1);
    if (!bad || !clu || !k0 || !v0 || !k1 || !v1 || !cnt2 || !len || !total) return SIVF_ERR_INVALID_ARG;

    int bits_t = bits_for((uint64_t)(D - 1));
    if (bits_t < 1) bits_t = 1;
    // the scratch keeps the previous call's contents: clear the flag and the counters
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return SIVF_ERR_CUDA;
    if (cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * 2 * (size_t)D, s) != cudaSuccess) return SIVF_ERR_CUDA;
    na_check<<<grid_for(k, 256), 256, 0, s>>>(k, n_entries, coff, bad);
    na_cluster_of<<<grid_for((int64_t)k * 32, 256), 256, 0, s>>>(k, n_entries, coff, clu, bad);
    if (n_entries > 0)
        na_keys<<<grid_for(n_entries, 256), 256, 0, s>>>(n_entries, D, cterm, clu, lam, k0, v0, cnt2, bad);
    na_lens<<<grid_for(D, 256), 256, 0, s>>>(D, cnt2, len, if_mf0);
    note_launch(n_entries > 0 ? 4 : 3);
    if (cudaGetLastError() != cudaSuccess) return SIVF_ERR_CUDA;
    if (scan_exclusive_i64(len, if_off, D, total, ws, s) != cudaSuccess) return SIVF_ERR_CUDA;
    if (cudaMemcpyAsync(if_off + D, total, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SIVF_ERR_CUDA;
    bool alt = false;
    if (radix_sort_pairs(k0, v0, k1, v1, n_entries, bits_t + 1, &alt, ws, s) != cudaSuccess) return SIVF_ERR_CUDA;
    if (n_entries > 0) {
        na_fill<<<grid_for(n_entries, 256), 256, 0, s>>>(n_entries, alt ? v1 : v0, clu, cval, if_cid, if_u, bad);
        note_launch();
    }
    if (cudaGetLastError() != cudaSuccess) return SIVF_ERR_CUDA;
    // the device-side check decides the status: wait for it
    int bad_h = 0;
    if (cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SIVF_ERR_CUDA;
    return bad_h ? SIVF_ERR_INVALID_ARG : SIVF_OK;
}
