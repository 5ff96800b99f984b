// Device-wide primitives used by the update step: exclusive prefix sums and a
// stable LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Scan: reduce-then-scan in three launches (tile sums, one-CTA scan of the
// tile sums, tile-local scan plus carry-in).
// Every tile kernel loops over tiles with a grid of at most TILE_GRID blocks,
// and when the element count is on the device it stops at the live tiles, so
// a launch sized by a capacity costs no empty blocks.
// Radix sort: digits of up to 10 bits (fewest passes for the key width), per
// pass (1) per-tile digit histograms stored digit-major, (2) an exclusive
// scan of that table, (3) a stable scatter whose in-tile ranks come from
// warp-level __match_any_sync on the digit.
#include "sivf_internal.cuh"

namespace sivf {

unsigned long long g_launches = 0;

int bits_for(uint64_t max_value) {
    int b = 0;
    while (b < 64 && (max_value >> b) != 0) ++b;
    return b;
}

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int64_t TILE_GRID = 2048;
inline unsigned tile_grid(int64_t tiles) { return (unsigned)(tiles < TILE_GRID ? (tiles > 0 ? tiles : 1) : TILE_GRID); }
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T x, T *smem_warp, T *block_total) {
    // x: this thread's value; returns exclusive prefix within the block.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T w = lane < nw ? smem_warp[lane] : T(0);
        T winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        if (lane < nw) smem_warp[lane] = winc - w;
        if (lane == nw - 1) *block_total = winc;
    }
    __syncthreads();
    T r = smem_warp[warp] + inc - x;
    return r;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_sums(const T *in, int64_t n, const int64_t *n_dev,
                                                               T *tile_sums) {
    __shared__ T warp_s[32];
    __shared__ T total;
    if (n_dev) n = min(*n_dev, n);  // never past the launch bound
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {  // block-uniform
        const int64_t base = t * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        T s = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (base + i < n) s += in[base + i];
        block_exclusive_scan<T>(s, warp_s, &total);
        if (threadIdx.x == 0) tile_sums[t] = total;
        __syncthreads();
    }
}

// n: tile sums, or the tile count of the element bound when n_dev (element
// count on the device) is given; only the live tiles are scanned.
template <typename T>
__global__ void __launch_bounds__(1024) scan_single_block(T *data, int64_t n, const int64_t *n_dev, int64_t nmax,
                                                          T *total_out) {
    __shared__ T warp_s[32];
    __shared__ T total;
    if (n_dev) n = (min(*n_dev, nmax) + SCAN_TILE - 1) / SCAN_TILE;
    T carry = 0;
    for (int64_t b = 0; b < n; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        T x = i < n ? data[i] : T(0);
        T ex = block_exclusive_scan<T>(x, warp_s, &total);
        if (i < n) data[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles(const T *in, T *out, int64_t n, const int64_t *n_dev,
                                                           const T *tile_offs) {
    __shared__ T warp_s[32];
    __shared__ T total;
    if (n_dev) n = min(*n_dev, n);  // never past the launch bound
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {  // block-uniform
        const int64_t base = t * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        T v[SCAN_ITEMS];
        T s = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            v[i] = base + i < n ? in[base + i] : T(0);
            s += v[i];
        }
        T ex = block_exclusive_scan<T>(s, warp_s, &total) + tile_offs[t];
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            if (base + i < n) out[base + i] = ex;
            ex += v[i];
        }
        __syncthreads();
    }
}

// n: element count, or its upper bound when n_dev (device count) is given.
template <typename T>
cudaError_t scan_exclusive_impl(const T *in, T *out, int64_t n, T *total, Workspace &ws, cudaStream_t s,
                                const int64_t *n_dev = nullptr) {
    if (n <= 0) {
        if (total) SIVF_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(T), s));
        return cudaSuccess;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    size_t mark = ws.used;
    T *sums = ws.take<T>((size_t)tiles);
    if (!sums) return cudaErrorMemoryAllocation;
    scan_tile_sums<T><<<tile_grid(tiles), SCAN_THREADS, 0, s>>>(in, n, n_dev, sums);
    scan_single_block<T><<<1, 1024, 0, s>>>(sums, tiles, n_dev, n, total);
    scan_tiles<T><<<tile_grid(tiles), SCAN_THREADS, 0, s>>>(in, out, n, n_dev, sums);
    note_launch(3);
    ws.used = mark;
    return cudaGetLastError();
}

// ---------------- radix sort ----------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096
constexpr int RS_MAX_BITS = 10;                 // digit width of one pass (<= 1024 buckets)

// Histograms are stored digit-major with the live tile count as the stride
// (tiles past the live element count write nothing), and the table size is
// left in *scan_n for the scan that follows.
template <int BITS>
__global__ void __launch_bounds__(RS_THREADS) radix_hist(const uint32_t *keys, int64_t n, const int64_t *n_dev,
                                                         int shift, uint32_t *counts, int64_t *scan_n) {
    constexpr int R = 1 << BITS;
    constexpr uint32_t mask = R - 1;
    __shared__ uint32_t h[R];
    if (n_dev) n = min(*n_dev, n);  // never past the launch bound
    const int64_t live = (n + RS_TILE - 1) / RS_TILE;
    if (blockIdx.x == 0 && threadIdx.x == 0) *scan_n = live * R;
    for (int64_t t = blockIdx.x; t < live; t += gridDim.x) {  // block-uniform
        for (int d = threadIdx.x; d < R; d += RS_THREADS) h[d] = 0;
        __syncthreads();
        const int64_t base = t * RS_TILE;
        for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
            const int64_t p = base + i;
            if (p < n) atomicAdd(&h[(keys[p] >> shift) & mask], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < R; d += RS_THREADS) counts[(int64_t)d * live + t] = h[d];
        __syncthreads();
    }
}

template <int BITS>
__global__ void __launch_bounds__(RS_THREADS) radix_scatter(const uint32_t *__restrict__ kin,
                                                            const uint32_t *__restrict__ vin,
                                                            uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                            int64_t n, const int64_t *__restrict__ n_dev, int shift,
                                                            const uint32_t *__restrict__ offs, int64_t tiles) {
    constexpr int R = 1 << BITS;
    constexpr uint32_t mask = R - 1;
    __shared__ uint32_t wcnt[RS_WARPS][R];
    __shared__ uint32_t toff[R];
    if (n_dev) n = min(*n_dev, n);  // never past the launch bound
    const int64_t live = (n + RS_TILE - 1) / RS_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < live; t += gridDim.x) {  // block-uniform
        for (int d = threadIdx.x; d < R; d += RS_THREADS) {
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) wcnt[w][d] = 0;
            toff[d] = offs[(int64_t)d * live + t];
        }
        __syncthreads();
        const int64_t wbase = t * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
        uint32_t kk[RS_ITEMS], vv[RS_ITEMS], rk[RS_ITEMS];
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            int64_t p = wbase + r * 32 + lane;
            bool valid = p < n;
            uint32_t key = valid ? kin[p] : 0u;
            kk[r] = key;
            vv[r] = valid ? vin[p] : 0u;
            uint32_t d = valid ? ((key >> shift) & mask) : (uint32_t)R;  // sentinel groups invalid lanes
            unsigned peers = __match_any_sync(0xffffffffu, d);
            uint32_t old = valid ? wcnt[warp][d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) wcnt[warp][d] = old + (uint32_t)__popc(peers);
            __syncwarp();
            rk[r] = old + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < R; d += RS_THREADS) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            int64_t p = wbase + r * 32 + lane;
            if (p < n) {
                uint32_t d = (kk[r] >> shift) & mask;
                uint32_t pos = toff[d] + wcnt[warp][d] + rk[r];
                kout[pos] = kk[r];
                vout[pos] = vv[r];
            }
        }
        __syncthreads();  // wcnt and toff are rewritten for the next tile
    }
}

template <int BITS>
void radix_pass(const uint32_t *ka, const uint32_t *va, uint32_t *kb, uint32_t *vb, int64_t n, const int64_t *n_dev,
                int shift, uint32_t *counts, int64_t *scan_n, int64_t tiles, Workspace &ws, cudaStream_t s,
                cudaError_t *err) {
    radix_hist<BITS><<<tile_grid(tiles), RS_THREADS, 0, s>>>(ka, n, n_dev, shift, counts, scan_n);
    cudaError_t e = scan_exclusive_impl<uint32_t>(counts, counts, tiles * (1 << BITS), nullptr, ws, s, scan_n);
    if (e != cudaSuccess) {
        *err = e;
        return;
    }
    radix_scatter<BITS><<<tile_grid(tiles), RS_THREADS, 0, s>>>(ka, va, kb, vb, n, n_dev, shift, counts, tiles);
    note_launch(2);
}

}  // namespace

cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, Workspace &ws,
                               cudaStream_t s) {
    return scan_exclusive_impl<int64_t>(in, out, n, total, ws, s);
}

cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, Workspace &ws, cudaStream_t s) {
    return scan_exclusive_impl<uint32_t>(in, out, n, nullptr, ws, s);
}

cudaError_t scan_exclusive_u32_dev(const uint32_t *in, uint32_t *out, int64_t nmax, const int64_t *n_dev,
                                   uint32_t *total, Workspace &ws, cudaStream_t s) {
    return scan_exclusive_impl<uint32_t>(in, out, nmax, total, ws, s, n_dev);
}

cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n, int nbits,
                             bool *result_in_alt, Workspace &ws, cudaStream_t s) {
    return radix_sort_pairs_dev(k0, v0, k1, v1, n, nullptr, nbits, result_in_alt, ws, s);
}

cudaError_t radix_sort_pairs_dev(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n,
                                 const int64_t *n_dev, int nbits, bool *result_in_alt, Workspace &ws, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 0 || nbits <= 0 || (n == 1 && !n_dev)) return cudaSuccess;
    if (n > (int64_t)0xFFFFFFFFll || nbits > 32) return cudaErrorInvalidValue;
    // fewest passes of at most RS_MAX_BITS bits, widths as equal as possible
    const int passes = (nbits + RS_MAX_BITS - 1) / RS_MAX_BITS;
    const int width = (nbits + passes - 1) / passes;
    int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    size_t mark = ws.used;
    uint32_t *counts = ws.take<uint32_t>((size_t)tiles << width);
    int64_t *scan_n = ws.take<int64_t>(1);
    if (!counts || !scan_n) return cudaErrorMemoryAllocation;
    uint32_t *ka = k0, *va = v0, *kb = k1, *vb = v1;
    cudaError_t err = cudaSuccess;
    for (int shift = 0; shift < nbits; shift += width) {
        switch (width) {
            case 1: radix_pass<1>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 2: radix_pass<2>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 3: radix_pass<3>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 4: radix_pass<4>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 5: radix_pass<5>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 6: radix_pass<6>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 7: radix_pass<7>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 8: radix_pass<8>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            case 9: radix_pass<9>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
            default: radix_pass<10>(ka, va, kb, vb, n, n_dev, shift, counts, scan_n, tiles, ws, s, &err); break;
        }
        if (err != cudaSuccess) return err;
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
        *result_in_alt = !*result_in_alt;
    }
    ws.used = mark;
    return cudaGetLastError();
}

}  // namespace sivf
