// Update step of SIVF (Algorithm 5, Section 4.2) on sm_103a, plus the
// set-up kernels (CSR validation, seed centroids).
//
// Pipeline for iteration r (lambda = lambda^[r] from the assignment), in the
// default dense form:
//  u1  per-cluster member counts from the labels.
//  u2  an int64 fixed-point accumulator row of the instance's D terms per
//      cluster, kept across iterations: every object whose label changed
//      moves its q(x) = ceil(x 2^shift) values from its old cluster's row to
//      the new one with integer atomics (k_acc_scatter). Integer sums are
//      exact, so each entry is the sum over the current members whatever the
//      history, and the result is deterministic.
//  u3  pass 1 (k_acc_rows1): new row sizes, ||s_j|| from the exact 128-bit
//      sum of the squared integer sums (one rounding to FP64), and the
//      objective pieces <s_j, mu_j^[r-1]>; pass 2 (k_acc_rows2): the row
//      compacted in ascending term order, u = S (2^-shift / ||s_j||) in FP32.
//      Dividing by |C_j| first cancels exactly and is skipped.
//  u4  invariant and empty clusters keep their centroid row (copied).
//  u5  the scan structures of the structured inverted file, counted per term
//      and part (k_if_count) and written in one scatter pass over the
//      centroid entries (k_scan_fill): the scan order (moving
//      clusters first), the dense head rows and the sparse scan copy, whose
//      lists hold the moving centroids first and the invariant ones after
//      (Algorithm 5, lines 1-14 and 21-30). The canonical sorted file (ids
//      ascending in each part) is built by a stable radix sort only when a
//      getter asks for it.
// The sort form replaces u1-u3 by a stable radix sort of (label, object id),
// an expansion of the recomputed clusters' members' (term, value) pairs sorted
// by (cluster rank, term) and reduced sequentially in FP64, in ascending
// object id, the order of the plain definition (Algorithm 5, lines 17-20).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "sivf_internal.cuh"

namespace sivf {
namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(int64_t n, int tpb = TPB) {
    int64_t b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    if (b > 0x7FFFFFFF) b = 0x7FFFFFFF;
    return (unsigned)b;
}

// Grid of a grid-stride kernel: enough blocks to fill the GPU a few times
// over, not one per element, so that a launch bounded by a capacity (with the
// live count on the device) costs no empty blocks.
constexpr unsigned GS_MAX_BLOCKS = 4096;
inline unsigned blocks_gs(int64_t n, int tpb = TPB) {
    const unsigned b = blocks_for(n, tpb);
    return b < GS_MAX_BLOCKS ? b : GS_MAX_BLOCKS;
}

// ---------------- validation and set-up ----------------

// bad bits: 1 row_ptr, 2 idx range/order, 4 value, 8 norm
__global__ void k_validate(int64_t N, int32_t D, int64_t nnz, const int64_t *row_ptr, const int32_t *idx,
                           const float *val, float *sumv, int *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < N; i += nw) {
        const int64_t b = row_ptr[i], e = row_ptr[i + 1];
        int flags = 0;
        if (b < 0 || e < b || e > nnz) flags |= 1;
        double ss = 0.0, sv = 0.0;
        if (!(flags & 1)) {
            for (int64_t h = b + lane; h < e; h += 32) {
                const int t = idx[h];
                const float v = val[h];
                if (t < 0 || t >= D) flags |= 2;
                if (h > b && idx[h - 1] >= t) flags |= 2;
                if (!(v > 0.0f) || !isfinite(v)) flags |= 4;
                ss += (double)v * (double)v;
                sv += (double)v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
            flags |= __shfl_xor_sync(0xffffffffu, flags, o);
        }
        if (lane == 0) {
            if (!(flags & 1) && e > b && fabs(sqrt(ss) - 1.0) > 1e-4) flags |= 8;
            sumv[i] = (float)(sv * (1.0 + 1e-6));  // rounded up: the bound needs S >= sum v
            if (flags) atomicOr(bad, flags);
        }
    }
}

__global__ void k_seed_sizes(int32_t k, const int32_t *init_ids, const int64_t *row_ptr, int64_t *sz) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) {
        int64_t d = init_ids[j];
        sz[j] = row_ptr[d + 1] - row_ptr[d];
    }
}

__global__ void k_seed_rows(int32_t k, const int32_t *init_ids, const int64_t *row_ptr, const int32_t *idx,
                            const float *val, const int64_t *coff, int32_t *cterm, float *cval, int32_t *cclu) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wid >= k) return;
    const int j = (int)wid;
    const int64_t d = init_ids[j];
    const int64_t b = row_ptr[d], e = row_ptr[d + 1], o = coff[j];
    for (int64_t h = b + lane; h < e; h += 32) {
        cterm[o + (h - b)] = idx[h];
        cval[o + (h - b)] = val[h];
        cclu[o + (h - b)] = j;
    }
}

// Replace a^[r] by src. lambda^[r] is recomputed against a^[r-1] (every
// cluster moving before the second assignment); an object whose label
// changes loses its stored own-cluster score.
__global__ void k_set_labels(int64_t N, const int32_t *src, int32_t *labels, const int32_t *labels_prev,
                             uint32_t *own, uint8_t *moving) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[i];
        if (labels[i] != a) {
            labels[i] = a;
            own[i] = OWN_INVALID;
        }
        const int32_t prev = labels_prev[i];
        if (a != prev) {
            moving[a] = 1;
            if (prev >= 0) moving[prev] = 1;
        }
    }
}

__global__ void k_check_labels(int64_t N, int32_t k, const int32_t *src, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[i];
        if (a < 0 || a >= k) atomicOr(bad, 1);
    }
}

// ---------------- u1: group objects by label ----------------

__global__ void k_label_keys(int64_t N, const int32_t *labels, uint32_t *keys, uint32_t *vals, int64_t *cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = labels[i];
        keys[i] = (uint32_t)a;
        vals[i] = (uint32_t)i;
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt + a), 1ull);
    }
}

// recompute flag: moving (lambda = 0) and non-empty
__global__ void k_recompute_flags(int32_t k, const uint8_t *lam, const int64_t *cnt, int64_t *flag) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) flag[j] = (lam[j] == 0 && cnt[j] > 0) ? 1 : 0;
}

// ---------------- u2: cluster sums ----------------

__global__ void k_member_tuples(int64_t N, const uint32_t *perm, const int32_t *labels, const int64_t *flag,
                                const int64_t *row_ptr, int64_t *tc) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[p];
        tc[p] = flag[labels[i]] ? row_ptr[i + 1] - row_ptr[i] : 0;
    }
}

// One warp per member (in cluster, then object order): its (term, value)
// pairs become tuples t = toff[p] + h with the cluster's rank.
__global__ void k_expand(int64_t N, const uint32_t *perm, const int32_t *labels, const int64_t *rrank,
                         const int64_t *tc, const int64_t *toff, const int64_t *row_ptr, const int32_t *idx,
                         const float *val, uint32_t *kterm, uint32_t *vtup, uint32_t *tterm, float *tval,
                         uint32_t *trank) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = wid; p < N; p += nw) {
        if (tc[p] == 0) continue;
        const int64_t i = perm[p];
        const uint32_t rk = (uint32_t)rrank[labels[i]];
        const int64_t b = row_ptr[i], e = row_ptr[i + 1], o = toff[p];
        for (int64_t h = b + lane; h < e; h += 32) {
            const uint32_t t = (uint32_t)(o + (h - b));
            kterm[t] = (uint32_t)idx[h];
            vtup[t] = t;
            tterm[t] = (uint32_t)idx[h];
            tval[t] = val[h];
            trank[t] = rk;
        }
    }
}

// One 32-bit key per tuple when it fits: (cluster rank, instance-local term),
// with the value's bits as the payload.
__global__ void k_expand_packed(int64_t N, const uint32_t *perm, const int32_t *labels, const int64_t *rrank,
                                const int64_t *tc, const int64_t *toff, const int64_t *row_ptr, const int32_t *idx,
                                const float *val, const int32_t *clu_doff, int bits_tl, uint32_t *key,
                                uint32_t *vbits) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = wid; p < N; p += nw) {
        if (tc[p] == 0) continue;
        const int64_t i = perm[p];
        const int32_t j = labels[i];
        const uint32_t hi = (uint32_t)rrank[j] << bits_tl;
        const int32_t doff = clu_doff[j];
        const int64_t b = row_ptr[i], e = row_ptr[i + 1], o = toff[p];
        for (int64_t h = b + lane; h < e; h += 32) {
            key[o + (h - b)] = hi | (uint32_t)(idx[h] - doff);
            vbits[o + (h - b)] = __float_as_uint(val[h]);
        }
    }
}

// packed keys back to (rank << 32 | global term) and float values
__global__ void k_unpack(int64_t nmax, const int64_t *n_dev, const uint32_t *key, const uint32_t *vbits,
                         int bits_tl, const int32_t *rank2clu, const int32_t *clu_doff, unsigned long long *key64,
                         float *sval) {
    const int64_t n = *n_dev;
    const uint32_t tmask = (1u << bits_tl) - 1u;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t kk = key[q];
        const uint32_t r = kk >> bits_tl;
        const uint32_t t = (kk & tmask) + (uint32_t)clu_doff[rank2clu[r]];
        key64[q] = ((unsigned long long)r << 32) | (unsigned long long)t;
        sval[q] = __uint_as_float(vbits[q]);
    }
}

// cluster of each rank (inverse of rrank on the recomputed clusters)
__global__ void k_rank2clu(int32_t k, const int64_t *flag, const int64_t *rrank, int32_t *rank2clu) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k && flag[j]) rank2clu[rrank[j]] = j;
}

// after the stable sort by term: rank keys for the stable sort by rank
__global__ void k_rank_keys(int64_t nmax, const int64_t *n_dev, const uint32_t *vtup_sorted, const uint32_t *trank,
                            uint32_t *krank, uint32_t *vrank) {
    const int64_t n = *n_dev;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = vtup_sorted[q];
        krank[q] = trank[t];
        vrank[q] = t;
    }
}

// tuples in (rank, term, object) order: composite key and value
__global__ void k_compose(int64_t nmax, const int64_t *n_dev, const uint32_t *krank, const uint32_t *vtup,
                          const uint32_t *tterm, const float *tval, unsigned long long *key64, float *sval) {
    const int64_t n = *n_dev;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = vtup[q];
        key64[q] = ((unsigned long long)krank[q] << 32) | (unsigned long long)tterm[t];
        sval[q] = tval[t];
    }
}

__global__ void k_heads(int64_t nmax, const int64_t *n_dev, const unsigned long long *key, uint32_t *head) {
    const int64_t n = *n_dev;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        head[e] = (e == 0 || key[e] != key[e - 1]) ? 1u : 0u;
}

// position of each run of equal keys: hpos[u] = first element of run u
__global__ void k_head_pos(int64_t nmax, const int64_t *n_dev, const uint32_t *head, const uint32_t *uidx,
                           uint32_t *hpos) {
    const int64_t n = *n_dev;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (head[e]) hpos[uidx[e]] = (uint32_t)e;
}

// FP64 sum of each run of equal keys (a (cluster, term) pair), in two passes
// with a fixed order (reproducible bit for bit):
//  1. each warp takes 32 consecutive elements and forms, by a segmented
//     inclusive scan over the lanes, the sum of every run piece inside those
//     32 elements, stored at the piece's last element;
//  2. one thread per run adds its pieces in ascending position.
__global__ void k_seg_pieces(int64_t nmax, const int64_t *n_dev, const unsigned long long *keys, const float *vals,
                             double *part) {
    const int64_t n = *n_dev;
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = wid * 32; base < n; base += nw * 32) {
        const int64_t e = base + lane;
        const bool valid = e < n;
        const unsigned long long key = valid ? keys[e] : ~0ull;
        double x = valid ? (double)vals[e] : 0.0;
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
        bool flag = lane == 0 || prev != key;  // a piece starts here
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            const bool f = __shfl_up_sync(0xffffffffu, flag, o);
            if (lane >= o && !flag) x = y + x;
            if (lane >= o) flag = flag || f;
        }
        const unsigned long long next = __shfl_down_sync(0xffffffffu, key, 1);
        const bool last = valid && (lane == 31 || e == n - 1 || next != key);
        if (last) part[e] = x;
    }
}

// Runs arrive sorted by (cluster rank, term): the first and the last run of
// each cluster record where its unique entries begin and end (no atomics).
__global__ void k_seg_runs(int64_t nmax, const int64_t *n_dev, const uint32_t *U_dev,
                           const unsigned long long *keys, const uint32_t *hpos, const double *part, int32_t *uterm,
                           double *usum, int64_t *ubeg, int64_t *uend) {
    const int64_t n = *n_dev;
    const int64_t U = n > 0 ? (int64_t)*U_dev : 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = hpos[u];
        const int64_t e = (u + 1 < U) ? (int64_t)hpos[u + 1] : n;
        double acc = 0.0;
        for (int64_t c = b >> 5; c <= ((e - 1) >> 5); ++c) {
            const int64_t end = ((c + 1) << 5) < e ? ((c + 1) << 5) : e;
            acc += part[end - 1];
        }
        const unsigned long long key = keys[b];
        const uint32_t r = (uint32_t)(key >> 32);
        uterm[u] = (int32_t)(key & 0xFFFFFFFFull);
        usum[u] = acc;
        if (u == 0 || (uint32_t)(keys[hpos[u - 1]] >> 32) != r) ubeg[r] = u;
        if (u + 1 == U || (uint32_t)(keys[e] >> 32) != r) uend[r] = u + 1;
    }
}

// ---------------- u3 / u4: new centroid rows ----------------

__global__ void k_new_sizes(int32_t k, const int64_t *flag, const int64_t *rrank, const int64_t *supoff,
                            const int64_t *supend, const int64_t *coff_old, int64_t *sz) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) sz[j] = flag[j] ? supend[rrank[j]] - supoff[rrank[j]] : coff_old[j + 1] - coff_old[j];
}

// One CTA (WR_THREADS) per cluster. Recomputed clusters: ||s|| in FP64 with
// strided per-thread sums and a fixed tree, u = s / ||s|| as FP32, and
// <s_j, mu_j^[r-1]> by binary search of each term in the previous row.
// Other clusters copy their previous row.
constexpr int WR_THREADS = 256;

__device__ __forceinline__ double block_sum_fixed(double x, double *sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int s = WR_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(WR_THREADS) k_write_rows(
    int32_t k, const int64_t *flag, const int64_t *rrank, const int64_t *supoff, const int64_t *supend,
    const int32_t *uterm, const double *usum, const int64_t *cnt, const int64_t *coff_old, const int32_t *cterm_old,
    const float *cval_old, const double *snorm_old, const int64_t *coff_new, int32_t *cterm_new, float *cval_new,
    int32_t *cclu_new, double *snorm_new, double *jA, double *jU, int64_t cap, unsigned long long *error) {
    __shared__ double sh[WR_THREADS];
    const int j = blockIdx.x;
    if (j >= k) return;
    const int64_t o = coff_new[j];
    const int64_t cb = coff_old[j], ce = coff_old[j + 1];
    if (coff_new[k] > cap) {  // more centroid entries than the buffers hold: write nothing, report
        if (j == 0 && threadIdx.x == 0) atomicOr(error, 1ull);
        return;
    }
    if (flag[j]) {
        const int64_t r = rrank[j];
        const int64_t ub = supoff[r], n = supend[r] - supoff[r];
        double ss = 0.0;
        for (int64_t q = threadIdx.x; q < n; q += WR_THREADS) ss += usum[ub + q] * usum[ub + q];
        const double nrm = sqrt(block_sum_fixed(ss, sh));
        double dot = 0.0;
        for (int64_t q = threadIdx.x; q < n; q += WR_THREADS) {
            const int32_t t = uterm[ub + q];
            const double sv = usum[ub + q];
            cterm_new[o + q] = t;
            cval_new[o + q] = (float)(sv / nrm);
            cclu_new[o + q] = j;
            int64_t lo = cb, hi = ce;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (cterm_old[mid] < t) lo = mid + 1; else hi = mid;
            }
            if (lo < ce && cterm_old[lo] == t) dot += sv * (double)cval_old[lo];
        }
        dot = block_sum_fixed(dot, sh);
        if (threadIdx.x == 0) {
            snorm_new[j] = nrm;
            jA[j] = dot;
            jU[j] = nrm;
        }
    } else {
        for (int64_t q = cb + threadIdx.x; q < ce; q += WR_THREADS) {
            cterm_new[o + (q - cb)] = cterm_old[q];
            cval_new[o + (q - cb)] = cval_old[q];
            cclu_new[o + (q - cb)] = j;
        }
        if (threadIdx.x == 0) {
            const double sn = cnt[j] > 0 ? snorm_old[j] : 0.0;
            snorm_new[j] = sn;
            jA[j] = sn;  // unchanged members: <s_j, s_j / ||s_j||> = ||s_j||
            jU[j] = sn;
        }
    }
}

// Copy the new rows back over the current ones (fixed buffers for graph replay).
__global__ void k_copy_back(int32_t k, int64_t cap, const int64_t *coff_src, const int32_t *term_src,
                            const float *val_src, const double *sn_src, int64_t *coff_dst, int32_t *term_dst,
                            float *val_dst, double *sn_dst) {
    const int64_t n = min(coff_src[k], cap);
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = g; e < n; e += st) {
        term_dst[e] = term_src[e];
        val_dst[e] = val_src[e];
    }
    for (int64_t j = g; j <= k; j += st) coff_dst[j] = coff_src[j];
    for (int64_t j = g; j < k; j += st) sn_dst[j] = sn_src[j];
}

// Per-instance objective sums (one CTA per instance), fixed order:
// per-thread strided partial sums, then a tree.
__global__ void __launch_bounds__(1024) k_sum_inst(const int32_t *inst_k, const double *a, const double *b,
                                                   double *out) {
    __shared__ double sa[1024], sb[1024];
    const int m = blockIdx.x;
    const int j0 = inst_k[m], j1 = inst_k[m + 1];
    double x = 0.0, y = 0.0;
    for (int j = j0 + threadIdx.x; j < j1; j += 1024) {
        x += a[j];
        y += b[j];
    }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = y;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * m] = sa[0];
        out[2 * m + 1] = sb[0];
    }
}

// ---------------- u2-u4, dense accumulator form ----------------
//
// Cluster sums in fixed point: every member value x contributes
// q(x) = ceil(x * 2^shift) to the cluster's accumulator entry of its term.
// The accumulator is kept across steps and updated incrementally: an object
// whose label differs from the one it was last added under (acc_lab) has its
// q values subtracted from the old cluster and added to the new one, with
// integer atomics. Integer sums do not depend on the order of the adds, so
// every entry equals the sum of q over the cluster's current members exactly,
// whatever the history; it exceeds the exact sum by less than one unit
// 2^-shift per member. The clusters touched are exactly the moving ones; their
// rows are then read in ascending term order.

__global__ void k_label_counts(int64_t N, const int32_t *labels, int64_t *cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt + labels[i]), 1ull);
}

// One warp per object whose label changed since it was last added: its q
// values move from the old cluster's row to the new one's.
__global__ void k_acc_scatter(int64_t N, const int32_t *labels, int32_t *acc_lab, const int64_t *row_ptr,
                              const int32_t *idx, const float *val, const int32_t *clu_doff, const int64_t *acc_off,
                              float fscale, int64_t *acc, int64_t *moved) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    long long mv = 0;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < N; i += nw) {
        const int32_t jn = labels[i], jo = acc_lab[i];
        if (jn == jo) continue;
        const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
        unsigned long long *rn = reinterpret_cast<unsigned long long *>(acc + acc_off[jn] - clu_doff[jn]);
        unsigned long long *ro =
            jo >= 0 ? reinterpret_cast<unsigned long long *>(acc + acc_off[jo] - clu_doff[jo]) : nullptr;
        for (int64_t h = rb + lane; h < re; h += 32) {
            const unsigned long long q = (unsigned long long)__float2ll_ru(val[h] * fscale);
            atomicAdd(rn + idx[h], q);
            if (ro) atomicAdd(ro + idx[h], 0ull - q);  // two's complement: subtracts q
        }
        mv += (re - rb) * (jo >= 0 ? 2 : 1);
        __syncwarp();
        if (lane == 0) acc_lab[i] = jn;
    }
    if (lane == 0 && mv) atomicAdd(reinterpret_cast<unsigned long long *>(moved), (unsigned long long)mv);
}

__device__ __forceinline__ long long block_sum_ll(long long x, long long *sh) {
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int s = WR_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const long long r = sh[0];
    __syncthreads();
    return r;
}

// Sum of (hi, lo) 128-bit unsigned values over the block (fixed tree, exact);
// every thread receives the total.
__device__ __forceinline__ void block_sum_u128(unsigned long long &hi, unsigned long long &lo,
                                               unsigned long long (*sh)[WR_THREADS]) {
    sh[0][threadIdx.x] = hi;
    sh[1][threadIdx.x] = lo;
    __syncthreads();
    for (int s = WR_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const unsigned long long l = sh[1][threadIdx.x] + sh[1][threadIdx.x + s];
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s] + (l < sh[1][threadIdx.x] ? 1ull : 0ull);
            sh[1][threadIdx.x] = l;
        }
        __syncthreads();
    }
    hi = sh[0][0];
    lo = sh[1][0];
    __syncthreads();
}

// Pass 1, one CTA per cluster: size of the new row, ||s_j|| (the squared
// integer sums added exactly in 128 bits, one rounding to FP64) and
// <s_j, mu_j^[r-1]> in FP64 over the previous row.
// Other clusters keep their row (sizes and objective pieces as in k_write_rows).
__global__ void __launch_bounds__(WR_THREADS) k_acc_rows1(
    int32_t k, const int64_t *flag, const int64_t *cnt, const int64_t *acc_off, const int32_t *clu_doff,
    const int64_t *acc, double inv_scale, const int64_t *coff_old, const int32_t *cterm_old, const float *cval_old,
    const double *snorm_old, int64_t *sz, double *snorm_new, double *jA, double *jU) {
    __shared__ double sh[WR_THREADS];
    __shared__ long long shl[WR_THREADS];
    __shared__ unsigned long long sh128[2][WR_THREADS];
    const int j = blockIdx.x;
    if (j >= k) return;
    const int64_t cb = coff_old[j], ce = coff_old[j + 1];
    if (!flag[j]) {
        if (threadIdx.x == 0) {
            const double sn = cnt[j] > 0 ? snorm_old[j] : 0.0;
            sz[j] = ce - cb;
            snorm_new[j] = sn;
            jA[j] = sn;  // unchanged members: <s_j, s_j / ||s_j||> = ||s_j||
            jU[j] = sn;
        }
        return;
    }
    const int64_t base = acc_off[j], L = acc_off[j + 1] - base;
    long long nz = 0;
    // ||S||^2 of the integer sums, exactly, as a 128-bit integer: the FP64 pipe
    // of this GPU retires about one operation per clock and SM, the integer
    // pipe dozens. Entries are non-negative (sums of positive member values)
    // and ||S|| = ||s_j|| 2^shift <= |C_j| 2^shift < 2^63, so the sum of
    // squares stays below 2^126.
    unsigned long long ss_hi = 0ull, ss_lo = 0ull;
    // rows start at even entries and have even lengths: 16-byte loads, two
    // of them in flight per thread
    const longlong2 *row = reinterpret_cast<const longlong2 *>(acc + base);
    const int64_t L2 = L >> 1;
    auto take = [&](long long v) {
        if (v) {
            ++nz;
            const unsigned long long u = (unsigned long long)v;
            const unsigned long long lo = u * u;
            ss_lo += lo;
            ss_hi += __umul64hi(u, u) + (ss_lo < lo ? 1ull : 0ull);
        }
    };
    for (int64_t p = threadIdx.x; p < L2; p += 2 * WR_THREADS) {
        const longlong2 a = row[p];
        const longlong2 b = p + WR_THREADS < L2 ? row[p + WR_THREADS] : make_longlong2(0, 0);
        take(a.x);
        take(a.y);
        take(b.x);
        take(b.y);
    }
    nz = block_sum_ll(nz, shl);
    block_sum_u128(ss_hi, ss_lo, sh128);
    // the exact sum to FP64 (one rounding of each half), then the power-of-two scale
    const double nrm = sqrt(((double)ss_hi * 18446744073709551616.0 + (double)ss_lo) * (inv_scale * inv_scale));
    double dot = 0.0;
    const int32_t doff = clu_doff[j];
    for (int64_t q = cb + threadIdx.x; q < ce; q += WR_THREADS)
        dot += (double)acc[base + (cterm_old[q] - doff)] * (double)cval_old[q];
    dot = block_sum_fixed(dot, sh) * inv_scale;
    if (threadIdx.x == 0) {
        sz[j] = nz;
        snorm_new[j] = nrm;
        jA[j] = dot;
        jU[j] = nrm;
    }
}

// Pass 2, one CTA per cluster: the new row in ascending term order (block
// compaction of the non-zero entries) and u = s * (2^-shift / ||s||) as FP32.
// Other clusters copy their row.
__global__ void __launch_bounds__(WR_THREADS) k_acc_rows2(
    int32_t k, const int64_t *flag, const int64_t *acc_off, const int32_t *clu_doff, const int64_t *acc,
    double inv_scale, const int64_t *coff_old, const int32_t *cterm_old, const float *cval_old,
    const double *snorm_new, const int64_t *coff_new, int32_t *cterm_new, float *cval_new, int32_t *cclu_new,
    int64_t cap, unsigned long long *error) {
    constexpr int PER = 2;  // sub-chunks of WR_THREADS entry pairs per chunk
    constexpr int NWR = WR_THREADS / 32;
    __shared__ int warp_n[PER][NWR];
    const int j = blockIdx.x;
    if (j >= k) return;
    const bool over = coff_new[k] > cap;  // more entries than the buffers hold: write nothing, report
    if (over && j == 0 && threadIdx.x == 0) atomicOr(error, 1ull);
    const int64_t o0 = coff_new[j];
    if (!flag[j]) {
        if (over) return;
        const int64_t cb = coff_old[j], ce = coff_old[j + 1];
        for (int64_t q = cb + threadIdx.x; q < ce; q += WR_THREADS) {
            cterm_new[o0 + (q - cb)] = cterm_old[q];
            cval_new[o0 + (q - cb)] = cval_old[q];
            cclu_new[o0 + (q - cb)] = j;
        }
        return;
    }
    const int64_t base = acc_off[j], L2 = (acc_off[j + 1] - base) >> 1;  // entry pairs (even rows)
    const longlong2 *row = reinterpret_cast<const longlong2 *>(acc + base);
    const int32_t doff = clu_doff[j];
    // u = S * (2^-shift / ||s_j||) in FP32 from the integer sum S (split in
    // 32-bit halves, each converted with one rounding): at most 4 roundings,
    // a relative error below 2.4e-7, with no FP64 operation per entry
    const float ff = (float)(inv_scale / snorm_new[j]);
    auto value = [&](long long v) {
        const unsigned long long u = (unsigned long long)v;
        const float fs = fmaf(__uint2float_rn((unsigned)(u >> 32)), 4294967296.0f, __uint2float_rn((unsigned)u));
        return fs * ff;
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t o = o0;
    for (int64_t c0 = 0; c0 < L2; c0 += (int64_t)WR_THREADS * PER) {
        // sub-chunk m holds pairs c0 + m*WR_THREADS + tid (coalesced 16-byte loads);
        // entries keep their order: pair by pair, and x before y inside a pair
        longlong2 v[PER];
        int ex[PER];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int64_t p = c0 + (int64_t)m * WR_THREADS + threadIdx.x;
            v[m] = p < L2 ? row[p] : make_longlong2(0, 0);
            const int n = (v[m].x != 0) + (v[m].y != 0);
            int inc = n;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
            ex[m] = inc - n;
            if (lane == 31) warp_n[m][warp] = inc;
        }
        __syncthreads();
        int total = 0;
#pragma unroll
        for (int m = 0; m < PER; ++m)
#pragma unroll
            for (int w = 0; w < NWR; ++w) total += warp_n[m][w];
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            if (v[m].x == 0 && v[m].y == 0) continue;
            int pre = 0;
            for (int mm = 0; mm < m; ++mm)
                for (int w = 0; w < NWR; ++w) pre += warp_n[mm][w];
            for (int w = 0; w < warp; ++w) pre += warp_n[m][w];
            int64_t pos = o + pre + ex[m];
            const int64_t t = 2 * (c0 + (int64_t)m * WR_THREADS + threadIdx.x);
            const long long pv[2] = {v[m].x, v[m].y};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (!pv[e]) continue;
                if (!over) {
                    cterm_new[pos] = (int32_t)(t + e) + doff;
                    cval_new[pos] = value(pv[e]);
                    cclu_new[pos] = j;
                }
                ++pos;
            }
        }
        o += total;
        __syncthreads();  // warp_n is rewritten by the next chunk
    }
}

// ---------------- u5: structured inverted file ----------------

// key = term << 1 | part (0 = front, moving; 1 = back, invariant). The
// unstructured file of IVF-CBICP keeps every posting in part 0.
__global__ void k_if_keys(const int64_t *n_dev, int64_t cap, const int32_t *cterm, const int32_t *cclu,
                          const uint8_t *lam, int structured, uint32_t *keys, uint32_t *vals, uint32_t *cnt2) {
    const int64_t n = min(*n_dev, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = ((uint32_t)cterm[e] << 1) | (uint32_t)(structured && lam[cclu[e]] ? 1 : 0);
        keys[e] = key;
        vals[e] = (uint32_t)e;
        atomicAdd(cnt2 + key, 1u);
    }
}

__global__ void k_if_lens(int32_t D, const uint32_t *cnt2, int64_t *len, int64_t *slen, int32_t *mf0) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < D) {
        const int64_t l = (int64_t)cnt2[2 * t] + (int64_t)cnt2[2 * t + 1];
        len[t] = l;
        slen[t] = (l + 3) & ~(int64_t)3;  // scan copy: lists start at multiples of 4 entries
        mf0[t] = (int32_t)cnt2[2 * t];
    }
}

// Position of entry p of a list of length L in the tiled scan layout: inside
// the list's full 128-entry blocks, entry 32m + l of a block sits at block
// position 4l + m; the ragged tail keeps canonical order.
__device__ __forceinline__ int64_t tiled_pos(int64_t p, int64_t L) {
    const int64_t fb = L & ~(int64_t)(SC_BLK - 1);
    if (p >= fb) return p;
    return (p & ~(int64_t)(SC_BLK - 1)) | ((p & 31) << 2) | ((p >> 5) & 3);
}

// Canonical arrays (if_cid: global cluster ids, if_val) in sorted order.
__global__ void k_if_fill(const int64_t *n_dev, int64_t cap, const uint32_t *order, const int32_t *cclu,
                          const float *cval, int32_t *if_cid, float *if_val) {
    const int64_t n = min(*n_dev, cap);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = order[q];
        if_cid[q] = cclu[e];
        if_val[q] = cval[e];
    }
}

// ---------------- scan order and dense head rows ----------------

// Scan position of every cluster: within its instance, the moving clusters of
// lambda^[r] (mov_list, ascending) take positions 0 .. n_mov - 1 and the
// invariant ones follow in ascending id; id_order (IVF-CBICP) keeps the ids.
__global__ void k_positions(int32_t k, int32_t n_inst, const int32_t *inst_k, const uint8_t *lam,
                            const int32_t *mov_list, const int32_t *mov_beg, int id_order, int32_t *clu_pos,
                            int32_t *pos_clu) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < k; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = (int32_t)g;
        int lo = 0, hi = n_inst - 1;  // instance: largest m with inst_k[m] <= j
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst_k[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int32_t koff = inst_k[lo], jl = j - koff;
        int32_t p = jl;
        if (!id_order) {
            const int32_t b = mov_beg[lo], e = mov_beg[lo + 1];
            int32_t a = b, z = e;  // first moving id >= j
            while (a < z) {
                const int32_t mid = (a + z) >> 1;
                if (mov_list[mid] < j) a = mid + 1; else z = mid;
            }
            p = lam[j] == 0 ? a - b : (e - b) + (jl - (a - b));
        }
        clu_pos[j] = p;
        pos_clu[koff + p] = jl;
    }
}

constexpr int DENSE_BINS = 64;      // list length / k in steps of 1/64
constexpr int DENSE_MIN_LEN = 32;   // shorter lists stay sparse whatever k

// instance of term t, its k, and the 1/64 bin of its list length
__device__ __forceinline__ void term_bin(int32_t t, int32_t n_inst, const int32_t *inst_d, const int32_t *inst_k,
                                         int64_t L, int32_t *kin, int *bin) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst_d[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int32_t km = inst_k[lo + 1] - inst_k[lo];
    *kin = km;
    const int64_t q = (L * DENSE_BINS) / (km > 0 ? km : 1);
    *bin = (int)(q < DENSE_BINS ? q : DENSE_BINS);
}

// Histogram of the dense-row entries each length bin would take (lists of at
// least min_len postings).
__global__ void k_dense_hist(int32_t D, int32_t n_inst, const int32_t *inst_d, const int32_t *inst_k,
                             const int64_t *len, int64_t min_len, unsigned long long *hist) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < D; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = len[g];
        if (L < min_len) continue;
        int32_t km;
        int bin;
        term_bin((int32_t)g, n_inst, inst_d, inst_k, L, &km, &bin);
        atomicAdd(hist + bin, (unsigned long long)((km + 7) & ~7));
    }
}

// Smallest bin >= bmin whose rows (with every longer bin's) fit in cap
// entries; DENSE_BINS + 1 = no dense rows.
__global__ void k_dense_threshold(const unsigned long long *hist, int bmin, unsigned long long cap, int32_t *thr) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long acc = 0;
    int b = DENSE_BINS + 1;
    for (int q = DENSE_BINS; q >= bmin; --q) {
        acc += hist[q];
        if (acc > cap) break;
        b = q;
    }
    *thr = b;
}

// Dense-row width (in 8-entry units) of every term; the sparse scan copy
// gives dense terms no room.
__global__ void k_dense_width(int32_t D, int32_t n_inst, const int32_t *inst_d, const int32_t *inst_k,
                              const int64_t *len, int64_t min_len, const int32_t *thr, int64_t *w8, int64_t *slen) {
    const int b = *thr;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < D; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = len[g];
        int64_t w = 0;
        if (L >= min_len) {
            int32_t km;
            int bin;
            term_bin((int32_t)g, n_inst, inst_d, inst_k, L, &km, &bin);
            if (bin >= b) w = (km + 7) >> 3;
        }
        w8[g] = w;
        if (w) slen[g] = 0;
    }
}

__global__ void k_dense_rows(int32_t D, const int64_t *w8, const int64_t *base8, int32_t *dense_row,
                             DevCounters *ctr) {
    long long n = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < D; g += (int64_t)gridDim.x * blockDim.x) {
        const bool d = w8[g] > 0;
        dense_row[g] = d ? (int32_t)base8[g] : -1;
        n += d;
    }
    if (n) atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->dense_terms), (unsigned long long)n);
}

// zero the entries in use (16 bytes at a time; rows are multiples of 8 entries)
__global__ void k_dense_zero(const int64_t *used8, int esize, uint4 *dense) {
    const int64_t n16 = used8[0] * 8 * esize / 16;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n16; q += (int64_t)gridDim.x * blockDim.x)
        dense[q] = make_uint4(0u, 0u, 0u, 0u);
}

// 16-bit stored value of a posting: BF16 (nearest, ties to even), or FP16 of
// u * 2^14 kept strictly positive
__device__ __forceinline__ uint16_t encode_lp(float u, int prec) {
    if (prec == SIVF_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(u));
    unsigned short h = __half_as_ushort(__float2half_rn(u * FP16_SCALE));
    if (h == 0 && u > 0.0f) h = 1;
    return h;
}

// per (term, part) posting counts of the current centroids
__global__ void k_if_count(const int64_t *n_dev, int64_t cap, const int32_t *cterm, const int32_t *cclu,
                           const uint8_t *lam, int structured, uint32_t *cnt2) {
    const int64_t n = min(*n_dev, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt2 + (((uint32_t)cterm[e] << 1) | (uint32_t)(structured && lam[cclu[e]] ? 1 : 0)), 1u);
}

// The scan structures read by the assignment, straight from the cluster-major
// centroid entries (one pass, no sort): an entry of a term with a dense row
// goes to the row at its cluster's scan position; any other entry takes the
// next free slot of its term's front (moving cluster) or back (invariant
// cluster) in the scan copy, stored at the slot's tiled position with the
// cluster's scan position as its id. The order of the postings inside a
// segment follows the atomic cursor; no score depends on it (each posting is
// one integer add).
__global__ void k_scan_fill(const int64_t *n_dev, int64_t cap, const int32_t *cterm, const int32_t *cclu,
                            const float *cval, const uint8_t *lam, int structured, const int32_t *clu_pos,
                            const int32_t *dense_row, const int64_t *if_off, const int32_t *if_mf0,
                            const int64_t *sc_off, uint32_t *cursor, int prec, void *dense, uint16_t *sc_id16,
                            int32_t *sc_id32, float *sc_val, uint32_t *sc_pack, uint16_t *sc_lp) {
    const int64_t n = min(*n_dev, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = cterm[e], j = cclu[e];
        const float u = cval[e];
        const uint32_t p = (uint32_t)clu_pos[j];
        const int32_t r = dense_row[t];
        if (r >= 0) {
            const int64_t d = (int64_t)r * 8 + p;
            if (prec == SIVF_FP32) static_cast<float *>(dense)[d] = u;
            else static_cast<uint16_t *>(dense)[d] = encode_lp(u, prec);
            continue;
        }
        const uint32_t part = (structured && lam[j]) ? 1u : 0u;
        const int64_t slot = (int64_t)atomicAdd(cursor + (((uint32_t)t << 1) | part), 1u) + (part ? if_mf0[t] : 0);
        const int64_t pos = sc_off[t] + tiled_pos(slot, if_off[t + 1] - if_off[t]);
        if (sc_id16) sc_id16[pos] = (uint16_t)p;
        if (sc_id32) sc_id32[pos] = (int32_t)p;
        if (prec == SIVF_FP32) {
            sc_val[pos] = u;
            continue;
        }
        const uint16_t lp = encode_lp(u, prec);
        if (sc_pack) sc_pack[pos] = (p << 16) | (uint32_t)lp;
        else sc_lp[pos] = lp;
    }
}

}  // namespace

cudaError_t validate_csr(sivf_ctx *c, int *bad_host) {
    int *bad = c->ws.take<int>(1);
    if (!bad) return cudaErrorMemoryAllocation;
    SIVF_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    k_validate<<<blocks_gs(c->N * 32), TPB, 0, c->stream>>>(c->N, c->D, c->nnz, c->row_ptr, c->idx, c->val,
                                                               c->sumv, bad);
    note_launch();
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(cudaMemcpyAsync(bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SIVF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->ws.reset();
    return cudaSuccess;
}

cudaError_t init_centroids(sivf_ctx *c, const int32_t *init_ids_dev) {
    const int cur = c->cur;
    int64_t *sz = c->ws.take<int64_t>((size_t)c->k + 1);
    int64_t *total = c->ws.take<int64_t>(1);
    if (!sz || !total) return cudaErrorMemoryAllocation;
    k_seed_sizes<<<blocks_for(c->k), TPB, 0, c->stream>>>(c->k, init_ids_dev, c->row_ptr, sz);
    note_launch();
    SIVF_CUDA_TRY(scan_exclusive_i64(sz, c->coff[cur], c->k, total, c->ws, c->stream));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->coff[cur] + c->k, total, sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream));
    int64_t tot = 0;
    SIVF_CUDA_TRY(cudaMemcpyAsync(&tot, total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    SIVF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (tot > c->cap_c) return cudaErrorMemoryAllocation;
    c->c_nnz = tot;
    c->if_nnz = tot;
    k_seed_rows<<<blocks_for((int64_t)c->k * 32), TPB, 0, c->stream>>>(c->k, init_ids_dev, c->row_ptr, c->idx,
                                                                       c->val, c->coff[cur], c->cterm[cur],
                                                                       c->cval[cur], c->cclu);
    note_launch();
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(cudaMemsetAsync(c->snorm, 0, sizeof(double) * c->k, c->stream));
    c->ws.reset();
    return cudaSuccess;
}

cudaError_t set_labels_dev(sivf_ctx *c, const int32_t *src) {
    // src must not live in the workspace region taken below
    int *bad = c->ws.take<int>(1);
    if (!bad) return cudaErrorMemoryAllocation;
    SIVF_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    k_check_labels<<<blocks_gs(c->N), TPB, 0, c->stream>>>(c->N, c->k, src, bad);
    note_launch();
    int bad_h = 0;
    SIVF_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SIVF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (bad_h) return cudaErrorInvalidValue;
    SIVF_CUDA_TRY(cudaMemsetAsync(c->moving, 0, c->k, c->stream));
    k_set_labels<<<blocks_gs(c->N), TPB, 0, c->stream>>>(c->N, src, c->labels, c->labels_prev, c->own, c->moving);
    note_launch();
    SIVF_CUDA_TRY(cudaGetLastError());
    if (c->iter == 0) c->iter = 1;  // first membership: every cluster is moving
    SIVF_CUDA_TRY(launch_finalize_assign(c));
    return cudaSuccess;
}

// Restart from new seeds: no labels, no own scores, every cluster moving,
// mu^[0] = seed rows, first inverted file.
cudaError_t reseed_dev(sivf_ctx *c, const int32_t *init_ids_dev) {
    const int64_t N = c->N;
    const int32_t k = c->k;
    SIVF_CUDA_TRY(cudaMemsetAsync(c->labels, 0xFF, sizeof(int32_t) * N, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->labels_prev, 0xFF, sizeof(int32_t) * N, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->own, 0xFF, sizeof(uint32_t) * N, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->lam, 0, k, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->lam_prev, 0, k, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->moving, 1, k, c->stream));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream));
    if (c->dense) {  // no member has been added yet
        SIVF_CUDA_TRY(cudaMemsetAsync(c->acc, 0, sizeof(int64_t) * (size_t)c->acc_total, c->stream));
        SIVF_CUDA_TRY(cudaMemsetAsync(c->acc_lab, 0xFF, sizeof(int32_t) * N, c->stream));
    }
    c->iter = 1;  // finalize below marks every cluster moving
    SIVF_CUDA_TRY(launch_finalize_assign(c));
    c->iter = 0;
    SIVF_CUDA_TRY(init_centroids(c, init_ids_dev));
    SIVF_CUDA_TRY(build_inverted_file(c));
    c->needs_update = false;
    return cudaSuccess;
}

// Scan structures of the structured inverted file of the current centroids
// (count in coff[k], on the device) with the current lambda: list offsets and
// front lengths, the scan order, the dense head rows and the sparse scan copy.
// No host synchronisation. The canonical file (ascending ids in each part,
// for the getters) is built on demand by build_canonical_if.
cudaError_t build_inverted_file(sivf_ctx *c) {
    const int64_t cap = c->cap_c;
    const int cur = c->cur;
    const int64_t *n_dev = c->coff[cur] + c->k;
    const int32_t D = c->D;
    Workspace &ws = c->ws;
    size_t mark = ws.used;
    uint32_t *cnt2 = ws.take<uint32_t>((size_t)2 * D);
    int64_t *len = ws.take<int64_t>((size_t)D + 1);
    int64_t *slen = ws.take<int64_t>((size_t)D + 1);
    int64_t *w8 = ws.take<int64_t>((size_t)D + 1);
    int64_t *base8 = ws.take<int64_t>((size_t)D + 1);
    unsigned long long *hist = ws.take<unsigned long long>(DENSE_BINS + 1);
    int64_t *total = ws.take<int64_t>(3);
    if (!cnt2 || !len || !slen || !w8 || !base8 || !hist || !total) return cudaErrorMemoryAllocation;
    cudaStream_t s = c->stream;
    const bool cb = c->cfg.icp == 2;
    c->canon_stale = true;
    SIVF_CUDA_TRY(cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * 2 * D, s));
    k_if_count<<<blocks_gs(cap), TPB, 0, s>>>(n_dev, cap, c->cterm[cur], c->cclu, c->lam, cb ? 0 : 1, cnt2);
    k_if_lens<<<blocks_for(D), TPB, 0, s>>>(D, cnt2, len, slen, c->if_mf0);
    // scan order of lambda^[r] (mov_list and mov_beg were computed from it)
    k_positions<<<blocks_gs(c->k), TPB, 0, s>>>(c->k, c->n_inst, c->inst_k, c->lam, c->mov_list, c->mov_beg,
                                                 cb ? 1 : 0, c->clu_pos, c->pos_clu);
    note_launch(3);
    // dense head rows: the longest lists (relative to their instance's k) that
    // fit in the row capacity, from dense_frac of k up; with dense_all every
    // list (the dense-mean variant: all of the centroids as dense rows)
    SIVF_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (DENSE_BINS + 1), s));
    const bool all = c->cfg.dense_all != 0;
    const int bmin = all ? 0 : std::max(1, (int)ceilf(c->dense_frac * DENSE_BINS));
    const int64_t min_len = all ? 1 : DENSE_MIN_LEN;
    const bool dense = c->cap_dense > 0 && !cb && bmin <= DENSE_BINS;
    if (dense) {
        k_dense_hist<<<blocks_gs(D), TPB, 0, s>>>(D, c->n_inst, c->inst_d, c->inst_k, len, min_len, hist);
        k_dense_threshold<<<1, 32, 0, s>>>(hist, bmin, (unsigned long long)c->cap_dense, c->dense_thr);
        note_launch(2);
    } else {  // no bin qualifies: the threshold becomes DENSE_BINS + 1 (no rows)
        k_dense_threshold<<<1, 32, 0, s>>>(hist, DENSE_BINS + 1, 0ull, c->dense_thr);
        note_launch();
    }
    k_dense_width<<<blocks_gs(D), TPB, 0, s>>>(D, c->n_inst, c->inst_d, c->inst_k, len, min_len, c->dense_thr, w8,
                                                slen);
    note_launch();
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(scan_exclusive_i64(len, c->if_off, D, total, ws, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->if_off + D, total, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(scan_exclusive_i64(slen, c->sc_off, D, total + 1, ws, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->sc_off + D, total + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(scan_exclusive_i64(w8, base8, D, total + 2, ws, s));
    SIVF_CUDA_TRY(cudaMemsetAsync(&c->ctr->dense_terms, 0, sizeof(long long), s));
    k_dense_rows<<<blocks_gs(D), TPB, 0, s>>>(D, w8, base8, c->dense_row, c->ctr);
    note_launch();
    if (dense) {
        const int esize = c->cfg.prec == SIVF_FP32 ? 4 : 2;
        k_dense_zero<<<blocks_gs(c->cap_dense * esize / 16), TPB, 0, s>>>(total + 2, esize,
                                                                            static_cast<uint4 *>(c->dense_val));
        note_launch();
    }
    // the counts are consumed: the same array now hands out the slots
    SIVF_CUDA_TRY(cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * 2 * D, s));
    k_scan_fill<<<blocks_gs(cap), TPB, 0, s>>>(n_dev, cap, c->cterm[cur], c->cclu, c->cval[cur], c->lam, cb ? 0 : 1,
                                                c->clu_pos, c->dense_row, c->if_off, c->if_mf0, c->sc_off, cnt2,
                                                (int)c->cfg.prec, c->dense_val, c->sc_id16, c->sc_id32, c->sc_val,
                                                c->sc_pack, c->sc_lp);
    note_launch();
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->dense_used, total + 2, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->sparse_entries, total + 1, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaGetLastError());
    ws.used = mark;
    return cudaSuccess;
}

// The canonical structured inverted file of the current centroids and lambda
// (Algorithm 5: for every term, the moving centroids first and the invariant
// ones after, ascending ids in each part) in if_cid / if_val, with the offsets
// and front lengths of the last build: a stable radix sort of the centroid
// entries by (term, part). Used by the getters only; synchronises the stream.
cudaError_t build_canonical_if(sivf_ctx *c) {
    if (!c->canon_stale) return cudaSuccess;
    const int64_t cap = c->cap_c;
    const int cur = c->cur;
    const int64_t *n_dev = c->coff[cur] + c->k;
    Workspace &ws = c->ws;
    ws.reset();
    uint32_t *cnt2 = ws.take<uint32_t>((size_t)2 * c->D);
    uint32_t *k0 = ws.take<uint32_t>((size_t)cap + 1), *v0 = ws.take<uint32_t>((size_t)cap + 1);
    uint32_t *k1 = ws.take<uint32_t>((size_t)cap + 1), *v1 = ws.take<uint32_t>((size_t)cap + 1);
    if (!cnt2 || !k0 || !v0 || !k1 || !v1) return cudaErrorMemoryAllocation;
    cudaStream_t s = c->stream;
    SIVF_CUDA_TRY(cudaMemsetAsync(cnt2, 0, sizeof(uint32_t) * 2 * c->D, s));
    k_if_keys<<<blocks_gs(cap), TPB, 0, s>>>(n_dev, cap, c->cterm[cur], c->cclu, c->lam, c->cfg.icp == 2 ? 0 : 1, k0,
                                              v0, cnt2);
    note_launch();
    bool alt = false;
    SIVF_CUDA_TRY(radix_sort_pairs_dev(k0, v0, k1, v1, cap, n_dev, c->bits_t + 1, &alt, ws, s));
    k_if_fill<<<blocks_gs(cap), TPB, 0, s>>>(n_dev, cap, alt ? v1 : v0, c->cclu, c->cval[cur], c->if_cid,
                                              c->if_val);
    note_launch();
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(cudaStreamSynchronize(s));
    ws.reset();
    c->canon_stale = false;
    return cudaSuccess;
}

// Update step with the dense accumulator (u1: member counts only; u2-u4 as
// above; u5 as in the sort form).
cudaError_t run_update_dense(sivf_ctx *c) {
    cudaStream_t s = c->stream;
    Workspace &ws = c->ws;
    ws.reset();
    const int64_t N = c->N;
    const int32_t k = c->k;
    const int cur = c->cur, nw = 1 - c->cur;
    int64_t *cnt = ws.take<int64_t>(k), *flag = ws.take<int64_t>(k);
    int64_t *sz = ws.take<int64_t>((size_t)k + 1), *newn_d = ws.take<int64_t>(1), *moved_d = ws.take<int64_t>(1);
    double *jAd = ws.take<double>(k), *jUd = ws.take<double>(k);
    if (!cnt || !flag || !sz || !newn_d || !moved_d || !jAd || !jUd) return cudaErrorMemoryAllocation;
    SIVF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * k, s));
    SIVF_CUDA_TRY(cudaMemsetAsync(moved_d, 0, sizeof(int64_t), s));
    k_label_counts<<<blocks_gs(N), TPB, 0, s>>>(N, c->labels, cnt);
    k_recompute_flags<<<blocks_for(k), TPB, 0, s>>>(k, c->lam, cnt, flag);
    const float fscale = ldexpf(1.0f, c->acc_shift);
    const double inv_scale = ldexp(1.0, -c->acc_shift);
    k_acc_scatter<<<blocks_gs(N * 32), TPB, 0, s>>>(N, c->labels, c->acc_lab, c->row_ptr, c->idx, c->val,
                                                     c->clu_doff, c->acc_off, fscale, c->acc, moved_d);
    k_acc_rows1<<<(unsigned)k, WR_THREADS, 0, s>>>(k, flag, cnt, c->acc_off, c->clu_doff, c->acc, inv_scale,
                                                   c->coff[cur], c->cterm[cur], c->cval[cur], c->snorm, sz,
                                                   c->snorm_new, jAd, jUd);
    note_launch(4);
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(scan_exclusive_i64(sz, c->coff[nw], k, newn_d, ws, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->coff[nw] + k, newn_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_acc_rows2<<<(unsigned)k, WR_THREADS, 0, s>>>(k, flag, c->acc_off, c->clu_doff, c->acc, inv_scale, c->coff[cur],
                                                   c->cterm[cur], c->cval[cur], c->snorm_new, c->coff[nw],
                                                   c->cterm[nw], c->cval[nw], c->cclu, c->cap_c, &c->ctr->error);
    k_sum_inst<<<(unsigned)c->n_inst, 1024, 0, s>>>(c->inst_k, jAd, jUd, c->obj_dev);
    k_copy_back<<<blocks_gs(c->cap_c), TPB, 0, s>>>(k, c->cap_c, c->coff[nw], c->cterm[nw], c->cval[nw],
                                                     c->snorm_new, c->coff[cur], c->cterm[cur], c->cval[cur],
                                                     c->snorm);
    note_launch(3);
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->moved, moved_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->c_nnz, newn_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ws.reset();
    SIVF_CUDA_TRY(build_inverted_file(c));
    ws.reset();
    return cudaSuccess;
}

// One update step (Algorithm 5). Every size that depends on the data stays on
// the device, so the whole step can be captured in a CUDA graph.
cudaError_t run_update(sivf_ctx *c) {
    cudaStream_t s = c->stream;
    Workspace &ws = c->ws;
    ws.reset();
    const int64_t N = c->N;
    const int32_t k = c->k;
    const int64_t Tmax = c->nnz > 0 ? c->nnz : 1;
    const int cur = c->cur, nw = 1 - c->cur;

    if (c->dense) return run_update_dense(c);

    // u1: members grouped by cluster, ascending object id
    uint32_t *lk0 = ws.take<uint32_t>(N), *lv0 = ws.take<uint32_t>(N);
    uint32_t *lk1 = ws.take<uint32_t>(N), *lv1 = ws.take<uint32_t>(N);
    int64_t *cnt = ws.take<int64_t>(k), *flag = ws.take<int64_t>(k), *rrank = ws.take<int64_t>(k);
    int64_t *nrec_d = ws.take<int64_t>(1), *T_d = ws.take<int64_t>(1), *newn_d = ws.take<int64_t>(1);
    uint32_t *U_d = ws.take<uint32_t>(1);
    int64_t *sz = ws.take<int64_t>((size_t)k + 1);
    double *jAd = ws.take<double>(k), *jUd = ws.take<double>(k);
    int64_t *tc = ws.take<int64_t>(N), *toff = ws.take<int64_t>(N);
    int64_t *ubeg = ws.take<int64_t>((size_t)k + 1), *uend = ws.take<int64_t>((size_t)k + 1);
    if (!lk0 || !lv0 || !lk1 || !lv1 || !cnt || !flag || !rrank || !nrec_d || !T_d || !newn_d || !U_d || !sz ||
        !jAd || !jUd || !tc || !toff || !ubeg || !uend)
        return cudaErrorMemoryAllocation;
    SIVF_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * k, s));
    k_label_keys<<<blocks_gs(N), TPB, 0, s>>>(N, c->labels, lk0, lv0, cnt);
    note_launch();
    bool alt = false;
    SIVF_CUDA_TRY(radix_sort_pairs(lk0, lv0, lk1, lv1, N, bits_for((uint64_t)(k - 1)), &alt, ws, s));
    const uint32_t *perm = alt ? lv1 : lv0;
    k_recompute_flags<<<blocks_for(k), TPB, 0, s>>>(k, c->lam, cnt, flag);
    note_launch();
    SIVF_CUDA_TRY(scan_exclusive_i64(flag, rrank, k, nrec_d, ws, s));

    // u2: tuples of the recomputed clusters' members, in member order; a
    // stable sort by term then a stable sort by cluster rank leave them in
    // (rank, term, object) order; equal (rank, term) runs are summed in FP64
    k_member_tuples<<<blocks_gs(N), TPB, 0, s>>>(N, perm, c->labels, flag, c->row_ptr, tc);
    note_launch();
    SIVF_CUDA_TRY(scan_exclusive_i64(tc, toff, N, T_d, ws, s));
    uint32_t *sa_k = ws.take<uint32_t>(Tmax), *sa_v = ws.take<uint32_t>(Tmax);
    uint32_t *sb_k = ws.take<uint32_t>(Tmax), *sb_v = ws.take<uint32_t>(Tmax);
    uint32_t *tterm = ws.take<uint32_t>(Tmax), *trank = ws.take<uint32_t>(Tmax);
    float *tval = ws.take<float>(Tmax), *sval = ws.take<float>(Tmax);
    unsigned long long *key64 = ws.take<unsigned long long>(Tmax);
    double *part = ws.take<double>(Tmax);
    int32_t *uterm = ws.take<int32_t>(Tmax);
    double *usum = ws.take<double>(Tmax);
    if (!sa_k || !sa_v || !sb_k || !sb_v || !tterm || !trank || !tval || !sval || !key64 || !part || !uterm || !usum)
        return cudaErrorMemoryAllocation;
    const int bits_r = bits_for((uint64_t)(k - 1));
    if (bits_r + c->bits_tl <= 32) {
        // one sort on (rank, local term) carrying the value bits
        int32_t *rank2clu = reinterpret_cast<int32_t *>(tterm);
        k_rank2clu<<<blocks_for(k), TPB, 0, s>>>(k, flag, rrank, rank2clu);
        k_expand_packed<<<blocks_gs(N * 32), TPB, 0, s>>>(N, perm, c->labels, rrank, tc, toff, c->row_ptr, c->idx,
                                                            c->val, c->clu_doff, c->bits_tl, sa_k, sa_v);
        note_launch(2);
        bool a1 = false;
        SIVF_CUDA_TRY(radix_sort_pairs_dev(sa_k, sa_v, sb_k, sb_v, Tmax, T_d, bits_r + c->bits_tl, &a1, ws, s));
        k_unpack<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, a1 ? sb_k : sa_k, a1 ? sb_v : sa_v, c->bits_tl, rank2clu,
                                                  c->clu_doff, key64, sval);
        note_launch();
    } else {
        // two stable sorts: by global term, then by rank
        k_expand<<<blocks_gs(N * 32), TPB, 0, s>>>(N, perm, c->labels, rrank, tc, toff, c->row_ptr, c->idx, c->val,
                                                     sa_k, sa_v, tterm, tval, trank);
        note_launch();
        bool a1 = false;
        SIVF_CUDA_TRY(radix_sort_pairs_dev(sa_k, sa_v, sb_k, sb_v, Tmax, T_d, c->bits_t, &a1, ws, s));
        uint32_t *x_v = a1 ? sb_v : sa_v;                           // tuple ids sorted by term
        uint32_t *y_k = a1 ? sa_k : sb_k, *y_v = a1 ? sa_v : sb_v;  // the free pair
        uint32_t *z_k = a1 ? sb_k : sa_k;                           // its ping-pong partner
        k_rank_keys<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, x_v, trank, y_k, y_v);
        note_launch();
        bool a2 = false;
        SIVF_CUDA_TRY(radix_sort_pairs_dev(y_k, y_v, z_k, x_v, Tmax, T_d, bits_r, &a2, ws, s));
        const uint32_t *r_k = a2 ? z_k : y_k, *r_v = a2 ? x_v : y_v;
        k_compose<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, r_k, r_v, tterm, tval, key64, sval);
        note_launch();
    }
    // the sort buffers are free again: run flags, run index, run position
    uint32_t *head = sa_k, *uidx = sa_v, *hpos = sb_k;
    k_heads<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, key64, head);
    note_launch();
    SIVF_CUDA_TRY(scan_exclusive_u32_dev(head, uidx, Tmax, T_d, U_d, ws, s));
    SIVF_CUDA_TRY(cudaMemsetAsync(ubeg, 0, sizeof(int64_t) * (k + 1), s));  // empty-row clusters: no entries
    SIVF_CUDA_TRY(cudaMemsetAsync(uend, 0, sizeof(int64_t) * (k + 1), s));
    k_head_pos<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, head, uidx, hpos);
    k_seg_pieces<<<blocks_gs((Tmax + 31) / 32 * 32), TPB, 0, s>>>(Tmax, T_d, key64, sval, part);
    k_seg_runs<<<blocks_gs(Tmax), TPB, 0, s>>>(Tmax, T_d, U_d, key64, hpos, part, uterm, usum, ubeg, uend);
    note_launch(3);
    SIVF_CUDA_TRY(cudaGetLastError());

    // u3/u4: new cluster-major rows (into the second buffer), copied back
    k_new_sizes<<<blocks_for(k), TPB, 0, s>>>(k, flag, rrank, ubeg, uend, c->coff[cur], sz);
    note_launch();
    SIVF_CUDA_TRY(scan_exclusive_i64(sz, c->coff[nw], k, newn_d, ws, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->coff[nw] + k, newn_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_write_rows<<<(unsigned)k, WR_THREADS, 0, s>>>(
        k, flag, rrank, ubeg, uend, uterm, usum, cnt, c->coff[cur], c->cterm[cur], c->cval[cur], c->snorm,
        c->coff[nw], c->cterm[nw], c->cval[nw], c->cclu, c->snorm_new, jAd, jUd, c->cap_c, &c->ctr->error);
    k_sum_inst<<<(unsigned)c->n_inst, 1024, 0, s>>>(c->inst_k, jAd, jUd, c->obj_dev);
    k_copy_back<<<blocks_gs(c->cap_c), TPB, 0, s>>>(k, c->cap_c, c->coff[nw], c->cterm[nw], c->cval[nw],
                                                     c->snorm_new, c->coff[cur], c->cterm[cur], c->cval[cur],
                                                     c->snorm);
    note_launch(3);
    SIVF_CUDA_TRY(cudaGetLastError());
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->moved, T_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(&c->ctr->c_nnz, newn_d, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ws.reset();

    // u5: rebuild the structured inverted file with lambda^[r]
    SIVF_CUDA_TRY(build_inverted_file(c));
    ws.reset();
    return cudaSuccess;
}
}  // namespace sivf
