// C ABI of the SIVF library (declared in include/sivf.h): argument checks,
// device memory ownership, step orchestration and error latching.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "sivf_internal.cuh"

using namespace sivf;

namespace {

const char *kNoCtx = "sivf: null context";

sivf_status fail(sivf_ctx *c, sivf_status st, const char *msg) {
    if (c) c->err = msg;
    return st;
}

sivf_status cuda_fail(sivf_ctx *c, cudaError_t e, const char *where) {
    if (c) {
        c->latched = true;
        c->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? SIVF_ERR_OOM : SIVF_ERR_CUDA;
}

#define API_CUDA(c, expr, where)                               \
    do {                                                       \
        cudaError_t e__ = (expr);                              \
        if (e__ != cudaSuccess) return cuda_fail(c, e__, where); \
    } while (0)

template <typename T>
cudaError_t dmalloc(sivf_ctx *c, T **p, size_t n) {
    size_t bytes = (n ? n : 1) * sizeof(T);
    if (c->cfg.mem_cap_bytes > 0 && c->owned_bytes + bytes > (size_t)c->cfg.mem_cap_bytes)
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e == cudaSuccess) c->owned_bytes += bytes;
    return e;
}

void free_all(sivf_ctx *c) {
    void *ptrs[] = {c->labels, c->labels_prev, c->own, c->sumv, c->lam, c->lam_prev, c->moving, c->mov_list,
                    c->n_mov_dev, c->snorm, c->snorm_new, c->coff[0], c->coff[1], c->cterm[0], c->cterm[1],
                    c->cval[0], c->cval[1], c->cclu, c->if_off, c->if_mf0, c->if_cid, c->if_cid16, c->if_pack, c->if_val, c->if_lp,
                    c->ctr, c->obj_dev, c->ws.base};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->ctr_host) cudaFreeHost(c->ctr_host);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
}

sivf_status check_usable(sivf_ctx *c) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    return SIVF_OK;
}

void pick_assign_config(sivf_ctx *c) {
    int T = c->cfg.threads;
    if (T != 64 && T != 128 && T != 256 && T != 512) T = 0;
    if (T == 0) T = c->k <= 256 ? 64 : (c->k <= 4096 ? 128 : 512);
    c->assign_threads = T;
    c->assign_ctas_per_sm = c->cfg.ctas_per_sm > 0 ? c->cfg.ctas_per_sm : 0;
}

}  // namespace

extern "C" {

sivf_status sivf_init(sivf_ctx **out, const sivf_config *cfg, int64_t N, int32_t D, int32_t k,
                      const int64_t *row_ptr, const int32_t *idx, const float *val, const int32_t *init_ids,
                      void *stream) {
    if (!out) return SIVF_ERR_INVALID_ARG;
    *out = nullptr;
    if (N < 1 || N > 0x7FFFFFFFll || D < 1 || D > (1 << 30) || k < 1 || (int64_t)k > N || !row_ptr || !idx || !val ||
        !init_ids)
        return SIVF_ERR_INVALID_ARG;
    if (cfg && (cfg->prec < SIVF_FP32 || cfg->prec > SIVF_FP16)) return SIVF_ERR_INVALID_ARG;
    {
        std::vector<char> seen((size_t)N, 0);
        for (int32_t j = 0; j < k; ++j) {
            int32_t d = init_ids[j];
            if (d < 0 || (int64_t)d >= N || seen[(size_t)d]) return SIVF_ERR_INVALID_ARG;
            seen[(size_t)d] = 1;
        }
    }
    sivf_ctx *c = new (std::nothrow) sivf_ctx();
    if (!c) return SIVF_ERR_OOM;
    if (cfg) {
        c->cfg = *cfg;
    } else {
        std::memset(&c->cfg, 0, sizeof(c->cfg));
        c->cfg.prec = SIVF_FP32;
        c->cfg.icp = 1;
    }
    c->N = N;
    c->D = D;
    c->k = k;
    c->stream = static_cast<cudaStream_t>(stream);
    c->row_ptr = row_ptr;
    c->idx = idx;
    c->val = val;
    c->bits_t = bits_for((uint64_t)(D - 1));
    if (c->bits_t < 1) c->bits_t = 1;
    if (c->bits_t > 30) {
        delete c;
        return SIVF_ERR_INVALID_ARG;
    }
    pick_assign_config(c);

    cudaError_t e;
#define INIT_CUDA(expr, where)                      \
    do {                                            \
        e = (expr);                                 \
        if (e != cudaSuccess) {                     \
            sivf_status st__ = cuda_fail(c, e, where); \
            free_all(c);                            \
            delete c;                               \
            return st__;                            \
        }                                           \
    } while (0)
    INIT_CUDA(cudaGetDevice(&c->device), "cudaGetDevice");
    INIT_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
    // nnz from row_ptr[N]
    int64_t nnz = 0, first = 0;
    INIT_CUDA(cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream), "read nnz");
    INIT_CUDA(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream), "read row_ptr");
    INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
    if (first != 0 || nnz < 0 || nnz >= 0x7FFFFFFFll) {
        delete c;
        return SIVF_ERR_BAD_CSR;
    }
    c->nnz = nnz;
    c->cap_c = 2 * nnz + 1024;
    const int64_t capc = c->cap_c;
    INIT_CUDA(dmalloc(c, &c->labels, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->labels_prev, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->own, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->sumv, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->lam, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->lam_prev, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->moving, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->mov_list, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->n_mov_dev, 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->snorm, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->snorm_new, k), "alloc");
    for (int b = 0; b < 2; ++b) {
        INIT_CUDA(dmalloc(c, &c->coff[b], (size_t)k + 1), "alloc");
        INIT_CUDA(dmalloc(c, &c->cterm[b], capc), "alloc");
        INIT_CUDA(dmalloc(c, &c->cval[b], capc), "alloc");
    }
    INIT_CUDA(dmalloc(c, &c->cclu, capc), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_off, (size_t)D + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_mf0, D), "alloc");
    // the scan reads aligned groups of 4 postings: up to 3 entries past the
    // last list, so the posting arrays carry a small tail pad
    INIT_CUDA(dmalloc(c, &c->if_cid, capc + IF_PAD), "alloc");
    if (k <= 65536) INIT_CUDA(dmalloc(c, &c->if_cid16, capc + IF_PAD), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_val, capc + IF_PAD), "alloc");
    if (c->cfg.prec != SIVF_FP32) INIT_CUDA(dmalloc(c, &c->if_lp, capc + IF_PAD), "alloc");
    if (c->cfg.prec != SIVF_FP32 && k <= 65536) INIT_CUDA(dmalloc(c, &c->if_pack, capc + IF_PAD), "alloc");
    INIT_CUDA(dmalloc(c, &c->ctr, 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->obj_dev, 2), "alloc");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->ctr_host), sizeof(DevCounters)), "alloc host");
    {
        // workspace: max of the update's two phases, plus primitive scratch
        const size_t n8 = (size_t)N * 8, k8 = (size_t)k * 8;
        // u1: 4 label key/value arrays (4 B x N), tuple counts/offsets (8 B x N),
        // per-cluster arrays; u2: unique (term, sum) pairs (12 B x nnz) and
        // per tuple 4 sort arrays, head/index/position and a piece sum (36 B)
        size_t phase1 = 4 * (size_t)N * 4 + 2 * n8 + 10 * k8 + 12 * ((size_t)nnz + 1) + 36 * ((size_t)nnz + 1) +
                        32 * 4096;
        size_t phase2 = 16 * ((size_t)capc + 1) + 24 * ((size_t)D + 1) + 16 * 4096;
        size_t ws = phase1 > phase2 ? phase1 : phase2;
        size_t maxn = (size_t)(capc > N ? capc : N);
        ws += (maxn / 4096 + 2) * 1024 * 4 + (maxn / 2048 + 2) * 16 + 64 * 256 + (1 << 20);
        c->ws_bytes = ws;
        INIT_CUDA(dmalloc(c, reinterpret_cast<char **>(&c->ws.base), ws), "alloc workspace");
        c->ws.cap = ws;
    }
    for (auto &ev : c->ev) INIT_CUDA(cudaEventCreate(&ev), "event");

    // validate the CSR and compute per-object value sums
    c->launch_base = g_launches;
    int bad = 0;
    INIT_CUDA(validate_csr(c, &bad), "validate");
    if (bad) {
        free_all(c);
        delete c;
        return SIVF_ERR_BAD_CSR;
    }
    // state: no labels, no own scores, every cluster moving
    INIT_CUDA(cudaMemsetAsync(c->labels, 0xFF, sizeof(int32_t) * N, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->labels_prev, 0xFF, sizeof(int32_t) * N, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->own, 0xFF, sizeof(uint32_t) * N, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->lam, 0, k, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->lam_prev, 0, k, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->moving, 1, k, c->stream), "memset");
    INIT_CUDA(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream), "memset");
    {
        std::vector<int32_t> ids((size_t)k);
        for (int32_t j = 0; j < k; ++j) ids[(size_t)j] = j;
        INIT_CUDA(cudaMemcpyAsync(c->mov_list, ids.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream),
                  "copy");
        INIT_CUDA(cudaMemcpyAsync(c->n_mov_dev, &k, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "copy");
        int32_t *ids_dev = c->ws.take<int32_t>((size_t)k);
        INIT_CUDA(ids_dev ? cudaSuccess : cudaErrorMemoryAllocation, "ws");
        INIT_CUDA(cudaMemcpyAsync(ids_dev, init_ids, sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream), "copy");
        INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
        // copy the seed rows (cluster-major), then the first inverted file
        INIT_CUDA(init_centroids(c, ids_dev), "init centroids");
    }
    INIT_CUDA(build_inverted_file(c), "build inverted file");
    INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
    c->stats.centroid_nnz = c->c_nnz;
#undef INIT_CUDA
    *out = c;
    return SIVF_OK;
}

sivf_status sivf_reseed(sivf_ctx *c, const int32_t *init_ids) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (!init_ids) return fail(c, SIVF_ERR_INVALID_ARG, "init_ids is NULL");
    {
        std::vector<char> seen((size_t)c->N, 0);
        for (int32_t j = 0; j < c->k; ++j) {
            int32_t d = init_ids[j];
            if (d < 0 || (int64_t)d >= c->N || seen[(size_t)d]) return fail(c, SIVF_ERR_INVALID_ARG, "bad init ids");
            seen[(size_t)d] = 1;
        }
    }
    c->ws.reset();
    int32_t *ids_dev = c->ws.take<int32_t>((size_t)c->k);
    if (!ids_dev) return cuda_fail(c, cudaErrorMemoryAllocation, "workspace");
    API_CUDA(c, cudaMemcpyAsync(ids_dev, init_ids, sizeof(int32_t) * c->k, cudaMemcpyHostToDevice, c->stream), "copy");
    c->launch_base = g_launches;
    API_CUDA(c, reseed_dev(c, ids_dev), "reseed");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    c->ws.reset();
    c->stats = sivf_stats{};
    c->stats.centroid_nnz = c->c_nnz;
    return SIVF_OK;
}

sivf_status sivf_assign(sivf_ctx *c, int64_t *n_changed) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    // a^[r-1] <- a^[r]; lambda^[r-1] <- lambda^[r]
    if (c->needs_update)
        return fail(c, SIVF_ERR_STATE,
                    "sivf_update must run between two assignments (and after sivf_set_labels)");
    std::swap(c->labels, c->labels_prev);
    std::swap(c->lam, c->lam_prev);
    c->iter += 1;
    API_CUDA(c, cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream), "memset");
    API_CUDA(c, cudaMemsetAsync(c->moving, 0, c->k, c->stream), "memset");
    int32_t nmp = 0;
    API_CUDA(c, cudaMemcpyAsync(&nmp, c->n_mov_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaEventRecord(c->ev[0], c->stream), "event");
    API_CUDA(c, launch_assign(c), "assign kernel");
    API_CUDA(c, launch_finalize_assign(c), "finalize kernel");
    API_CUDA(c, cudaEventRecord(c->ev[1], c->stream), "event");
    API_CUDA(c, cudaMemcpyAsync(c->ctr_host, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    float ms = 0.f;
    API_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]), "elapsed");
    const DevCounters &h = *c->ctr_host;
    if (h.error) {
        c->latched = true;
        c->err = "device-side check failed in the assignment";
        return SIVF_ERR_STATE;
    }
    sivf_stats &s = c->stats;
    s.iter = c->iter;
    s.changed = (int64_t)h.changed;
    s.n_moving = (int64_t)h.n_moving;
    s.n_moving_prev = nmp;
    s.filtered = (int64_t)h.filtered;
    s.simcalc = (int64_t)h.simcalc;
    s.postings = (int64_t)h.postings;
    s.rescored = (int64_t)h.rescored;
    s.rescore_cands = (int64_t)h.rescore_cands;
    s.ms_assign = ms;
    if (n_changed) *n_changed = s.changed;
    // the inverted file still has the lambda^[r-1] layout: the next
    // assignment needs the update that rebuilds it with lambda^[r]
    c->needs_update = true;
    return SIVF_OK;
}

sivf_status sivf_update(sivf_ctx *c) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (c->iter < 1) return fail(c, SIVF_ERR_STATE, "sivf_update needs an assignment (or sivf_set_labels) first");
    API_CUDA(c, cudaEventRecord(c->ev[2], c->stream), "event");
    API_CUDA(c, run_update(c), "update");
    API_CUDA(c, cudaEventRecord(c->ev[3], c->stream), "event");
    double obj[2] = {0, 0};
    API_CUDA(c, cudaMemcpyAsync(obj, c->obj_dev, sizeof(obj), cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    float ms = 0.f;
    API_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]), "elapsed");
    c->stats.objective_assign = obj[0];
    c->stats.objective_update = obj[1];
    c->stats.ms_update = ms;
    c->stats.centroid_nnz = c->c_nnz;
    c->needs_update = false;
    return SIVF_OK;
}

sivf_status sivf_run(sivf_ctx *c, int32_t max_iter, int32_t *iters_out, double *objective_out) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (max_iter < 0) return fail(c, SIVF_ERR_INVALID_ARG, "max_iter < 0");
    int32_t done = 0;
    double obj = 0.0;
    if (c->needs_update && max_iter > 0) {
        st = sivf_update(c);
        if (st != SIVF_OK) return st;
    }
    for (int32_t it = 0; it < max_iter; ++it) {
        int64_t changed = 0;
        st = sivf_assign(c, &changed);
        if (st != SIVF_OK) return st;
        ++done;
        if (c->iter > 1 && changed == 0) break;
        st = sivf_update(c);
        if (st != SIVF_OK) return st;
        obj = c->stats.objective_assign;
    }
    if (iters_out) *iters_out = done;
    if (objective_out) *objective_out = obj;
    return SIVF_OK;
}

sivf_status sivf_get_labels(sivf_ctx *c, int32_t *dst, int dst_is_device) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (!dst) return fail(c, SIVF_ERR_INVALID_ARG, "dst is NULL");
    if (c->latched) return SIVF_ERR_STATE;
    API_CUDA(c, cudaMemcpyAsync(dst, c->labels, sizeof(int32_t) * c->N,
                                dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
             "copy labels");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    return SIVF_OK;
}

sivf_status sivf_set_labels(sivf_ctx *c, const int32_t *src, int src_is_device) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (!src) return fail(c, SIVF_ERR_INVALID_ARG, "src is NULL");
    c->ws.reset();
    if (!src_is_device) {
        int32_t *tmp = c->ws.take<int32_t>((size_t)c->N);
        if (!tmp) return cuda_fail(c, cudaErrorMemoryAllocation, "workspace");
        API_CUDA(c, cudaMemcpyAsync(tmp, src, sizeof(int32_t) * c->N, cudaMemcpyHostToDevice, c->stream), "copy");
        src = tmp;
    }
    cudaError_t e = set_labels_dev(c, src);
    c->ws.reset();
    if (e == cudaErrorInvalidValue) return fail(c, SIVF_ERR_INVALID_ARG, "labels out of range");
    if (e != cudaSuccess) return cuda_fail(c, e, "set labels");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    c->needs_update = true;
    return SIVF_OK;
}

sivf_status sivf_get_centroids(sivf_ctx *c, int64_t *off, int32_t *term, float *u, int64_t cap, int64_t *nnz_out) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    if (!off) return fail(c, SIVF_ERR_INVALID_ARG, "off is NULL");
    const int cur = c->cur;
    API_CUDA(c, cudaMemcpyAsync(off, c->coff[cur], sizeof(int64_t) * (c->k + 1), cudaMemcpyDeviceToHost, c->stream),
             "copy");
    if (nnz_out) *nnz_out = c->c_nnz;
    if (cap < c->c_nnz || !term || !u) {
        API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
        return fail(c, SIVF_ERR_INVALID_ARG, "capacity below the centroid nnz");
    }
    API_CUDA(c, cudaMemcpyAsync(term, c->cterm[cur], sizeof(int32_t) * c->c_nnz, cudaMemcpyDeviceToHost, c->stream),
             "copy");
    API_CUDA(c, cudaMemcpyAsync(u, c->cval[cur], sizeof(float) * c->c_nnz, cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    return SIVF_OK;
}

sivf_status sivf_get_inverted_file(sivf_ctx *c, int64_t *off, int32_t *mf0, int32_t *cid, float *u, int64_t cap,
                                   int64_t *nnz_out) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    if (!off || !mf0) return fail(c, SIVF_ERR_INVALID_ARG, "off/mf0 is NULL");
    API_CUDA(c, cudaMemcpyAsync(off, c->if_off, sizeof(int64_t) * (c->D + 1), cudaMemcpyDeviceToHost, c->stream),
             "copy");
    API_CUDA(c, cudaMemcpyAsync(mf0, c->if_mf0, sizeof(int32_t) * c->D, cudaMemcpyDeviceToHost, c->stream), "copy");
    if (nnz_out) *nnz_out = c->if_nnz;
    if (cap < c->if_nnz || !cid || !u) {
        API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
        return fail(c, SIVF_ERR_INVALID_ARG, "capacity below the inverted-file nnz");
    }
    API_CUDA(c, cudaMemcpyAsync(cid, c->if_cid, sizeof(int32_t) * c->if_nnz, cudaMemcpyDeviceToHost, c->stream),
             "copy");
    API_CUDA(c, cudaMemcpyAsync(u, c->if_val, sizeof(float) * c->if_nnz, cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    return SIVF_OK;
}

sivf_status sivf_get_lambda(sivf_ctx *c, uint8_t *dst) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    if (!dst) return fail(c, SIVF_ERR_INVALID_ARG, "dst is NULL");
    API_CUDA(c, cudaMemcpyAsync(dst, c->lam, c->k, cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    return SIVF_OK;
}

sivf_status sivf_get_stats(sivf_ctx *c, sivf_stats *out) {
    if (!c || !out) return SIVF_ERR_INVALID_ARG;
    c->stats.launches = (int64_t)(g_launches - c->launch_base);
    *out = c->stats;
    return SIVF_OK;
}

const char *sivf_last_error(const sivf_ctx *c) {
    if (!c) return kNoCtx;
    return c->err.c_str();
}

void sivf_destroy(sivf_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
