// C ABI of the SIVF library (declared in include/sivf.h): argument checks,
// device memory ownership, step orchestration and error latching.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
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
                    c->cval[0], c->cval[1], c->cclu, c->if_off, c->if_mf0, c->if_cid, c->if_val, c->sc_off, c->sc_id16, c->sc_id32, c->sc_val, c->sc_pack, c->sc_lp,
                    c->ctr, c->obj_dev, c->ws.base, c->inst_obj, c->inst_k, c->mov_beg, c->clu_koff,
                    c->inst_changed, c->own_row_ptr, c->own_idx, c->own_val, c->clu_doff,
                    c->loop_dev, c->done_dev, c->objf_dev, c->grho, c->acc, c->acc_off, c->acc_lab,
                    c->clu_pos, c->pos_clu, c->dense_row, c->dense_val, c->inst_d, c->dense_thr,
                    c->heavy_ids, c->light_ids};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    destroy_loop_graph(c);
    void *pins[] = {c->ctr_host, c->inst_changed_pin, c->obj_pin, c->nmov_pin, c->loop_pin, c->objf_pin};
    for (void *p : pins)
        if (p) cudaFreeHost(p);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
}

sivf_status check_usable(sivf_ctx *c) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    return SIVF_OK;
}

// Dense-row counters of the inverted file built by sivf_init / sivf_reseed
// (later builds report them through the update step's counters).
cudaError_t read_file_counters(sivf_ctx *c) {
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->ctr_host, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
    SIVF_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->dense_terms_h = c->ctr_host->dense_terms;
    c->dense_used_h = c->ctr_host->dense_used * 8;
    c->sparse_entries_h = c->ctr_host->sparse_entries;
    return cudaSuccess;
}

void pick_assign_config(sivf_ctx *c) {
    int T = c->cfg.threads;
    if (T != 32 && T != 64 && T != 128 && T != 256 && T != 512) T = 0;
    if (T == 0) T = c->kmax <= 2048 ? 64 : (c->kmax <= 4096 ? 128 : 512);  // measured on the k = 1000 and k = 10,000 corpora
    c->assign_threads = T;
    c->assign_ctas_per_sm = c->cfg.ctas_per_sm > 0 ? c->cfg.ctas_per_sm : 0;
    int dev = 0, smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool fits = ((size_t)((c->kmax + 3) & ~3) * 4 + (size_t)T * ASSIGN_STAGE_BYTES) <= (size_t)smem;
    c->assign_global = c->cfg.score_buffer == 2 || (c->cfg.score_buffer == 0 && !fits) ? 1 : 0;
    if (c->cfg.icp == 2) {  // IVF-CBICP: 128 threads, shared score vector, no tuning
        c->assign_threads = 128;
        c->assign_global = 0;
    }
}

}  // namespace

namespace {

// Shared tail of sivf_init and sivf_batch_init: allocate every device array,
// validate the (possibly concatenated) CSR, seed the centroids and build the
// first inverted file. Instance tables are host vectors of n_inst + 1 offsets.
// owned_* (non-null for batch contexts) are adopted by the context.
sivf_status create_ctx(sivf_ctx **out, const sivf_config *cfg, int64_t N, int32_t D, int32_t k,
                       const int64_t *row_ptr, const int32_t *idx, const float *val, const int32_t *init_ids,
                       void *stream, const std::vector<int64_t> &inst_obj, const std::vector<int32_t> &inst_k,
                       const std::vector<int32_t> &inst_d, int64_t *owned_row_ptr, int32_t *owned_idx,
                       float *owned_val) {
    sivf_ctx *c = new (std::nothrow) sivf_ctx();
    if (!c) {
        cudaFree(owned_row_ptr);
        cudaFree(owned_idx);
        cudaFree(owned_val);
        return SIVF_ERR_OOM;
    }
    c->own_row_ptr = owned_row_ptr;
    c->own_idx = owned_idx;
    c->own_val = owned_val;
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
    c->n_inst = (int32_t)inst_obj.size() - 1;
    c->inst_obj_h = inst_obj;
    c->inst_k_h = inst_k;
    c->inst_d_h = inst_d;
    c->inst_changed_h.assign((size_t)c->n_inst, 0);
    c->inst_obj_assign_h.assign((size_t)c->n_inst, 0.0);
    c->inst_obj_update_h.assign((size_t)c->n_inst, 0.0);
    c->kmax = 0;
    for (int32_t m = 0; m < c->n_inst; ++m) c->kmax = std::max(c->kmax, inst_k[(size_t)m + 1] - inst_k[(size_t)m]);
    c->bits_t = bits_for((uint64_t)(D - 1));
    if (c->bits_t < 1) c->bits_t = 1;
    if (c->bits_t > 30) {
        free_all(c);
        delete c;
        return SIVF_ERR_INVALID_ARG;
    }
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
    pick_assign_config(c);
    if (c->cfg.icp == 2) {  // the IVF-CBICP kernel keeps the score vector and lambda bits in shared memory
        int smem = 0;
        INIT_CUDA(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device), "attr");
        const size_t need = (size_t)((c->kmax + 3) & ~3) * 4 + 128 * (size_t)ASSIGN_STAGE_BYTES +
                            (size_t)((k + 31) >> 5) * 4;
        if (need > (size_t)smem) {
            free_all(c);
            delete c;
            return SIVF_ERR_INVALID_ARG;
        }
    }
    // nnz from row_ptr[N]
    int64_t nnz = 0, first = 0;
    INIT_CUDA(cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream), "read nnz");
    INIT_CUDA(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream), "read row_ptr");
    INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
    if (first != 0 || nnz < 0 || nnz >= 0x7FFFFFFFll) {
        free_all(c);
        delete c;
        return SIVF_ERR_BAD_CSR;
    }
    // the scan addresses postings with 32-bit offsets
    if (2 * nnz + 1024 + 3 * (int64_t)D + IF_PAD >= 0x7FFFFFFFll) {
        free_all(c);
        delete c;
        return SIVF_ERR_INVALID_ARG;
    }
    c->nnz = nnz;
    c->cap_c = 2 * nnz + 1024;
    const int64_t capc = c->cap_c;
    const int32_t ni = c->n_inst;
    INIT_CUDA(dmalloc(c, &c->labels, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->heavy_ids, N), "alloc");
    INIT_CUDA(dmalloc(c, &c->light_ids, N), "alloc");
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
    INIT_CUDA(dmalloc(c, &c->inst_obj, (size_t)ni + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->inst_k, (size_t)ni + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->mov_beg, (size_t)ni + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->clu_koff, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->clu_doff, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->inst_changed, ni), "alloc");
    for (int b = 0; b < 2; ++b) {
        INIT_CUDA(dmalloc(c, &c->coff[b], (size_t)k + 1), "alloc");
        INIT_CUDA(dmalloc(c, &c->cterm[b], capc), "alloc");
        INIT_CUDA(dmalloc(c, &c->cval[b], capc), "alloc");
    }
    INIT_CUDA(dmalloc(c, &c->cclu, capc), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_off, (size_t)D + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_mf0, D), "alloc");
    // posting arrays carry a small tail pad; the scan copy also pads every
    // list to a multiple of 4 entries
    INIT_CUDA(dmalloc(c, &c->if_cid, capc + IF_PAD), "alloc");
    INIT_CUDA(dmalloc(c, &c->if_val, capc + IF_PAD), "alloc");
    c->cap_s = capc + 3 * (int64_t)D + IF_PAD;
    const size_t caps = (size_t)c->cap_s;
    const bool ids16 = c->kmax <= 65536;
    INIT_CUDA(dmalloc(c, &c->sc_off, (size_t)D + 1), "alloc");
    if (c->cfg.prec == SIVF_FP32) {
        if (ids16) INIT_CUDA(dmalloc(c, &c->sc_id16, caps), "alloc");
        else INIT_CUDA(dmalloc(c, &c->sc_id32, caps), "alloc");
        INIT_CUDA(dmalloc(c, &c->sc_val, caps), "alloc");
    } else if (ids16) {
        INIT_CUDA(dmalloc(c, &c->sc_pack, caps), "alloc");
    } else {
        INIT_CUDA(dmalloc(c, &c->sc_id32, caps), "alloc");
        INIT_CUDA(dmalloc(c, &c->sc_lp, caps), "alloc");
    }
    // scan order and dense head rows
    INIT_CUDA(dmalloc(c, &c->clu_pos, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->pos_clu, k), "alloc");
    INIT_CUDA(dmalloc(c, &c->dense_row, D), "alloc");
    INIT_CUDA(dmalloc(c, &c->inst_d, (size_t)ni + 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->dense_thr, 1), "alloc");
    {
        const int64_t esize = c->cfg.prec == SIVF_FP32 ? 4 : 2;
        const int64_t bytes = c->cfg.dense_max_bytes == 0 ? (int64_t)96 << 20 : c->cfg.dense_max_bytes;
        c->cap_dense = (c->cfg.icp == 2 || bytes < 0) ? 0 : (bytes / esize) & ~(int64_t)7;
        if (c->cfg.dense_all && c->cfg.icp != 2) {  // room for a row of every term
            c->cap_dense = 0;
            for (int32_t m = 0; m < ni; ++m)
                c->cap_dense += (int64_t)(inst_d[(size_t)m + 1] - inst_d[(size_t)m]) *
                                ((inst_k[(size_t)m + 1] - inst_k[(size_t)m] + 7) & ~7);
        }
        c->dense_frac = c->cfg.dense_min_fraction > 0.f ? c->cfg.dense_min_fraction : 0.25f;
        if (c->cap_dense / 8 >= 0x7FFFFFFFll) {  // rows are addressed in 8-entry units with 32 bits
            free_all(c);
            delete c;
            return SIVF_ERR_INVALID_ARG;
        }
        if (c->cap_dense > 0) INIT_CUDA(dmalloc(c, reinterpret_cast<uint16_t **>(&c->dense_val),
                                                (size_t)(c->cap_dense * esize / 2)), "alloc dense rows");
    }
    INIT_CUDA(dmalloc(c, &c->ctr, 1), "alloc");
    INIT_CUDA(dmalloc(c, &c->obj_dev, 2 * (size_t)ni), "alloc");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->ctr_host), sizeof(DevCounters)), "alloc host");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->inst_changed_pin), sizeof(unsigned long long) * ni),
              "alloc host");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->obj_pin), sizeof(double) * 2 * ni), "alloc host");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->nmov_pin), sizeof(int32_t)), "alloc host");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->loop_pin), sizeof(int32_t) * (4 + (size_t)ni)), "alloc host");
    INIT_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->objf_pin), sizeof(double) * ni), "alloc host");
    if (c->assign_global || c->cfg.autotune) {
        // global score vectors: one kmax slab per resident CTA (at most 16 per SM)
        c->grho_ctas = (int64_t)c->num_sms * 16;
        INIT_CUDA(dmalloc(c, &c->grho, (size_t)c->grho_ctas * ((c->kmax + 3) & ~3)), "alloc");
        INIT_CUDA(cudaMemsetAsync(c->grho, 0, sizeof(uint32_t) * (size_t)c->grho_ctas * ((c->kmax + 3) & ~3),
                                  c->stream), "memset");
    }
    INIT_CUDA(dmalloc(c, &c->loop_dev, 4), "alloc");
    INIT_CUDA(dmalloc(c, &c->done_dev, ni), "alloc");
    INIT_CUDA(dmalloc(c, &c->objf_dev, ni), "alloc");
    {
        // dense update accumulator: one row of the instance's D terms per cluster
        // (padded to an even length; the pad entry stays zero)
        std::vector<int64_t> aoff((size_t)k + 1, 0);
        int64_t nmax = 1;
        for (int32_t m = 0; m < ni; ++m) {
            nmax = std::max(nmax, inst_obj[(size_t)m + 1] - inst_obj[(size_t)m]);
            for (int32_t j = inst_k[(size_t)m]; j < inst_k[(size_t)m + 1]; ++j)
                aoff[(size_t)j + 1] = aoff[(size_t)j] + ((inst_d[(size_t)m + 1] - inst_d[(size_t)m] + 1) & ~1);  // rows 16-byte aligned
        }
        const size_t acc_bytes = 8 * (size_t)aoff[(size_t)k];
        bool dense = c->cfg.update_mode == 1;
        if (c->cfg.update_mode == 0) {
            size_t free_b = 0, total_b = 0;
            INIT_CUDA(cudaMemGetInfo(&free_b, &total_b), "mem info");
            dense = acc_bytes <= free_b / 2 &&
                    (c->cfg.mem_cap_bytes <= 0 || c->owned_bytes + acc_bytes <= (size_t)c->cfg.mem_cap_bytes);
        }
        if (dense) {
            INIT_CUDA(dmalloc(c, &c->acc, (size_t)aoff[(size_t)k]), "alloc accumulator");
            INIT_CUDA(dmalloc(c, &c->acc_off, (size_t)k + 1), "alloc");
            INIT_CUDA(dmalloc(c, &c->acc_lab, (size_t)N), "alloc");
            INIT_CUDA(cudaMemcpyAsync(c->acc_off, aoff.data(), sizeof(int64_t) * ((size_t)k + 1),
                                      cudaMemcpyHostToDevice, c->stream), "copy");
            INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
            // a cluster holds at most nmax objects of values <= 1, each rounded
            // up by less than one unit: sums stay below 2^62 + nmax
            c->acc_shift = 62 - bits_for((uint64_t)nmax);
            c->acc_total = aoff[(size_t)k];
            c->dense = true;
        }
    }
    {
        // workspace: max of the update's two phases, plus primitive scratch
        const size_t n8 = (size_t)N * 8, k8 = (size_t)k * 8;
        // u1: 4 label key/value arrays (4 B x N), tuple counts/offsets (8 B x N),
        // per-cluster arrays; u2 per tuple (sort mode only): 4 sort arrays,
        // term, rank, value, sorted value, 64-bit key, piece sum, unique term
        // and sum (60 B)
        size_t phase1 = 4 * (size_t)N * 4 + 2 * n8 + 14 * k8 + (c->dense ? 0 : 64 * ((size_t)nnz + 1)) + 32 * 4096;
        // u5: sort arrays (16 B x entries), per-term counts, lengths, dense widths
        // and offsets (40 B x terms), the dense-length histogram
        size_t phase2 = 16 * ((size_t)capc + 1) + 48 * ((size_t)D + 1) + 16 * 4096;
        size_t ws = phase1 > phase2 ? phase1 : phase2;
        size_t maxn = (size_t)(capc > N ? capc : N);
        ws += (maxn / 4096 + 2) * 1024 * 4 + (maxn / 2048 + 2) * 16 + 64 * 256 + (1 << 20);
        c->ws_bytes = ws;
        INIT_CUDA(dmalloc(c, reinterpret_cast<char **>(&c->ws.base), ws), "alloc workspace");
        c->ws.cap = ws;
    }
    for (auto &ev : c->ev) INIT_CUDA(cudaEventCreate(&ev), "event");
    {
        std::vector<int32_t> koff((size_t)k), doff((size_t)k);
        int32_t dmax = 1;
        for (int32_t m = 0; m < ni; ++m) {
            dmax = std::max(dmax, inst_d[(size_t)m + 1] - inst_d[(size_t)m]);
            for (int32_t j = inst_k[(size_t)m]; j < inst_k[(size_t)m + 1]; ++j) {
                koff[(size_t)j] = inst_k[(size_t)m];
                doff[(size_t)j] = inst_d[(size_t)m];
            }
        }
        c->bits_tl = std::max(1, bits_for((uint64_t)(dmax - 1)));
        INIT_CUDA(cudaMemcpyAsync(c->clu_doff, doff.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream),
                  "copy");
        INIT_CUDA(cudaMemcpyAsync(c->inst_obj, inst_obj.data(), sizeof(int64_t) * (ni + 1), cudaMemcpyHostToDevice,
                                  c->stream), "copy");
        INIT_CUDA(cudaMemcpyAsync(c->inst_k, inst_k.data(), sizeof(int32_t) * (ni + 1), cudaMemcpyHostToDevice,
                                  c->stream), "copy");
        INIT_CUDA(cudaMemcpyAsync(c->inst_d, inst_d.data(), sizeof(int32_t) * (ni + 1), cudaMemcpyHostToDevice,
                                  c->stream), "copy");
        INIT_CUDA(cudaMemcpyAsync(c->clu_koff, koff.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream),
                  "copy");
        INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
    }

    // validate the CSR and compute per-object value sums
    c->launch_base = g_launches;
    int bad = 0;
    INIT_CUDA(validate_csr(c, &bad), "validate");
    if (bad) {
        free_all(c);
        delete c;
        return SIVF_ERR_BAD_CSR;
    }
    {
        int32_t *ids_dev = c->ws.take<int32_t>((size_t)k);
        INIT_CUDA(ids_dev ? cudaSuccess : cudaErrorMemoryAllocation, "ws");
        INIT_CUDA(cudaMemcpyAsync(ids_dev, init_ids, sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream), "copy");
        // state: no labels, no own scores, every cluster moving; seed rows and
        // the first inverted file
        INIT_CUDA(reseed_dev(c, ids_dev), "seed");
    }
    INIT_CUDA(cudaStreamSynchronize(c->stream), "sync");
    INIT_CUDA(read_file_counters(c), "counters");
    c->ws.reset();
    c->stats.centroid_nnz = c->c_nnz;
#undef INIT_CUDA
    *out = c;
    return SIVF_OK;
}

bool distinct_ids(const int32_t *ids, int32_t k, int64_t N) {
    std::vector<char> seen((size_t)N, 0);
    for (int32_t j = 0; j < k; ++j) {
        const int32_t d = ids[j];
        if (d < 0 || (int64_t)d >= N || seen[(size_t)d]) return false;
        seen[(size_t)d] = 1;
    }
    return true;
}

__global__ void k_concat_rows(int64_t n, const int64_t *src, int64_t nnz_off, int64_t *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + nnz_off;
}

__global__ void k_concat_terms(int64_t n, const int32_t *src, int32_t d_off, int32_t D, int32_t *dst, int *bad) {
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < n; h += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = src[h];
        if (t < 0 || t >= D) atomicOr(bad, 1);
        dst[h] = (t < 0 || t >= D) ? -1 : t + d_off;  // -1 fails validation later
    }
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
    if (cfg && (cfg->prec < SIVF_FP32 || cfg->prec > SIVF_FP16 || cfg->icp < 0 || cfg->icp > 3 ||
                !(cfg->dense_min_fraction >= 0.f && cfg->dense_min_fraction <= 1.f) ||
                cfg->light_max_moving > 1472))
        return SIVF_ERR_INVALID_ARG;
    if (!distinct_ids(init_ids, k, N)) return SIVF_ERR_INVALID_ARG;
    if (cfg && cfg->inputs_on_host) {
        // host CSR: copy it into device buffers that the context adopts
        const int64_t nnz = row_ptr[N];
        if (row_ptr[0] != 0 || nnz < 0 || nnz >= 0x7FFFFFFFll) return SIVF_ERR_BAD_CSR;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int64_t *rp = nullptr;
        int32_t *ix = nullptr;
        float *vl = nullptr;
        const size_t nz = nnz > 0 ? (size_t)nnz : 1;
        if (cudaMalloc(reinterpret_cast<void **>(&rp), sizeof(int64_t) * (size_t)(N + 1)) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&ix), sizeof(int32_t) * nz) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&vl), sizeof(float) * nz) != cudaSuccess) {
            cudaFree(rp);
            cudaFree(ix);
            cudaFree(vl);
            cudaGetLastError();
            return SIVF_ERR_OOM;
        }
        if (cudaMemcpyAsync(rp, row_ptr, sizeof(int64_t) * (size_t)(N + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            (nnz > 0 && cudaMemcpyAsync(ix, idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            (nnz > 0 && cudaMemcpyAsync(vl, val, sizeof(float) * (size_t)nnz, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
            cudaStreamSynchronize(s);
            cudaFree(rp);
            cudaFree(ix);
            cudaFree(vl);
            return SIVF_ERR_CUDA;
        }
        // create_ctx synchronises the stream before it returns, so the host
        // arrays are no longer read once this call returns
        return create_ctx(out, cfg, N, D, k, rp, ix, vl, init_ids, stream, {0, N}, {0, k}, {0, D}, rp, ix, vl);
    }
    return create_ctx(out, cfg, N, D, k, row_ptr, idx, val, init_ids, stream, {0, N}, {0, k}, {0, D}, nullptr,
                      nullptr, nullptr);
}

sivf_status sivf_batch_init(sivf_ctx **out, const sivf_config *cfg, int32_t n_inst, const sivf_instance_desc *descs,
                            void *stream) {
    if (!out) return SIVF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_inst < 1 || n_inst > 65536 || !descs) return SIVF_ERR_INVALID_ARG;
    if (cfg && (cfg->prec < SIVF_FP32 || cfg->prec > SIVF_FP16 || cfg->inputs_on_host || cfg->icp < 0 || cfg->icp > 3 ||
                !(cfg->dense_min_fraction >= 0.f && cfg->dense_min_fraction <= 1.f) ||
                cfg->light_max_moving > 1472))
        return SIVF_ERR_INVALID_ARG;
    std::vector<int64_t> inst_obj(1, 0);
    std::vector<int32_t> inst_k(1, 0), inst_d(1, 0);
    for (int32_t m = 0; m < n_inst; ++m) {
        const sivf_instance_desc &d = descs[m];
        if (d.N < 1 || d.D < 1 || d.k < 1 || (int64_t)d.k > d.N || !d.row_ptr || !d.idx || !d.val || !d.init_ids)
            return SIVF_ERR_INVALID_ARG;
        if (!distinct_ids(d.init_ids, d.k, d.N)) return SIVF_ERR_INVALID_ARG;
        if (inst_obj.back() + d.N > 0x7FFFFFFFll || (int64_t)inst_k.back() + d.k > 0x7FFFFFFFll ||
            (int64_t)inst_d.back() + d.D > (1 << 30))
            return SIVF_ERR_INVALID_ARG;
        inst_obj.push_back(inst_obj.back() + d.N);
        inst_k.push_back(inst_k.back() + d.k);
        inst_d.push_back(inst_d.back() + d.D);
    }
    const int64_t N = inst_obj.back();
    const int32_t K = inst_k.back(), Dt = inst_d.back();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // instance sizes (nnz) from each row_ptr[N]
    std::vector<int64_t> nnz_off(1, 0);
    for (int32_t m = 0; m < n_inst; ++m) {
        int64_t nz = 0, f = 0;
        if (cudaMemcpyAsync(&nz, descs[m].row_ptr + descs[m].N, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&f, descs[m].row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SIVF_ERR_CUDA;
        if (f != 0 || nz < 0) return SIVF_ERR_BAD_CSR;
        nnz_off.push_back(nnz_off.back() + nz);
    }
    const int64_t nnz = nnz_off.back();
    if (nnz >= 0x7FFFFFFFll) return SIVF_ERR_INVALID_ARG;
    // concatenated CSR: terms of instance m shifted by its term offset
    int64_t *rp = nullptr;
    int32_t *ix = nullptr;
    float *vl = nullptr;
    int *bad = nullptr;
    auto cleanup = [&]() {
        cudaFree(rp);
        cudaFree(ix);
        cudaFree(vl);
        cudaFree(bad);
    };
    if (cudaMalloc(&rp, sizeof(int64_t) * (N + 1)) != cudaSuccess || cudaMalloc(&ix, sizeof(int32_t) * (nnz + 1)) != cudaSuccess ||
        cudaMalloc(&vl, sizeof(float) * (nnz + 1)) != cudaSuccess || cudaMalloc(&bad, sizeof(int)) != cudaSuccess) {
        cleanup();
        return SIVF_ERR_OOM;
    }
    bool ok = cudaMemsetAsync(bad, 0, sizeof(int), s) == cudaSuccess;
    for (int32_t m = 0; m < n_inst && ok; ++m) {
        const sivf_instance_desc &d = descs[m];
        const int64_t nz = nnz_off[(size_t)m + 1] - nnz_off[(size_t)m];
        k_concat_rows<<<(unsigned)std::min<int64_t>((d.N + 255) / 256 + 1, 65535), 256, 0, s>>>(
            d.N, d.row_ptr, nnz_off[(size_t)m], rp + inst_obj[(size_t)m]);
        if (nz > 0) {
            k_concat_terms<<<(unsigned)std::min<int64_t>((nz + 255) / 256, 65535), 256, 0, s>>>(
                nz, d.idx, inst_d[(size_t)m], d.D, ix + nnz_off[(size_t)m], bad);
            ok = cudaMemcpyAsync(vl + nnz_off[(size_t)m], d.val, sizeof(float) * nz, cudaMemcpyDeviceToDevice, s) ==
                 cudaSuccess;
        }
        note_launch(nz > 0 ? 2 : 1);
    }
    int bad_h = 0;
    ok = ok && cudaMemcpyAsync(rp + N, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    cudaFree(bad);
    bad = nullptr;
    if (!ok) {
        cleanup();
        return SIVF_ERR_CUDA;
    }
    if (bad_h) {
        cleanup();
        return SIVF_ERR_BAD_CSR;
    }
    std::vector<int32_t> ids((size_t)K);
    for (int32_t m = 0; m < n_inst; ++m)
        for (int32_t j = 0; j < descs[m].k; ++j)
            ids[(size_t)inst_k[(size_t)m] + j] = descs[m].init_ids[j] + (int32_t)inst_obj[(size_t)m];
    return create_ctx(out, cfg, N, Dt, K, rp, ix, vl, ids.data(), stream, inst_obj, inst_k, inst_d, rp, ix, vl);
}

sivf_status sivf_reseed(sivf_ctx *c, const int32_t *init_ids) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (!init_ids) return fail(c, SIVF_ERR_INVALID_ARG, "init_ids is NULL");
    if (!distinct_ids(init_ids, c->k, c->N)) return fail(c, SIVF_ERR_INVALID_ARG, "bad init ids");
    for (int32_t m = 0; m < c->n_inst; ++m)  // each seed must be an object of its cluster's instance
        for (int32_t j = c->inst_k_h[(size_t)m]; j < c->inst_k_h[(size_t)m + 1]; ++j)
            if (init_ids[j] < c->inst_obj_h[(size_t)m] || init_ids[j] >= c->inst_obj_h[(size_t)m + 1])
                return fail(c, SIVF_ERR_INVALID_ARG, "seed outside its instance");
    c->ws.reset();
    int32_t *ids_dev = c->ws.take<int32_t>((size_t)c->k);
    if (!ids_dev) return cuda_fail(c, cudaErrorMemoryAllocation, "workspace");
    API_CUDA(c, cudaMemcpyAsync(ids_dev, init_ids, sizeof(int32_t) * c->k, cudaMemcpyHostToDevice, c->stream), "copy");
    c->launch_base = g_launches;
    API_CUDA(c, reseed_dev(c, ids_dev), "reseed");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    API_CUDA(c, read_file_counters(c), "counters");
    c->ws.reset();
    c->stats = sivf_stats{};
    c->stats.centroid_nnz = c->c_nnz;
    // no update has run from these seeds: no objective yet
    std::fill(c->inst_obj_assign_h.begin(), c->inst_obj_assign_h.end(), 0.0);
    std::fill(c->inst_obj_update_h.begin(), c->inst_obj_update_h.end(), 0.0);
    std::fill(c->inst_changed_h.begin(), c->inst_changed_h.end(), 0ull);
    return SIVF_OK;
}

}  // extern "C"

namespace sivf {

// Stream operations of one assignment step (no host synchronisation). With
// timing, CUDA events bracket the kernels and the counters are copied to the
// pinned host mirrors; a graph body is captured without either.
cudaError_t enqueue_assign(sivf_ctx *c, bool timing) {
    cudaStream_t s = c->stream;
    // a^[r-1] <- a^[r], lambda^[r-1] <- lambda^[r] (copies keep every buffer
    // address fixed from one iteration to the next)
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->labels_prev, c->labels, sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaMemcpyAsync(c->lam_prev, c->lam, c->k, cudaMemcpyDeviceToDevice, s));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->moving, 0, c->k, s));
    SIVF_CUDA_TRY(cudaMemsetAsync(c->inst_changed, 0, sizeof(unsigned long long) * c->n_inst, s));
    if (timing) {
        SIVF_CUDA_TRY(cudaMemcpyAsync(c->nmov_pin, c->n_mov_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SIVF_CUDA_TRY(cudaEventRecord(c->ev[0], s));
    }
    SIVF_CUDA_TRY(launch_assign(c));
    SIVF_CUDA_TRY(launch_finalize_assign(c));
    if (timing) {
        SIVF_CUDA_TRY(cudaEventRecord(c->ev[1], s));
        SIVF_CUDA_TRY(cudaMemcpyAsync(c->ctr_host, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
        SIVF_CUDA_TRY(cudaMemcpyAsync(c->inst_changed_pin, c->inst_changed, sizeof(unsigned long long) * c->n_inst,
                                      cudaMemcpyDeviceToHost, s));
    }
    return cudaSuccess;
}

cudaError_t enqueue_update(sivf_ctx *c, bool timing) {
    cudaStream_t s = c->stream;
    if (timing) SIVF_CUDA_TRY(cudaEventRecord(c->ev[2], s));
    SIVF_CUDA_TRY(run_update(c));
    if (timing) {
        SIVF_CUDA_TRY(cudaEventRecord(c->ev[3], s));
        SIVF_CUDA_TRY(cudaMemcpyAsync(c->obj_pin, c->obj_dev, sizeof(double) * 2 * c->n_inst, cudaMemcpyDeviceToHost,
                                      s));
        SIVF_CUDA_TRY(cudaMemcpyAsync(c->ctr_host, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    }
    return cudaSuccess;
}

}  // namespace sivf

namespace {

// Host bookkeeping after an assignment whose counters are in the pinned mirrors.
sivf_status finish_assign(sivf_ctx *c, int64_t *n_changed, float ms) {
    const DevCounters &h = *c->ctr_host;
    if (h.error) {
        c->latched = true;
        c->err = (h.error & 1ull) ? "device-side check failed in the assignment: a row offset of the CSR is out of range"
                                  : "device-side check failed in the assignment: a term of the CSR is outside [0, D)";
        return SIVF_ERR_STATE;
    }
    for (int32_t m = 0; m < c->n_inst; ++m)
        c->inst_changed_h[(size_t)m] = c->n_inst == 1 ? h.changed : c->inst_changed_pin[m];
    sivf_stats &st = c->stats;
    st.iter = c->iter;
    st.changed = (int64_t)h.changed;
    st.n_moving = (int64_t)h.n_moving;
    st.n_moving_prev = *c->nmov_pin;
    st.filtered = (int64_t)h.filtered;
    st.simcalc = (int64_t)h.simcalc;
    st.postings = (int64_t)h.postings;
    st.rescored = (int64_t)h.rescored;
    st.rescore_cands = (int64_t)h.rescore_cands;
    st.dense_entries = (int64_t)h.dense_entries;
    st.dense_postings = (int64_t)h.dense_postings;
    st.light_objects = (int64_t)h.n_light;
    if (ms >= 0.f) st.ms_assign = ms;
    if (n_changed) *n_changed = st.changed;
    return SIVF_OK;
}

sivf_status finish_update(sivf_ctx *c, float ms) {
    if (c->ctr_host->error) {
        c->latched = true;
        c->err = "the centroids outgrew their buffers (more than 2 nnz + 1024 entries)";
        return SIVF_ERR_OOM;
    }
    c->c_nnz = c->ctr_host->c_nnz;
    c->if_nnz = c->c_nnz;
    c->dense_terms_h = c->ctr_host->dense_terms;
    c->dense_used_h = c->ctr_host->dense_used * 8;
    c->sparse_entries_h = c->ctr_host->sparse_entries;
    c->stats.moved_nnz = c->ctr_host->moved;
    double ja = 0.0, ju = 0.0;
    for (int32_t m = 0; m < c->n_inst; ++m) {
        c->inst_obj_assign_h[(size_t)m] = c->obj_pin[2 * m];
        c->inst_obj_update_h[(size_t)m] = c->obj_pin[2 * m + 1];
        ja += c->obj_pin[2 * m];
        ju += c->obj_pin[2 * m + 1];
    }
    c->stats.objective_assign = ja;
    c->stats.objective_update = ju;
    if (ms >= 0.f) c->stats.ms_update = ms;
    c->stats.centroid_nnz = c->c_nnz;
    c->needs_update = false;
    return SIVF_OK;
}

// Runs iterations on the device until every instance has converged or c->iter
// reaches max_total. done/objf: host arrays (n_inst), updated in place.
// Requires c->iter >= 2 and no pending update.
sivf_status graph_loop(sivf_ctx *c, int32_t max_total, std::vector<int32_t> &done, std::vector<double> &objf) {
    const int32_t ni = c->n_inst;
    if (!c->graph_exec) {
        cudaError_t e = build_loop_graph(c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->cfg.use_graph = 0;  // keep working with host-launched steps
            c->err = std::string("graph capture unavailable (") + c->err + "), stepping from the host: " +
                     cudaGetErrorString(e);
            return SIVF_ERR_CUDA;
        }
    }
    cudaStream_t s = c->stream;
    int32_t *lp = c->loop_pin;
    lp[0] = c->iter;
    lp[1] = max_total;
    lp[2] = 0;
    lp[3] = 0;
    for (int32_t m = 0; m < ni; ++m) {
        lp[4 + m] = done[(size_t)m];
        c->objf_pin[m] = objf[(size_t)m];
    }
    API_CUDA(c, cudaMemcpyAsync(c->loop_dev, lp, sizeof(int32_t) * 4, cudaMemcpyHostToDevice, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->done_dev, lp + 4, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->objf_dev, c->objf_pin, sizeof(double) * ni, cudaMemcpyHostToDevice, s), "copy");
    const int32_t iter0 = c->iter;
    API_CUDA(c, cudaGraphLaunch(c->graph_exec, s), "graph launch");
    c->canon_stale = true;  // the replayed updates rebuilt the file
    API_CUDA(c, cudaMemcpyAsync(lp, c->loop_dev, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(lp + 4, c->done_dev, sizeof(int32_t) * ni, cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->objf_pin, c->objf_dev, sizeof(double) * ni, cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->nmov_pin, c->n_mov_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->ctr_host, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->inst_changed_pin, c->inst_changed, sizeof(unsigned long long) * ni,
                                cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaMemcpyAsync(c->obj_pin, c->obj_dev, sizeof(double) * 2 * ni, cudaMemcpyDeviceToHost, s), "copy");
    API_CUDA(c, cudaStreamSynchronize(s), "sync");
    c->iter = lp[0];
    for (int32_t m = 0; m < ni; ++m) {
        done[(size_t)m] = lp[4 + m];
        objf[(size_t)m] = c->objf_pin[m];
    }
    __atomic_fetch_add(&g_launches, c->launches_per_iter * (unsigned long long)(c->iter - iter0), __ATOMIC_RELAXED);
    c->stats.graph_iters += c->iter - iter0;
    sivf_status st = finish_assign(c, nullptr, -1.f);
    if (st != SIVF_OK) return st;
    return finish_update(c, -1.f);  // the body ends with an update
}

}  // namespace

extern "C" {

sivf_status sivf_assign(sivf_ctx *c, int64_t *n_changed) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (c->needs_update)
        return fail(c, SIVF_ERR_STATE,
                    "sivf_update must run between two assignments (and after sivf_set_labels)");
    c->iter += 1;
    if (c->cfg.autotune && c->cfg.icp != 2 && !c->tuned && c->iter == 2) API_CUDA(c, autotune_assign(c), "autotune");
    API_CUDA(c, enqueue_assign(c, true), "assignment");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    float ms = 0.f;
    API_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]), "elapsed");
    st = finish_assign(c, n_changed, ms);
    if (st != SIVF_OK) return st;
    // the inverted file still has the lambda^[r-1] layout: the next
    // assignment needs the update that rebuilds it with lambda^[r]
    c->needs_update = true;
    return SIVF_OK;
}

sivf_status sivf_update(sivf_ctx *c) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (c->iter < 1) return fail(c, SIVF_ERR_STATE, "sivf_update needs an assignment (or sivf_set_labels) first");
    API_CUDA(c, enqueue_update(c, true), "update");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    float ms = 0.f;
    API_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]), "elapsed");
    return finish_update(c, ms);
}

// Shared by sivf_run and sivf_batch_run: iterate until every instance has
// converged or max_iter assignments ran in this call. done[m] = iteration of
// convergence (0 = not converged), objf[m] = objective at the last update.
static sivf_status run_loop(sivf_ctx *c, int32_t max_iter, std::vector<int32_t> &done, std::vector<double> &objf) {
    sivf_status st;
    const size_t ni = (size_t)c->n_inst;
    const int32_t max_total = c->iter + max_iter;
    c->stats.graph_iters = 0;
    size_t remaining = 0;
    for (size_t m = 0; m < ni; ++m) remaining += done[m] == 0;
    if (c->needs_update && max_iter > 0) {
        st = sivf_update(c);
        if (st != SIVF_OK) return st;
        for (size_t m = 0; m < ni; ++m) objf[m] = c->inst_obj_update_h[m];
    }
    while (c->iter < max_total && remaining > 0) {
        if (c->cfg.use_graph && !c->cfg.checked && c->iter >= 2 && !c->needs_update) {
            st = graph_loop(c, max_total, done, objf);
            if (st == SIVF_OK) break;
            if (c->latched) return st;  // a real failure; otherwise fall back to host-launched steps
        }
        st = sivf_assign(c, nullptr);
        if (st != SIVF_OK) return st;
        // an instance converges at its first assignment (r > 1) that changes no
        // label; later iterations leave it untouched (every cluster invariant)
        for (size_t m = 0; m < ni; ++m) {
            if (!done[m] && c->iter > 1 && c->inst_changed_h[m] == 0) {
                done[m] = c->iter;
                --remaining;
            }
        }
        if (remaining == 0) break;
        st = sivf_update(c);
        if (st != SIVF_OK) return st;
        for (size_t m = 0; m < ni; ++m)
            if (!done[m]) objf[m] = c->inst_obj_update_h[m];
    }
    return SIVF_OK;
}

sivf_status sivf_run(sivf_ctx *c, int32_t max_iter, int32_t *iters_out, double *objective_out) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (max_iter < 0) return fail(c, SIVF_ERR_INVALID_ARG, "max_iter < 0");
    const int32_t iter0 = c->iter;
    std::vector<int32_t> done((size_t)c->n_inst, 0);
    std::vector<double> objf(c->inst_obj_update_h);  // a call that runs no update reports the last one
    st = run_loop(c, max_iter, done, objf);
    if (st != SIVF_OK) return st;
    if (iters_out) *iters_out = c->n_inst == 1 && done[0] ? done[0] - iter0 : c->iter - iter0;
    if (objective_out) *objective_out = c->n_inst == 1 ? objf[0] : c->stats.objective_update;
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
    API_CUDA(c, build_canonical_if(c), "canonical inverted file");
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
    c->stats.assign_threads = c->assign_threads;
    c->stats.assign_global = c->assign_global;
    c->stats.update_dense = c->dense ? 1 : 0;
    c->stats.dense_terms = c->dense_terms_h;
    c->stats.dense_row_entries = c->dense_used_h;
    *out = c->stats;
    return SIVF_OK;
}

const char *sivf_last_error(const sivf_ctx *c) {
    if (!c) return kNoCtx;
    return c->err.c_str();
}

sivf_status sivf_batch_run(sivf_ctx *c, int32_t max_iter, int32_t *iters_out, double *objective_out) {
    sivf_status st = check_usable(c);
    if (st != SIVF_OK) return st;
    if (max_iter < 0) return fail(c, SIVF_ERR_INVALID_ARG, "max_iter < 0");
    const size_t ni = (size_t)c->n_inst;
    std::vector<int32_t> done(ni, 0);
    std::vector<double> objf(c->inst_obj_update_h);  // a call that runs no update reports the last one
    st = run_loop(c, max_iter, done, objf);
    if (st != SIVF_OK) return st;
    for (size_t m = 0; m < ni; ++m) {
        if (iters_out) iters_out[m] = done[m] ? done[m] : c->iter;
        if (objective_out) objective_out[m] = objf[m];
    }
    return SIVF_OK;
}

sivf_status sivf_batch_get_labels(sivf_ctx *c, int32_t inst, int32_t *dst) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (c->latched) return SIVF_ERR_STATE;
    if (inst < 0 || inst >= c->n_inst || !dst) return fail(c, SIVF_ERR_INVALID_ARG, "bad instance or dst");
    const int64_t b = c->inst_obj_h[(size_t)inst], n = c->inst_obj_h[(size_t)inst + 1] - b;
    API_CUDA(c, cudaMemcpyAsync(dst, c->labels + b, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream), "copy");
    API_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
    const int32_t koff = c->inst_k_h[(size_t)inst];
    for (int64_t i = 0; i < n; ++i)
        if (dst[i] >= 0) dst[i] -= koff;
    return SIVF_OK;
}

sivf_status sivf_batch_instance_stats(sivf_ctx *c, int32_t inst, int64_t *changed, double *objective_assign,
                                      double *objective_update) {
    if (!c) return SIVF_ERR_INVALID_ARG;
    if (inst < 0 || inst >= c->n_inst) return fail(c, SIVF_ERR_INVALID_ARG, "bad instance");
    if (changed) *changed = (int64_t)c->inst_changed_h[(size_t)inst];
    if (objective_assign) *objective_assign = c->inst_obj_assign_h[(size_t)inst];
    if (objective_update) *objective_update = c->inst_obj_update_h[(size_t)inst];
    return SIVF_OK;
}

void sivf_destroy(sivf_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
