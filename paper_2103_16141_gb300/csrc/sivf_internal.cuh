// Internal declarations of the SIVF GB300 library (not part of the C ABI).
//
// Data layout in HBM (all device arrays owned by the context unless noted):
//   object CSR            row_ptr int64[N+1], idx int32[nnz], val f32[nnz]  (borrowed)
//   labels, labels_prev   int32[N]      a^[r], a^[r-1]
//   own                   uint32[N]     fixed-point (2^-31) score of the object's own
//                                        cluster from its last scan; OWN_INVALID = none
//   sumv                  f32[N]        sum of the object's values (error bound)
//   lam, lam_prev         uint8[k]      lambda^[r], lambda^[r-1] (1 = invariant)
//   mov_list              int32[k]      ids j with lambda^[r] = 0 (ascending)
//   centroids (x2)        coff int64[k+1], cterm int32[cap], cval f32[cap], cclu int32[cap]
//                                        cluster-major FP32 master copy, ascending terms
//   snorm                 f64[k]        ||s_j|| of the sum behind each centroid
//   inverted file         if_off int64[D+1], if_mf0 int32[D]; if_cid int32[cap],
//                                        if_val f32[cap]: canonical order (front ids
//                                        ascending, then back ids ascending), built
//                                        on demand for the getters
//   scan copy of the file sc_off int64[D+1]: each list starts at a multiple of 4
//                                        entries; a list's full 128-entry blocks are
//                                        stored transposed (entry 32m + l of a block at
//                                        block position 4l + m), so that lane l reads
//                                        entries l, 32+l, 64+l, 96+l with one vector
//                                        load; the ragged tail keeps list order. Inside
//                                        a segment the postings are in the order the
//                                        build's atomic cursor handed out.
//                                        Arrays (scan positions): sc_id16 u16 or
//                                        sc_id32 int32, plus sc_val f32 (FP32), or
//                                        sc_pack u32 = id << 16 | bf16/fp16 value
//                                        (16-bit ids and values), or sc_lp u16
//                                        Ids in the scan copy are scan positions (below).
//   scan order            clu_pos int32[k]: position of cluster j in its instance's
//                                        scan order (moving clusters of lambda^[r] first,
//                                        ascending id, then the invariant ones, ascending
//                                        id); pos_clu int32[k]: the inverse (instance
//                                        offset + position -> local id). Score vectors are
//                                        indexed by position. IVF-CBICP keeps id order.
//   dense head rows       dense_row int32[D]: first entry / 8 of term t's dense row, or
//                                        -1 (the term is scanned from the sparse copy);
//                                        dense_val (u16 or f32) [cap_dense]: one row per dense
//                                        term, the term's value for every cluster of its
//                                        instance at the cluster's scan position (0 where
//                                        the cluster lacks the term), padded to a multiple
//                                        of 8 entries; a term's list becomes a row when it
//                                        holds at least dense_frac of its instance's k
//                                        (raised while the rows would exceed cap_dense).
//   update accumulator    acc int64 (dense form): one row of the instance's D terms per
//                                        cluster (acc_off), the fixed-point sums
//                                        q(x) = ceil(x 2^shift) of the current members,
//                                        kept across iterations
//   object lists          heavy_ids, light_ids int32[N]: the objects of the CTA and the
//                                        warp-per-object assignment kernels
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sivf.h"

namespace sivf {

constexpr uint32_t OWN_INVALID = 0xFFFFFFFFu;
// tail padding (entries) of the inverted-file posting arrays
constexpr int64_t IF_PAD = 256;
// block of the tiled scan layout: 32 lanes x 4 entries
constexpr int SC_BLK = 128;
// shared memory the assignment kernel stages per thread besides the score
// vector: list start, full-block end, end of the full scanned blocks, scaled
// value, scanned length, item prefix, row-posting prefix, dense row and value
constexpr int ASSIGN_STAGE_BYTES = 36;
// Scores are accumulated as unsigned fixed point with quantum 2^-31:
// q = ceil(fl(v * u) * 2^31). Cosine scores are <= 1 (+ rounding), so the
// sum of an object's terms stays below 2^32.
constexpr float FIX_SCALE = 2147483648.0f;  // 2^31
constexpr double FIX_QUANTUM = 4.656612873077392578125e-10;  // 2^-31
// FP16 postings store u * 2^14 so that every centroid value >= 2^-28 is a
// normal half-precision number.
constexpr float FP16_SCALE = 16384.0f;
constexpr float FP16_INV_SCALE = 1.0f / 16384.0f;

struct DevCounters {
    unsigned long long changed;
    unsigned long long filtered;
    unsigned long long simcalc;
    unsigned long long postings;
    unsigned long long rescored;
    unsigned long long rescore_cands;
    unsigned long long n_moving;     // lambda^[r] = 0 count (written by finalize)
    unsigned long long work;         // object work counter of the assignment kernel
    unsigned long long error;        // nonzero: device-side check failed (code)
    long long moved;                 // object non-zeros gathered by the last update
    long long c_nnz;                 // centroid non-zeros after the last update
    unsigned long long dense_entries;   // dense-row entries read by the assignment
    unsigned long long dense_postings;  // postings of the scanned segments held in dense rows
    long long dense_terms;              // terms with a dense row (last inverted-file build)
    long long dense_used;               // dense-row entries in use / 8 (last build)
    unsigned long long work_light;   // object work counter of the light (warp-per-object) kernel
    unsigned int n_heavy, n_light;   // objects in the two lists of the assignment
    long long sparse_entries;        // entries of the sparse scan copy (last build)
};

// Bump allocator over one device block (scratch that lives for one step).
struct Workspace {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    void reset() { used = 0; }
    template <typename T>
    T *take(size_t n) {
        size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

}  // namespace sivf

struct sivf_ctx {
    sivf_config cfg;
    int64_t N = 0;
    int32_t D = 0, k = 0;
    int64_t nnz = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    const int64_t *row_ptr = nullptr;
    const int32_t *idx = nullptr;
    const float *val = nullptr;

    bool latched = false;
    bool needs_update = false;  // an assignment or set_labels since the last update
    std::string err;
    int32_t iter = 0;
    int bits_t = 0;  // bits of a term id

    // object state
    int32_t *labels = nullptr, *labels_prev = nullptr;
    uint32_t *own = nullptr;
    float *sumv = nullptr;

    // cluster state
    uint8_t *lam = nullptr, *lam_prev = nullptr, *moving = nullptr;
    int32_t *mov_list = nullptr;
    int32_t *n_mov_dev = nullptr;
    double *snorm = nullptr, *snorm_new = nullptr;

    // centroids, double-buffered
    int64_t *coff[2] = {nullptr, nullptr};
    int32_t *cterm[2] = {nullptr, nullptr};
    float *cval[2] = {nullptr, nullptr};
    int32_t *cclu = nullptr;  // cluster id of each entry of the current buffer
    int cur = 0;
    int64_t cap_c = 0;
    int64_t c_nnz = 0;

    // structured inverted file
    int64_t *if_off = nullptr;
    int32_t *if_mf0 = nullptr;
    int32_t *if_cid = nullptr;
    float *if_val = nullptr;
    int64_t if_nnz = 0;
    bool canon_stale = true;  // if_cid / if_val predate the last inverted-file build
    // scan copy (tiled layout, local ids); which arrays exist depends on the
    // id width (16 bits when every instance has k <= 65536) and the precision
    int64_t *sc_off = nullptr;
    uint16_t *sc_id16 = nullptr;
    int32_t *sc_id32 = nullptr;
    float *sc_val = nullptr;      // FP32 postings
    uint32_t *sc_pack = nullptr;  // 16-bit ids and 16-bit values
    uint16_t *sc_lp = nullptr;    // 32-bit ids and 16-bit values
    int64_t cap_s = 0;            // entries of each scan array
    // scan order and dense head rows (see the layout above)
    int32_t *clu_pos = nullptr, *pos_clu = nullptr;
    int32_t *dense_row = nullptr;
    void *dense_val = nullptr;    // dense rows: u16 (BF16/FP16) or f32 entries
    int64_t cap_dense = 0;        // entries of dense (0: no dense rows)
    float dense_frac = 0.f;       // list length / k from which a term gets a dense row
    int32_t *inst_d = nullptr;    // device [n_inst+1]: first term of each instance
    int32_t *dense_thr = nullptr; // device [1]: threshold bin chosen by the last build
    long long dense_terms_h = 0, dense_used_h = 0;

    // dense update accumulator: cluster j owns acc[acc_off[j] .. acc_off[j+1]),
    // one int64 per term of its instance, in units of 2^-acc_shift. It holds
    // the fixed-point sums of the members recorded in acc_lab (the label each
    // object was last added under, -1 = none) and is updated incrementally.
    bool dense = false;
    int64_t *acc = nullptr;
    int64_t *acc_off = nullptr;
    int32_t *acc_lab = nullptr;
    int64_t acc_total = 0;  // entries of acc
    int acc_shift = 0;

    // counters and step scratch
    sivf::DevCounters *ctr = nullptr;
    sivf::DevCounters *ctr_host = nullptr;  // pinned mirror
    double *obj_dev = nullptr;              // [2 * n_inst]: J_assign, J_update per instance
    sivf::Workspace ws;
    size_t ws_bytes = 0;
    size_t owned_bytes = 0;
    sivf_stats stats{};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int assign_threads = 0, assign_ctas_per_sm = 0;
    int64_t assign_grid = 0;  // cached launch grid of the assignment kernel (0 = not yet chosen)
    int assign_global = 0;    // 1: score vectors in global memory (grho), else shared memory
    bool tuned = false;       // the autotuner has picked the assignment configuration
    uint32_t *grho = nullptr; // global score vectors: grho_ctas slabs of kmax (zero between objects)
    int64_t grho_ctas = 0;
    unsigned long long launch_base = 0;  // g_launches at init / reseed
    // object lists of the assignment: filtered objects of instances with few
    // moving clusters take the warp-per-object kernel (light), the rest the
    // CTA-per-object kernel (heavy)
    int32_t *heavy_ids = nullptr, *light_ids = nullptr;
    long long sparse_entries_h = 0;  // entries of the sparse scan copy (host copy, for the L2 hint)

    // independent instances sharing one context: objects [inst_obj[m],
    // inst_obj[m+1]), clusters [inst_k[m], inst_k[m+1]), terms [inst_d[m],
    // inst_d[m+1]) belong to instance m (one instance for sivf_init)
    int32_t n_inst = 1;
    int32_t kmax = 0;                  // largest instance k (shared-memory score vector)
    int64_t *inst_obj = nullptr;       // device [n_inst+1]
    int32_t *inst_k = nullptr;         // device [n_inst+1]
    int32_t *mov_beg = nullptr;        // device [n_inst+1]
    int32_t *clu_koff = nullptr;       // device [k]: first cluster of the cluster's instance
    int32_t *clu_doff = nullptr;       // device [k]: first term of the cluster's instance
    int bits_tl = 0;                   // bits of an instance-local term id
    unsigned long long *inst_changed = nullptr;  // device [n_inst]
    std::vector<int64_t> inst_obj_h;
    std::vector<int32_t> inst_k_h, inst_d_h;
    std::vector<unsigned long long> inst_changed_h;
    std::vector<double> inst_obj_assign_h, inst_obj_update_h;
    // pinned host mirrors (read after a stream synchronisation)
    unsigned long long *inst_changed_pin = nullptr;  // [n_inst]
    double *obj_pin = nullptr;                      // [2 * n_inst]
    int32_t *nmov_pin = nullptr;                    // [1] moving count before the assignment
    // device-side Lloyd loop (use_graph): WHILE conditional node around one iteration
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int32_t *loop_dev = nullptr;      // [4]: iter, max_iter, remaining, pad
    int32_t *done_dev = nullptr;      // [n_inst]: iteration of convergence (0 = not yet)
    double *objf_dev = nullptr;       // [n_inst]: objective at the instance's last update
    int32_t *loop_pin = nullptr;      // pinned [4 + n_inst] mirror of loop_dev and done_dev
    double *objf_pin = nullptr;       // pinned [n_inst]
    unsigned long long launches_per_iter = 0;
    // concatenated object CSR owned by a batch context (null for sivf_init)
    int64_t *own_row_ptr = nullptr;
    int32_t *own_idx = nullptr;
    float *own_val = nullptr;
};

namespace sivf {

// Kernel launches issued by the library (host-side count, all contexts).
extern unsigned long long g_launches;
inline void note_launch(unsigned long long n = 1) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }

// ---- primitives.cu ----
// Exclusive prefix sum of n elements (in may equal out). Optional total.
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, Workspace &ws,
                               cudaStream_t s);
cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, Workspace &ws, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `nbits` bits of the
// keys. Input in (k0, v0); (k1, v1) is scratch of the same size. Returns, via
// *result_in_alt, whether the sorted output ended in (k1, v1).
cudaError_t radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n, int nbits,
                             bool *result_in_alt, Workspace &ws, cudaStream_t s);
// Same with the live element count in device memory (n = its upper bound):
// no host synchronisation, so it can be captured in a CUDA graph.
cudaError_t radix_sort_pairs_dev(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t n,
                                 const int64_t *n_dev, int nbits, bool *result_in_alt, Workspace &ws, cudaStream_t s);
cudaError_t scan_exclusive_u32_dev(const uint32_t *in, uint32_t *out, int64_t nmax, const int64_t *n_dev,
                                   uint32_t *total, Workspace &ws, cudaStream_t s);
int bits_for(uint64_t max_value);  // number of bits to hold values in [0, max_value]

// ---- assign.cu ----
cudaError_t launch_assign(sivf_ctx *c);
cudaError_t launch_finalize_assign(sivf_ctx *c);
cudaError_t autotune_assign(sivf_ctx *c);

// ---- graph.cu ----
cudaError_t build_loop_graph(sivf_ctx *c);
void destroy_loop_graph(sivf_ctx *c);

// ---- api.cu (step enqueue without host synchronisation) ----
cudaError_t enqueue_assign(sivf_ctx *c, bool timing);
cudaError_t enqueue_update(sivf_ctx *c, bool timing);

// ---- update.cu ----
cudaError_t run_update(sivf_ctx *c);
cudaError_t build_inverted_file(sivf_ctx *c);
cudaError_t build_canonical_if(sivf_ctx *c);
cudaError_t validate_csr(sivf_ctx *c, int *bad);
cudaError_t init_centroids(sivf_ctx *c, const int32_t *init_ids_dev);
cudaError_t set_labels_dev(sivf_ctx *c, const int32_t *src_dev);
cudaError_t reseed_dev(sivf_ctx *c, const int32_t *init_ids_dev);

}  // namespace sivf

#define SIVF_CUDA_TRY(expr)                    \
    do {                                       \
        cudaError_t e__ = (expr);              \
        if (e__ != cudaSuccess) return e__;    \
    } while (0)
