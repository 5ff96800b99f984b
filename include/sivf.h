/*
 * sivf.h — C ABI of the GB300 (sm_103a) implementation of SIVF spherical
 * k-means: the structured inverted-file assignment step with the invariant
 * centroid-pair (ICP) filter, and the update step that rebuilds the file.
 *
 * Method: Aoyama & Saito, "Structured Inverted-File k-Means Clustering for
 * High-Dimensional Sparse Data", arXiv 2103.16141.
 *   - problem and objective: Section 1 (spherical k-means: unit-length
 *     objects and means, cosine similarity), Section 2.1 Eq. (1) and
 *     Algorithm 1 (Lloyd iteration);
 *   - assignment step: Algorithm 4 (Section 4.1), with the unfiltered
 *     inverted-file assignment of Algorithm 2 (Section 3.2) as the icp = 0 mode;
 *   - update step and structured inverted file: Algorithm 5 (Section 4.2).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a sivf_status and never aborts or traps.
 *   - An invalid argument returns SIVF_ERR_INVALID_ARG (or SIVF_ERR_BAD_CSR)
 *     and leaves the context unchanged.
 *   - A CUDA failure returns SIVF_ERR_CUDA; after it the context is latched:
 *     every later call except the getters of sivf_last_error and
 *     sivf_destroy returns SIVF_ERR_STATE.
 *   - All device work is ordered on the stream passed to sivf_init. Calls
 *     that return host values synchronise that stream.
 *   - Labels are 0-based cluster ids in [0, k).
 *   - "DEVICE" pointers are CUDA device (or managed) memory; "HOST" pointers
 *     are ordinary host memory.
 */
#ifndef SIVF_H
#define SIVF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIVF_OK = 0,
    SIVF_ERR_INVALID_ARG = 1,
    SIVF_ERR_BAD_CSR = 2,
    SIVF_ERR_OOM = 3,
    SIVF_ERR_CUDA = 4,
    SIVF_ERR_TIMEOUT = 5,
    SIVF_ERR_STATE = 6
} sivf_status;

/* Storage precision of the inverted-file posting values used by the
 * assignment scan. Products are formed in FP32 and accumulated exactly in
 * fixed point; objects whose top-2 margin is inside the derived error bound
 * are re-scored in FP64 from the FP32 centroid values, so the labels do not
 * depend on this choice. */
typedef enum { SIVF_FP32 = 0, SIVF_BF16 = 1, SIVF_FP16 = 2 } sivf_precision;

typedef struct {
    sivf_precision prec; /* posting value precision for the scan */
    int icp;             /* 1: SIVF with the ICP filter (Algorithm 4); 0: unfiltered
                            (Algorithm 2); 2: IVF-CBICP (Algorithm 3), the paper's
                            branch-based baseline over an unstructured file (ascending
                            centroid ids in every list, mf0 = list length), kept for
                            ablation: 128 threads, shared score vector, no tuning;
                            3: SIVF with the relaxed filter (an object whose own
                            cluster moved also keeps to the moving centroids when its
                            similarity to its own centroid did not decrease, tested
                            with the error bound after the front scan; tried while at
                            most half of its instance's clusters are moving). It pays
                            off with FP32 postings; with BF16/FP16 the bound is too wide
                            for the test to pass often */
    int threads;         /* threads per CTA of the assignment kernel (32, 64, 128, 256 or
                            512); 0 = automatic */
    int ctas_per_sm;     /* resident CTAs per SM of the assignment kernel; 0 = automatic */
    int64_t mem_cap_bytes; /* cap on library-owned device memory; 0 = no cap */
    int use_graph;       /* 1: after the first two iterations, sivf_run / sivf_batch_run
                            replay one CUDA graph whose conditional WHILE node runs the
                            remaining iterations on the device (no per-iteration host
                            round trip); 0: every step launched from the host */
    int autotune;        /* 1: at the second assignment, time every feasible assignment
                            kernel configuration (threads per CTA x score vector in shared
                            or global memory; a shared score vector that lets fewer than
                            512 threads reside per SM is not tried) on the live state and
                            keep the fastest;
                            threads / ctas_per_sm then only seed the search. The choice
                            is remembered for the process (per device and problem
                            shape), so later contexts of the same shape skip the trials */
    int score_buffer;    /* 0: automatic (shared memory when k fits), 1: shared, 2: global */
    int update_mode;     /* cluster sums of the update step: 0 automatic (dense when the
                            accumulator takes at most half of the free device memory
                            and fits mem_cap_bytes), 1 dense, 2 sort. Dense: one int64
                            fixed-point accumulator row of D entries per cluster
                            (8 k D bytes; per instance for batches), kept across
                            steps and updated with integer atomics for the objects
                            whose label changed, then compacted in ascending term
                            order for the moving clusters.
                            Sort: the members' (cluster, term, value) tuples are
                            radix-sorted and equal (cluster, term) runs summed in
                            FP64 in member order. Both are deterministic. */
    int inputs_on_host;  /* sivf_init only. 1: row_ptr / idx / val are HOST memory; the
                            library copies them (on the stream, asynchronously when the host
                            memory is pinned) into device buffers it owns and frees in
                            sivf_destroy, and the host arrays may be released once
                            sivf_init returns. 0: DEVICE memory, borrowed. sivf_batch_init
                            rejects 1 (its descriptors are DEVICE). */
    int checked;         /* 1: the assignment step checks every object's row offsets
                            (0 <= row_ptr[i] <= row_ptr[i+1] <= nnz) and terms (in
                            [0, D)) before using them, as the borrowed CSR may have
                            changed since sivf_init validated it. A failed check reads
                            nothing through the bad value, records a device-side status
                            word, and the assignment then returns SIVF_ERR_STATE with
                            the context latched. Checked contexts step every iteration
                            from the host (no CUDA-graph loop), so no update runs on
                            unchecked data. 0: the CSR is trusted after validation. */
    int64_t dense_max_bytes;  /* device memory for dense head-term rows. The posting
                            lists that hold a large share of their instance's k
                            centroids are stored as dense rows (one value per cluster,
                            0 where a cluster lacks the term, in scan order: moving
                            clusters first) and read with vector loads into FP32
                            registers instead of per-posting score atomics. Rows take
                            k x 2 bytes (BF16/FP16) or k x 4 bytes (FP32) each.
                            0 = automatic (96 MB, below the L2 size), < 0 = none */
    float dense_min_fraction; /* a list becomes a dense row when it holds at least this
                            fraction of its instance's k (the threshold rises while the
                            rows would exceed dense_max_bytes); 0 = automatic (0.25).
                            Must be in [0, 1]. IVF-CBICP (icp = 2) uses no dense rows */
    int light_max_moving;     /* filtered objects (own cluster invariant) of an instance with
                            at most this many moving clusters are scored by one warp each
                            instead of one CTA each (same scores, labels and counts; no
                            block-wide barrier per object). 0 = automatic (1472, the
                            largest allowed), < 0 = every object in the CTA kernel. Used
                            with icp = 1 and 3 */
    int dense_all;            /* 1: every term gets a dense row, whatever its length: the
                            centroids are held as a dense matrix (k x 2 or k x 4 bytes per
                            term, in scan order), the dense-mean variant of the scan
                            (Lloyd-ICP with full-expression means, as the paper's
                            comparison systems keep them; Section 3). Same labels;
                            dense_max_bytes and dense_min_fraction are then ignored */
} sivf_config;

/* Counters of the most recent assignment / update (host copy). */
typedef struct {
    int32_t iter;            /* r: number of assignment steps done */
    int64_t changed;         /* objects whose label changed at r (N at r = 1) */
    int64_t n_moving;        /* clusters with lambda^[r] = 0 */
    int64_t n_moving_prev;   /* clusters with lambda^[r-1] = 0 (candidates of a filtered object) */
    int64_t filtered;        /* objects that took the filtered (front-only) branch */
    int64_t simcalc;         /* similarity calculations: k per unfiltered, n_moving_prev per filtered object */
    int64_t postings;        /* postings visited by the scan (the method's count: the
                                scanned segments' lengths, whichever layout held them) */
    int64_t rescored;        /* objects re-scored in FP64 (top-2 margin inside the error bound) */
    int64_t rescore_cands;   /* candidate centroids re-scored in FP64 */
    int64_t centroid_nnz;    /* non-zeros of the centroid set M^[r] after the last update */
    int64_t moved_nnz;       /* object non-zeros the last update read: sort form, every member
                                of a recomputed cluster; dense form, the objects whose label
                                changed, counted once per cluster row touched */
    double objective_assign; /* J^[r] = sum_i <x_i, mu_{a(i)}^[r-1]> (FP64) for the labels of
                                assignment r, evaluated by the update step that follows it as
                                sum_j <s_j, mu_j^[r-1]>: current after sivf_update, still the
                                previous value between sivf_assign and sivf_update */
    double objective_update; /* sum_j ||s_j^[r]||, s_j = sum of members (FP64), of the last update */
    double ms_assign;        /* device time of the last assignment step */
    double ms_update;        /* device time of the last update step */
    int64_t launches;        /* kernels launched by the library since sivf_init / sivf_reseed */
    int64_t graph_iters;     /* iterations the last sivf_run / sivf_batch_run ran inside its CUDA graph */
    int32_t assign_threads;  /* threads per CTA of the assignment kernel in use */
    int32_t assign_global;   /* 1 if its score vectors live in global memory */
    int32_t update_dense;    /* 1 if the update step sums into the dense accumulator */
    int64_t dense_entries;   /* dense-row entries read by the last assignment */
    int64_t dense_postings;  /* of `postings`, those of terms read from dense rows (the
                                rest were read one posting at a time) */
    int64_t dense_terms;     /* terms with a dense row in the current inverted file */
    int64_t dense_row_entries; /* entries of those rows (padded to multiples of 8) */
    int64_t light_objects;   /* objects of the last assignment scored one warp each (filtered
                                objects of instances with few moving clusters) */
} sivf_stats;

typedef struct sivf_ctx sivf_ctx; /* opaque, library-owned */

/*
 * sivf_init — validate the object set, copy the initial centroids and build
 * the first inverted file (Algorithm 1 input M^[0]; Algorithm 5 layout with
 * every centroid moving, since lambda^[0] = 0).
 *   out      : HOST, receives the new context (NULL on failure).
 *   cfg      : HOST, copied; NULL means defaults (FP32, icp = 1).
 *   N, D, k  : objects, vocabulary size, clusters; 1 <= k <= N, D >= 1.
 *   row_ptr  : DEVICE int64[N+1], CSR row offsets, row_ptr[0] = 0, non-decreasing.
 *   idx      : DEVICE int32[nnz], term ids in [0, D), strictly ascending in each row.
 *   val      : DEVICE float[nnz], tf-idf values > 0, each row of unit L2 norm.
 *              row_ptr / idx / val are BORROWED: they must stay valid and
 *              unchanged until sivf_destroy. With cfg->inputs_on_host = 1 all
 *              three are HOST arrays instead, copied at init.
 *   init_ids : HOST int32[k], distinct object ids; mu_j^[0] = x_{init_ids[j]}. Copied.
 *   stream   : cudaStream_t (may be NULL = legacy default stream).
 * Errors: SIVF_ERR_INVALID_ARG (sizes, ids; 2 nnz + 3 D + 1280 must stay
 * below 2^31 - 1, the range of the scan's 32-bit posting offsets),
 * SIVF_ERR_BAD_CSR (row_ptr not
 * monotone, idx out of range or not ascending, val not finite and positive,
 * a row norm off 1 by more than 1e-4), SIVF_ERR_OOM, SIVF_ERR_CUDA.
 */
sivf_status sivf_init(sivf_ctx **out, const sivf_config *cfg, int64_t N, int32_t D, int32_t k,
                      const int64_t *row_ptr, const int32_t *idx, const float *val,
                      const int32_t *init_ids, void *stream);

/*
 * sivf_reseed — restart the context from new initial centroids without
 * reallocating: mu_j^[0] = x_{init_ids[j]}, no labels, every cluster moving,
 * first inverted file rebuilt (same as the tail of sivf_init).
 *   init_ids : HOST int32[k], distinct object ids. Copied.
 * Errors: SIVF_ERR_INVALID_ARG (ids), SIVF_ERR_CUDA.
 */
sivf_status sivf_reseed(sivf_ctx *ctx, const int32_t *init_ids);

/*
 * sivf_assign — one assignment step (Algorithm 4; Algorithm 2 when icp = 0,
 * Algorithm 3 when icp = 2, Algorithm 4 with the relaxed filter when icp = 3):
 * scores every object against the structured inverted file, takes the argmax
 * (largest score, lowest index on ties), and marks invariant clusters
 * (lambda_j^[r] = 1 iff no object entered or left cluster j).
 *   n_changed : HOST out, may be NULL; objects whose label changed.
 * Synchronises the stream. Two assignments must be separated by an update
 * (the inverted file is laid out for the lambda of the previous step):
 * otherwise SIVF_ERR_STATE, context unchanged.
 */
sivf_status sivf_assign(sivf_ctx *ctx, int64_t *n_changed);

/*
 * sivf_update — one update step (Algorithm 5): means of the moving clusters,
 * normalised to unit length and stored as FP32 (norm in FP64: dense form from
 * the exact 128-bit sum of the squared integer sums, values scaled in FP32
 * within 2.4e-7 of the exactly rounded quotient; sort form in FP64 throughout);
 * invariant and empty
 * clusters keep their centroid; the structured inverted file is rebuilt
 * (moving centroids in front, invariant behind, ascending ids in each part).
 * Requires at least one assignment (or sivf_set_labels) since sivf_init.
 */
sivf_status sivf_update(sivf_ctx *ctx);

/*
 * sivf_run — Algorithm 1 loop: assign, then update, until an assignment
 * (r > 1) changes no label or max_iter assignments have run. With use_graph,
 * iterations after the second run inside one CUDA graph (per-step device
 * times in sivf_stats are then those of the last host-launched step).
 *   iters_out     : HOST out, may be NULL; assignment steps run by this call.
 *   objective_out : HOST out, may be NULL; sum_j ||s_j|| of the last update
 *                   (the objective with the final centroids). At convergence
 *                   it equals J of the last assignment, which kept every label.
 */
sivf_status sivf_run(sivf_ctx *ctx, int32_t max_iter, int32_t *iters_out, double *objective_out);

/* sivf_get_labels — copy N labels to dst (DEVICE if dst_is_device, else HOST). */
sivf_status sivf_get_labels(sivf_ctx *ctx, int32_t *dst, int dst_is_device);

/*
 * sivf_set_labels — replace the labels (resume from a checkpoint, or lockstep
 * resynchronisation). src: N labels in [0, k) (DEVICE if src_is_device).
 * Clusters whose membership changes become moving; objects whose label
 * changes lose their stored own-cluster score and take the unfiltered branch
 * at the next assignment. Call sivf_update afterwards to rebuild the means.
 */
sivf_status sivf_set_labels(sivf_ctx *ctx, const int32_t *src, int src_is_device);

/*
 * sivf_get_centroids — cluster-major FP32 centroids (the master copy):
 *   off  : HOST int64[k+1] (always written),
 *   term : HOST int32[cap], u : HOST float[cap] (written if cap >= nnz),
 *   nnz_out : HOST, receives the centroid non-zero count.
 * Returns SIVF_ERR_INVALID_ARG (after writing off and nnz_out) if cap < nnz.
 */
sivf_status sivf_get_centroids(sivf_ctx *ctx, int64_t *off, int32_t *term, float *u, int64_t cap,
                               int64_t *nnz_out);

/*
 * sivf_get_inverted_file — the structured inverted file (Algorithm 5 output;
 * with icp = 2 the unstructured file of Algorithm 3, one part per list):
 *   off : HOST int64[D+1], mf0 : HOST int32[D] (front length),
 *   cid : HOST int32[cap], u : HOST float[cap] (FP32 values), nnz_out.
 * Same capacity rule as sivf_get_centroids.
 */
sivf_status sivf_get_inverted_file(sivf_ctx *ctx, int64_t *off, int32_t *mf0, int32_t *cid, float *u,
                                   int64_t cap, int64_t *nnz_out);

/* sivf_get_lambda — copy lambda^[r] (k bytes, 1 = invariant) to HOST dst. */
sivf_status sivf_get_lambda(sivf_ctx *ctx, uint8_t *dst);

/* sivf_get_stats — counters of the last assignment and update (HOST out). */
sivf_status sivf_get_stats(sivf_ctx *ctx, sivf_stats *out);

/* sivf_last_error — context-owned message of the last failure ("" if none);
 * valid until the next call on ctx. Accepts NULL (returns a static string). */
const char *sivf_last_error(const sivf_ctx *ctx);

/*
 * Batched independent instances (one context, one assignment launch and one
 * update per iteration for all of them).
 *
 * sivf_instance_desc — one clustering problem: N objects over D terms, k
 * clusters, its own CSR (DEVICE, same rules as sivf_init; copied at init,
 * so the caller may free it afterwards) and k distinct seed object ids
 * (HOST, local to the instance, copied).
 */
typedef struct {
    int64_t N;
    int32_t D;
    int32_t k;
    const int64_t *row_ptr;
    const int32_t *idx;
    const float *val;
    const int32_t *init_ids;
} sivf_instance_desc;

/*
 * sivf_batch_init — one context for n_inst independent instances. Internally
 * the instances are laid side by side (disjoint object, term and cluster
 * ranges); every assignment and update step covers all of them, and each
 * object is only compared with its own instance's centroids. sivf_assign,
 * sivf_update, sivf_get_stats and sivf_reseed (global seed ids, instance by
 * instance) work on the whole batch; the other getters see the concatenation.
 * Errors as sivf_init.
 */
sivf_status sivf_batch_init(sivf_ctx **out, const sivf_config *cfg, int32_t n_inst, const sivf_instance_desc *descs,
                            void *stream);

/*
 * sivf_batch_run — Algorithm 1 for every instance at once: iterate until each
 * instance has had an assignment (r > 1) that changes none of its labels, or
 * max_iter assignments. An instance that converged stays converged (all its
 * clusters are invariant, so its objects keep their labels at no scan cost).
 *   iters_out     : HOST int32[n_inst], may be NULL; the iteration r at which
 *                   the instance converged, counted from sivf_batch_init or
 *                   sivf_reseed (not from this call), or the context's
 *                   iteration count if it has not converged.
 *   objective_out : HOST double[n_inst], may be NULL; the instance's objective
 *                   sum of cosines at its last update.
 */
sivf_status sivf_batch_run(sivf_ctx *ctx, int32_t max_iter, int32_t *iters_out, double *objective_out);

/* sivf_batch_get_labels — instance inst's N labels, local cluster ids, to HOST dst. */
sivf_status sivf_batch_get_labels(sivf_ctx *ctx, int32_t inst, int32_t *dst);

/* sivf_batch_instance_stats — instance inst's changed count of the last
 * assignment and its objectives of the last update (HOST outs, may be NULL). */
sivf_status sivf_batch_instance_stats(sivf_ctx *ctx, int32_t inst, int64_t *changed, double *objective_assign,
                                      double *objective_update);

/* sivf_destroy — free all library-owned device memory. Accepts NULL. */
void sivf_destroy(sivf_ctx *ctx);

/*
 * Allocation-free inverted-file build. The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, such as
 * an inference-engine plugin whose execution step must not allocate, or a
 * service that reserves a fixed device-memory budget at start-up and cannot
 * call cudaMalloc on a request path (the call can fail under that budget and
 * it synchronises the device).
 *
 * sivf_build_inverted_file_noalloc — the structured inverted file that
 * sivf_update builds: for every term, the centroids holding it, moving ones
 * (lam[j] == 0) first and invariant ones (lam[j] == 1) after, ascending ids in
 * each part, with their values. It allocates nothing: its scratch is a
 * file-scope static device array of SIVF_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits.
 *   k, D      : clusters and terms; 1 <= k <= SIVF_NOALLOC_MAX_CLUSTERS,
 *               1 <= D <= SIVF_NOALLOC_MAX_TERMS.
 *   n_entries : HOST, total centroid non-zeros = coff[k];
 *               0 <= n_entries <= SIVF_NOALLOC_MAX_ENTRIES.
 *   coff      : DEVICE int64[k+1], cterm : DEVICE int32[n_entries] (ascending
 *               terms in each row, each in [0, D)), cval : DEVICE
 *               float[n_entries] — the cluster-major centroids
 *               (sivf_get_centroids layout).
 *   lam       : DEVICE uint8[k], 1 = invariant.
 *   if_off    : DEVICE int64[D+1] out, if_mf0 : DEVICE int32[D] out (front
 *               length), if_cid : DEVICE int32[n_entries] out,
 *               if_u : DEVICE float[n_entries] out. Caller-owned.
 *   stream    : cudaStream_t; all work is ordered on it. The call waits for
 *               the stream once, at its end, to read the result of its
 *               device-side checks.
 * Errors: SIVF_ERR_INVALID_ARG, with nothing launched, when a size is beyond
 * the limits above or a pointer is NULL; SIVF_ERR_INVALID_ARG after the
 * device-side checks when coff is not a valid offset array (coff[0] = 0,
 * non-decreasing, coff[k] = n_entries) or a term lies outside [0, D): the
 * outputs are then unspecified, and nothing outside the arrays above and the
 * scratch is touched; SIVF_ERR_CUDA on a CUDA failure.
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture begins. Every call reuses the same array and clears what
 * must start at zero; calls that overlap on the GPU race on it.
 */
#define SIVF_NOALLOC_MAX_ENTRIES (1 << 20)
#define SIVF_NOALLOC_MAX_TERMS (1 << 18)
#define SIVF_NOALLOC_MAX_CLUSTERS (1 << 20)
#define SIVF_NOALLOC_SCRATCH_BYTES (26u << 20)
sivf_status sivf_build_inverted_file_noalloc(int32_t k, int32_t D, int64_t n_entries, const int64_t *coff,
                                             const int32_t *cterm, const float *cval, const uint8_t *lam,
                                             int64_t *if_off, int32_t *if_mf0, int32_t *if_cid, float *if_u,
                                             void *stream);

/*
 * sivf_measure_read_bandwidth — streaming-read bandwidth of a device buffer,
 * measured with CUDA events on `stream`: the denominator of the assignment
 * scan's roofline when its posting stream is served by L2. The paper has no
 * counterpart (it measures on CPUs).
 *   buf     : DEVICE, 16-byte aligned, `bytes` readable bytes (only read).
 *   bytes   : >= 16; whole 16-byte vectors are read. A buffer that fits in L2
 *             (129 MB on GB300) measures L2 -> SM delivery, a larger one HBM.
 *   passes  : >= 1 timed passes over the buffer, after one untimed warm pass.
 *             Loads bypass L1 (ld.global.cg), and every SM reads a different
 *             slice in consecutive passes.
 *   gbs_out : HOST out, bytes read per second / 1e9; ms_out: HOST out (may be
 *             NULL), the timed duration.
 * Synchronises the stream. Errors: SIVF_ERR_INVALID_ARG (NULL, misaligned or
 * too small), SIVF_ERR_CUDA.
 */
sivf_status sivf_measure_read_bandwidth(const void *buf, int64_t bytes, int32_t passes, void *stream,
                                        double *gbs_out, double *ms_out);

#ifdef __cplusplus
}
#endif
#endif /* SIVF_H */
