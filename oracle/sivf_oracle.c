/*
 * FP64 CPU oracle for SIVF spherical k-means (Aoyama & Saito, arXiv 2103.16141).
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct
 * restatement of what the method computes. Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it. It shares no code, header
 * or helper with the CUDA implementation.
 *
 * Everything is double precision; input values (fp32) are promoted exactly.
 *
 * Two assignment modes:
 *   icp = 0 : inverted-file assignment without a filter (Algorithm 2): every
 *             posting of every term of the object is scored, argmax over all k.
 *   icp = 1 : SIVF assignment (Algorithm 4): if the object's cluster was
 *             invariant at the previous iteration, only the front (moving)
 *             segment of each posting list is scanned.
 *   icp = 2 : IVF-CBICP assignment (Algorithm 3): the same objects are
 *             filtered, but they traverse every posting of each list and a
 *             second branch, per posting, skips the invariant centroids. It
 *             reaches the same scores and labels; only the traversal differs.
 *   icp = 3 : SIVF with the relaxed filter the paper cites in Section 3
 *             (Bottesch et al.): an object whose own cluster moved is also
 *             restricted to the moving centroids when its similarity to its
 *             own centroid did not decrease (rho_new >= rho_old; the
 *             invariant centroids' similarities are unchanged, so none of
 *             them can overtake it). Tried while at most half of the
 *             clusters are moving. Same labels, fewer similarities.
 * The update step (Algorithm 5) is shared by both modes and always lays the
 * inverted file out in the structured form (moving centroids in front,
 * invariant centroids behind, ascending centroid id inside each part).
 *
 * Readings of places where the paper is silent or ambiguous:
 *   - Argmax ties go to the lowest centroid index; an all-zero score vector
 *     yields label 0 (the paper's strict ">" scan from j = 1 starting at
 *     rho_max = 0 leaves the label undefined in that case).
 *   - A filtered object keeps its own (invariant) cluster as a candidate, with
 *     the score carried from the previous iteration; otherwise Algorithm 4
 *     would never compare against the object's current centroid. The stored
 *     score is exact because that centroid has not changed.
 *   - lambda^[0] = lambda^[1] = 0 (no membership history yet).
 *   - An empty cluster keeps its previous centroid.
 *   - Algorithm 5 counts the parts of the file with lambda^[r] and places the
 *     postings with lambda^[r-1]; both use lambda^[r] here (otherwise the
 *     front/back counters overrun their parts).
 *   - Convergence: an assignment (r > 1) that changes no label.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct orc {
    int64_t N;
    int32_t D, k;
    const int64_t *row_ptr; /* borrowed */
    const int32_t *idx;
    const float *val;
    int icp;
    int iter; /* number of assignment steps done */

    /* centroids M^[r], cluster-major: row j = terms cen_term[cen_off[j]..cen_off[j+1]) */
    int64_t *cen_off;
    int32_t *cen_term;
    double *cen_val;
    double *cen_snorm; /* ||s_j|| of the last update (0 for seeds / empty) */

    /* structured inverted file of M^[r] */
    int64_t *if_off; /* D+1 */
    int32_t *if_mf0; /* D: length of the front (moving) part */
    int32_t *if_cid;
    double *if_u;

    uint8_t *lambda;    /* lambda^[r]: 1 = invariant */
    int32_t *labels;    /* a^[r], -1 before the first assignment */
    int32_t *prev_labels;
    double *own;        /* score of the object's own cluster, from its last assignment */
    uint8_t *own_ok;
    double *best, *second; /* top-2 candidate scores of the last assignment */
    uint8_t *filtered;  /* 1 if the object took the filtered branch */
} orc;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* Build the structured inverted file from the cluster-major centroids and
 * lambda (Algorithm 5, lines 1-14 for the counts, 21-30 for the placement). */
static int build_if(orc *o) {
    int32_t D = o->D, k = o->k;
    int32_t *mf0 = (int32_t *)xcalloc((size_t)D, sizeof(int32_t));
    int32_t *mf1 = (int32_t *)xcalloc((size_t)D, sizeof(int32_t));
    if (!mf0 || !mf1) { free(mf0); free(mf1); return -1; }
    for (int32_t j = 0; j < k; ++j) {
        for (int64_t q = o->cen_off[j]; q < o->cen_off[j + 1]; ++q) {
            int32_t p = o->cen_term[q];
            if (o->lambda[j] == 0) mf0[p] += 1; else mf1[p] += 1;
        }
    }
    int64_t *off = (int64_t *)xcalloc((size_t)D + 1, sizeof(int64_t));
    if (!off) { free(mf0); free(mf1); return -1; }
    for (int32_t p = 0; p < D; ++p) off[p + 1] = off[p] + mf0[p] + mf1[p];
    int64_t nnz = off[D];
    int32_t *cid = (int32_t *)xcalloc((size_t)nnz, sizeof(int32_t));
    double *u = (double *)xcalloc((size_t)nnz, sizeof(double));
    int64_t *q0 = (int64_t *)xcalloc((size_t)D, sizeof(int64_t));
    int64_t *q1 = (int64_t *)xcalloc((size_t)D, sizeof(int64_t));
    if (!cid || !u || !q0 || !q1) { free(mf0); free(mf1); free(off); free(cid); free(u); free(q0); free(q1); return -1; }
    for (int32_t p = 0; p < D; ++p) {
        q0[p] = off[p];
        q1[p] = off[p] + mf0[p];
    }
    for (int32_t j = 0; j < k; ++j) {
        for (int64_t q = o->cen_off[j]; q < o->cen_off[j + 1]; ++q) {
            int32_t p = o->cen_term[q];
            int64_t *pos = (o->lambda[j] == 0) ? &q0[p] : &q1[p];
            cid[*pos] = j;
            u[*pos] = o->cen_val[q];
            *pos += 1;
        }
    }
    free(o->if_off); free(o->if_mf0); free(o->if_cid); free(o->if_u);
    o->if_off = off;
    o->if_mf0 = mf0;
    o->if_cid = cid;
    o->if_u = u;
    free(mf1); free(q0); free(q1);
    return 0;
}

void orc_destroy(orc *o) {
    if (!o) return;
    free(o->cen_off); free(o->cen_term); free(o->cen_val); free(o->cen_snorm);
    free(o->if_off); free(o->if_mf0); free(o->if_cid); free(o->if_u);
    free(o->lambda); free(o->labels); free(o->prev_labels); free(o->own); free(o->own_ok);
    free(o->best); free(o->second); free(o->filtered);
    free(o);
}

/* Iteration 0: mu_j^[0] = x_{init_ids[j]} (Algorithm 1 input M^[0]). */
orc *orc_create(int64_t N, int32_t D, int32_t k, const int64_t *row_ptr, const int32_t *idx,
                const float *val, const int32_t *init_ids, int icp) {
    if (N < 1 || D < 1 || k < 1 || (int64_t)k > N || icp < 0 || icp > 3) return NULL;
    orc *o = (orc *)xcalloc(1, sizeof(orc));
    if (!o) return NULL;
    o->N = N; o->D = D; o->k = k;
    o->row_ptr = row_ptr; o->idx = idx; o->val = val;
    o->icp = icp;
    o->cen_off = (int64_t *)xcalloc((size_t)k + 1, sizeof(int64_t));
    o->cen_snorm = (double *)xcalloc((size_t)k, sizeof(double));
    o->lambda = (uint8_t *)xcalloc((size_t)k, 1);
    o->labels = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    o->prev_labels = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    o->own = (double *)xcalloc((size_t)N, sizeof(double));
    o->own_ok = (uint8_t *)xcalloc((size_t)N, 1);
    o->best = (double *)xcalloc((size_t)N, sizeof(double));
    o->second = (double *)xcalloc((size_t)N, sizeof(double));
    o->filtered = (uint8_t *)xcalloc((size_t)N, 1);
    if (!o->cen_off || !o->cen_snorm || !o->lambda || !o->labels || !o->prev_labels || !o->own ||
        !o->own_ok || !o->best || !o->second || !o->filtered) { orc_destroy(o); return NULL; }
    for (int32_t j = 0; j < k; ++j) {
        int32_t d = init_ids[j];
        if (d < 0 || d >= N) { orc_destroy(o); return NULL; }
        o->cen_off[j + 1] = o->cen_off[j] + (row_ptr[d + 1] - row_ptr[d]);
    }
    o->cen_term = (int32_t *)xcalloc((size_t)o->cen_off[k], sizeof(int32_t));
    o->cen_val = (double *)xcalloc((size_t)o->cen_off[k], sizeof(double));
    if (!o->cen_term || !o->cen_val) { orc_destroy(o); return NULL; }
    for (int32_t j = 0; j < k; ++j) {
        int32_t d = init_ids[j];
        int64_t w = o->cen_off[j];
        for (int64_t q = row_ptr[d]; q < row_ptr[d + 1]; ++q, ++w) {
            o->cen_term[w] = idx[q];
            o->cen_val[w] = (double)val[q];
        }
    }
    for (int64_t i = 0; i < N; ++i) o->labels[i] = -1;
    /* lambda^[0] = 0: every centroid sits in the front part */
    if (build_if(o) != 0) { orc_destroy(o); return NULL; }
    return o;
}

/*
 * Assignment step at iteration r (Algorithm 2 when icp = 0, Algorithm 4 when
 * icp = 1, Algorithm 3 when icp = 2). stats[0..7] = changed, n_moving
 * (lambda^[r] = 0 count), sim-calcs, postings visited (traversed, whether or
 * not accumulated), objective sum_i rho_{i,a(i)}, filtered objects, n_moving at
 * r-1, iteration r.
 */
int orc_assign(orc *o, double *stats) {
    const int64_t N = o->N;
    const int32_t k = o->k;
    const int r = o->iter + 1;
    int64_t n_moving_prev = 0;
    for (int32_t j = 0; j < k; ++j) n_moving_prev += (o->lambda[j] == 0);
    memcpy(o->prev_labels, o->labels, sizeof(int32_t) * (size_t)N);
    int64_t simcalc = 0, postings = 0, nfilt = 0;
    int err = 0;
#pragma omp parallel reduction(+ : simcalc, postings, nfilt)
    {
        double *rho = (double *)xcalloc((size_t)k, sizeof(double));
        if (!rho) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            if (!rho) continue;
            int32_t a_prev = o->prev_labels[i];
            /* Algorithm 4, line 6: branch once per object on lambda_{a(x_i)} */
            int filt = o->icp && a_prev >= 0 && o->own_ok[i] && o->lambda[a_prev] == 1;
            /* Relaxed filter (icp = 3): the own cluster moved, but the object
             * keeps to the moving centroids if its similarity to its own
             * centroid did not decrease; the own centroid is moving, so its new
             * score comes out of the front scan. Otherwise everything is
             * scanned again. It is tried only while at most half of the
             * clusters are moving (a rejected try scans the fronts twice). */
            int relax = o->icp == 3 && !filt && a_prev >= 0 && o->own_ok[i] && 2 * n_moving_prev <= k;
            for (int pass = 0; pass < 2; ++pass) {
                const int front = (filt || relax) && pass == 0;
                for (int32_t j = 0; j < k; ++j) rho[j] = 0.0;
                for (int64_t h = o->row_ptr[i]; h < o->row_ptr[i + 1]; ++h) {
                    int32_t s = o->idx[h];
                    double v = (double)o->val[h];
                    int64_t b = o->if_off[s];
                    if (filt && o->icp == 2) {
                        /* Algorithm 3: every posting, a branch on lambda of its centroid */
                        int64_t e = o->if_off[s + 1];
                        for (int64_t q = b; q < e; ++q)
                            if (o->lambda[o->if_cid[q]] == 0) rho[o->if_cid[q]] += v * o->if_u[q];
                        postings += e - b;
                        continue;
                    }
                    int64_t e = front ? b + o->if_mf0[s] : o->if_off[s + 1];
                    for (int64_t q = b; q < e; ++q) rho[o->if_cid[q]] += v * o->if_u[q];
                    postings += e - b;
                }
                if (relax && pass == 0) {
                    if (rho[a_prev] >= o->own[i]) break; /* accepted */
                    simcalc += n_moving_prev;            /* the front scan was wasted */
                    relax = 0;
                    continue;
                }
                break;
            }
            /* argmax: largest score, lowest index among equal scores */
            int32_t a = -1;
            double bst = 0.0, snd = -1.0;
            for (int32_t j = 0; j < k; ++j) {
                double x;
                if (filt) {
                    if (j == a_prev) x = o->own[i];
                    else if (o->lambda[j] == 0) x = rho[j];
                    else continue; /* invariant centroid: not a candidate */
                } else if (relax) {
                    if (o->lambda[j] == 0) x = rho[j];
                    else continue; /* the own centroid is among the moving ones */
                } else {
                    x = rho[j];
                }
                if (a < 0 || x > bst) {
                    if (a >= 0) snd = bst;
                    a = j;
                    bst = x;
                } else if (x > snd) {
                    snd = x;
                }
            }
            o->labels[i] = a;
            o->best[i] = bst;
            o->second[i] = snd;
            o->own[i] = bst;
            o->own_ok[i] = 1;
            o->filtered[i] = (uint8_t)(filt || relax);
            simcalc += (filt || relax) ? n_moving_prev : k;
            nfilt += filt || relax;
        }
        free(rho);
    }
    if (err) return -1;
    /* Algorithm 4, lines 17-19: lambda_j^[r] = 1 iff C_j^[r] = C_j^[r-1].
     * A cluster changes exactly when some object enters or leaves it. */
    int64_t changed = 0;
    if (r == 1) {
        memset(o->lambda, 0, (size_t)k);
        changed = N;
    } else {
        memset(o->lambda, 1, (size_t)k);
        for (int64_t i = 0; i < N; ++i) {
            int32_t a0 = o->prev_labels[i], a1 = o->labels[i];
            if (a0 != a1) {
                changed += 1;
                if (a0 >= 0) o->lambda[a0] = 0;
                o->lambda[a1] = 0;
            }
        }
    }
    int64_t n_moving = 0;
    for (int32_t j = 0; j < k; ++j) n_moving += (o->lambda[j] == 0);
    double obj = 0.0;
    for (int64_t i = 0; i < N; ++i) obj += o->best[i];
    o->iter = r;
    if (stats) {
        stats[0] = (double)changed;
        stats[1] = (double)n_moving;
        stats[2] = (double)simcalc;
        stats[3] = (double)postings;
        stats[4] = obj;
        stats[5] = (double)nfilt;
        stats[6] = (double)n_moving_prev;
        stats[7] = (double)r;
    }
    return 0;
}

/*
 * Update step (Algorithm 5). For each non-empty cluster j the mean of its
 * members is formed (lines 17-20) and normalised to unit length; the
 * structured inverted file is then rebuilt with lambda^[r]. An empty cluster
 * keeps its previous centroid. stats[0] = sum_j ||s_j|| (the objective after
 * the update, s_j = sum of the members of C_j), stats[1] = centroid nnz,
 * stats[2] = empty clusters.
 */
int orc_update(orc *o, double *stats) {
    const int64_t N = o->N;
    const int32_t D = o->D, k = o->k;
    /* members of each cluster in ascending object id */
    int64_t *moff = (int64_t *)xcalloc((size_t)k + 1, sizeof(int64_t));
    int64_t *mem = (int64_t *)xcalloc((size_t)N, sizeof(int64_t));
    int64_t *cur = (int64_t *)xcalloc((size_t)k, sizeof(int64_t));
    if (!moff || !mem || !cur) { free(moff); free(mem); free(cur); return -1; }
    for (int64_t i = 0; i < N; ++i) moff[o->labels[i] + 1] += 1;
    for (int32_t j = 0; j < k; ++j) moff[j + 1] += moff[j];
    for (int32_t j = 0; j < k; ++j) cur[j] = moff[j];
    for (int64_t i = 0; i < N; ++i) mem[cur[o->labels[i]]++] = i;
    free(cur);

    /* pass 1: support size of each new centroid */
    int64_t *noff = (int64_t *)xcalloc((size_t)k + 1, sizeof(int64_t));
    if (!noff) { free(moff); free(mem); return -1; }
    int err = 0;
#pragma omp parallel
    {
        uint8_t *mark = (uint8_t *)xcalloc((size_t)D, 1);
        if (!mark) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int32_t j = 0; j < k; ++j) {
            if (!mark) continue;
            if (moff[j + 1] == moff[j]) { /* empty: keep the previous centroid */
                noff[j + 1] = o->cen_off[j + 1] - o->cen_off[j];
                continue;
            }
            int64_t c = 0;
            for (int64_t m = moff[j]; m < moff[j + 1]; ++m) {
                int64_t i = mem[m];
                for (int64_t h = o->row_ptr[i]; h < o->row_ptr[i + 1]; ++h) {
                    int32_t s = o->idx[h];
                    if (!mark[s]) { mark[s] = 1; c += 1; }
                }
            }
            for (int64_t m = moff[j]; m < moff[j + 1]; ++m) {
                int64_t i = mem[m];
                for (int64_t h = o->row_ptr[i]; h < o->row_ptr[i + 1]; ++h) mark[o->idx[h]] = 0;
            }
            noff[j + 1] = c;
        }
        free(mark);
    }
    if (err) { free(moff); free(mem); free(noff); return -1; }
    for (int32_t j = 0; j < k; ++j) noff[j + 1] += noff[j];
    int32_t *nterm = (int32_t *)xcalloc((size_t)noff[k], sizeof(int32_t));
    double *nval = (double *)xcalloc((size_t)noff[k], sizeof(double));
    double *snorm = (double *)xcalloc((size_t)k, sizeof(double));
    if (!nterm || !nval || !snorm) { free(moff); free(mem); free(noff); free(nterm); free(nval); free(snorm); return -1; }

    /* pass 2: means (Algorithm 5, lines 17-20) and unit-length centroids */
#pragma omp parallel
    {
        double *w = (double *)xcalloc((size_t)D, sizeof(double));
        if (!w) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int32_t j = 0; j < k; ++j) {
            if (!w) continue;
            int64_t cnt = moff[j + 1] - moff[j];
            if (cnt == 0) {
                int64_t d = noff[j];
                for (int64_t q = o->cen_off[j]; q < o->cen_off[j + 1]; ++q, ++d) {
                    nterm[d] = o->cen_term[q];
                    nval[d] = o->cen_val[q];
                }
                snorm[j] = 0.0;
                continue;
            }
            for (int32_t p = 0; p < D; ++p) w[p] = 0.0;
            for (int64_t m = moff[j]; m < moff[j + 1]; ++m) { /* ascending object id */
                int64_t i = mem[m];
                for (int64_t h = o->row_ptr[i]; h < o->row_ptr[i + 1]; ++h) w[o->idx[h]] += (double)o->val[h];
            }
            /* ||s_j|| of the plain sum, accumulated over ascending term id */
            double ss = 0.0;
            for (int32_t p = 0; p < D; ++p) ss += w[p] * w[p];
            snorm[j] = sqrt(ss);
            /* mean w / |C_j|, then u = w / ||w|| (Algorithm 5, lines 20, 24, 29) */
            double wn = 0.0;
            for (int32_t p = 0; p < D; ++p) {
                w[p] = w[p] / (double)cnt;
                wn += w[p] * w[p];
            }
            wn = sqrt(wn);
            int64_t d = noff[j];
            for (int32_t p = 0; p < D; ++p) {
                if (w[p] != 0.0) {
                    nterm[d] = p;
                    nval[d] = w[p] / wn;
                    d += 1;
                }
            }
        }
        free(w);
    }
    if (err) { free(moff); free(mem); free(noff); free(nterm); free(nval); free(snorm); return -1; }
    int64_t nempty = 0;
    for (int32_t j = 0; j < k; ++j) nempty += (moff[j + 1] == moff[j]);
    free(o->cen_off); free(o->cen_term); free(o->cen_val); free(o->cen_snorm);
    o->cen_off = noff;
    o->cen_term = nterm;
    o->cen_val = nval;
    o->cen_snorm = snorm;
    free(moff);
    free(mem);
    if (build_if(o) != 0) return -1;
    if (stats) {
        double obj = 0.0;
        for (int32_t j = 0; j < k; ++j) obj += snorm[j];
        stats[0] = obj;
        stats[1] = (double)o->cen_off[k];
        stats[2] = (double)nempty;
    }
    return 0;
}

/* Replace a^[r] (resume / lockstep resynchronisation). lambda^[r] is
 * recomputed against a^[r-1] (every cluster moving before the second
 * assignment); objects whose label changes lose their stored own score and
 * take the unfiltered branch next time. */
int orc_set_labels(orc *o, const int32_t *labels) {
    for (int64_t i = 0; i < o->N; ++i)
        if (labels[i] < 0 || labels[i] >= o->k) return -1;
    for (int64_t i = 0; i < o->N; ++i) {
        if (o->labels[i] != labels[i]) {
            o->labels[i] = labels[i];
            /* its stored score belongs to the old cluster (the new one is
             * marked moving below, so the object is not filtered next time
             * in any case) */
            o->own_ok[i] = 0;
        }
    }
    if (o->iter <= 1) {
        memset(o->lambda, 0, (size_t)o->k);
        o->iter = 1;
        return 0;
    }
    memset(o->lambda, 1, (size_t)o->k);
    for (int64_t i = 0; i < o->N; ++i) {
        int32_t a0 = o->prev_labels[i], a1 = o->labels[i];
        if (a0 != a1) {
            if (a0 >= 0) o->lambda[a0] = 0;
            o->lambda[a1] = 0;
        }
    }
    return 0;
}

/* ---- accessors ---- */
int32_t orc_iter(const orc *o) { return o->iter; }
void orc_get_labels(const orc *o, int32_t *out) { memcpy(out, o->labels, sizeof(int32_t) * (size_t)o->N); }
void orc_get_scores(const orc *o, double *best, double *second, uint8_t *filtered) {
    memcpy(best, o->best, sizeof(double) * (size_t)o->N);
    memcpy(second, o->second, sizeof(double) * (size_t)o->N);
    memcpy(filtered, o->filtered, (size_t)o->N);
}
void orc_get_lambda(const orc *o, uint8_t *out) { memcpy(out, o->lambda, (size_t)o->k); }
int64_t orc_centroid_nnz(const orc *o) { return o->cen_off[o->k]; }
void orc_get_centroids(const orc *o, int64_t *off, int32_t *term, double *val, double *snorm) {
    memcpy(off, o->cen_off, sizeof(int64_t) * ((size_t)o->k + 1));
    memcpy(term, o->cen_term, sizeof(int32_t) * (size_t)o->cen_off[o->k]);
    memcpy(val, o->cen_val, sizeof(double) * (size_t)o->cen_off[o->k]);
    memcpy(snorm, o->cen_snorm, sizeof(double) * (size_t)o->k);
}
int64_t orc_if_nnz(const orc *o) { return o->if_off[o->D]; }
void orc_get_if(const orc *o, int64_t *off, int32_t *mf0, int32_t *cid, double *u) {
    memcpy(off, o->if_off, sizeof(int64_t) * ((size_t)o->D + 1));
    memcpy(mf0, o->if_mf0, sizeof(int32_t) * (size_t)o->D);
    memcpy(cid, o->if_cid, sizeof(int32_t) * (size_t)o->if_off[o->D]);
    memcpy(u, o->if_u, sizeof(double) * (size_t)o->if_off[o->D]);
}
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Unfiltered scores of selected objects against the current centroids
 * (Algorithm 2 scoring, no state change). For each listed object: label
 * (largest score, lowest index on ties), best and second-best score. */
int orc_score_objects(const orc *o, const int64_t *ids, int64_t n, int32_t *label, double *best,
                      double *second) {
    const int32_t k = o->k;
    int err = 0;
#pragma omp parallel
    {
        double *rho = (double *)xcalloc((size_t)k, sizeof(double));
        if (!rho) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t m = 0; m < n; ++m) {
            if (!rho) continue;
            int64_t i = ids[m];
            for (int32_t j = 0; j < k; ++j) rho[j] = 0.0;
            for (int64_t h = o->row_ptr[i]; h < o->row_ptr[i + 1]; ++h) {
                int32_t s = o->idx[h];
                double v = (double)o->val[h];
                for (int64_t q = o->if_off[s]; q < o->if_off[s + 1]; ++q) rho[o->if_cid[q]] += v * o->if_u[q];
            }
            int32_t a = 0;
            double bst = rho[0], snd = -1.0;
            for (int32_t j = 1; j < k; ++j) {
                if (rho[j] > bst) { snd = bst; bst = rho[j]; a = j; }
                else if (rho[j] > snd) snd = rho[j];
            }
            label[m] = a;
            best[m] = bst;
            second[m] = snd;
        }
        free(rho);
    }
    return err ? -1 : 0;
}
