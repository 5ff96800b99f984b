/*
 * Seeded synthetic tf-idf corpus generator (input preparation only).
 *
 * Produces sparse, L2-normalised document vectors shaped like the paper's
 * PubMed / NYT tf-idf sets (Section 5.1): a vocabulary of D terms whose
 * frequencies follow Zipf(s), document lengths drawn from a lognormal,
 * tf = 1 + Poisson(1), value = tf * ln(N / df), rows sorted by term id and
 * normalised in double precision, stored as float.
 *
 * This file holds no clustering arithmetic. Both the FP64 oracle and the
 * CUDA path consume the arrays it writes.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Each document draws from its
 * own stream, seeded from (seed, document id), so results do not depend on the
 * thread count or on the host architecture.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *g) {
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, 1): 53 random bits, offset by half an ulp so 0 never occurs */
static double sm64_unif(sm64 *g) {
    return ((double)(sm64_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static sm64 stream_for(uint64_t seed, uint64_t salt, uint64_t id) {
    sm64 g;
    g.s = seed * 0xD1B54A32D192ED03ULL ^ (salt * 0x8CB92BA72F3D8DD7ULL) ^ (id + 0x632BE59BD9B4E019ULL);
    /* decorrelate nearby ids */
    (void)sm64_next(&g);
    (void)sm64_next(&g);
    return g;
}

/* standard normal by the Box-Muller transform */
static double normal01(sm64 *g) {
    double u1 = sm64_unif(g), u2 = sm64_unif(g);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Poisson(1) by sequential inversion of its CDF */
static int poisson1(sm64 *g) {
    double u = sm64_unif(g);
    double p = exp(-1.0), c = p;
    int k = 0;
    while (u > c && k < 64) {
        k += 1;
        p /= (double)k;
        c += p;
    }
    return k;
}

/*
 * Document lengths: L = round(exp(mu + sigma * Z)), clipped to [lo, hi] and
 * to at most D / 2 distinct terms.
 */
void synth_lengths(int64_t N, int32_t D, double mu, double sigma, int32_t lo, int32_t hi,
                   uint64_t seed, int32_t *len_out) {
    int32_t cap = D / 2 > 1 ? D / 2 : 1;
    if (hi > cap) hi = cap;
    if (lo > hi) lo = hi;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        sm64 g = stream_for(seed, 1, (uint64_t)i);
        double L = floor(exp(mu + sigma * normal01(&g)) + 0.5);
        if (L < lo) L = lo;
        if (L > hi) L = hi;
        len_out[i] = (int32_t)L;
    }
}

/* k distinct ids from [0, N): partial Fisher-Yates over an index array */
int synth_init_ids(int64_t N, int32_t k, uint64_t seed, int32_t *out) {
    if (k < 0 || (int64_t)k > N) return -1;
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!a) return -2;
    for (int64_t i = 0; i < N; ++i) a[i] = (int32_t)i;
    sm64 g = stream_for(seed, 7, 0);
    for (int32_t j = 0; j < k; ++j) {
        uint64_t r = sm64_next(&g) % (uint64_t)(N - j);
        int64_t p = j + (int64_t)r;
        int32_t t = a[j];
        a[j] = a[p];
        a[p] = t;
        out[j] = a[j];
    }
    free(a);
    return 0;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Fill rows. row_ptr has N+1 entries built from synth_lengths. Writes sorted
 * term ids into idx and tf counts into tf (int32, same length as idx).
 * Term frequencies follow Zipf(s) over ranks 1..D; a seeded random
 * permutation maps ranks to term ids so frequent terms are not contiguous.
 */
int synth_terms(int64_t N, int32_t D, double s, uint64_t seed, const int64_t *row_ptr,
                int32_t *idx, int32_t *tf) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)D);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)D);
    if (!cdf || !perm) {
        free(cdf);
        free(perm);
        return -2;
    }
    double acc = 0.0;
    for (int32_t r = 0; r < D; ++r) {
        acc += pow((double)(r + 1), -s);
        cdf[r] = acc;
    }
    for (int32_t r = 0; r < D; ++r) cdf[r] /= acc;
    cdf[D - 1] = 1.0;
    for (int32_t r = 0; r < D; ++r) perm[r] = r;
    {
        sm64 g = stream_for(seed, 3, 0);
        for (int32_t r = D - 1; r > 0; --r) {
            int32_t p = (int32_t)(sm64_next(&g) % (uint64_t)(r + 1));
            int32_t t = perm[r];
            perm[r] = perm[p];
            perm[p] = t;
        }
    }
    int err = 0;
#pragma omp parallel
    {
        uint8_t *seen = (uint8_t *)calloc((size_t)D, 1);
        if (!seen) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < N; ++i) {
            if (!seen) continue;
            sm64 g = stream_for(seed, 2, (uint64_t)i);
            int64_t b = row_ptr[i], e = row_ptr[i + 1];
            int64_t n = 0;
            while (b + n < e) {
                double u = sm64_unif(&g);
                /* smallest rank r with cdf[r] >= u */
                int32_t lo = 0, hi = D - 1;
                while (lo < hi) {
                    int32_t mid = lo + (hi - lo) / 2;
                    if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
                }
                int32_t t = perm[lo];
                if (seen[t]) continue; /* rejection of repeats */
                seen[t] = 1;
                idx[b + n] = t;
                n += 1;
            }
            for (int64_t q = b; q < e; ++q) seen[idx[q]] = 0;
            qsort(idx + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
            for (int64_t q = b; q < e; ++q) tf[q] = 1 + poisson1(&g);
        }
        free(seen);
    }
    free(cdf);
    free(perm);
    return err;
}

/*
 * tf-idf weighting and row normalisation. df[t] = number of rows holding t.
 * value = tf * ln(N / df); a term held by every row has value 0 and is dropped,
 * so every stored value is strictly positive. Rows are compacted in place:
 * new_row_ptr receives the compacted offsets. Each row is L2-normalised in
 * double precision and stored as float. Returns the new nnz.
 */
int64_t synth_tfidf(int64_t N, int32_t D, const int64_t *row_ptr, int32_t *idx, const int32_t *tf,
                    float *val, int64_t *new_row_ptr) {
    int64_t *df = (int64_t *)calloc((size_t)D, sizeof(int64_t));
    if (!df) return -2;
    int64_t nnz = row_ptr[N];
    for (int64_t q = 0; q < nnz; ++q) df[idx[q]] += 1;
    /* pass 1: surviving entries per row */
    new_row_ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t c = 0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) c += (df[idx[q]] < N);
        new_row_ptr[i + 1] = new_row_ptr[i] + c;
    }
    /* pass 2: weight, normalise in double, compact (entries only move toward
     * the front, and each is read before its slot can be overwritten) */
    for (int64_t i = 0; i < N; ++i) {
        double ss = 0.0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            int32_t t = idx[q];
            if (df[t] >= N) continue;
            double x = (double)tf[q] * log((double)N / (double)df[t]);
            ss += x * x;
        }
        double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
        int64_t w = new_row_ptr[i];
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            int32_t t = idx[q];
            if (df[t] >= N) continue;
            double x = (double)tf[q] * log((double)N / (double)df[t]);
            idx[w] = t;
            val[w] = (float)(x * inv);
            w += 1;
        }
    }
    free(df);
    return new_row_ptr[N];
}
