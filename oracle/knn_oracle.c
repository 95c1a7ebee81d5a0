/*
 * knn_oracle.c -- the brute-force k-nearest-neighbour ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library; it reads plain float arrays and writes plain double/int arrays.
 *
 * What it computes (Garcia, Debreuve, Barlaud, "Fast k Nearest Neighbor Search
 * using GPU", Sec. 2.1 "Problem definition" and the brute-force algorithm
 * listed right after it):
 *
 *   R = {r_1..r_m}, Q = {q_1..q_n} in R^d.  For each query q_i:
 *     1. compute the distance from q_i to every r_j, j in [1, m];
 *     2. sort the m distances;
 *     3. keep the k reference points with the smallest distances;
 *     4. repeat for every query.
 *
 * Readings of points the paper leaves open (each one is listed with its
 * reason in the design notes of the repository):
 *   - arithmetic: every coordinate is widened to double and the distance is
 *     accumulated in double, coordinate 0 first, with no fused multiply-add
 *     (the build passes -ffp-contract=off), so the value is reproducible
 *     bit for bit on any IEEE-754 host;
 *   - Euclidean distance is sqrt(sum_t (q_t - r_t)^2); the sort compares the
 *     squared value (sqrt is monotone, but it can round two different squares
 *     to one double, so ordering on the square is the exact order);
 *   - Manhattan distance is sum_t |q_t - r_t|; infinity-norm distance is
 *     max_t |q_t - r_t| (the paper names both as admissible distances);
 *   - Mahalanobis distance (also named there) is sqrt(delta^T M delta) for
 *     delta = q - r and a given symmetric positive definite M (the inverse
 *     covariance), evaluated straight from that definition in double:
 *     sum over a of delta_a * (sum over b of M[a][b] * delta_b), both sums in
 *     ascending index order; the sort compares the quadratic form;
 *   - step 2 is a FULL sort of all m pairs (key, j) with ties broken by the
 *     smaller index j -- the paper's step 2 sorts everything, and the
 *     tie rule makes the result unique;
 *   - indices are 0-based (the paper's r_1..r_m is 1-based notation).
 *
 * Parity of its values is pinned by tests/test_oracle.py against hand-built
 * lattice cases (tests/golden/), brute force over permutations on tiny inputs,
 * closed forms and invariants; see that file.
 *
 * Mutants: building with -DORACLE_MUTANT=N plants one deliberate mistake so the
 * tests can show that the pins catch it.  A normal build defines nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

enum { ORACLE_L2 = 0, ORACLE_L1 = 1, ORACLE_LINF = 2 };

typedef struct {
    double key; /* squared L2, or L1, or Linf */
    int32_t j;  /* reference index, 0-based */
} oracle_pair;

/* Ascending by key, ties by the smaller reference index (reading c1). */
/* Threads of one call: nthreads when positive, else the OpenMP default.  Passed
 * to the parallel region alone, so one call's count does not carry over to the
 * next (omp_set_num_threads would). */
static int oracle_team(int32_t nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

static int oracle_pair_cmp(const void* a, const void* b) {
    const oracle_pair* x = (const oracle_pair*)a;
    const oracle_pair* y = (const oracle_pair*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
#if ORACLE_MUTANT == 3
    /* mutant 3: reversed tie-break */
    return (x->j < y->j) ? 1 : (x->j > y->j ? -1 : 0);
#else
    return (x->j < y->j) ? -1 : (x->j > y->j ? 1 : 0);
#endif
}

/* Distance key between one query and one reference (step 1 of the algorithm). */
static double oracle_key(const float* q, const float* r, int32_t d, int metric) {
    double acc = 0.0;
#if ORACLE_MUTANT == 1
    d = d - 1; /* mutant 1: drops the last coordinate's term */
#endif
    for (int32_t t = 0; t < d; ++t) {
#if ORACLE_MUTANT == 2
        double diff = (double)q[t] + (double)r[t]; /* mutant 2: wrong sign */
#else
        double diff = (double)q[t] - (double)r[t];
#endif
        if (metric == ORACLE_L2) {
            acc = acc + diff * diff;
        } else if (metric == ORACLE_L1) {
            acc = acc + fabs(diff);
        } else {
            double a = fabs(diff);
            if (a > acc) acc = a;
        }
    }
    return acc;
}

/*
 * oracle_knn: the brute-force algorithm above for n queries against m
 * references.  R is m x d and Q is n x d, row-major float.  Writes, for each
 * query i, the first k entries of the fully sorted list into
 * dist_out[i*k + s] (the distance, i.e. sqrt of the key for L2) and
 * idx_out[i*k + s].  Returns 0 on success, -1 on invalid arguments, -2 when
 * a scratch allocation fails.  nthreads <= 0 uses the OpenMP default.
 */
int oracle_knn(const float* R, int64_t m, const float* Q, int64_t n, int32_t d,
               int32_t k, int32_t metric, double* dist_out, int32_t* idx_out,
               int32_t nthreads) {
    if (m < 1 || n < 0 || d < 1 || k < 1 || k > m) return -1;
    if (metric < ORACLE_L2 || metric > ORACLE_LINF) return -1;
    if (n == 0) return 0;
    if (!R || !Q || !dist_out || !idx_out) return -1;
    int failed = 0;
    const int team = oracle_team(nthreads);
    (void)team;
#pragma omp parallel num_threads(team)
    {
        oracle_pair* pairs = (oracle_pair*)malloc((size_t)m * sizeof(oracle_pair));
        if (!pairs) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; ++i) {
            if (!pairs) continue;
#if ORACLE_MUTANT == 4
            const float* q = R + (i % m) * d; /* mutant 4: operands swapped */
#else
            const float* q = Q + i * d;
#endif
            for (int64_t j = 0; j < m; ++j) {
                pairs[j].key = oracle_key(q, R + j * d, d, metric);
                pairs[j].j = (int32_t)j;
            }
            qsort(pairs, (size_t)m, sizeof(oracle_pair), oracle_pair_cmp);
            for (int32_t s = 0; s < k; ++s) {
                double key = pairs[s].key;
                dist_out[i * k + s] = (metric == ORACLE_L2) ? sqrt(key) : key;
                idx_out[i * k + s] = pairs[s].j;
            }
        }
        free(pairs);
    }
    return failed ? -2 : 0;
}

/*
 * oracle_key_pairs: the raw key (squared L2, L1 or Linf, in double) for an
 * explicit list of (query, reference) pairs.  Used by the tests to sample
 * single distances of a large problem without sorting all of it.
 */
int oracle_key_pairs(const float* R, int64_t m, const float* Q, int64_t n, int32_t d,
                     int32_t metric, const int64_t* qi, const int64_t* rj,
                     int64_t npairs, double* key_out) {
    if (m < 1 || n < 1 || d < 1 || npairs < 0) return -1;
    for (int64_t p = 0; p < npairs; ++p) {
        if (qi[p] < 0 || qi[p] >= n || rj[p] < 0 || rj[p] >= m) return -1;
        key_out[p] = oracle_key(Q + qi[p] * d, R + rj[p] * d, d, metric);
    }
    return 0;
}

/*
 * oracle_knn_subset: oracle_knn for the queries listed in qsel only (each a
 * row index into Q).  Output rows follow the order of qsel.  This is how the
 * tests check sampled queries of a full-size problem.
 */
int oracle_knn_subset(const float* R, int64_t m, const float* Q, int64_t n, int32_t d,
                      int32_t k, int32_t metric, const int64_t* qsel, int64_t nsel,
                      double* dist_out, int32_t* idx_out, int32_t nthreads) {
    if (nsel < 0 || n < 1) return -1;
    if (nsel == 0) return 0;
    float* Qs = (float*)malloc((size_t)nsel * (size_t)d * sizeof(float));
    if (!Qs) return -2;
    for (int64_t s = 0; s < nsel; ++s) {
        if (qsel[s] < 0 || qsel[s] >= n) { free(Qs); return -1; }
        memcpy(Qs + s * d, Q + qsel[s] * d, (size_t)d * sizeof(float));
    }
    int rc = oracle_knn(R, m, Qs, nsel, d, k, metric, dist_out, idx_out, nthreads);
    free(Qs);
    return rc;
}

/* The quadratic form delta^T M delta of one query and one reference, M a
 * d x d row-major double matrix (the Mahalanobis key; see the header). */
static double oracle_mahalanobis_key(const float* q, const float* r, int32_t d, const double* M) {
    double acc = 0.0;
    for (int32_t a = 0; a < d; ++a) {
        const double da = (double)q[a] - (double)r[a];
        double inner = 0.0;
        for (int32_t b = 0; b < d; ++b) {
#if ORACLE_MUTANT == 5
            /* mutant 5: off-diagonal terms dropped */
            const double mab = (a == b) ? M[(size_t)a * d + b] : 0.0;
#else
            const double mab = M[(size_t)a * d + b];
#endif
            inner = inner + mab * ((double)q[b] - (double)r[b]);
        }
        acc = acc + da * inner;
    }
    return acc;
}

/*
 * oracle_knn_mahalanobis: the brute-force algorithm under the Mahalanobis
 * distance with matrix M (d x d, row-major double, symmetric positive
 * definite).  Outputs as oracle_knn: dist = sqrt(key), ascending by (key,
 * index).  Returns 0, -1 on invalid arguments, -2 on allocation failure.
 */
int oracle_knn_mahalanobis(const float* R, int64_t m, const float* Q, int64_t n, int32_t d,
                           const double* M, int32_t k, double* dist_out, int32_t* idx_out,
                           int32_t nthreads) {
    if (m < 1 || n < 0 || d < 1 || k < 1 || k > m) return -1;
    if (n == 0) return 0;
    if (!R || !Q || !M || !dist_out || !idx_out) return -1;
    int failed = 0;
    const int team = oracle_team(nthreads);
    (void)team;
#pragma omp parallel num_threads(team)
    {
        oracle_pair* pairs = (oracle_pair*)malloc((size_t)m * sizeof(oracle_pair));
        if (!pairs) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; ++i) {
            if (!pairs) continue;
            const float* q = Q + i * d;
            for (int64_t j = 0; j < m; ++j) {
                pairs[j].key = oracle_mahalanobis_key(q, R + j * d, d, M);
                pairs[j].j = (int32_t)j;
            }
            qsort(pairs, (size_t)m, sizeof(oracle_pair), oracle_pair_cmp);
            for (int32_t s = 0; s < k; ++s) {
                dist_out[i * k + s] = sqrt(pairs[s].key);
                idx_out[i * k + s] = pairs[s].j;
            }
        }
        free(pairs);
    }
    return failed ? -2 : 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
