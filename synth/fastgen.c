/*
 * Fast member draws for the seeded synthetic hypergraphs (input generation
 * only; no s-line arithmetic). Shared by the tests, the oracle's inputs and the
 * benchmark, like the rest of the synth package.
 *
 * Row r takes the first size[r] distinct vertices of an i.i.d. sequence drawn
 * with probability proportional to weight[v] (sequential weighted sampling
 * without replacement, i.e. rejection of repeats), then is sorted. Draws use
 * Walker's alias method (Vose's construction); the random stream of row r is
 * SplitMix64 (Steele, Lea, Flood 2014) started from mix(key ^ mix(r + 1)), so
 * rows can be drawn in any order on any number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t fg_mix(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    uint64_t state;
} fg_rng;

static uint64_t fg_next(fg_rng* r) {
    r->state += 0x9E3779B97F4A7C15ull;
    uint64_t z = r->state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double fg_uniform(fg_rng* r) { return (double)(fg_next(r) >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    int32_t n;
    double* prob;   /* acceptance probability of column v */
    int32_t* alias; /* alternative of column v */
} fg_alias;

/* Vose's alias construction over weights w[0..n). Returns 0 on success. */
static int fg_alias_build(fg_alias* A, const double* w, int32_t n) {
    A->n = n;
    A->prob = (double*)malloc(sizeof(double) * (size_t)n);
    A->alias = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* small = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* large = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!A->prob || !A->alias || !p || !small || !large) return 1;
    double total = 0;
    for (int32_t v = 0; v < n; ++v) total += w[v];
    int32_t ns = 0, nl = 0;
    for (int32_t v = 0; v < n; ++v) {
        p[v] = w[v] * (double)n / total;
        if (p[v] < 1.0)
            small[ns++] = v;
        else
            large[nl++] = v;
    }
    while (ns > 0 && nl > 0) {
        const int32_t s = small[--ns], l = large[--nl];
        A->prob[s] = p[s];
        A->alias[s] = l;
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0)
            small[ns++] = l;
        else
            large[nl++] = l;
    }
    while (nl > 0) {
        const int32_t l = large[--nl];
        A->prob[l] = 1.0;
        A->alias[l] = l;
    }
    while (ns > 0) { /* rounding leftovers */
        const int32_t s = small[--ns];
        A->prob[s] = 1.0;
        A->alias[s] = s;
    }
    free(p);
    free(small);
    free(large);
    return 0;
}

static int32_t fg_alias_draw(const fg_alias* A, fg_rng* r) {
    const uint64_t x = fg_next(r);
    const int32_t col = (int32_t)(((x >> 32) * (uint64_t)A->n) >> 32);
    const double u = (double)(x & 0xffffffffu) * (1.0 / 4294967296.0);
    return u < A->prob[col] ? col : A->alias[col];
}

static int fg_cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

typedef struct {
    const fg_alias* A;
    const int64_t* sizes;
    const int64_t* off;
    int32_t* idx;
    int64_t m;
    uint64_t key;
    int64_t next;
    pthread_mutex_t lock;
    int64_t max_size;
} fg_job;

static void* fg_worker(void* arg) {
    fg_job* J = (fg_job*)arg;
    size_t cap = 16;
    while ((int64_t)cap < 2 * J->max_size + 2) cap <<= 1;
    int32_t* set = (int32_t*)malloc(sizeof(int32_t) * cap);
    const int64_t CH = 256;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        const int64_t r0 = J->next;
        J->next += CH;
        pthread_mutex_unlock(&J->lock);
        if (r0 >= J->m) break;
        const int64_t r1 = r0 + CH < J->m ? r0 + CH : J->m;
        for (int64_t r = r0; r < r1; ++r) {
            const int64_t k = J->sizes[r];
            int32_t* out = J->idx + J->off[r];
            if (k <= 0) continue;
            size_t hc = 16;
            while ((int64_t)hc < 2 * k) hc <<= 1;
            memset(set, 0xff, sizeof(int32_t) * hc);
            fg_rng g = {fg_mix(J->key ^ fg_mix((uint64_t)r + 1))};
            int64_t have = 0;
            while (have < k) {
                const int32_t v = fg_alias_draw(J->A, &g);
                size_t h = ((uint64_t)(uint32_t)v * 0x9E3779B97F4A7C15ull) >> 40;
                h &= hc - 1;
                for (;;) {
                    if (set[h] == v) break; /* repeat: rejected */
                    if (set[h] < 0) {
                        set[h] = v;
                        out[have++] = v;
                        break;
                    }
                    h = (h + 1) & (hc - 1);
                }
            }
            qsort(out, (size_t)k, sizeof(int32_t), fg_cmp_i32);
        }
    }
    free(set);
    return NULL;
}

/* Draws the members of m rows. sizes[r] <= number of vertices with positive
 * weight is required (the caller clamps sizes to n). off has m+1 entries and
 * must already hold the prefix sums of sizes. Returns 0 on success. */
int fastgen_members(int64_t m, const int64_t* sizes, const int64_t* off, const double* weights,
                    int32_t n, uint64_t key, int32_t* idx, int nthreads) {
    fg_alias A;
    if (fg_alias_build(&A, weights, n)) return 1;
    fg_job J;
    memset(&J, 0, sizeof(J));
    J.A = &A;
    J.sizes = sizes;
    J.off = off;
    J.idx = idx;
    J.m = m;
    J.key = key;
    for (int64_t r = 0; r < m; ++r)
        if (sizes[r] > J.max_size) J.max_size = sizes[r];
    if (nthreads < 1) nthreads = 1;
    pthread_mutex_init(&J.lock, NULL);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, fg_worker, &J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    free(A.prob);
    free(A.alias);
    return 0;
}
