/*
 * CPU oracle for s-line graphs of hypergraphs -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. The GPU library shares no code, header or table with it.
 *
 * What it computes, written out from the definitions of the paper
 * (Liu et al., "High-order Line Graphs of Non-uniform Hypergraphs"):
 *
 *   inc(e,f) = |e ∩ f|                                    (Section II-A)
 *   e, f are s-incident iff |e ∩ f| >= s, s >= 1          (Section II-B)
 *   L_s(H) has an edge {e_i, e_j} iff e_i, e_j s-incident (Section II-B)
 *   L = H^T H holds inc(e_i, e_j) off the diagonal        (Section II-B)
 *
 * The oracle's output is the strict upper triangle (i < j, the orientation
 * used throughout Section III and Stage 1 of Section IV) as triples
 * (i, j, |e_i ∩ e_j|) with overlap >= s, sorted by (i, j). Every overlap is
 * computed as the plain intersection size of two sorted vertex lists, i.e. the
 * "ijk" dot-product order of Section III-B / the naive all-pairs algorithm:
 * no hashing, no wedges, no pruning, no blocking. Rows are spread over POSIX
 * threads; each row's arithmetic is independent of the thread that runs it.
 *
 * Also here, each by its definition:
 *   - validation of the CSR input (hyperedges are sets, Section I);
 *   - the dual / transposed incidence H^T (Section II-A): adj(v) ascending;
 *   - the row digest used to compare TB-scale outputs by sampled rows:
 *       D_i = sum_k mix(mix((i<<32)|k) ^ ((j_k<<32)|o_k))   (mod 2^64)
 *     over the row's output entries k = 0..c_i-1 in ascending j, where mix is
 *     the SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ECAP 2

/* ---------------------------------------------------------------- helpers */

static uint64_t orc_mix(uint64_t x) {
    /* SplitMix64: add the golden-ratio increment, then two xor-shift-multiply
     * rounds and a final xor-shift. */
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t oracle_mix(uint64_t x) { return orc_mix(x); }

uint64_t oracle_pair_hash(int32_t i, int64_t k, int32_t j, int32_t o) {
    uint64_t a = orc_mix(((uint64_t)(uint32_t)i << 32) | (uint64_t)(uint32_t)k);
    return orc_mix(a ^ (((uint64_t)(uint32_t)j << 32) | (uint64_t)(uint32_t)o));
}

/* |a ∩ b| for two strictly increasing lists (merge of sorted lists). */
static int32_t orc_intersect(const int32_t* a, int32_t na, const int32_t* b, int32_t nb) {
    int32_t p = 0, q = 0, c = 0;
    while (p < na && q < nb) {
        if (a[p] < b[q]) {
            ++p;
        } else if (b[q] < a[p]) {
            ++q;
        } else {
            ++c;
            ++p;
            ++q;
        }
    }
    return c;
}

/* ------------------------------------------------------------- validation */

/* Returns 0 when off/idx describe m hyperedges over n vertices with every row
 * strictly increasing (a set, no repeated vertex), else ORC_EINVAL. */
int oracle_validate(const int32_t* off, const int32_t* idx, int32_t m, int32_t n) {
    if (m < 0 || n < 0 || off == NULL) return ORC_EINVAL;
    if (off[0] != 0) return ORC_EINVAL;
    for (int32_t i = 0; i < m; ++i) {
        if (off[i + 1] < off[i]) return ORC_EINVAL;
        for (int32_t p = off[i]; p < off[i + 1]; ++p) {
            if (idx[p] < 0 || idx[p] >= n) return ORC_EINVAL;
            if (p > off[i] && idx[p] <= idx[p - 1]) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ dual / H^T */

/* adj(v) = { i : v in e_i } in ascending i. offT has n+1 entries. */
void oracle_transpose(const int32_t* off, const int32_t* idx, int32_t m, int32_t n,
                      int32_t* offT, int32_t* idxT) {
    memset(offT, 0, sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < m; ++i)
        for (int32_t p = off[i]; p < off[i + 1]; ++p) offT[idx[p] + 1]++;
    for (int32_t v = 0; v < n; ++v) offT[v + 1] += offT[v];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    memcpy(fill, offT, sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < m; ++i) /* rows visited in ascending i */
        for (int32_t p = off[i]; p < off[i + 1]; ++p) idxT[fill[idx[p]]++] = i;
    free(fill);
}

/* ---------------------------------------------------- threaded row driver */

typedef struct {
    const int32_t* off;
    const int32_t* idx;
    int32_t m;
    const int32_t* rows; /* rows to evaluate (NULL = all rows 0..m-1) */
    int64_t nrows;
    const int32_t* s_list;
    int32_t ns;
    int32_t s_min;
    /* outputs, indexed [r * ns + t] for row r of the list and s_list[t] */
    int64_t* counts;    /* number of j > i with overlap >= s */
    uint64_t* digests;  /* row digest (see header) */
    int64_t* osum;      /* sum of overlaps over j > i with |e_j| >= s when |e_i| >= s */
    /* shared work cursor */
    int64_t next;
    pthread_mutex_t lock;
} orc_rows_job;

static void orc_one_row(orc_rows_job* J, int64_t r, int32_t* obuf, int32_t* jbuf) {
    const int32_t i = J->rows ? J->rows[r] : (int32_t)r;
    const int32_t* ei = J->idx + J->off[i];
    const int32_t ni = J->off[i + 1] - J->off[i];
    /* overlaps with every later hyperedge, ascending j */
    int32_t c = 0;
    for (int32_t j = i + 1; j < J->m; ++j) {
        const int32_t o = orc_intersect(ei, ni, J->idx + J->off[j], J->off[j + 1] - J->off[j]);
        if (o >= 1) {
            jbuf[c] = j;
            obuf[c] = o;
            ++c;
        }
    }
    for (int32_t t = 0; t < J->ns; ++t) {
        const int32_t s = J->s_list[t];
        int64_t cnt = 0, sum = 0;
        uint64_t d = 0;
        for (int32_t k = 0; k < c; ++k) {
            const int32_t j = jbuf[k];
            const int32_t o = obuf[k];
            if (o >= s) {
                d += oracle_pair_hash(i, cnt, j, o);
                ++cnt;
            }
            if (ni >= s && (J->off[j + 1] - J->off[j]) >= s) sum += o;
        }
        if (J->counts) J->counts[r * J->ns + t] = cnt;
        if (J->digests) J->digests[r * J->ns + t] = d;
        if (J->osum) J->osum[r * J->ns + t] = sum;
    }
}

static void* orc_rows_worker(void* arg) {
    orc_rows_job* J = (orc_rows_job*)arg;
    int32_t* obuf = (int32_t*)malloc(sizeof(int32_t) * ((size_t)J->m + 1));
    int32_t* jbuf = (int32_t*)malloc(sizeof(int32_t) * ((size_t)J->m + 1));
    for (;;) {
        pthread_mutex_lock(&J->lock);
        const int64_t r = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (r >= J->nrows) break;
        orc_one_row(J, r, obuf, jbuf);
    }
    free(obuf);
    free(jbuf);
    return NULL;
}

static void orc_run(orc_rows_job* J, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    pthread_mutex_init(&J->lock, NULL);
    J->next = 0;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_rows_worker, J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J->lock);
}

/* Per-row results for a list of rows (or all rows when rows == NULL) and for
 * every s in s_list at once: counts c_i(s), digests D_i(s) and the overlap sum
 * over E_s (equal to the row's wedge count W_{s,i} by double counting). Any
 * output pointer may be NULL. */
void oracle_rows(const int32_t* off, const int32_t* idx, int32_t m, const int32_t* rows,
                 int64_t nrows, const int32_t* s_list, int32_t ns, int64_t* counts,
                 uint64_t* digests, int64_t* osum, int nthreads) {
    orc_rows_job J;
    memset(&J, 0, sizeof(J));
    J.off = off;
    J.idx = idx;
    J.m = m;
    J.rows = rows;
    J.nrows = rows ? nrows : m;
    J.s_list = s_list;
    J.ns = ns;
    J.counts = counts;
    J.digests = digests;
    J.osum = osum;
    orc_run(&J, nthreads);
}

/* The full s-line graph edge list, sorted by (i, j): rows are emitted one
 * after another in ascending i, each in ascending j. Writes at most cap
 * triples; returns the total number of triples (so a short buffer can be
 * detected and the call repeated), or -1 on invalid arguments. */
int64_t oracle_slg(const int32_t* off, const int32_t* idx, int32_t m, int32_t s, int32_t* I,
                   int32_t* Jo, int32_t* O, int64_t cap) {
    if (s < 1) return -1;
    int64_t p = 0;
    for (int32_t i = 0; i < m; ++i) {
        const int32_t* ei = idx + off[i];
        const int32_t ni = off[i + 1] - off[i];
        for (int32_t j = i + 1; j < m; ++j) {
            const int32_t o = orc_intersect(ei, ni, idx + off[j], off[j + 1] - off[j]);
            if (o >= s) {
                if (p < cap) {
                    I[p] = i;
                    Jo[p] = j;
                    O[p] = o;
                }
                ++p;
            }
        }
    }
    return p;
}

/* One row's list (j ascending, overlap) at threshold s. Returns the row's
 * count; writes at most cap entries. */
int64_t oracle_row_list(const int32_t* off, const int32_t* idx, int32_t m, int32_t i, int32_t s,
                        int32_t* Jo, int32_t* O, int64_t cap) {
    const int32_t* ei = idx + off[i];
    const int32_t ni = off[i + 1] - off[i];
    int64_t p = 0;
    for (int32_t j = i + 1; j < m; ++j) {
        const int32_t o = orc_intersect(ei, ni, idx + off[j], off[j + 1] - off[j]);
        if (o >= s) {
            if (p < cap) {
                Jo[p] = j;
                O[p] = o;
            }
            ++p;
        }
    }
    return p;
}

/* Digest of an explicit (I, J, O) list: sum over entries of the pair hash,
 * with k the position of the entry inside its row (entries of a row must be
 * contiguous). Lets a test digest a list it holds in memory. */
uint64_t oracle_list_digest(const int32_t* I, const int32_t* Jo, const int32_t* O, int64_t P) {
    uint64_t d = 0;
    int64_t k = 0;
    for (int64_t p = 0; p < P; ++p) {
        k = (p > 0 && I[p] == I[p - 1]) ? k + 1 : 0;
        d += oracle_pair_hash(I[p], k, Jo[p], O[p]);
    }
    return d;
}

/* ----------------------------------------------- threaded full edge list */

typedef struct {
    const int32_t* off;
    const int32_t* idx;
    int32_t m;
    int32_t s;
    const int64_t* rowoff; /* where row i's list starts (from per-row counts) */
    int32_t* I;
    int32_t* J;
    int32_t* O;
    int64_t next;
    pthread_mutex_t lock;
} orc_fill_job;

static void* orc_fill_worker(void* arg) {
    orc_fill_job* F = (orc_fill_job*)arg;
    for (;;) {
        pthread_mutex_lock(&F->lock);
        const int64_t i = F->next++;
        pthread_mutex_unlock(&F->lock);
        if (i >= F->m) break;
        const int32_t* ei = F->idx + F->off[i];
        const int32_t ni = F->off[i + 1] - F->off[i];
        int64_t p = F->rowoff[i];
        for (int32_t j = (int32_t)i + 1; j < F->m; ++j) {
            const int32_t o = orc_intersect(ei, ni, F->idx + F->off[j], F->off[j + 1] - F->off[j]);
            if (o >= F->s) {
                F->I[p] = (int32_t)i;
                F->J[p] = j;
                F->O[p] = o;
                ++p;
            }
        }
    }
    return NULL;
}

/* Same list as oracle_slg, rows spread over threads: row i writes its
 * (i, j, overlap) triples, ascending j, from rowoff[i] on. rowoff comes from
 * the per-row counts of oracle_rows. */
void oracle_slg_fill_rows(const int32_t* off, const int32_t* idx, int32_t m, int32_t s,
                          const int64_t* rowoff, int32_t* I, int32_t* Jo, int32_t* O,
                          int nthreads) {
    orc_fill_job F;
    memset(&F, 0, sizeof(F));
    F.off = off;
    F.idx = idx;
    F.m = m;
    F.s = s;
    F.rowoff = rowoff;
    F.I = I;
    F.J = Jo;
    F.O = O;
    if (nthreads < 1) nthreads = 1;
    pthread_mutex_init(&F.lock, NULL);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_fill_worker, &F);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&F.lock);
}
