/*
 * libslg -- s-line graphs of non-uniform hypergraphs on one GB300 (sm_103a).
 *
 * C ABI. Plain pointers and sizes only; no C++ or framework types cross this
 * boundary. Every call returns an slg_status (0 = SLG_OK); on failure the
 * calling thread's message is available from slg_last_error().
 *
 * The problem (Liu et al., "High-order Line Graphs of Non-uniform
 * Hypergraphs", arXiv 2201.11326):
 *   - a hypergraph H = <V, E> has n vertices and an indexable family of m
 *     hyperedges e_0..e_{m-1}, each a subset of V; two hyperedges with equal
 *     vertex sets are distinct by index (Section I);
 *   - e_i and e_j are s-incident when |e_i ∩ e_j| >= s, s >= 1 (Section II-B);
 *   - the s-line graph L_s(H) joins every s-incident pair; its weighted form
 *     is L = H^T H with the diagonal ignored (Section II-B);
 *   - Algorithm 2 (Section III-C) states the computation: input (H, s),
 *     output the edge list of L_s(H), each pair once (i < j).
 *
 * Conventions shared by every call:
 *   - Input incidence: int32 CSR over hyperedges. off[m+1] with off[0] = 0
 *     and off non-decreasing; idx[off[m]] with row i = idx[off[i]..off[i+1])
 *     listing the vertices of e_i in strictly increasing order, each in
 *     [0, n). Rows may be empty; vertices need not be covered.
 *   - Output: the canonical edge list of L_s(H): triples (I[p], J[p], O[p])
 *     with I[p] < J[p], O[p] = |e_I ∩ e_J| >= s (the exact overlap, not capped
 *     at s), sorted by (I, J), as three int32 arrays (structure of arrays).
 *     Hyperedge ids are the caller's 0-based ids; there is no relabelling.
 *   - Pointers to arrays may be host memory (pageable or pinned) or device
 *     memory of the current device; the library detects which. The caller
 *     keeps ownership of every array it passes in; the library never frees
 *     or retains them past the call.
 *   - All device work of a graph runs on the CUDA stream given to slg_load
 *     (NULL = the legacy default stream). Calls that return host-visible
 *     results synchronise that stream before returning.
 *   - A graph handle is not thread-safe; distinct handles are independent.
 */
#ifndef SLG_H
#define SLG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t slg_status;

#define SLG_OK 0
#define SLG_EINVAL 1    /* bad argument: malformed CSR, s < 1, bad range, NULL */
#define SLG_ENOMEM 2    /* device memory exhausted */
#define SLG_ECUDA 3     /* a CUDA runtime error (message in slg_last_error) */
#define SLG_ETIMEOUT 4  /* a bounded device wait gave up */
#define SLG_ECAPACITY 5 /* caller's output buffer too small; *pairs holds the need */
#define SLG_EBUSY 6     /* resource in use */
#define SLG_EINTERNAL 7 /* an internal consistency check failed */

typedef struct slg_graph slg_graph;

/* Message describing the last failure on the calling thread ("" if none).
 * The string stays valid until the next libslg call on the same thread. */
const char* slg_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t slg_version(void);

/*
 * slg_load -- upload and validate a hypergraph, build its dual.
 *
 * Implements the input side of Algorithm 2 (Section III-C) and the dual /
 * transposed incidence H^T of Section II-A, which the "ikj" order of
 * Section III-B walks (for k in H^T.Adj[i], for j in H.Adj[k]).
 *
 *   off, idx  : CSR as described above (m+1 and off[m] int32 entries), host
 *               or device memory; copied, the caller may free them after.
 *   m, n      : number of hyperedges and vertices (m, n >= 0).
 *   stream    : cudaStream_t (as void*) for all device work of this graph.
 *   out       : receives the new handle (release with slg_free).
 *
 * Errors: SLG_EINVAL if the CSR is malformed (off[0] != 0, a decreasing
 * offset, an id outside [0, n), a row not strictly increasing -- which
 * includes a repeated vertex, since hyperedges are sets), SLG_ENOMEM,
 * SLG_ECUDA. On error *out is NULL and nothing is retained.
 */
slg_status slg_load(const int32_t* off, const int32_t* idx, int32_t m, int32_t n,
                    void* stream, slg_graph** out);

/* Release a handle and all its device memory. NULL is ignored. */
void slg_free(slg_graph* g);

/* Sizes of a loaded graph (any output may be NULL). */
slg_status slg_graph_info(const slg_graph* g, int32_t* m, int32_t* n, int64_t* nnz);

/*
 * slg_transpose_copy -- copy out the dual incidence H^T (Section II-A):
 * offT[n+1] and idxT[nnz] where adj(v) = idxT[offT[v]..offT[v+1]) lists the
 * hyperedges containing v in increasing id. Host or device destinations.
 */
slg_status slg_transpose_copy(slg_graph* g, int32_t* offT, int32_t* idxT);

/*
 * slg_dual -- the dual hypergraph H* (Section II-A: vertices and hyperedges
 * swap roles, incidence H^T) as a new handle. Its s-line graphs are the
 * s-clique graphs of H (Section III-H: vertices u, v joined when they share at
 * least s hyperedges, i.e. the off-diagonal of W = H H^T - D_V thresholded at
 * s), with vertex ids as row ids. Built from the device-resident transpose
 * (no host copy); release with slg_free. Errors as slg_load; SLG_EINVAL for a
 * batch.
 */
slg_status slg_dual(slg_graph* g, void* stream, slg_graph** out);

/*
 * slg_count -- exact size of L_s(H) and the algorithmic work, without
 * writing the list (the counting half of Algorithm 2, Section III-C).
 *
 *   pairs  : receives |L_s(H)|, the number of pairs i < j with
 *            |e_i ∩ e_j| >= s (may be NULL).
 *   wedges : receives W_s = sum over v of C(d_s(v), 2), where d_s(v) counts
 *            the hyperedges of size >= s containing v: the number of
 *            increments of the overlap counters of Algorithm 2 when both
 *            sides are pruned to E_s (Section III-E) (may be NULL).
 * Errors: SLG_EINVAL for s < 1.
 */
slg_status slg_count(slg_graph* g, int32_t s, int64_t* pairs, int64_t* wedges);

/*
 * slg_bound -- cheap upper bound floor(W_s / s) on |L_s(H)|: every s-incident
 * pair accounts for at least s wedges (Section III-E). Needs no counting pass.
 */
slg_status slg_bound(slg_graph* g, int32_t s, int64_t* pairs_ub);

/*
 * slg_row_offsets -- per-row output offsets of L_s(H): rowoff[i] is the
 * position of row i's first pair in the canonical list, rowoff[m] = |L_s|.
 * rowoff has m+1 int64 entries (host or device).
 */
slg_status slg_row_offsets(slg_graph* g, int32_t s, int64_t* rowoff);

/*
 * slg_build -- the whole edge list of L_s(H) (Algorithm 2, Section III-C).
 *
 *   I, J, O : output arrays of at least cap int32 entries each, host or
 *             device memory (all three of the same kind).
 *   cap     : capacity in pairs.
 *   pairs   : receives |L_s(H)|.
 * Errors: SLG_ECAPACITY when |L_s(H)| > cap (*pairs is set, nothing is
 * written), SLG_EINVAL for s < 1.
 */
slg_status slg_build(slg_graph* g, int32_t s, int32_t* I, int32_t* J, int32_t* O, int64_t cap,
                     int64_t* pairs);

/*
 * slg_build_window -- the pairs of rows [row_begin, row_end) only: the
 * contiguous slice rowoff[row_begin]..rowoff[row_end] of the canonical list.
 * Lets a list larger than device memory be produced in pieces; rows are the
 * independent units of Algorithm 2's parallel loop (Section III-C).
 *
 *   digest      : if not NULL, receives the sum over the slice of
 *                 mix(mix((i<<32)|k) ^ ((j<<32)|o)) mod 2^64, with k the
 *                 position of the pair inside its row and mix the SplitMix64
 *                 output function (Steele, Lea, Flood 2014).
 *   row_digests : if not NULL, receives the same sum per row
 *                 (row_end - row_begin uint64 entries, host or device).
 * Errors: SLG_EINVAL for a bad range or s < 1; SLG_ECAPACITY as slg_build.
 */
slg_status slg_build_window(slg_graph* g, int32_t s, int32_t row_begin, int32_t row_end,
                            int32_t* I, int32_t* J, int32_t* O, int64_t cap, int64_t* pairs,
                            uint64_t* digest, uint64_t* row_digests);

/*
 * slg_plan_windows -- split rows [0, m) into consecutive windows whose pair
 * count is at most cap each: row_splits[0] = 0 < ... < row_splits[w] = m.
 * A single row with more than cap pairs makes the call fail with
 * SLG_ECAPACITY (*nwindows = 0). row_splits (host) holds max_windows + 1
 * entries; SLG_ECAPACITY also when more than max_windows windows are needed
 * (*nwindows is then set to the number needed).
 */
slg_status slg_plan_windows(slg_graph* g, int32_t s, int64_t cap, int32_t* row_splits,
                            int32_t max_windows, int32_t* nwindows);

/*
 * Ensembles (Algorithm 3, Section III-D): the s-line graphs of one hypergraph
 * for several thresholds s_list[0] < s_list[1] < ... < s_list[k-1]. Algorithm
 * 3 counts the overlaps once (pruned by the smallest s) and then filters the
 * counted pairs once per threshold. Here one plan, pruned by s_list[0], serves
 * every list: one counting pass counts every list, and the fills write the
 * lists of a row window one after another, or one selected list.
 *
 * Every ensemble call takes the same (s_list, k), with 1 <= k <=
 * SLG_ENSEMBLE_MAX and s_list strictly ascending, s_list[0] >= 1. The counts
 * are cached per handle until another s or list is used. Errors: SLG_EINVAL for
 * a bad list or a batch handle.
 *
 * slg_ensemble_count -- pairs[t] = |L_{s_list[t]}(H)| (k entries, may be
 * NULL); wedges = W_{s_list[0]} (may be NULL).
 */
#define SLG_ENSEMBLE_MAX 16
slg_status slg_ensemble_count(slg_graph* g, const int32_t* s_list, int32_t k, int64_t* pairs,
                              int64_t* wedges);

/*
 * slg_ensemble_row_offsets -- rowoff[t*(m+1) + i] is row i's first position in
 * the canonical list of L_{s_list[t]}(H) (k*(m+1) int64 entries, host or
 * device).
 */
slg_status slg_ensemble_row_offsets(slg_graph* g, const int32_t* s_list, int32_t k,
                                    int64_t* rowoff);

/*
 * slg_ensemble_plan_windows -- as slg_plan_windows for the lists selected by
 * `which`: SLG_ENSEMBLE_ALL (-1) sizes a window by the sum of its pairs over
 * the k lists, t in [0, k) by list t alone.
 */
#define SLG_ENSEMBLE_ALL (-1)
slg_status slg_ensemble_plan_windows(slg_graph* g, const int32_t* s_list, int32_t k, int32_t which,
                                     int64_t cap, int32_t* row_splits, int32_t max_windows,
                                     int32_t* nwindows);

/*
 * slg_ensemble_build_window -- the pairs of rows [row_begin, row_end).
 *
 * which = SLG_ENSEMBLE_ALL: every list, back to back in I, J, O (cap entries
 * each, host or device, all of one kind): list t occupies positions seg_t ..
 * seg_t + pairs[t] - 1, seg_t = pairs[0] + ... + pairs[t-1]. Each list is
 * filled from the shared plan and counts by its own pass.
 * which = t in [0, k): list t alone, at positions 0 .. pairs[0] - 1.
 * Each list is the contiguous slice of its canonical list (sorted by (i, j)).
 *
 *   pairs       : k entries (ALL) or 1 entry (one list): the pair counts.
 *   digests     : NULL or as many entries as pairs: digests as in
 *                 slg_build_window.
 *   row_digests : NULL or (entries of pairs) * (row_end - row_begin) entries,
 *                 list-major.
 * Errors: SLG_ECAPACITY when the selected lists together exceed cap (pairs is
 * set, nothing is written); SLG_EINVAL as above, for a bad range or a bad
 * `which`.
 */
slg_status slg_ensemble_build_window(slg_graph* g, const int32_t* s_list, int32_t k, int32_t which,
                                     int32_t row_begin, int32_t row_end, int32_t* I, int32_t* J,
                                     int32_t* O, int64_t cap, int64_t* pairs, uint64_t* digests,
                                     uint64_t* row_digests);

/*
 * slg_ensemble_stream_window -- the lists window after window, each
 * sparse-accumulator and hub-pair row walked once (Algorithm 2, Section
 * III-C, counts a row's pairs and emits them from one pass over its wedges;
 * Algorithm 3, Section III-D, gives every threshold from one count).
 *
 * No counting pass over the whole graph comes first: the rows of a window are
 * chosen before they are walked, from an upper bound on their pairs (the
 * exact count for table and dense rows, counted once before the first window;
 * W_i / s_list[0] for sparse-accumulator rows; walked entries / (s_list[0] - 1)
 * for hub-pair rows), scaled by what the windows before observed. The
 * window's sparse-accumulator and hub-pair items are walked once, counting and
 * staging their pairs in a pool (slg_set_staging; 5 bytes per pair, about
 * 5 * cap bytes); their offsets are a scan of the window's counts; the pairs
 * are then copied into place (items the pool could not hold are walked again).
 * List t > 0 of the window is list t-1 filtered by s_list[t] (the lists are
 * nested and in the same order). If the rows' pairs exceed cap after all, the
 * window ends at the last row that fits.
 *
 *   s_list, k : 1 <= k <= SLG_ENSEMBLE_MAX ascending thresholds >= 1 (one
 *               graph, not a batch).
 *   r0        : the window's first row: 0, then the previous call's *r1.
 *   I, J, O   : device arrays (of the current device) of cap pairs, written
 *               with every list of rows [r0, *r1) back to back, each in
 *               canonical (i, j) order; the caller owns them.
 *   r1        : out: the end of the window's rows; r0 < *r1 <= m unless r0 == m
 *               (then *r1 == m and nothing is written).
 *   pairs     : out: k entries, the pairs of each list in the window.
 * Windows of consecutive calls cover the rows once each, in order, and their
 * lists concatenated are the lists of slg_ensemble_build. The plan for
 * s_list[0] and the bounds are built by the first call and kept with the graph
 * (another s, another call on the graph's plan, slg_set_bins, slg_free release
 * them); the counts of the regular calls are recomputed after this one.
 * Errors: SLG_EINVAL (NULL argument, bad s_list or r0, cap < 1, host or another
 * GPU's arrays, a batch); SLG_ECAPACITY when one row's lists exceed cap
 * (nothing is returned for it); SLG_ENOMEM; SLG_ECUDA; SLG_EINTERNAL when a
 * device consistency check fails.
 */
slg_status slg_ensemble_stream_window(slg_graph* g, const int32_t* s_list, int32_t k, int32_t r0,
                                      int32_t* I, int32_t* J, int32_t* O, int64_t cap,
                                      int32_t* r1, int64_t* pairs);

/* slg_stream_window -- slg_ensemble_stream_window for the one threshold s. */
slg_status slg_stream_window(slg_graph* g, int32_t s, int32_t r0, int32_t* I, int32_t* J,
                             int32_t* O, int64_t cap, int32_t* r1, int64_t* pairs);

/*
 * Phase timing. When enabled, the library records CUDA events on the graph's
 * stream around each phase; slg_last_timing then returns, for the last
 * counting pass and the last fill, ms[0..4] = planning (pruning, per-row
 * work, binning), counting pass, scan of the counts, fill pass, digest.
 */
slg_status slg_set_timing(slg_graph* g, int32_t enable);
slg_status slg_last_timing(slg_graph* g, float* ms5);

/*
 * Number of handlers (SLG_NMODES): 0 = warp table, 1 = CTA table, 2 = CTA
 * dense tiles, 3 = warp dense tiles, 4 = CTA sparse accumulator, 5 = warp
 * sparse accumulator (hash rounds), 6 = hub pairs (see slg_set_hub_pairs).
 *
 * Per-handler kernel time accumulated while timing is enabled:
 * ms[pass*SLG_NMODES + mode] and launches[pass*SLG_NMODES + mode] (2 *
 * SLG_NMODES entries each), pass 0 = counting, 1 = fill. reset != 0 zeroes
 * the totals after reading. Either output may be NULL.
 */
#define SLG_NMODES 7
slg_status slg_kernel_stats(slg_graph* g, int32_t reset, float* ms, int64_t* launches);

/*
 * Work per handler for s (runs the counting pass if needed):
 * out[mode * SLG_MODE_STATS_COLS + c] (SLG_MODE_STATS_COLS * SLG_NMODES
 * entries), summed over the rows the handler takes, with c =
 *   0 rows, 1 wedges, 2 incidences (sum of |e_i|), 3 output pairs,
 *   4 wedges through non-hub vertices (the dense handlers read adj_s entries
 *     for these only; a hub's share of an overlap is a popcount of two hub
 *     masks),
 *   5 candidate partners the dense handlers' extraction scans in the counting
 *     pass (one 4-byte hub mask read each; 0 for the other handlers),
 *   6 the same for the fill, which skips work items without pairs.
 * The wedge total over the handlers is W_s.
 */
#define SLG_MODE_STATS_COLS 7
slg_status slg_mode_stats(slg_graph* g, int32_t s, int64_t* out);

/* The same per handler for list `which` of an ensemble (Algorithm 3, Section
 * III-D; see slg_ensemble_count): rows and wedges of the shared plan (built for
 * s_list[0]), that list's pairs, and the partners its fill scans. Column 5 is
 * the one counting pass shared by every list. */
slg_status slg_ensemble_mode_stats(slg_graph* g, const int32_t* s_list, int32_t k, int32_t which,
                                   int64_t* out);

/*
 * slg_batch_load -- many hypergraphs, each with its own s, as one handle.
 *
 * Rows are the independent units of Algorithm 2's parallel loop (Section
 * III-C), and hyperedges of different members share no vertex, so the s-line
 * graph of the members' disjoint union is the union of their s-line graphs,
 * each member with its own threshold. The union is assembled on the device
 * from the members' already-built incidence and dual; one plan, one counting
 * pass and one fill per window then serve all members.
 *
 *   gs     : k loaded member graphs (they stay owned by the caller and must
 *            outlive the call; the batch copies what it needs).
 *   s      : k thresholds (host), each >= 1.
 *   stream : cudaStream_t (as void*) for the batch's device work.
 *   out    : receives the batch handle (release with slg_free).
 *
 * On a batch handle every call that takes s must be given s = 0 ("each
 * member's own s"); any other value is SLG_EINVAL. Rows are numbered member by
 * member (member b's rows start at row_base[b], see slg_batch_info), so the
 * batch's canonical list is the members' lists one after another; inside it
 * I and J hold member-local hyperedge ids, and digests hash member-local ids,
 * so a member's slice is identical to what its own handle produces.
 * Errors: SLG_EINVAL (k < 1, NULL member, s < 1, more than 2^31 rows,
 * vertices or incidences in total), SLG_ENOMEM, SLG_ECUDA.
 */
slg_status slg_batch_load(slg_graph* const* gs, const int32_t* s, int32_t k, void* stream,
                          slg_graph** out);

/* Members of a batch: *k and row_base[0..k] (host), member b owning rows
 * row_base[b] .. row_base[b+1]-1 of the batch. SLG_EINVAL if not a batch. */
slg_status slg_batch_info(const slg_graph* b, int32_t* k, int32_t* row_base);

/* pair_base[0..k] (host): member b's pairs occupy positions pair_base[b] ..
 * pair_base[b+1]-1 of the batch's list. Runs the counting pass if needed. */
slg_status slg_batch_pair_offsets(slg_graph* b, int64_t* pair_base);

/*
 * slg_batch -- the s-line graphs of k hypergraphs, each with its own
 * threshold, in one call: for every member b, Algorithm 2's statement (input
 * (H_b, s[b]), output the edge list of L_{s[b]}(H_b), Section III-C), with the
 * members run together as one batch (slg_batch_load: one plan, one counting
 * pass and one fill per window over all members).
 *
 *   gs, s, k : as slg_batch_load; the device work runs on gs[0]'s stream.
 *   results  : k entries. Before the call the caller sets want_list (nonzero:
 *              return the member's list); the call fills in the rest.
 *
 * Per member: pairs = |L_s|, wedges = W_s, digest = the digest of the whole
 * list as slg_build_window defines it (member-local ids, so it equals what
 * the member's own handle gives). With want_list, I/J/O receive host arrays of
 * `pairs` int32 entries allocated by the library (canonical order, member-local
 * ids; NULL when pairs = 0); release them with slg_result_free. Lists pass
 * through a device window of at most 2^27 pairs (or the largest row).
 * Errors: as slg_batch_load; SLG_ENOMEM also when a wanted list does not fit
 * host memory (no member then keeps a list). On any error every result's
 * status holds the error and no list is kept.
 */
typedef struct {
    int32_t want_list;  /* in: nonzero to receive the list in I/J/O */
    slg_status status;  /* out */
    int64_t pairs;      /* out: |L_s(H)| */
    int64_t wedges;     /* out: W_s */
    uint64_t digest;    /* out: digest of the whole list */
    int32_t* I;         /* out: host arrays (library-allocated) or NULL */
    int32_t* J;
    int32_t* O;
} slg_result;

slg_status slg_batch(slg_graph* const* gs, const int32_t* s, int32_t k, slg_result* results);

/* Release the lists of a result (I, J, O become NULL). NULL is ignored. */
void slg_result_free(slg_result* r);

/*
 * Serving: s-line queries (graph, s) over resident hypergraphs.
 *
 * The paper's ensembles compute many s-line graphs of one hypergraph
 * (Algorithm 3, Section III-D; Section V). A server keeps registered graphs on
 * the device and runs queries on `workers` threads, each with its own CUDA
 * stream and streaming window, so queries overlap on the device (a query uses
 * a private plan over the shared graph arrays). A query whose predicted result
 * 12 * floor(W_s / s) bytes (every s-incident pair accounts for at least s
 * wedges, Section III-E) is at most max_result_pairs pairs is kept on the
 * device until released, and is admitted only when its prediction fits in
 * memory_budget minus the results already held; larger results are streamed
 * through the worker's window (window_pairs pairs, allocated at creation,
 * outside the budget) and return counts and digest only. Pending queries are
 * taken in submission order (policy 0) or smallest predicted W_s first
 * (policy 1), skipping one that does not fit yet; small_workers of the workers
 * take only queries predicted at most small_wedges wedges, so that short
 * queries are not queued behind long ones. With batch_max > 1, a worker that
 * takes a small query (W_s <= small_wedges, s <= max_s) also takes up to
 * batch_max - 1 more pending small queries that fit, of any graphs and s, and
 * runs them as one batch (slg_batch_load: one plan, one counting pass, one
 * fill); each query's result, counts and digest are the same as when it runs
 * alone. A batch finishes as a whole, so its members are the smallest pending
 * small queries, each predicted at most 4 times the first query's W_s (or at
 * most 2^26 wedges). Queries that arrive while others run join the next batch
 * (continuous batching).
 */
typedef struct slg_server slg_server;

typedef struct {
    int64_t memory_budget;    /* bytes for kept results */
    int64_t window_pairs;     /* pairs per streaming window, one window per worker */
    int64_t max_result_pairs; /* larger results are streamed, not kept */
    int32_t workers;          /* concurrent queries (host threads, CUDA streams) */
    int32_t max_s;            /* W_s is precomputed for s = 1..max_s at registration */
    int32_t digest;           /* nonzero: compute each result's digest (slg_build_window) */
    int32_t policy;           /* 0: submission order; 1: smallest predicted W_s first */
    int32_t small_workers;    /* workers that only take queries with W_s <= small_wedges */
    int32_t batch_max;        /* small queries run together, at most this many (<= 1: none) */
    int64_t small_wedges;     /* threshold of small queries (small workers, batching) */
} slg_serve_cfg;

typedef struct {
    slg_status status;
    int32_t materialized; /* 1: the list is kept (slg_serve_fetch); 0: streamed */
    int64_t pairs;        /* |L_s| */
    int64_t wedges;       /* W_s */
    uint64_t digest;      /* digest of the whole list (if cfg.digest) */
    double latency_us;    /* submit -> done */
    double queue_us;      /* submit -> start */
    int32_t batch_size;   /* queries of the batch it ran in (1: it ran alone) */
} slg_serve_result;

typedef struct {
    int64_t completed;
    double p50_us, p99_us, mean_us, max_us; /* latency, submit -> done */
    double span_s;                          /* first submit -> last completion */
    double queries_per_s, pairs_per_s, wedges_per_s;
    int64_t peak_memory;                    /* bytes of kept results, at most */
    int64_t pending;
    int64_t running;
    int64_t batched;          /* queries completed inside a batch of two or more */
    int64_t batches;          /* such batches */
    int64_t batch_overflows;  /* batches whose lists exceeded the window: run one by one */
    int64_t batch_failures;   /* batches that failed and were run one by one (the last
                                 reason is then in slg_last_error after this call) */
} slg_serve_stats_t;

/* Create a server on the current device (starts the worker threads). */
slg_status slg_serve_create(const slg_serve_cfg* cfg, slg_server** out);
/* Stop the workers (queries still pending are dropped) and free everything. */
void slg_serve_destroy(slg_server* srv);
/* Register a loaded graph (not a batch); it must outlive the server. Computes
 * W_s for s = 1..max_s. */
slg_status slg_serve_register(slg_server* srv, slg_graph* g, int32_t* graph_id);
/* Queue a query; SLG_ECAPACITY if its kept result could never fit the budget. */
slg_status slg_serve_submit(slg_server* srv, int32_t graph_id, int32_t s, uint64_t* ticket);
/* Wait up to timeout_ms for a query; SLG_ETIMEOUT if it has not finished. */
slg_status slg_serve_poll(slg_server* srv, uint64_t ticket, int32_t timeout_ms,
                          slg_serve_result* out);
/* Copy a kept result (canonical list) into I/J/O (host or device, cap pairs). */
slg_status slg_serve_fetch(slg_server* srv, uint64_t ticket, int32_t* I, int32_t* J, int32_t* O,
                           int64_t cap);
/* Forget a finished query and free its kept result. */
slg_status slg_serve_release(slg_server* srv, uint64_t ticket);
/* Latency percentiles and throughput of the queries finished since the last
 * reset (reset != 0 starts a new period). */
slg_status slg_serve_stats(slg_server* srv, int32_t reset, slg_serve_stats_t* out);

/* Number of CUDA kernels this library has launched in this process. */
int64_t slg_kernel_launches(void);

/*
 * slg_scan_counts_noalloc -- exclusive prefix sum of per-row pair counts
 * into int64 output offsets (offsets[0] = 0, offsets[n] = total), the step
 * that places each row's pairs in a count-then-fill list, for callers that
 * cannot allocate device memory. The paper has no counterpart: its output
 * lists are merged host-side containers.
 *
 * Who needs it: a caller whose process has handed all device memory to
 * another allocator (a serving runtime or framework that reserves HBM up
 * front, so a further cudaMalloc fails or steals its budget), or a caller
 * on a latency-critical path that cannot afford cudaMalloc/cudaFree, which
 * may synchronise the whole device. This call performs no device
 * allocation of any kind: its scratch (the per-tile sums) is a fixed
 * 264 KiB array compiled into the library, present on every GPU that loads
 * it until the process exits.
 *
 *   counts  : n int32 per-row counts, memory of the current device.
 *   offsets : n+1 int64 outputs, memory of the current device (caller-owned).
 *   n       : 0 <= n <= 67,108,864; larger n fails with SLG_EINVAL and
 *             launches nothing.
 *   stream  : cudaStream_t (as void*) for the kernels; the call returns
 *             after enqueueing them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture begins. The address is cached for the life of
 * the process: do not use this call after resetting the device
 * (cudaDeviceReset), which invalidates it. All calls on a device share the one
 * array: every call writes each tile sum before reading it, so nothing needs
 * clearing, but calls whose kernels overlap on the GPU (e.g. on two
 * streams) race on it and must be serialised by the caller.
 * Errors: SLG_EINVAL (size above the limit, NULL or host pointers, or
 * memory of a device other than the current one), SLG_ECUDA.
 */
slg_status slg_scan_counts_noalloc(const int32_t* counts, int64_t* offsets, int64_t n,
                                   void* stream);

/*
 * Binning of rows into work items (replaces the relabel-by-degree and the
 * blocked/cyclic ranges of Sections III-F and IV). A row with W_i wedges and
 * candidate span S_i (last minus first partner id, plus one) is handled
 *   - by one warp with a 256-slot table when W_i <= warp_max_wedges (<= 128);
 *   - by a dense j-tiled handler when 256 * W_i >= dense_min_density * S_i
 *     (or S_i <= 4096); dense_min_density < 0 disables it. A dense row with
 *     at most wdense_max_ranges (<= 32; 0 disables) wedge ranges through
 *     non-hub vertices goes to the warp-level dense handler (items of
 *     8192 * dense_item_tiles ids), other dense rows to the CTA-level one
 *     (items of 32768 * dense_item_tiles ids);
 *   - by a sparse accumulator (8-bit counters over id tiles and a list of the
 *     counters touched) when |e_i| <= 255 and W_i >= sparse_min_per_tile *
 *     ceil(S_i / 65536) (< 0 disables it), in items of about
 *     sparse_item_wedges wedges: one warp with 4096-id tiles when |e_i| <=
 *     wsparse_max_size (<= 32; 0 disables it), 32 * W_i < S_i and s >= 2,
 *     else one CTA with 65536-id tiles;
 *   - otherwise by CTA hash tables, about block_item_wedges wedges per item.
 * Results do not depend on these values; only speed does. Resets the plan.
 * SLG_ECAPACITY from a later call when a binning needs 2^31 items or more.
 */
slg_status slg_set_bins(slg_graph* g, int32_t warp_max_wedges, int32_t block_item_wedges,
                        int32_t dense_min_density, int32_t dense_item_tiles,
                        int32_t wdense_max_ranges, int32_t sparse_min_per_tile,
                        int32_t sparse_item_wedges, int32_t wsparse_max_size);

/*
 * slg_set_hub_pairs -- the hub-pair handler for sparse rows at s >= 2.
 *
 * Algorithm 2 (Section III-C) counts every wedge (i, v, j). A pair with
 * overlap >= s >= 2 shares either a vertex outside the max_hubs highest-degree
 * vertices ("hubs") or at least two hubs. So for s >= 2 a row's partners can be
 * taken from its wedges through non-hub vertices and from the lists of rows
 * holding a pair of its hubs (built once per graph: the transpose of every
 * row's hub pairs); a partner sharing t hubs appears in t(t-1)/2 of those
 * lists, which gives t, and one look at the partner's hubs settles t <= 1.
 * Pairs that share a single hub and nothing else are never visited. The result
 * is the same list; only the work changes. A row (|e_i| <= 255, not dense)
 * uses the handler when its hub-pair work is at most half its wedges.
 *
 *   max_hubs          : hubs of the index, at most 4096 (fewer when the index
 *                       would exceed about 1.9e9 entries or the free device
 *                       memory); 0 disables the handler. Default 4096.
 *   min_sparse_wedges : the index is built by the first plan for s >= 2 whose
 *                       table and sparse-accumulator rows carry at least this
 *                       many wedges (default 2^33); 0 builds it whenever such
 *                       rows exist.
 * Releases the plan and any index built before. Not available on batches or
 * on a server's views.
 */
slg_status slg_set_hub_pairs(slg_graph* g, int32_t max_hubs, int64_t min_sparse_wedges);

/*
 * slg_set_ensemble_filter -- how slg_ensemble_build_window with which =
 * SLG_ENSEMBLE_ALL produces the lists after the first.
 *
 * Algorithm 3's lists are nested and in the same (i, j) order, so list t holds
 * exactly the pairs of list t-1 with overlap >= s_list[t]. In a window holding
 * every list, list t can be taken from list t-1's segment by a filter (16
 * bytes read per pair of list t-1) instead of walking the window's rows again
 * (about 4 bytes per entry read: wedges through vertices that are not mask
 * hubs, and the walked entries of hub-pair rows).
 *   mode : -1 (default) whichever reads less: the filter when 6 * (pairs of list
 *          t-1 in the window) < the entries a walk of the window's rows reads;
 *          0 always walk; 1 always filter.
 * The lists are the same either way.
 */
slg_status slg_set_ensemble_filter(slg_graph* g, int32_t mode);

/*
 * slg_ensemble_fill_stats -- how the windows of every list (slg_ensemble_build_
 * window with which = SLG_ENSEMBLE_ALL, and slg_ensemble_stream_window, whose
 * list 0 counts as walked) made each list since the handle was loaded or last
 * reset: out[6 * t + c] for list index t < SLG_ENSEMBLE_MAX
 * (6 * SLG_ENSEMBLE_MAX entries, caller-owned host memory; NULL skips the
 * copy), c = 0 windows walked by the fill, 1 pairs they wrote, 2 windows
 * filtered from list t-1, 3 pairs the filter wrote, 4 the filter's device
 * time in microseconds (count, scan and write, CUDA events on the graph's
 * stream), accumulated only while slg_set_timing is on, 5 pairs of list t-1
 * the filter read. reset != 0 zeroes
 * the counters after the copy. Host-side counters: no device work, no error
 * besides a NULL graph (SLG_EINVAL).
 */
slg_status slg_ensemble_fill_stats(slg_graph* g, int32_t reset, int64_t* out);

/*
 * slg_set_staging -- one walk instead of two for the sparse-accumulator and
 * hub-pair rows.
 *
 * Algorithm 2 (Section III-C) counts each row's pairs, the offsets are a scan
 * of the counts, and each row is then walked again to write its pairs. For the
 * sparse-accumulator and hub-pair rows the counting pass may instead run their
 * writing kernels: each item's pairs go, in canonical order, into a staging
 * pool on the device (in chunks of 2^20 pairs per CTA) along with its count;
 * once the pool is spent the remaining items are counted as usual. A window
 * (slg_build_window, slg_build) then copies its staged items into place and
 * walks only the others. Results are identical with or without staging.
 *
 *   max_bytes : -1 (default) automatic: three quarters of the free device
 *               memory beyond 6 GiB (5 bytes per pair plus 8 bytes per work
 *               item), at most 2^34 pairs, and no more than the rows can fill
 *               (the entries they walk, plus a chunk per CTA); made only when
 *               the rows can fill at least 2^26 pairs, and only while the
 *               automatic pools of all handles stay under a quarter of the
 *               device's memory; 0 disables staging; > 0 caps the pool at this
 *               many bytes (made at any size).
 * CTAs take chunks of 2^12 to 2^20 pairs (a quarter CTA's share of what the
 * rows can fill); no pool is made below 16 chunks (automatic) or one chunk
 * (capped). The pool is allocated by each counting pass of a plan that has
 * such rows and released with the plan (a new s, slg_set_bins, slg_free). A
 * server's queries and batch handles (slg_batch_load, slg_batch) do not stage
 * unless this call turns it on. Releases the current plan.
 */
slg_status slg_set_staging(slg_graph* g, int64_t max_bytes);

/*
 * slg_staging_stats -- the last counting pass's staging: out4 = {pool size
 * in pairs, chunk size in pairs, items staged, work items of the plan}; zeros
 * (but the items) when it staged nothing or the plan is not counted.
 */
slg_status slg_staging_stats(slg_graph* g, int64_t* out4);

/*
 * slg_autotune -- choose the binning thresholds of slg_set_bins for s on this
 * graph by measurement (the paper tunes its ranges, chunking and relabelling by
 * hand, Sections III-F and IV). Coordinate descent from the current thresholds:
 * each knob in turn is tried over a short list of values, keeping any value
 * that lowers the time. A trial times, with CUDA events on the graph's stream,
 * the planning, the counting pass and the fill of sample row windows spread over
 * the graph (at most 2^26 pairs, written to a 768 MiB scratch buffer).
 *
 *   s          : the threshold to tune for (0 for a batch handle).
 *   max_trials : at most this many trials (the first times the current
 *                thresholds); a trial costs about one counting pass.
 *   bins_out   : NULL or 8 int32 entries: the chosen thresholds, in
 *                slg_set_bins' argument order.
 *   ms_out     : NULL or the chosen thresholds' trial time in ms.
 * The thresholds stay set on the handle; results never depend on them.
 * Errors: SLG_EINVAL for a bad s or max_trials < 1.
 */
slg_status slg_autotune(slg_graph* g, int32_t s, int32_t max_trials, int32_t* bins_out,
                        float* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* SLG_H */
