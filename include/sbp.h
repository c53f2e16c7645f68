/*
 * sbp.h -- C ABI of libsbp, a single-GPU (sm_103a) implementation of the
 * hot path of stochastic block partitioning (SBP) on directed graphs under
 * the degree-corrected stochastic blockmodel (DCSBM).
 *
 * Method (Wanye, Gleyzer, Kao, Feng, "Exact Distributed Stochastic Block
 * Partitioning", Section II):
 *   - blockmodel M[r][s] = number of edges from block r to block s, with
 *     block degrees dout_r = sum_s M[r][s] and din_s = sum_r M[r][s];
 *   - log-likelihood L (Eq. 1) and description length DL (Eq. 2);
 *   - MCMC phase (Alg. 2) run as an asynchronous-Gibbs pass: every vertex
 *     proposes a block against a frozen blockmodel, the change in DL is
 *     computed over the affected rows and columns only (Section III-A (c)),
 *     a Hastings-corrected Metropolis test decides, then M is rebuilt from
 *     the new assignments (Alg. 5: apply all moves, then the blockmodel is
 *     consistent again);
 *   - block merge phase (Alg. 1, Alg. 4): per block, x merge proposals,
 *     keep the best Delta DL, sort, merge until C is reduced;
 *   - golden-ratio search over the number of blocks C (Section II-B).
 *
 * Conventions shared by every call:
 *   - return value: SBP_OK (0) or a negative SBP_E* code; the message of
 *     the last failure on the calling thread is read with sbp_last_error();
 *   - handles are opaque; the library owns every device allocation it makes
 *     and frees it in sbp_free_model / sbp_free_graph;
 *   - input arrays are borrowed for the duration of the call only;
 *   - a pointer documented "host or device" may be either; the library asks
 *     the CUDA runtime which one it is;
 *   - device work runs on the stream given to sbp_build_blockmodel (0 = the
 *     legacy default stream); calls that return values to the host
 *     synchronise that stream, the others only enqueue work;
 *   - no call is thread-safe on the same handle; different handles are
 *     independent;
 *   - vertex ids are int32 in [0, n); edge count m < 2^30.
 */
#ifndef SBP_H
#define SBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBP_OK 0
#define SBP_EINVAL (-1)    /* bad argument: size, range, label, pointer kind */
#define SBP_ENOMEM (-2)    /* device or host allocation failed */
#define SBP_EHASHFULL (-3) /* a hash table ran out of slots */
#define SBP_EPROBE (-4)    /* a bounded probe or wait gave up */
#define SBP_ECUDA (-5)     /* a CUDA runtime call failed */
#define SBP_ESTATE (-6)    /* call not valid in the handle's current state */

typedef struct sbp_graph sbp_graph_t;
typedef struct sbp_model sbp_model_t;

/* Run parameters.  beta: inverse temperature of the Metropolis test;
 * merge_proposals: x of Alg. 1; reduction: share of blocks merged per merge
 * phase before the golden-ratio bracket exists; t_pre / t_post: convergence
 * threshold t of Alg. 2 before / after the bracket exists; max_sweeps: x of
 * Alg. 2; dense_max_B: largest B held as a dense B x B matrix;
 * full_rebuild: 0 lets a commit update the block counts (dense M, or the
 * cell counts behind sparse rows when B * B is small) from the moved
 * vertices' rows when they hold at most E/4 edge ends (the apply step of
 * Alg. 5, same result), 1 always recounts them from all edges;
 * dl_fp32: 1 evaluates the x ln x terms of Delta DL in FP32 with a rigorous
 * error bound and redoes them exactly (fixed point and FP64) only for the
 * proposals whose log(u) falls within the resulting band of logA, so every
 * decision equals the FP64 one (Eq. 1-2; the precision form); 0 evaluates
 * them exactly for every proposal;
 * hybrid_h: 0 for the asynchronous-Gibbs pass; h > 0 for the hybrid pass of
 * the hybrid SBP the paper adopts (Section III-B): the h vertices of largest
 * degree (ties: lower id first) are decided one after another against the
 * current blockmodel, each accepted move applied at once, then the others by
 * asynchronous Gibbs against the result.  Full-range passes of a dense model
 * only (sparse models and vertex ranges use the asynchronous pass). */
typedef struct sbp_params {
    uint64_t seed;
    double beta;
    int32_t merge_proposals;
    int32_t max_sweeps;
    double reduction;
    double t_pre;
    double t_post;
    int32_t dense_max_B;
    int32_t full_rebuild;
    int32_t dl_fp32;
    int32_t hybrid_h;
    int32_t reserved;
} sbp_params;

/* Counters of one nodal pass.  n_proposed: vertices with at least one edge
 * (they draw a proposal); n_moves: proposals with s != current block;
 * n_accepted: moves taken; n_margin: proposals whose log acceptance ratio
 * lies within 1e-9 * max(|logA|, 1) of log(u) (decided, and reported so a
 * comparison with another FP64 implementation can excuse them);
 * n_move_edges: sum of the degrees of the vertices with s != current block
 * (the rows the pass had to aggregate); dl_before / dl_after: DL (Eq. 2)
 * before and after the rebuild; n_recheck: moves decided by the exact
 * (FP64) evaluation because the fast one could not settle them; n_entries:
 * the distinct neighbour blocks of those vertices, summed (each is one
 * entry of the sparse vector of changes, Section III-A (c), and costs four
 * blockmodel lookups and two degree lookups). */
typedef struct sbp_sweep_stats {
    int64_t n_proposed;
    int64_t n_moves;
    int64_t n_accepted;
    int64_t n_margin;
    int64_t n_move_edges;
    double dl_before;
    double dl_after;
    int64_t n_recheck;
    int64_t n_entries;
} sbp_sweep_stats;

/* Optional per-vertex outputs of a nodal decision pass: each member is NULL
 * or a DEVICE pointer to n elements; entries outside [v_begin, v_end) are
 * left untouched.  s: proposed block (current block when there was no
 * proposal); flags: bit 0 proposed, bit 1 accepted, bit 2 margin case;
 * dH: Delta DL of the proposed move (0 when s equals the current block);
 * logA: log acceptance ratio -beta*dH + ln(p_bwd / p_fwd). */
typedef struct sbp_vertex_trace {
    int32_t *s;
    int32_t *flags;
    double *dH;
    double *logA;
} sbp_vertex_trace;

/* Copies the message of the last failure on this thread (NUL-terminated,
 * truncated to len) and returns its full length. */
size_t sbp_last_error(char *buf, size_t len);

/* Fills p with the defaults: seed 0, beta 3, 10 merge proposals, 100
 * sweeps, reduction 0.5, t 5e-4 / 1e-4, dense_max_B 4096, full_rebuild 0,
 * dl_fp32 1, hybrid_h 0. */
int sbp_default_params(sbp_params *p);

/* Loads a directed graph given as COO (src[e] -> dst[e], e < m; host or
 * device pointers) onto the current CUDA device: CSR of out-edges and CSR
 * of in-edges, each row ascending by neighbour id, duplicates kept,
 * self-loops kept (listed in both rows of their vertex).  The graph is the
 * "Graph G" input of Alg. 1-2.  Errors: SBP_EINVAL for n < 1, m < 0,
 * m >= 2^30 or an id outside [0, n); SBP_ENOMEM. */
int sbp_load_graph(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, sbp_graph_t **out);

int sbp_graph_info(const sbp_graph_t *g, int64_t *n, int64_t *m);
void sbp_free_graph(sbp_graph_t *g);

/* Creates a blockmodel handle for assignment b (n labels in [0, B), host or
 * device) and builds M, block degrees and DL (Eq. 1-2, Section II-A).
 * stream: a cudaStream_t (may be NULL) that every later call on this model
 * orders its work on (the decision pass of a graph with 2^22 edges or more
 * runs part of its kernels on two side streams of the model, forked from and
 * joined back into this stream within the call).  p may be NULL
 * (defaults).  The graph must outlive the model.
 * Errors: SBP_EINVAL for B < 1, B > n or a label outside [0, B);
 * SBP_ENOMEM. */
int sbp_build_blockmodel(const sbp_graph_t *g, int32_t B, const int32_t *b, const sbp_params *p, void *stream,
                         sbp_model_t **out);

/* Replaces the assignment of an existing model (labels in [0, B), host or
 * device) and rebuilds M and DL.  The labels are checked on the device
 * before they replace the current ones: on SBP_EINVAL (a label outside
 * [0, B), the smallest such vertex named in the message) the model keeps its
 * assignment.  With the model's own B (after its first nodal pass, unless
 * full_rebuild is set) the change is applied like the moves of a pass: the
 * counts are updated from the changed vertices' rows when those hold at most
 * a quarter of the edges, else recounted; either way M, the degrees and DL
 * are those of a rebuild from scratch.  Discards pending decisions.  Other
 * errors as sbp_build_blockmodel. */
int sbp_set_assignment(sbp_model_t *m, int32_t B, const int32_t *b);

/* One asynchronous-Gibbs nodal pass restricted to the vertices of
 * [v_begin, v_end) (Alg. 2 / Alg. 5 with one rank per vertex): each of them
 * proposes a block and is accepted or rejected against the frozen (b, M);
 * then b takes the decisions and M, the block degrees and DL are rebuilt.
 * sweep_id keys the random draws (Philox4x64-10 counter (sweep_id, v)).
 * stats may be NULL: the call then only enqueues work.  Errors: SBP_EINVAL
 * for a bad range; SBP_EHASHFULL / SBP_EPROBE from the kernels' bounded
 * tables (reported when stats are read). */
int sbp_nodal_sweep(sbp_model_t *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end, sbp_sweep_stats *stats);

/* The decision half of sbp_nodal_sweep: decides [v_begin, v_end) into the
 * model's pending assignment without changing (b, M).  Several calls on
 * disjoint ranges followed by sbp_commit give exactly sbp_nodal_sweep over
 * their union (the per-rank pass and exchange of Alg. 5).  trace may be
 * NULL. */
int sbp_nodal_decide(sbp_model_t *m, uint64_t sweep_id, int64_t v_begin, int64_t v_end, const sbp_vertex_trace *trace);

/* Exchange of the pending assignment between ranks that decided disjoint
 * ranges (the allgather of the new labels in Alg. 5).  sbp_get_pending copies
 * the pending labels of [v_begin, v_end) to out (v_end - v_begin entries,
 * host or device; synchronises the model's stream).  sbp_set_pending writes
 * them from in (host or device) so that the next sbp_commit applies them.
 * Labels must lie in [0, B): host input is checked before the copy
 * (SBP_EINVAL, nothing written); on device input a label outside it keeps
 * the vertex in its current block and the next status check reports
 * SBP_EINVAL.  Errors: SBP_EINVAL for a NULL pointer or a bad range. */
int sbp_get_pending(const sbp_model_t *m, int64_t v_begin, int64_t v_end, int32_t *out);
int sbp_set_pending(sbp_model_t *m, int64_t v_begin, int64_t v_end, const int32_t *in);

/* Applies the pending assignment, rebuilds M and DL, and resets the pending
 * assignment to the new b.  stats may be NULL (counters accumulated by the
 * decide calls since the previous commit). */
int sbp_commit(sbp_model_t *m, sbp_sweep_stats *stats);

/* Merge proposals of Alg. 1 / Alg. 4: for every block r, x proposals s != r
 * (x = merge_proposals), each scored by the Delta DL of merging r into s;
 * the best (smallest score, earliest proposal on a tie at 2^-20 nats) is
 * written to best_s[r], best_dDL[r] (B entries each, host or device).
 * round_id keys the draws.  Requires B >= 2. */
int sbp_merge_proposals(sbp_model_t *m, uint64_t round_id, int32_t *best_s, double *best_dDL);

/* Merge phase (Alg. 1): proposals, then merges in ascending (score, r)
 * order, each linking r's group under s's group unless they are already
 * one, until n_merges links are made; a further proposal round (next
 * round_id) runs when the list is exhausted first.  Blocks are relabelled
 * densely by their smallest member and M is rebuilt.  *rounds_used (may be
 * NULL) receives the number of round_ids consumed.  Requires
 * 1 <= n_merges < B. */
int sbp_merge_blocks(sbp_model_t *m, uint64_t round_id, int32_t n_merges, int32_t *B_out, int32_t *rounds_used);

/* Drops labels that no vertex holds and renumbers the rest densely in
 * ascending order; rebuilds M.  *B_out receives the new B. */
int sbp_compact(sbp_model_t *m, int32_t *B_out);

/* Full run (Fig. 1, Section II-B): start with one block per vertex,
 * alternate merge and MCMC phases under the golden-ratio search until the
 * bracket closes.  Writes the best assignment (n labels, host or device),
 * its B and DL.  p may be NULL (defaults).  stream as in
 * sbp_build_blockmodel. *n_sweeps (may be NULL) receives the number of
 * nodal passes run. */
int sbp_partition(const sbp_graph_t *g, const sbp_params *p, void *stream, int32_t *b_out, int32_t *B_out,
                  double *dl_out, int64_t *n_sweeps);

/* Read-back.  b_out: n labels; M_out: B*B row-major counts (dense models
 * only, SBP_ESTATE otherwise); dout/din: B entries each.  Host or device
 * pointers; these calls synchronise the model's stream and report any
 * error a kernel recorded since the last check. */
int sbp_get_assignment(const sbp_model_t *m, int32_t *b_out);
int sbp_get_B(const sbp_model_t *m, int32_t *B_out);
int sbp_get_dl(const sbp_model_t *m, double *dl_out);
int sbp_get_blockmodel_dense(const sbp_model_t *m, int32_t *M_out);
int sbp_get_degrees(const sbp_model_t *m, int32_t *dout, int32_t *din);

/* The nonzeros of M in either form, as ascending keys r*B + c (int64) with
 * their counts (int32), written to host buffers of `capacity` entries.
 * *nnz receives the number of nonzeros; when it exceeds capacity nothing is
 * written and SBP_EINVAL is returned. */
int sbp_get_blockmodel_coo(const sbp_model_t *m, int64_t capacity, int64_t *keys, int32_t *counts, int64_t *nnz);
int sbp_sync(const sbp_model_t *m);
void sbp_free_model(sbp_model_t *m);

/* Description length (Eq. 2) of a dense blockmodel, computed without
 * allocating any device memory.  The paper has no counterpart: this exists
 * for callers that must not allocate once they are running (for example a
 * serving process whose memory pool owns the device, or code that cannot
 * accept cudaMalloc's implicit synchronisation or a late allocation
 * failure).  Inputs are DEVICE pointers the caller owns: M, B*B row-major
 * counts; dout and din, B block degrees each; E and N are the graph's edge
 * and vertex counts; dl_out is a DEVICE pointer to one double, written
 * asynchronously on `stream` (a cudaStream_t, may be NULL).
 * Scratch: a fixed 128 KB array of device memory inside the library (16384
 * partial sums), so B is limited to 4096; larger B is rejected with
 * SBP_EINVAL.  Every call shares that array: calls whose GPU work overlaps
 * (on different streams) race and must be ordered by the caller.  The first
 * call on each device looks up the array's device address with that device
 * current; make that first call before any stream capture.  That address is
 * kept for the rest of the process: it does not survive cudaDeviceReset, so
 * after a reset of a device this entry point must not be called on it.
 * Results agree
 * with sbp_get_dl to about 1e-13 relative (x ln x from FP64 log here). */
int sbp_dense_dl_noalloc(const int32_t *M, int32_t B, const int32_t *dout, const int32_t *din, int64_t E, int64_t N,
                         double *dl_out, void *stream);

/* Philox4x64-10 of the device code, for known-answer tests: writes 4*count
 * words for counters (c0 + i, c1, c2, c3), i < count, under key (k0, k1);
 * out is a host pointer. */
int sbp_philox_check(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1, int32_t count,
                     uint64_t *out);

/* ---------------------------------------------------------------------
 * Batching form: many graphs partitioned together.
 *
 * Every graph runs the same golden-ratio search as sbp_partition (Section
 * II-B; Alg. 1, 2) and ends with the same assignment, B, DL and sweep count.
 * A graph whose next phase starts at B <= 1024 on a dense model and merges
 * to B <= max_B hands its search to a persistent launch over all waiting
 * graphs: a CTA runs that graph's phases (start state, merge rounds, sweeps
 * with the convergence test, compaction, bracket update) until the search
 * ends or a phase is out of those bounds.  This overlaps with the
 * per-graph work (set-up, larger-B phases) that `workers` host threads
 * drive on their graphs' streams.  Graphs are admitted in input order
 * while their estimated device memory fits mem_fraction of the free
 * memory, and each model is freed when its graph finishes.
 *
 * workers: host threads (1..256); max_B: largest B a batched phase merges
 * to (1..1024); max_n: largest graph (vertices) whose searches are batched
 * (a CTA runs a whole search, so the biggest graphs can be better served by
 * the per-graph kernels); dense_max_B: dense/sparse switch of the batch's models
 * (max_B..16384); ctas_per_sm: persistent CTAs per SM (1..8);
 * movers_per_warp: movers a warp of the persistent kernel evaluates at once
 * (1, 2 or 4: 32, 16 or 8 lanes each; fewer when their per-mover count rows
 * would not fit shared memory); mem_fraction: (0, 0.95].  No option changes
 * a result. */
typedef struct sbp_batch_options {
    int32_t workers;
    int32_t max_B;
    int32_t dense_max_B;
    int32_t ctas_per_sm;
    int32_t max_n;
    int32_t movers_per_warp;
    double mem_fraction;
} sbp_batch_options;

/* Per-graph result: B, DL and sweeps as sbp_partition returns them;
 * t_submit, t_admit, t_done: seconds from the start of the call (or of the
 * server) to the graph's submission, admission and result. */
typedef struct sbp_batch_result {
    int32_t B;
    int32_t reserved;
    double dl;
    int64_t n_sweeps;
    double t_submit;
    double t_admit;
    double t_done;
} sbp_batch_result;

/* Where a batch call spent its time: rounds: persistent launches;
 * s_per_graph: worker-seconds of per-graph work (summed over the workers),
 * of which s_merge in set-up, merge phases and compaction and s_sweeps in
 * per-graph MCMC sweeps; s_batched: wall seconds of the persistent launches,
 * summed over launches (up to 16 are in flight at once);
 * phases_batched: phases run in the persistent launches, of which
 * merges_batched with their merge phase (the others had theirs run per
 * graph) and starts_batched from a search state the model no longer held;
 * phases_per_graph: MCMC phases run per graph. */
typedef struct sbp_batch_stats {
    int64_t rounds;
    double s_per_graph;
    double s_batched;
    int64_t phases_batched;
    int64_t phases_per_graph;
    double s_merge;
    double s_sweeps;
    int64_t merges_batched;
    int64_t starts_batched;
} sbp_batch_stats;

/* Fills o with the defaults: 32 workers, max_B 512, max_n 65536, dense_max_B
 * 1024, 2 CTAs per SM, 2 movers per warp, mem_fraction 0.5. */
int sbp_default_batch_options(sbp_batch_options *o);

/* Partitions graphs[0..count).  p: NULL for the defaults (shared by every
 * graph); o: NULL for the defaults.  b_out: NULL, or count pointers (host or
 * device) to n_i labels each; res: count results (host); stats: NULL or
 * the call's time split.  Fails with the first error of any graph; partial
 * results are then undefined. */
int sbp_partition_batch(const sbp_graph_t *const *graphs, int32_t count, const sbp_params *p,
                        const sbp_batch_options *o, int32_t *const *b_out, sbp_batch_result *res,
                        sbp_batch_stats *stats);

/* Autotuner of the batching form: times sbp_partition_batch on a sample of
 * graphs (`sample` of them, evenly spaced in size order; all when sample <= 0
 * or >= count) under candidate options and returns the fastest in *best.
 * The search starts from *best when `start` is nonzero (else from the
 * defaults) and tunes one option at a time, in this order:
 * movers_per_warp {1, 2, 4}, ctas_per_sm {1, 2, 3, 4}, max_B {128, 256,
 * 512, 1024}, max_n {1024, 4096, 16384, 65536}, dense_max_B {1024, 4096};
 * workers (the caller's host threads) and mem_fraction are kept.  A
 * sample runs far from the full batch's load (its host workers are mostly
 * idle), so options that favour per-graph work can win on it and lose on
 * the whole batch.  *graphs_per_s (may be NULL) receives the best rate on
 * the sample, *trials (may be NULL) the number of timed runs.
 * Every run must give the same B and DL for every graph; SBP_ESTATE
 * otherwise.  p: NULL for the defaults. */
int sbp_autotune_batch(const sbp_graph_t *const *graphs, int32_t count, const sbp_params *p, int32_t sample,
                       int32_t start, sbp_batch_options *best, double *graphs_per_s, int32_t *trials);

/* ---------------------------------------------------------------------
 * Serving form: the batch engine fed while it runs (continuous batching).
 * sbp_server_create starts the engine (host worker threads and a launcher
 * thread); requests submitted while others run are admitted as their
 * memory fits (memory freed by finished requests admits the next), and
 * their work overlaps on the device with the others'.  Free host workers
 * take the oldest admitted request's next step first (a batch call takes
 * the largest graph's), so requests finish close to arrival order.  Every
 * request's
 * result equals sbp_partition of its graph alone.  A graph and its b_out
 * buffer (host or device, n labels, or NULL) must stay valid until the
 * request is done.  sbp_server_wait blocks until the request is done and
 * returns its result (the request's own failure, if it failed);
 * sbp_server_poll sets *done without blocking; sbp_server_destroy finishes
 * every submitted request, then stops the threads and frees the engine. */
typedef struct sbp_server sbp_server_t;

int sbp_server_create(const sbp_params *p, const sbp_batch_options *o, sbp_server_t **out);
int sbp_server_submit(sbp_server_t *s, const sbp_graph_t *g, int32_t *b_out, int64_t *request);
int sbp_server_poll(sbp_server_t *s, int64_t request, int32_t *done);
int sbp_server_wait(sbp_server_t *s, int64_t request, sbp_batch_result *res);
int sbp_server_stats(sbp_server_t *s, sbp_batch_stats *stats);
void sbp_server_destroy(sbp_server_t *s);

/* The FP32 x ln x term of the precision form, for known-answer tests:
 * val[i] = f(x[i] + k[i]) - f(x[i]) with f(x) = x ln x as the FP32 Delta DL
 * evaluation computes it, am[i] the magnitude its error bound is
 * proportional to (|val - exact| <= 28 * 2^-24 * am); host arrays; x >= 0,
 * 0 <= x + k < 2^31. */
int sbp_dxlogx32_check(const int32_t *x, const int32_t *k, int32_t count, float *val, float *am);

/* Number of kernel launches the library has issued in this process, over
 * all handles and devices (a host-side counter, incremented as each launch
 * is enqueued, whether or not the kernel then finds work to do).  For
 * accounting only: read it before and after a region of calls. */
int sbp_kernel_launches(uint64_t *out);

#ifdef __cplusplus
}
#endif

#endif /* SBP_H */
