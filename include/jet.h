/*
 * libjet -- deterministic Jet refinement for the connectivity metric on one
 * GB300 (sm_103a), after "Deterministic Parallel High-Quality Hypergraph
 * Partitioning" (arXiv 2504.12013).
 *
 * C ABI.  Plain pointers and sizes only.  Unless a function says otherwise:
 *   - every pointer argument is a DEVICE pointer owned by the caller; the
 *     library never frees it and never keeps it beyond the call, except the
 *     hypergraph arrays, which must stay valid and unchanged for the lifetime
 *     of the context;
 *   - work is enqueued on the context's stream; the call returns without
 *     waiting for the GPU unless its comment says it synchronizes;
 *   - the return value is JET_OK (0) or a negative JET_ERR_* code, and
 *     jet_last_error() gives a one-line reason.  On error nothing has been
 *     written to caller buffers, except where the comment says so.
 *   - results are bit-identical from run to run: all accumulation is integer
 *     and order-independent.
 *
 * Notation (Section 2 of the paper): H = (V, E, c, omega), n = |V|, m = |E|,
 * P = sum of |e| (pins), k blocks, Pi : V -> {0..k-1} (blocks are 0-based),
 * phi_e[i] = |e cap V_i|, lambda(e) = |{i : phi_e[i] > 0}|,
 * (lambda-1)(Pi) = sum_e (lambda(e) - 1) omega(e),
 * L_max = floor((1 + eps) * ceil(c(V)/k)).
 */
#ifndef JET_H
#define JET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JET_OK 0
#define JET_ERR_INVALID_ARG (-1) /* bad size, pointer, parameter or unsupported k        */
#define JET_ERR_OOM (-2)         /* device allocation failed                              */
#define JET_ERR_CUDA (-3)        /* a CUDA call failed (message in jet_last_error)        */
#define JET_ERR_OVERFLOW (-4)    /* a weight sum would leave the exact integer ranges     */
#define JET_ERR_DATA (-5)        /* device check found a bad index/weight in the inputs   */

/*
 * Hypergraph in two CSR views (Section 2).  All arrays are device memory.
 *   eptr[m+1], pins[P]   pins of edge e are pins[eptr[e] .. eptr[e+1]),
 *                        distinct vertex ids in [0, n), any order
 *   vptr[n+1], inc[P]    incident edges I(v) are inc[vptr[v] .. vptr[v+1]);
 *                        must be the exact transpose of (eptr, pins)
 *   vwgt[n]              c(v) >= 1
 *   ewgt[m]              omega(e) >= 1
 * Empty edges are allowed and contribute 0 to (lambda-1).
 */
typedef struct {
  int32_t n, m;
  int64_t P;
  const int64_t *eptr;
  const int32_t *pins;
  const int64_t *vptr;
  const int32_t *inc;
  const int32_t *vwgt;
  const int32_t *ewgt;
} jet_hypergraph;

/*
 * Parameters.  eps = eps_num/eps_den (the balance bound, Section 2; 3/100 in
 * Section 7.1); d = d_num/d_den (deadzone size, Section 4.3; 1/10).  The
 * rebalancer runs at most max_rebalance_rounds rounds per call.
 * k must be in [2, 256].
 */
typedef struct {
  int32_t k;
  int32_t eps_num, eps_den;
  int32_t d_num, d_den;
  int32_t max_rebalance_rounds;
} jet_params;

/*
 * Per-iteration statistics, written to DEVICE memory by jet_refine_round and
 * jet_rebalance (eight int64 fields, 64 bytes).
 */
typedef struct {
  int64_t candidates;       /* |M| after the temperature filter (Section 4.1)     */
  int64_t approved;         /* moves kept by the afterburner (Algorithm 2)        */
  int64_t rebalance_rounds; /* rebalancing rounds that found an overloaded block  */
  int64_t rebalance_moves;  /* vertices moved by the rebalancer (Section 4.3)     */
  int64_t objective;        /* (lambda-1) after the iteration                     */
  int64_t max_block_weight; /* max_i c(V_i) after the iteration                    */
  int64_t imbalanced;       /* 1 if max_i c(V_i) > L_max                           */
  int64_t reserved;
} jet_round_stats;

/* Summary of jet_refine, written to HOST memory. */
typedef struct {
  int64_t iterations;           /* Jet iterations executed over all phases            */
  int64_t objective;            /* (lambda-1) of the returned partition               */
  int64_t initial_objective;    /* (lambda-1) of the input partition                  */
  int64_t balanced;             /* 1 if the returned partition satisfies L_max        */
  int64_t phase_iterations[8];  /* iterations per temperature (first 8 phases)        */
} jet_refine_result;

typedef struct jet_ctx jet_ctx;

/*
 * Create a context for one hypergraph: validates the arguments, checks the
 * CSR arrays on the device (index ranges, monotone offsets, positive
 * weights, the transpose degree counts), computes c(V), ceil(c(V)/k), L_max
 * and the deadzone bound, classifies vertices and edges by size, and
 * allocates the library-owned workspace (about m*ceil(k/32)*4 + 48*n bytes
 * plus the class lists).  `stream` is a cudaStream_t (NULL = legacy default
 * stream).  SYNCHRONIZES the stream.  Errors: JET_ERR_INVALID_ARG (k outside
 * [2,256], negative sizes, NULL arrays with nonzero sizes, eps/d
 * denominators <= 0, negative numerators), JET_ERR_DATA (bad CSR or
 * weights), JET_ERR_OVERFLOW (some sum of omega over I(v) >= 2^31, c(v) >
 * 32767, or c(V) >= 2^50), JET_ERR_OOM, JET_ERR_CUDA.  *out is NULL on error.
 */
int jet_ctx_create(jet_ctx **out, const jet_hypergraph *hg, const jet_params *params, void *stream);

/* Free the workspace.  Synchronizes the stream first.  NULL is ignored. */
void jet_ctx_destroy(jet_ctx *ctx);

/* One-line reason of the last error on this context (static string if ctx is NULL). */
const char *jet_last_error(const jet_ctx *ctx);

/*
 * Pin counts (Section 2; the table that makes gains linear, Section 4.2):
 * phi[e*k + i] = |e cap V_i| (int32, row-major m x k, fully overwritten) and
 * block_w[i] = c(V_i) (int64[k], overwritten) for the partition part[n]
 * (values in [0,k)).  Also rebuilds the context's connectivity bitmasks of
 * phi.  A part value outside [0,k) is reported as JET_ERR_DATA by the next
 * synchronizing call on this context (the affected pins are skipped).
 */
int jet_build_pincounts(jet_ctx *ctx, const int32_t *part, int32_t *phi, int64_t *block_w);

/*
 * Connectivity metric (Section 2): *objective_out = sum_e (lambda(e)-1)
 * omega(e), lambda(e) = number of nonzero entries of row e of phi.
 * objective_out is one device int64.  Reads phi densely; does not use or
 * change the context's bitmasks.
 */
int jet_connectivity(jet_ctx *ctx, const int32_t *phi, int64_t *objective_out);

/*
 * One Jet iteration, the body of Algorithm 1 (Section 4.1): move candidates
 * with temperature tau = tau_num/tau_den in [0,1) (the unlocked vertices
 * whose best adjacent target t(v) has gain >= -tau * A(v)); the hypergraph
 * afterburner (Algorithm 2), keeping candidates whose recomputed gain in the
 * order (gain desc, vertex id asc) is > 0; ApplyMoves of the kept moves;
 * locked[v] := 1 exactly for the moved vertices; then, if some block exceeds
 * L_max, deterministic rebalancing rounds (Section 4.3) as in
 * jet_rebalance.  part[n], phi[m*k], block_w[k], locked[n] (uint8) are
 * updated in place and must describe one consistent state (as left by
 * jet_build_pincounts or a previous call).  stats (device, may be NULL)
 * receives the iteration's statistics.
 * Synchronization: in graph mode (the default, see jet_set_graph_mode) the
 * call does NOT synchronize (one graph launch; the first call with a new
 * argument set also captures and instantiates the graph).  In the
 * kernel-by-kernel mode it SYNCHRONIZES the stream once after ApplyMoves
 * (to learn whether a block is overloaded) and once per rebalancing round.
 * Errors: JET_ERR_INVALID_ARG for tau outside [0,1) or NULL state arrays.
 */
int jet_refine_round(jet_ctx *ctx, int32_t tau_num, int32_t tau_den, int32_t *part, int32_t *phi,
                     int64_t *block_w, uint8_t *locked, jet_round_stats *stats);

/*
 * Execution form of jet_refine_round (default enable = 1): a CUDA graph per
 * argument set (captured on first use and cached, up to 6 per context), whose
 * rebalancing rounds run in a conditional WHILE node decided on the device,
 * so the call returns without synchronizing and device-detected data errors
 * surface at the next synchronizing call.  enable = 0 runs the same kernels
 * one by one with a stream synchronization per rebalancing round; results
 * are identical.
 */
int jet_set_graph_mode(jet_ctx *ctx, int enable);

/*
 * Graph path (default off; the paper notes that graphs get a specialised
 * implementation, Section 7).  Allowed only when every edge has exactly two
 * distinct pins (JET_ERR_INVALID_ARG otherwise).  For an edge e = {v, u},
 * Lambda(e) = {Pi(v), Pi(u)} and |e cap V_Pi(v)| > 1 iff Pi(u) = Pi(v), so
 * gains, rebalancing targets and (lambda-1) (the weighted edge cut) are read
 * from the neighbours' blocks through an adjacency array built here
 * (4 bytes per incidence, context-owned), and moves change only Pi and the
 * block weights: phi and the edge bitmasks are not maintained.  Results are
 * identical to the hypergraph path.  While the graph path is on: phi
 * arguments may be NULL; jet_refine_round, jet_rebalance and the rollback
 * leave phi as it was; jet_refine, batches and jet_uncoarsen rebuild phi
 * (when not NULL) from the final partition; jet_build_pincounts builds
 * block_w (and phi when not NULL); jet_quotient_schedule is refused.  After
 * turning it off, call jet_build_pincounts before the next round.
 * Switching drops the context's captured graphs; do it before building a
 * batch of this context.  Synchronizes.
 */
int jet_set_graph_path(jet_ctx *ctx, int enable);

/*
 * Deterministic rebalancing (Section 4.3) until no block exceeds L_max, a
 * round moves nothing, or params.max_rebalance_rounds rounds ran.  Per
 * round, from the state at its start: every vertex v of an overloaded block
 * s with 2c(v) <= 3(c(V_s) - ceil(c(V)/k)) takes its best target b != s
 * with c(V_b) + c(v) <= L_max outside the deadzone (c(V_b) >= L_max_real -
 * d*eps*ceil(c(V)/k)), ties to the smaller block id; priority gain*c(v) for
 * gain >= 0, gain/c(v) below, ties to the smaller vertex id; per overloaded
 * block the minimal prefix of that order whose weight reaches the excess
 * moves, all at once.  Locks are ignored and unchanged.  stats (device, may
 * be NULL) receives rebalance_rounds, rebalance_moves, objective,
 * max_block_weight and imbalanced (other fields 0).  SYNCHRONIZES the
 * stream once before the first round (to learn whether a block is
 * overloaded) and once per round (the stop rule is read on the host); it is
 * the only call of the round's steps that always synchronizes.
 */
int jet_rebalance(jet_ctx *ctx, int32_t *part, int32_t *phi, int64_t *block_w, jet_round_stats *stats);

/*
 * Algorithm 1 to convergence with a temperature schedule (Section 7.2: three
 * temperatures 3/4, 3/8, 0 and an iteration limit of 8): builds phi and
 * block_w from part, then for every tau in tau_pairs (HOST array of n_tau
 * (num, den) pairs) clears the locks and iterates jet_refine_round until
 * `limit` iterations in a row bring no strictly better balanced partition,
 * then rolls back to the best balanced partition seen.  part (device, n)
 * is updated in place; phi/block_w (device, caller-sized m*k and k) hold the
 * final state.  *result (HOST) receives the summary.  Synchronizes.  In graph
 * mode (the default, see jet_set_graph_mode) the whole schedule runs as one
 * CUDA graph with the loop control on the device and one synchronization at
 * the end; the kernel-by-kernel form reads each iteration's statistics.
 */
int jet_refine(jet_ctx *ctx, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part, int32_t *phi,
               int64_t *block_w, jet_refine_result *result);

/*
 * Batches: many independent instances refined by ONE CUDA-graph launch
 * (Algorithm 1 per instance, as in jet_refine).  Each instance has its own
 * context (its own hypergraph, k and eps); jet_batch_create takes `count`
 * distinct contexts (HOST array) and a stream for the launches (NULL =
 * legacy default stream).  The batch graph holds every instance's refinement
 * as an independent branch, so their kernels overlap on the device; results
 * are identical to running jet_refine on each context alone.
 *
 * jet_batch_refine: part[i], phi[i], block_w[i] (HOST arrays of DEVICE
 * pointers, one per instance, sized as for jet_refine) are refined in place;
 * results (HOST, count entries, may be NULL) receive the summaries.  The
 * graph is built on the first call and reused while the schedule, limit and
 * state pointers are unchanged.  Synchronizes.  Errors as jet_refine, for
 * the first failing instance; the message is in jet_batch_last_error.
 *
 * Work split: with split s = 0 every instance sizes its grids for all SMs;
 * with s > 0 instance i sizes them for max(1, s * num_SMs * P_i / sum P)
 * SMs (P = pins), so many small instances share the device instead of each
 * asking for all of it.  jet_batch_tune runs the batch once per candidate
 * split (splits, HOST, n_splits entries, each in [0, 64]), restoring every
 * part[i] before each run, keeps the fastest split, and leaves the
 * partitions as they were; ms_out (HOST, may be NULL) gets each run's
 * device time.  The contexts' grid sizes return to all SMs when the batch
 * is destroyed.  The paper has no batched form; this is the serving-side
 * pattern of running many refinements on one GPU.
 */
typedef struct jet_batch jet_batch;

int jet_batch_create(jet_batch **out, jet_ctx *const *ctxs, int32_t count, void *stream);
void jet_batch_destroy(jet_batch *batch);
const char *jet_batch_last_error(const jet_batch *batch);
int jet_batch_refine(jet_batch *batch, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                     int32_t *const *phi, int64_t *const *block_w, jet_refine_result *results);
int jet_batch_set_split(jet_batch *batch, int32_t split);
int jet_batch_get_split(const jet_batch *batch);
int jet_batch_tune(jet_batch *batch, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                   int32_t *const *phi, int64_t *const *block_w, const int32_t *splits, int32_t n_splits,
                   float *ms_out);

/*
 * Persistent form of a batch (the north star's "one persistent launch"):
 * jet_batch_set_team(batch, ctas, threads, split_pins) with ctas in {1, 2, 4,
 * 8} and threads a multiple of 32 in [128, 1024] makes jet_batch_refine run
 * ONE persistent kernel (captured in a CUDA graph with the reset of its work
 * queue and the copy of the summaries): teams of `ctas` thread blocks (a
 * thread-block cluster when ctas > 1) of `threads` threads each take the next
 * instance from a device work queue (instances grouped by ceil(k/32), largest
 * first) and run all of Algorithm 1 on it, with the team's barrier between
 * phases, so every instance advances at its own pace.  With ctas > 1 and
 * split_pins > 0, once the queue reaches instances of fewer than split_pins
 * pins, each block of a cluster takes instances on its own (small instances
 * are bound by barrier latency, which a single block pays least).  ctas = 0
 * returns to the branch-graph form.  Results are identical to jet_refine on
 * each instance alone, whatever the shape.  Every context must be on the
 * hypergraph path (JET_ERR_INVALID_ARG otherwise); a partition value outside
 * [0, k) is JET_ERR_DATA for that instance (naming it in
 * jet_batch_last_error), and that instance is not refined.
 *
 * jet_batch_autotune chooses the team shape: for each of the n_shapes
 * (ctas, threads, split_pins) triples of `shapes` (HOST) it runs the
 * persistent kernel on `sample` instances spread over the sizes of the batch,
 * each stopped after trial_iterations Jet iterations, from the same
 * partitions (restored before each trial and at the end), and keeps the
 * shape with the most (pins x iterations) per second; ms_out and rate_out
 * (HOST, n_shapes entries, may be NULL) receive each trial's device time and
 * rate.  The arguments are those of jet_batch_refine.  Synchronizes.
 */
int jet_batch_set_team(jet_batch *batch, int32_t ctas, int32_t threads, int32_t split_pins);
int jet_batch_get_team(const jet_batch *batch, int32_t *ctas, int32_t *threads, int32_t *split_pins);
int jet_batch_autotune(jet_batch *batch, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                       int32_t *const *phi, int64_t *const *block_w, const int32_t *shapes, int32_t n_shapes,
                       int32_t sample, int32_t trial_iterations, float *ms_out, double *rate_out);

/*
 * Uncoarsening (the refinement phase of the multilevel scheme, §7.2: the
 * partition of the coarsest level is projected level by level to the input
 * and refined with Algorithm 1 at every level) as ONE CUDA graph.
 * levels[0..n_levels) are contexts of the hierarchy's hypergraphs from the
 * coarsest (0) to the finest, all with the same k; maps[l] (device int32, one
 * entry per vertex of level l+1) gives each vertex of level l+1 its vertex of
 * level l.  part[0] (device) holds the coarsest level's initial partition;
 * part[l] for l >= 1 receive the projections; every part[l], phi[l],
 * block_w[l] (HOST arrays of DEVICE pointers, sized as for jet_refine) end
 * refined.  results (HOST, n_levels entries, may be NULL) receive the
 * per-level summaries.  `stream` runs the graph.  Synchronizes.  A map value
 * outside [0, n of level l) is JET_ERR_DATA; other errors as jet_refine.
 * The hierarchy itself (coarsening, Section 6) is the caller's.
 */
int jet_uncoarsen(jet_ctx *const *levels, int32_t n_levels, const int32_t *const *maps, const int32_t *tau_pairs,
                  int32_t n_tau, int32_t limit, int32_t *const *part, int32_t *const *phi, int64_t *const *block_w,
                  jet_refine_result *results, void *stream);

/*
 * Coarsening (Section 6, Algorithm 4): one level of deterministic
 * synchronous clustering, then the contraction of its clusters.
 *
 * jet_cluster.  Clusters are label classes; label[v] (DEVICE, n, out)
 * starts as v.  The vertices are visited in sub-rounds of order (DEVICE, n,
 * a permutation of [0, n): the random split of Algorithm 4, an input so
 * that the result is reproducible): single_subrounds sub-rounds of one
 * vertex, then sizes 2, 4, 8, ... up to max(1, floor(n / subround_cap_div))
 * (prefix doubling, Section 6; the paper uses 100 and 100).  Within a
 * sub-round, from the state at its start, each vertex still in a singleton
 * cluster rates the clusters C of its neighbours, sum over its edges e with
 * 2 <= |e| <= rating_max_edge that touch C of omega(e)/(|e|-1) (the
 * corrected heavy-edge rating: once per edge and cluster; 32.32 fixed point,
 * each term rounded down), over the clusters with
 * c(C) + c(u) <= max_cluster_weight, and proposes the best (ties to the
 * smaller label).  Mutual proposals u <-> v go towards the heavier would-be
 * cluster (its weight plus its other proposers; ties: the smaller id stays),
 * each target accepts the longest prefix of its proposers in (c(u), u)
 * order that keeps it within max_cluster_weight, and the accepted vertices
 * move at once.  Synchronizes.  Errors: JET_ERR_INVALID_ARG (NULL pointers,
 * max_cluster_weight < 1, rating_max_edge < 2, single_subrounds < 0,
 * subround_cap_div < 1), JET_ERR_DATA (malformed CSR, or order not a
 * permutation), JET_ERR_OVERFLOW (a vertex's rating sum reaches 2^63, or
 * its rated edges hold more than 2^27 pins), JET_ERR_OOM, JET_ERR_CUDA.
 *
 * jet_contract.  The non-empty label classes of label (DEVICE, n, values in
 * [0, n)) become the coarse vertices, numbered in increasing label order,
 * weighing the sum of their members; map (DEVICE, n, out) gives each vertex
 * its coarse vertex.  Every edge keeps its distinct coarse pins in
 * increasing order and is dropped below two; edges with equal pin sets merge
 * into the one of smallest id with their weights summed; coarse edges keep
 * the order of those ids; the incidences of a coarse vertex are in
 * increasing coarse-edge id.  out holds DEVICE buffers owned by the caller,
 * sized as the input's (eptr m+1, pins P, vptr n+1, inc P, vwgt n, ewgt m);
 * *n_out, *m_out, *P_out (HOST) get the coarse sizes.  Synchronizes.
 * Errors: JET_ERR_INVALID_ARG, JET_ERR_DATA (malformed CSR or a label
 * outside [0, n)), JET_ERR_OVERFLOW (a coarse weight leaves int32),
 * JET_ERR_OOM, JET_ERR_CUDA.
 *
 * Both allocate stream-ordered scratch and free it before returning; both
 * report errors through jet_last_error(NULL); `stream` is a cudaStream_t.
 */
/*
 * max_cluster_weight also bounds the coarse vertex weights of the next level
 * (a cluster of several vertices never exceeds it; a single vertex keeps its
 * own weight).  jet_ctx_create accepts c(v) <= 32767 only (JET_ERR_OVERFLOW
 * otherwise), so a hierarchy meant for jet_uncoarsen should use
 * max_cluster_weight <= 32767.
 */
typedef struct {
  int64_t max_cluster_weight; /* bound on the weight of a cluster              */
  int32_t rating_max_edge;    /* edges with more pins add nothing to a rating  */
  int32_t single_subrounds;   /* one-vertex sub-rounds at the start            */
  int32_t subround_cap_div;   /* sub-rounds grow to floor(n / this) vertices   */
} jet_coarsen_params;

typedef struct { /* DEVICE buffers owned by the caller */
  int64_t *eptr;
  int32_t *pins;
  int64_t *vptr;
  int32_t *inc;
  int32_t *vwgt;
  int32_t *ewgt;
} jet_hypergraph_out;

int jet_cluster(const jet_hypergraph *hg, const jet_coarsen_params *params, const int32_t *order, int32_t *label,
                void *stream);
int jet_contract(const jet_hypergraph *hg, const int32_t *label, int32_t *map, const jet_hypergraph_out *out,
                 int32_t *n_out, int32_t *m_out, int64_t *P_out, void *stream);

/*
 * Serving: a request loop that refines submitted jobs (each = jet_refine_host
 * on the job's host buffers: upload, Algorithm 1 as one graph, download) with
 * up to max_active jobs on the device at once, each on its own stream and
 * worker thread.  Jobs are admitted in submission order while a slot is free
 * and the sum of the admitted jobs' device footprints (jet_job_footprint)
 * stays within hbm_budget bytes, so a job that arrives while others run
 * starts as soon as a slot and enough memory are free, and its kernels
 * overlap with theirs.  A job's result is the same as running it alone.
 *
 * jet_server_submit copies the job description (not the arrays): hg_host's
 * arrays and part_host (HOST, n; refined in place) must stay valid and
 * untouched until jet_server_wait reports the job.  Errors:
 * JET_ERR_INVALID_ARG (bad arguments), JET_ERR_OOM (the footprint exceeds
 * the whole budget).  *id_out gets the job id (1, 2, ...).
 *
 * jet_server_wait moves up to max_done finished jobs into done (HOST) and
 * sets *n_done; it blocks until at least one job is done or timeout_ms
 * passes (0: no wait, < 0: no limit).  A job's own failure is in its status
 * and its message.  latency_ms runs from submission to the partition being
 * back in host memory; queue_ms from submission to admission (so the
 * service time is latency_ms - queue_ms).  device_start_ms / device_end_ms
 * place the job on the GPU timeline: CUDA events recorded on the job's
 * stream before its first upload and after its partition's download,
 * measured from an event recorded when the server was created; two jobs
 * whose intervals intersect had work in flight on the device at the same
 * time.
 *
 * jet_server_load reports the jobs waiting for admission, the jobs admitted
 * or running, and the reserved bytes.  jet_server_destroy waits for every
 * submitted job, then stops the workers; reports not yet collected are
 * dropped.  The paper has no serving loop; this is the project's runtime
 * around the refinement.
 */
typedef struct jet_server jet_server;

typedef struct {
  int64_t id;
  int32_t status;            /* JET_OK or the job's error code              */
  int32_t reserved;
  double latency_ms;         /* submission -> result in host memory          */
  double queue_ms;           /* submission -> admission                      */
  double device_start_ms;    /* GPU timeline: before the first upload        */
  double device_end_ms;      /* GPU timeline: after the partition's download */
  jet_refine_result result;  /* summary of the job's refinement              */
  char message[128];         /* reason of a failed job ("" on success)       */
} jet_job_done;

size_t jet_job_footprint(int32_t n, int32_t m, int64_t P, int32_t k);
int jet_server_create(jet_server **out, size_t hbm_budget, int32_t max_active);
int jet_server_submit(jet_server *server, const jet_hypergraph *hg_host, const jet_params *params,
                      const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part_host, int64_t *id_out);
int jet_server_wait(jet_server *server, jet_job_done *done, int32_t max_done, int32_t *n_done, int32_t timeout_ms);
int jet_server_load(jet_server *server, int32_t *pending, int32_t *running, size_t *reserved_bytes);
const char *jet_server_last_error(const jet_server *server);
void jet_server_destroy(jet_server *server);

/*
 * The candidate step of jet_refine_round alone (Section 4.1), for
 * inspection: in_m[v] (uint8) = 1 for v in M, and for those v target[v] =
 * t(v) and gain[v] = gain(v, t(v)) (int32); other entries are -1 / 0.  The
 * candidates stay in the context for a following jet_afterburner call.
 */
int jet_candidates(jet_ctx *ctx, int32_t tau_num, int32_t tau_den, const int32_t *part, const int32_t *phi,
                   const uint8_t *locked, int32_t *target, int32_t *gain, uint8_t *in_m);

/*
 * The afterburner of Algorithm 2 alone, on the candidates of the last
 * jet_candidates call on this context with the same part/phi:
 * rg[v] (int32) = recomputed gain, approved[v] (uint8) = v in M and rg > 0.
 * Nothing is moved.
 */
int jet_afterburner(jet_ctx *ctx, const int32_t *part, const int32_t *phi, int32_t *rg, uint8_t *approved);

/*
 * End-to-end call on HOST buffers: copies the hypergraph (the same arrays as
 * jet_hypergraph, in host memory; pinned memory gives the fastest copies) and
 * part[n] to the device, runs jet_refine with the given schedule, and copies
 * the refined partition back into part.  Allocates and frees its own device
 * memory.  Synchronizes.  *result (host, may be NULL) gets the summary.
 */
int jet_refine_host(const jet_hypergraph *hg_host, const jet_params *params, const int32_t *tau_pairs,
                    int32_t n_tau, int32_t limit, int32_t *part, jet_refine_result *result);

/*
 * End-to-end call on HOST buffers for a fixed number of iterations: copies
 * the hypergraph (as for jet_refine_host) and part[n] to the device, builds
 * phi and the block weights (jet_build_pincounts), clears the locks, runs
 * n_rounds iterations of jet_refine_round at tau = tau_num/tau_den (the body
 * of Algorithm 1, Section 4.1, without the loop control), and copies the
 * partition back into part.  *stats (HOST, may be NULL) gets the last
 * iteration's statistics.  Allocates and frees its own device memory.
 * Synchronizes.  Errors as jet_ctx_create and jet_refine_round, and
 * JET_ERR_INVALID_ARG for n_rounds < 0.
 */
int jet_rounds_host(const jet_hypergraph *hg_host, const jet_params *params, int32_t tau_num, int32_t tau_den,
                    int32_t n_rounds, int32_t *part, jet_round_stats *stats);

/*
 * Device memory of the library (no counterpart in the paper).  The library's
 * stream-ordered allocations (context workspace, the device copies of the
 * host-buffer calls above, batch plans, coarsening pools) come from a memory
 * pool of its own, one per device, that keeps what the library frees for its
 * next calls instead of returning it to the driver at every synchronization:
 * a call on host buffers would otherwise map its gigabytes afresh each time.
 * So after a call the process keeps up to the largest working set the library
 * has needed on that device.  jet_release_memory returns the kept memory of
 * every device's pool to the driver (cudaMemPoolTrimTo); call it when no
 * library work is in flight.  Returns JET_OK or JET_ERR_CUDA.
 */
int jet_release_memory(void);

/*
 * Profiling.  The library's kernels fall into JET_PROF_FAMILIES families:
 *   0 pin counts and bitmasks    1 move candidates         2 afterburner
 *   3 approval and locks         4 apply moves             5 rebalancing targets
 *   6 rebalancing selection      7 rebalancing control     8 objective and stats
 *   9 other (connectivity, rollback, exports)
 * Kernel launches are always counted per family.  While profiling is enabled
 * (jet_profile_enable(ctx, 1)), each family's launches on the context's
 * stream are also bracketed by CUDA events.  jet_profile_read synchronizes the
 * stream and writes, per family (HOST arrays of JET_PROF_FAMILIES entries,
 * any may be NULL): ms_out = summed device time in milliseconds, calls_out =
 * timed launcher invocations, launches_out = kernels launched; reset != 0
 * clears everything afterwards.  Profiling records events only and does not
 * change results.
 */
#define JET_PROF_FAMILIES 10
int jet_profile_enable(jet_ctx *ctx, int enable);
int jet_profile_read(jet_ctx *ctx, double *ms_out, int64_t *calls_out, int64_t *launches_out, int reset);

/*
 * Matching schedule of k-way refinement (Section 5, "K-Way Refinement:
 * Matching Schedule"): the quotient graph Q of the partition whose pin
 * counts are phi (device, m*k) has the blocks as vertices and an edge {i, j}
 * when some hyperedge has pins in both V_i and V_j.  The block pairs of Q are
 * scheduled in rounds; each round is a maximal matching in the pairs not
 * scheduled yet, so a block takes part in one two-way refinement at a time.
 * Per round the blocks go in order of their degree among the unscheduled
 * pairs (descending, ties to the smaller id), and a block still unmatched
 * takes its unmatched neighbour of the largest such degree (ties to the
 * smaller id).  Writes, in selection order, pairs[2p], pairs[2p+1] (device
 * int32, room for k(k-1) entries) = the block whose turn it was and its
 * partner, and round_of[p] (device int32, room for k(k-1)/2 entries);
 * *n_pairs and *n_rounds (HOST) get the counts.  Synchronizes.  The two-way
 * flow refinements themselves are not part of this library.
 */
int jet_quotient_schedule(jet_ctx *ctx, const int32_t *phi, int32_t *pairs, int32_t *round_of, int32_t *n_pairs,
                          int32_t *n_rounds);

/*
 * Work counts of the last jet_refine_round or jet_rebalance call (for byte
 * models of the kernels; always counted, no events).  Synchronizes.  Writes
 * up to n (<= 5) entries of out (HOST): [0] vertices of overloaded blocks
 * met by the rebalancing target passes, summed over the rounds; [1] vertices
 * they evaluated (one record each); [2] the incidences of those vertices;
 * [3] incidences of all moved vertices (Jet and rebalancing moves); [4] the
 * levels of the rebalancing selection's radix select (a property of the
 * context: every record is read once per level after the first).
 */
int jet_profile_work(jet_ctx *ctx, int64_t *out, int32_t n);

/*
 * Block weights without any device allocation (the paper has no counterpart;
 * this is a deployment variant of the block-weight pass of
 * jet_build_pincounts).  For callers that must not allocate device memory:
 * applications that give the whole device to their own pool, and loops where
 * a cudaMalloc/cudaFree would stall the device too long.  No context is
 * needed.
 *   part[n] (device, values in [0,k)), vwgt[n] (device, c(v)) in;
 *   block_w[k] (device int64, overwritten) = c(V_i);
 *   block_count[k] (device int32, may be NULL) = |V_i|;
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * Scratch: a file-scope device array of 1.25 KiB per GPU, resident until
 * process exit, limits k to [2, 256] (JET_ERR_INVALID_ARG otherwise).  The
 * first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it for the rest of the
 * process, so do not keep calling it across a cudaDeviceReset of that device
 * (the cached address would be stale).  Every call clears the array first;
 * calls that overlap on the GPU share it and race.  Allocates nothing (no
 * cudaMalloc, cudaFree or allocating library call).  SYNCHRONIZES the stream
 * (it copies the data-error flag to the host and waits), so it must not be
 * called while that stream is being captured into a CUDA graph.  A value of
 * part outside [0,k) or a weight vwgt[v] < 1 returns JET_ERR_DATA (block_w
 * and block_count are then not meaningful).  Errors are reported by
 * jet_last_error(NULL).
 */
int jet_block_weights_noalloc(const int32_t *part, const int32_t *vwgt, int32_t n, int32_t k, int64_t *block_w,
                              int32_t *block_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* JET_H */
