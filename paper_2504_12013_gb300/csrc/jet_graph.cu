// Algorithm 1 (the temperature schedule of Section 7.2 with the improvement
// counter, the best-partition snapshot and the rollback) as ONE CUDA graph,
// and batches of independent instances refined by one graph launch.
//
// Per temperature phase the graph holds a WHILE node over Jet iterations.
// Its body is one iteration (the same nodes as jet_refine_round, including
// the nested WHILE node of the rebalancing rounds) followed by a control
// kernel that applies Algorithm 1's rule: a balanced iteration with a
// strictly smaller (lambda-1) than the best so far resets the counter and
// snapshots the partition; the loop runs while the counter is below the
// limit.  After the phase the partition is rolled back to the snapshot by
// moves.  Nothing is read on the host until the graph has finished.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "jet_internal.cuh"

namespace jet {
namespace {

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

// Statistics of the input partition: the first candidate for the best one.
__global__ void k_refine_begin(const jet_round_stats *st, RefineState *rs) {
  RefineState r;
  memset(&r, 0, sizeof(r));
  r.res.initial_objective = st->objective;
  r.have_best = st->imbalanced ? 0 : 1;
  r.best = st->objective;
  r.snap = r.have_best;
  *rs = r;
}

// best = part when the last step improved (every thread reads the flag).
__global__ void k_snapshot(int32_t *best, const int32_t *part, int32_t n, const RefineState *rs) {
  if (!rs->snap) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    best[v] = part[v];
}

__global__ void k_phase_begin(RefineState *rs, int32_t limit, cudaGraphConditionalHandle h) {
  rs->it = 0;
  rs->in_phase = 0;
  rs->snap = 0;
  cudaGraphSetConditional(h, limit > 0 ? 1u : 0u);
}

// Algorithm 1's loop control after one iteration.
__global__ void k_iteration_end(const jet_round_stats *st, RefineState *rs, int32_t limit,
                                cudaGraphConditionalHandle h) {
  rs->res.iterations += 1;
  rs->in_phase += 1;
  rs->it += 1;
  int snap = 0;
  if (!st->imbalanced && (!rs->have_best || st->objective < rs->best)) {
    rs->have_best = 1;
    rs->best = st->objective;
    rs->it = 0;
    snap = 1;
  }
  rs->snap = snap;
  cudaGraphSetConditional(h, rs->it < limit ? 1u : 0u);
}

__global__ void k_phase_end(RefineState *rs, int32_t phase) {
  if (phase < 8) rs->res.phase_iterations[phase] = rs->in_phase;
}

__global__ void k_refine_end(const jet_round_stats *st, RefineState *rs) {
  rs->res.objective = st->objective;
  rs->res.balanced = st->imbalanced ? 0 : 1;
}

// Projection of a partition to the next finer level of a hierarchy:
// part_fine[v] = part_coarse[map[v]]; a map value outside [0, n_coarse) is
// reported as a data error and gives block 0.
__global__ void k_project(const int32_t *part_coarse, const int32_t *map, int32_t n_fine, int32_t n_coarse,
                          int32_t *part_fine, Counters *cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_fine; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = map[v];
    if ((unsigned)u < (unsigned)n_coarse) {
      part_fine[v] = part_coarse[u];
    } else {
      part_fine[v] = 0;
      atomicOr(&cnt->err, kErrMapRange);
    }
  }
}

bool same_key(const jet_ctx::RefineGraph &g, const int32_t *tau, int32_t n_tau, int32_t limit, const void *part,
              const void *phi, const void *bw, const void *res) {
  if (!g.exec || g.limit != limit || g.part != part || g.phi != phi || g.bw != bw || g.res != res) return false;
  if ((int)g.tau.size() != 2 * n_tau) return false;
  return n_tau == 0 || memcmp(g.tau.data(), tau, sizeof(int32_t) * 2 * n_tau) == 0;
}

}  // namespace

// Captures the whole refinement onto c->cap_stream[0], which must be
// capturing; the iteration bodies use cap_stream[1] and the rebalancing
// bodies cap_stream[2].  result_dst receives the summary at the end (host
// pinned or device memory).
cudaError_t capture_refine(jet_ctx *c, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part,
                           int32_t *phi, int64_t *block_w, jet_refine_result *result_dst) {
  cudaStream_t s0 = c->cap_stream[0], s1 = c->cap_stream[1], s2 = c->cap_stream[2];
  cudaStream_t saved = c->stream;
  c->stream = s0;
  RefineState *rs = c->rstate;
  const int gn = grid_for(c->n, 256, c->launch_sms);
  cudaError_t e = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = launch_pincounts(c, part, phi, block_w)) != cudaSuccess) return e;
    if ((e = reset_counters(c)) != cudaSuccess) return e;
    if ((e = launch_objective(c, part)) != cudaSuccess) return e;
    if ((e = launch_stats(c, block_w, c->stats_scratch, 1)) != cudaSuccess) return e;
    k_refine_begin<<<1, 1, 0, s0>>>(c->stats_scratch, rs);
    k_snapshot<<<gn, 256, 0, s0>>>(c->best_part, part, c->n, rs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int ti = 0; ti < n_tau; ++ti) {
      if (c->n > 0 && (e = cudaMemsetAsync(c->locked_ws, 0, c->n, s0)) != cudaSuccess) return e;
      cudaStreamCaptureStatus st;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t *deps = nullptr;
      const cudaGraphEdgeData *ed = nullptr;
      size_t nd = 0;
      if ((e = cudaStreamGetCaptureInfo(s0, &st, nullptr, &cg, &deps, &ed, &nd)) != cudaSuccess) return e;
      cudaGraphConditionalHandle h;
      if ((e = cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
      k_phase_begin<<<1, 1, 0, s0>>>(rs, limit, h);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = cudaStreamGetCaptureInfo(s0, &st, nullptr, &cg, &deps, &ed, &nd)) != cudaSuccess) return e;
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cn;
      if ((e = cudaGraphAddNode(&cn, cg, deps, ed, nd, &cp)) != cudaSuccess) return e;
      if ((e = cudaStreamUpdateCaptureDependencies(s0, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamBeginCaptureToGraph(s1, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
      cudaError_t eb = capture_iteration(c, s1, s2, tau_pairs[2 * ti], tau_pairs[2 * ti + 1], part, phi, block_w,
                                         c->locked_ws, c->stats_scratch, nullptr, nullptr);
      if (eb == cudaSuccess) {
        k_iteration_end<<<1, 1, 0, s1>>>(c->stats_scratch, rs, limit, h);
        k_snapshot<<<gn, 256, 0, s1>>>(c->best_part, part, c->n, rs);
        eb = cudaGetLastError();
      }
      cudaGraph_t tmp = nullptr;
      e = cudaStreamEndCapture(s1, &tmp);
      if (eb != cudaSuccess) return eb;
      if (e != cudaSuccess) return e;
      k_phase_end<<<1, 1, 0, s0>>>(rs, ti);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // rollback to the best balanced partition (no moves when there is none)
      if ((e = launch_rollback_moves(c, part, c->best_part, &rs->have_best)) != cudaSuccess) return e;
      if ((e = launch_apply(c, part, phi, block_w)) != cudaSuccess) return e;
    }
    if (c->graph_path && phi && (e = launch_pincounts(c, part, phi, block_w)) != cudaSuccess) return e;  // final phi
    if ((e = reset_counters(c)) != cudaSuccess) return e;
    if ((e = launch_objective(c, part)) != cudaSuccess) return e;
    if ((e = launch_stats(c, block_w, c->stats_scratch, 1)) != cudaSuccess) return e;
    k_refine_end<<<1, 1, 0, s0>>>(c->stats_scratch, rs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(result_dst, &rs->res, sizeof(jet_refine_result), cudaMemcpyDefault, s0);
  }();
  c->stream = saved;
  return e;
}

void destroy_refine_graph(jet_ctx *c) {
  if (c->refine_graph.exec) cudaGraphExecDestroy(c->refine_graph.exec);
  c->refine_graph.exec = nullptr;
  if (c->rstate) cudaFree(c->rstate);
  c->rstate = nullptr;
  if (c->res_host) cudaFreeHost(c->res_host);
  c->res_host = nullptr;
}

static cudaError_t ensure_refine_state(jet_ctx *c) {
  cudaError_t e = cudaSuccess;
  if (!c->rstate) e = cudaMalloc(reinterpret_cast<void **>(&c->rstate), sizeof(RefineState));
  if (e == cudaSuccess && !c->res_host)
    e = cudaMallocHost(reinterpret_cast<void **>(&c->res_host), sizeof(jet_refine_result));
  if (e == cudaSuccess) e = ensure_capture_streams(c);
  return e;
}

// jet_refine in graph mode: build (or reuse) the graph, launch, wait, report.
int refine_graph(jet_ctx *c, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part, int32_t *phi,
                 int64_t *block_w, jet_refine_result *result) {
  CK(ensure_refine_state(c), "refine state");
  jet_ctx::RefineGraph &G = c->refine_graph;
  if (!same_key(G, tau_pairs, n_tau, limit, part, phi, block_w, c->res_host)) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "graph");
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap_stream[0], g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      c->capturing = 1;
      cudaError_t ec = capture_refine(c, tau_pairs, n_tau, limit, part, phi, block_w, c->res_host);
      c->capturing = 0;
      cudaGraph_t done = nullptr;
      e = cudaStreamEndCapture(c->cap_stream[0], &done);
      if (ec != cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      G.exec = nullptr;
      return cuda_fail(c, e, "refine graph");
    }
    G.tau.assign(tau_pairs, tau_pairs + 2 * n_tau);
    G.limit = limit;
    G.part = part;
    G.phi = phi;
    G.bw = block_w;
    G.res = c->res_host;
  }
  CK(cudaGraphLaunch(G.exec, c->stream), "refine graph launch");
  int rc = sync_counters(c);  // synchronizes; reports data errors found on the device
  if (rc) return rc;
  *result = *c->res_host;
  return JET_OK;
}

}  // namespace jet

// ---------------------------------------------------------------- batches
// A batch refines many independent instances (one context each) with one
// graph launch: every instance's refinement graph is captured on its own
// streams, forked from and joined back into the batch stream, so the
// instances are parallel branches of one graph and their kernels overlap on
// the device.  The work split is the number of SMs each instance's grids are
// sized for; jet_batch_tune measures a few splits and keeps the fastest.
struct jet_batch {
  std::vector<jet_ctx *> ctx;
  cudaStream_t stream = nullptr;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int32_t> tau;
  int32_t limit = 0;
  std::vector<const void *> args;  // part, phi, block_w of every instance
  jet_refine_result *res_host = nullptr;
  int split = 0;        // 0: every instance sizes its grids for all SMs; s > 0: see jet_batch_set_split
  int built_split = -1;
  // persistent form (team_ctas > 0): one kernel whose teams of team_ctas blocks of team_threads threads each
  // refine one instance at a time from a device queue
  int team_ctas = 0, team_threads = 0;
  int32_t team_split = 0;  // instances of fewer pins run on single blocks of a cluster
  jet::TeamPlan *plan = nullptr;
  std::vector<const void *> plan_args;  // part, phi, block_w of every instance, the schedule and the limit the
  std::vector<int32_t> plan_tau;        // plan and its graph were built for
  int32_t plan_limit = 0;
  cudaGraphExec_t team_exec = nullptr;
  int team_exec_ctas = 0, team_exec_threads = 0, team_exec_split = -1;
  char err[256] = {0};
};

namespace {

int bfail(jet_batch *b, int code, const char *msg, cudaError_t e = cudaSuccess) {
  if (b) snprintf(b->err, sizeof(b->err), "%.160s%s%.80s", msg, e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
  jet::set_global_error("%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
  return code;
}

// SMs instance i's grids are sized for under split s: s = 0 keeps all SMs;
// otherwise the instance gets a share proportional to its pins, scaled by s,
// and at least one SM.
void apply_split(jet_batch *b, int s) {
  long long total = 0;
  for (jet_ctx *c : b->ctx) total += c->P > 0 ? c->P : 1;
  for (jet_ctx *c : b->ctx) {
    if (s == 0) {
      c->launch_sms = c->num_sms;
      continue;
    }
    const long long p = c->P > 0 ? c->P : 1;
    long long share = (long long)c->num_sms * s * p / (total > 0 ? total : 1);
    if (share < 1) share = 1;
    if (share > c->num_sms) share = c->num_sms;
    c->launch_sms = (int)share;
  }
}

int build_batch(jet_batch *b, const int32_t *tau, int32_t n_tau, int32_t limit, int32_t *const *part,
                int32_t *const *phi, int64_t *const *block_w) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  apply_split(b, b->split);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return bfail(b, JET_ERR_CUDA, "batch graph", e);
  e = cudaStreamBeginCaptureToGraph(b->origin, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
  int rc = JET_OK;
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess && rc == JET_OK; ++i) {
    jet_ctx *c = b->ctx[i];
    e = jet::ensure_capture_streams(c);
    if (e == cudaSuccess && !c->rstate) e = cudaMalloc(reinterpret_cast<void **>(&c->rstate), sizeof(jet::RefineState));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cap_stream[0], b->fork, 0);  // joins the capture
    if (e != cudaSuccess) break;
    c->capturing = 1;
    e = jet::capture_refine(c, tau, n_tau, limit, part[i], phi[i], block_w[i], &b->res_host[i]);
    c->capturing = 0;
    // join the branch back even after a failed capture, so that the origin's capture ends with every
    // forked stream joined (and is then discarded) instead of leaving a stream in an open capture
    cudaError_t ej = cudaEventRecord(b->join, c->cap_stream[0]);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->origin, b->join, 0);
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) rc = bfail(b, JET_ERR_CUDA, c->err[0] ? c->err : "batch capture", e);
  }
  cudaGraph_t done = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->origin, &done);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return rc != JET_OK ? rc : bfail(b, JET_ERR_CUDA, "batch graph", e);
  }
  b->tau.assign(tau, tau + 2 * n_tau);
  b->limit = limit;
  b->args.clear();
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    b->args.push_back(part[i]);
    b->args.push_back(phi[i]);
    b->args.push_back(block_w[i]);
  }
  b->built_split = b->split;
  return JET_OK;
}

bool batch_key_matches(const jet_batch *b, const int32_t *tau, int32_t n_tau, int32_t limit, int32_t *const *part,
                       int32_t *const *phi, int64_t *const *block_w) {
  if (!b->exec || b->built_split != b->split || b->limit != limit || (int)b->tau.size() != 2 * n_tau) return false;
  if (n_tau && memcmp(b->tau.data(), tau, sizeof(int32_t) * 2 * n_tau)) return false;
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (b->args[3 * i] != part[i] || b->args[3 * i + 1] != phi[i] || b->args[3 * i + 2] != block_w[i]) return false;
  return true;
}

int check_batch_args(jet_batch *b, const int32_t *tau, int32_t n_tau, int32_t limit, int32_t *const *part,
                     int32_t *const *phi, int64_t *const *block_w) {
  if (!b) return bfail(nullptr, JET_ERR_INVALID_ARG, "batch is NULL");
  if (n_tau < 0 || (n_tau > 0 && !tau) || limit < 1) return bfail(b, JET_ERR_INVALID_ARG, "bad schedule");
  for (int i = 0; i < n_tau; ++i)
    if (tau[2 * i + 1] <= 0 || tau[2 * i] < 0 || tau[2 * i] >= tau[2 * i + 1])
      return bfail(b, JET_ERR_INVALID_ARG, "a temperature is outside [0, 1)");
  if (!part || !phi || !block_w) return bfail(b, JET_ERR_INVALID_ARG, "NULL state array list");
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const jet_ctx *c = b->ctx[i];
    if ((c->n > 0 && !part[i]) || (c->m > 0 && !phi[i] && !c->graph_path) || !block_w[i])
      return bfail(b, JET_ERR_INVALID_ARG, "NULL state array of an instance");
  }
  return JET_OK;
}

// The device plan of the persistent form for this schedule and these state arrays (rebuilt when they change).
int ensure_plan(jet_batch *b, const int32_t *tau, int32_t n_tau, int32_t limit, int32_t *const *part,
                int32_t *const *phi, int64_t *const *block_w) {
  std::vector<const void *> args;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    args.push_back(part[i]);
    args.push_back(phi[i]);
    args.push_back(block_w[i]);
  }
  std::vector<int32_t> t(tau, tau + 2 * n_tau);
  if (b->plan && args == b->plan_args && t == b->plan_tau && limit == b->plan_limit) return JET_OK;
  if (b->team_exec) cudaGraphExecDestroy(b->team_exec);
  b->team_exec = nullptr;
  if (b->plan) jet::team_plan_destroy(b->plan, b->stream);
  b->plan = nullptr;
  for (jet_ctx *c : b->ctx) {
    if (c->graph_path) return bfail(b, JET_ERR_INVALID_ARG, "the persistent form needs every instance on the hypergraph path");
    cudaStreamSynchronize(c->stream);
  }
  int rc = jet::team_plan_build(&b->plan, b->ctx.data(), (int32_t)b->ctx.size(), part, phi, block_w, tau, n_tau,
                                b->stream);
  if (rc) return bfail(b, rc, jet_last_error(nullptr));
  b->plan_args = args;
  b->plan_tau = t;
  b->plan_limit = limit;
  return JET_OK;
}

// The persistent form: one graph (queue reset, the persistent launches, the summaries to the host), launched on
// b->stream; waits and reports.
int run_team(jet_batch *b, int32_t limit, jet_refine_result *results) {
  if (!b->team_exec || b->team_exec_ctas != b->team_ctas || b->team_exec_threads != b->team_threads ||
      b->team_exec_split != b->team_split) {
    if (b->team_exec) cudaGraphExecDestroy(b->team_exec);
    b->team_exec = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ec =
          jet::team_launch(b->plan, b->team_ctas, b->team_threads, b->team_split, limit, 0, b->origin, nullptr, 0);
      if (ec == cudaSuccess) ec = jet::team_results(b->plan, b->res_host, b->origin);
      e = cudaStreamEndCapture(b->origin, &g);
      if (ec != cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->team_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->team_exec = nullptr;
      return bfail(b, JET_ERR_CUDA, "persistent batch graph", e);
    }
    b->team_exec_ctas = b->team_ctas;
    b->team_exec_threads = b->team_threads;
    b->team_exec_split = b->team_split;
  }
  cudaError_t e = cudaGraphLaunch(b->team_exec, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, JET_ERR_CUDA, "persistent batch launch", e);
  const int bad = jet::team_first_error(b->plan, b->stream);
  if (bad == -2) return bfail(b, JET_ERR_CUDA, "persistent batch error check");
  if (bad >= 0) {
    char msg[160];
    snprintf(msg, sizeof(msg), "instance %d: a partition value is outside [0, k)", bad);
    return bfail(b, JET_ERR_DATA, msg);
  }
  for (size_t i = 0; i < b->ctx.size(); ++i) b->ctx[i]->phi_owner = static_cast<const int32_t *>(b->plan_args[3 * i + 1]);
  if (results) memcpy(results, b->res_host, sizeof(jet_refine_result) * b->ctx.size());
  return JET_OK;
}

// Launch the batch graph on b->stream and wait; report per-instance errors.
int run_batch(jet_batch *b, jet_refine_result *results) {
  cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, JET_ERR_CUDA, "batch launch", e);
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    int rc = jet::sync_counters(b->ctx[i]);
    if (rc) return bfail(b, rc, b->ctx[i]->err);
  }
  if (results) memcpy(results, b->res_host, sizeof(jet_refine_result) * b->ctx.size());
  return JET_OK;
}

}  // namespace

extern "C" {

int jet_batch_create(jet_batch **out, jet_ctx *const *ctxs, int32_t count, void *stream) {
  if (!out) return bfail(nullptr, JET_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !ctxs) return bfail(nullptr, JET_ERR_INVALID_ARG, "a batch needs at least one context");
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return bfail(nullptr, JET_ERR_INVALID_ARG, "a context of the batch is NULL");
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (ctxs[i] == ctxs[j]) return bfail(nullptr, JET_ERR_INVALID_ARG, "a context appears twice in the batch");
  jet_batch *b = new (std::nothrow) jet_batch;
  if (!b) return bfail(nullptr, JET_ERR_OOM, "host allocation failed");
  b->ctx.assign(ctxs, ctxs + count);
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMallocHost(reinterpret_cast<void **>(&b->res_host), sizeof(jet_refine_result) * (size_t)count);
  if (e != cudaSuccess) {
    int rc = bfail(nullptr, JET_ERR_CUDA, "batch set-up", e);
    jet_batch_destroy(b);
    return rc;
  }
  // the contexts' own streams must be idle before their graphs are used from the batch stream
  for (jet_ctx *c : b->ctx) cudaStreamSynchronize(c->stream);
  *out = b;
  return JET_OK;
}

void jet_batch_destroy(jet_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->team_exec) cudaGraphExecDestroy(b->team_exec);
  if (b->plan) jet::team_plan_destroy(b->plan, b->stream);
  for (jet_ctx *c : b->ctx) c->launch_sms = c->num_sms;
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->res_host) cudaFreeHost(b->res_host);
  delete b;
}

const char *jet_batch_last_error(const jet_batch *b) { return b ? b->err : jet_last_error(nullptr); }

int jet_batch_set_split(jet_batch *b, int32_t split) {
  if (!b) return bfail(nullptr, JET_ERR_INVALID_ARG, "batch is NULL");
  if (split < 0 || split > 64) return bfail(b, JET_ERR_INVALID_ARG, "split must be in [0, 64]");
  b->split = split;
  return JET_OK;
}

int jet_batch_get_split(const jet_batch *b) { return b ? b->split : -1; }

int jet_batch_set_team(jet_batch *b, int32_t ctas, int32_t threads, int32_t split_pins) {
  if (!b) return bfail(nullptr, JET_ERR_INVALID_ARG, "batch is NULL");
  if (ctas == 0) {
    b->team_ctas = b->team_threads = b->team_split = 0;
    return JET_OK;
  }
  if (split_pins < 0) return bfail(b, JET_ERR_INVALID_ARG, "split_pins must be >= 0");
  if (!(ctas == 1 || ctas == 2 || ctas == 4 || ctas == 8))
    return bfail(b, JET_ERR_INVALID_ARG, "team blocks must be 1, 2, 4 or 8");
  if (threads < 128 || threads > 1024 || threads % 32)
    return bfail(b, JET_ERR_INVALID_ARG, "team threads must be a multiple of 32 in [128, 1024]");
  for (jet_ctx *c : b->ctx)
    if (c->graph_path) return bfail(b, JET_ERR_INVALID_ARG, "the persistent form needs every instance on the hypergraph path");
  b->team_ctas = ctas;
  b->team_threads = threads;
  b->team_split = split_pins;
  return JET_OK;
}

int jet_batch_get_team(const jet_batch *b, int32_t *ctas, int32_t *threads, int32_t *split_pins) {
  if (!b || !ctas || !threads || !split_pins) return bfail(nullptr, JET_ERR_INVALID_ARG, "NULL argument");
  *ctas = b->team_ctas;
  *threads = b->team_threads;
  *split_pins = b->team_split;
  return JET_OK;
}

int jet_batch_autotune(jet_batch *b, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                       int32_t *const *phi, int64_t *const *block_w, const int32_t *shapes, int32_t n_shapes,
                       int32_t sample, int32_t trial_iterations, float *ms_out, double *rate_out) {
  int rc = check_batch_args(b, tau_pairs, n_tau, limit, part, phi, block_w);
  if (rc) return rc;
  if (n_shapes < 1 || !shapes) return bfail(b, JET_ERR_INVALID_ARG, "no team shapes to try");
  if (sample < 1 || trial_iterations < 1) return bfail(b, JET_ERR_INVALID_ARG, "sample and trial_iterations must be >= 1");
  for (int i = 0; i < n_shapes; ++i) {
    const int c = shapes[3 * i], t = shapes[3 * i + 1];
    if (!(c == 1 || c == 2 || c == 4 || c == 8) || t < 128 || t > 1024 || t % 32 || shapes[3 * i + 2] < 0)
      return bfail(b, JET_ERR_INVALID_ARG,
                   "a team shape is outside {1,2,4,8} x [128, 1024] (multiples of 32) x [0, 2^31)");
  }
  if ((rc = ensure_plan(b, tau_pairs, n_tau, limit, part, phi, block_w))) return rc;
  const std::vector<int32_t> smp = jet::team_sample(b->plan, sample);
  // every trial starts from the sample's partitions: keep device copies
  std::vector<int32_t *> saved(smp.size(), nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < smp.size() && e == cudaSuccess; ++i) {
    const jet_ctx *c = b->ctx[smp[i]];
    if (c->n == 0) continue;
    e = cudaMalloc(reinterpret_cast<void **>(&saved[i]), sizeof(int32_t) * c->n);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(saved[i], part[smp[i]], sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, b->stream);
  }
  auto restore = [&]() {
    for (size_t i = 0; i < smp.size() && e == cudaSuccess; ++i)
      if (saved[i])
        e = cudaMemcpyAsync(part[smp[i]], saved[i], sizeof(int32_t) * b->ctx[smp[i]]->n, cudaMemcpyDeviceToDevice,
                            b->stream);
  };
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  std::vector<jet_refine_result> res(b->ctx.size());
  int best = -1;
  double best_rate = 0.0;
  for (int t = 0; t < n_shapes && e == cudaSuccess; ++t) {
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {  // an untimed run (first launch of this shape), a timed one
      restore();
      if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
      if (e == cudaSuccess)
        e = jet::team_launch(b->plan, shapes[3 * t], shapes[3 * t + 1], shapes[3 * t + 2], limit, trial_iterations,
                             b->stream, smp.data(), (int32_t)smp.size());
      if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
      if (e == cudaSuccess) e = jet::team_results(b->plan, res.data(), b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    double work = 0.0;
    for (int32_t i : smp) work += (double)jet::team_pins(b->plan, i) * (double)res[i].iterations;
    const double rate = ms > 0.f ? work / (ms * 1e-3) : 0.0;
    if (ms_out) ms_out[t] = ms;
    if (rate_out) rate_out[t] = rate;
    if (e == cudaSuccess && (best < 0 || rate > best_rate)) {
      best = t;
      best_rate = rate;
    }
  }
  restore();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  for (int32_t *q : saved)
    if (q) cudaFree(q);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return bfail(b, JET_ERR_CUDA, "persistent batch tuning", e);
  b->team_ctas = shapes[3 * best];
  b->team_threads = shapes[3 * best + 1];
  b->team_split = shapes[3 * best + 2];
  return JET_OK;
}

int jet_batch_refine(jet_batch *b, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                     int32_t *const *phi, int64_t *const *block_w, jet_refine_result *results) {
  int rc = check_batch_args(b, tau_pairs, n_tau, limit, part, phi, block_w);
  if (rc) return rc;
  if (b->team_ctas > 0) {
    if ((rc = ensure_plan(b, tau_pairs, n_tau, limit, part, phi, block_w))) return rc;
    return run_team(b, limit, results);
  }
  if (!batch_key_matches(b, tau_pairs, n_tau, limit, part, phi, block_w) &&
      (rc = build_batch(b, tau_pairs, n_tau, limit, part, phi, block_w)))
    return rc;
  return run_batch(b, results);
}

int jet_batch_tune(jet_batch *b, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *const *part,
                   int32_t *const *phi, int64_t *const *block_w, const int32_t *splits, int32_t n_splits,
                   float *ms_out) {
  int rc = check_batch_args(b, tau_pairs, n_tau, limit, part, phi, block_w);
  if (rc) return rc;
  if (n_splits < 1 || !splits) return bfail(b, JET_ERR_INVALID_ARG, "no splits to try");
  for (int i = 0; i < n_splits; ++i)
    if (splits[i] < 0 || splits[i] > 64) return bfail(b, JET_ERR_INVALID_ARG, "split must be in [0, 64]");
  // every trial starts from the same partitions: keep a device copy of each
  std::vector<int32_t *> saved(b->ctx.size(), nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i)
    if (b->ctx[i]->n > 0) {
      e = cudaMalloc(reinterpret_cast<void **>(&saved[i]), sizeof(int32_t) * b->ctx[i]->n);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(saved[i], part[i], sizeof(int32_t) * b->ctx[i]->n, cudaMemcpyDeviceToDevice, b->stream);
    }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  auto restore = [&]() {
    for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i)
      if (saved[i])
        e = cudaMemcpyAsync(part[i], saved[i], sizeof(int32_t) * b->ctx[i]->n, cudaMemcpyDeviceToDevice, b->stream);
  };
  int best = -1;
  float best_ms = 0.f;
  for (int t = 0; t < n_splits && e == cudaSuccess && rc == JET_OK; ++t) {
    b->split = splits[t];
    rc = build_batch(b, tau_pairs, n_tau, limit, part, phi, block_w);
    if (rc) break;
    // one untimed run (first launch of a new graph), then a timed one
    for (int r = 0; r < 2 && e == cudaSuccess && rc == JET_OK; ++r) {
      restore();
      if (e != cudaSuccess) break;
      if (r == 1) e = cudaEventRecord(t0, b->stream);
      if (e == cudaSuccess) rc = run_batch(b, nullptr);
      if (r == 1 && e == cudaSuccess && rc == JET_OK) {
        e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (ms_out) ms_out[t] = ms;
        if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
          best = t;
          best_ms = ms;
        }
      }
    }
  }
  restore();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  for (int32_t *p : saved)
    if (p) cudaFree(p);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (rc) return rc;
  if (e != cudaSuccess) return bfail(b, JET_ERR_CUDA, "batch tuning", e);
  b->split = splits[best];
  return JET_OK;
}

int jet_uncoarsen(jet_ctx *const *levels, int32_t n_levels, const int32_t *const *maps, const int32_t *tau_pairs,
                  int32_t n_tau, int32_t limit, int32_t *const *part, int32_t *const *phi, int64_t *const *block_w,
                  jet_refine_result *results, void *stream) {
  if (!levels || n_levels < 1) return bfail(nullptr, JET_ERR_INVALID_ARG, "no levels");
  if (n_levels > 1 && !maps) return bfail(nullptr, JET_ERR_INVALID_ARG, "maps is NULL");
  if (!part || !phi || !block_w) return bfail(nullptr, JET_ERR_INVALID_ARG, "NULL state array list");
  if (n_tau < 0 || (n_tau > 0 && !tau_pairs) || limit < 1) return bfail(nullptr, JET_ERR_INVALID_ARG, "bad schedule");
  for (int i = 0; i < n_tau; ++i)
    if (tau_pairs[2 * i + 1] <= 0 || tau_pairs[2 * i] < 0 || tau_pairs[2 * i] >= tau_pairs[2 * i + 1])
      return bfail(nullptr, JET_ERR_INVALID_ARG, "a temperature is outside [0, 1)");
  for (int l = 0; l < n_levels; ++l) {
    const jet_ctx *c = levels[l];
    if (!c) return bfail(nullptr, JET_ERR_INVALID_ARG, "a level's context is NULL");
    if (c->k != levels[0]->k) return bfail(nullptr, JET_ERR_INVALID_ARG, "the levels have different k");
    if ((c->n > 0 && !part[l]) || (c->m > 0 && !phi[l] && !c->graph_path) || !block_w[l])
      return bfail(nullptr, JET_ERR_INVALID_ARG, "NULL state array of a level");
    if (l > 0 && c->n > 0 && !maps[l - 1]) return bfail(nullptr, JET_ERR_INVALID_ARG, "NULL map of a level");
    for (int j = 0; j < l; ++j)
      if (levels[j] == c) return bfail(nullptr, JET_ERR_INVALID_ARG, "a context appears twice");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t origin = nullptr;
  cudaEvent_t ev = nullptr;
  jet_refine_result *res = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&res), sizeof(jet_refine_result) * n_levels);
  for (int l = 0; l < n_levels && e == cudaSuccess; ++l) {
    cudaStreamSynchronize(levels[l]->stream);
    e = jet::ensure_capture_streams(levels[l]);
    if (e == cudaSuccess && !levels[l]->rstate)
      e = cudaMalloc(reinterpret_cast<void **>(&levels[l]->rstate), sizeof(jet::RefineState));
  }
  if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(origin, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t ec = cudaEventRecord(ev, origin);
    // a chain: level l waits for level l-1, projects its partition, refines
    for (int l = 0; l < n_levels && ec == cudaSuccess; ++l) {
      jet_ctx *c = levels[l];
      cudaStream_t s0 = c->cap_stream[0];
      ec = cudaStreamWaitEvent(s0, ev, 0);
      if (ec == cudaSuccess && l > 0 && c->n > 0) {
        jet::k_project<<<jet::grid_for(c->n, 256, c->launch_sms), 256, 0, s0>>>(part[l - 1], maps[l - 1], c->n,
                                                                                  levels[l - 1]->n, part[l], c->cnt);
        ec = cudaGetLastError();
      }
      if (ec == cudaSuccess) {
        c->capturing = 1;
        ec = jet::capture_refine(c, tau_pairs, n_tau, limit, part[l], phi[l], block_w[l], &res[l]);
        c->capturing = 0;
      }
      if (ec == cudaSuccess) ec = cudaEventRecord(ev, s0);
    }
    if (ec == cudaSuccess) ec = cudaStreamWaitEvent(origin, ev, 0);
    cudaGraph_t done = nullptr;
    e = cudaStreamEndCapture(origin, &done);
    if (ec != cudaSuccess) e = ec;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int rc = e == cudaSuccess ? JET_OK : bfail(nullptr, JET_ERR_CUDA, "uncoarsening graph", e);
  for (int l = 0; l < n_levels && rc == JET_OK; ++l) {
    const int r = jet::sync_counters(levels[l]);
    if (r) rc = bfail(nullptr, r, levels[l]->err);
  }
  if (rc == JET_OK && results) memcpy(results, res, sizeof(jet_refine_result) * n_levels);
  if (exec) cudaGraphExecDestroy(exec);
  if (g) cudaGraphDestroy(g);
  if (res) cudaFreeHost(res);
  if (ev) cudaEventDestroy(ev);
  if (origin) cudaStreamDestroy(origin);
  return rc;
}

}  // extern "C"
