// C ABI of libjet: argument checks, context and workspace, and the host-side
// order of the kernels of one Jet iteration (Algorithm 1) and of the
// temperature schedule (Section 7.2).
#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "jet_internal.cuh"

using namespace jet;

namespace {
thread_local char g_err[256] = {0};

// The library's device memory pools, one per device (created on first use).
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

namespace jet {

int fail(jet_ctx *c, int code, const char *fmt, ...) {
  char *dst = c ? c->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 256, fmt, ap);
  va_end(ap);
  return code;
}

cudaError_t pool_alloc_bytes(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
      uint64_t keep = ~0ull;  // never release at synchronization; jet_release_memory trims
      if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
      }
      g_pools[dev] = pool;
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int cuda_fail(jet_ctx *c, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, JET_ERR_OOM, "%s: out of device memory", where);
  return fail(c, JET_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                 \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

template <class T>
cudaError_t dalloc(jet_ctx *c, T **p, size_t count) {
  return jet::pool_alloc(reinterpret_cast<void **>(p), sizeof(T) * (count > 0 ? count : 1), c->stream);
}

void dfree(jet_ctx *c, void *p) {
  if (p) cudaFreeAsync(p, c->stream);
}

// floor(a / b) and ceil(a / b) for b > 0
__int128 floor_div(__int128 a, __int128 b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__int128 ceil_div(__int128 a, __int128 b) { return -floor_div(-a, b); }

const char *data_error_text(int err) {
  if (err & kErrOffsets) return "CSR offsets are not monotone or do not span [0, P]";
  if (err & kErrWeight) return "a vertex or edge weight is < 1";
  if (err & kErrPinRange) return "a pin id is outside [0, n)";
  if (err & kErrIncRange) return "an incidence (edge id) is outside [0, m)";
  if (err & kErrTranspose) return "vptr/inc is not the transpose of eptr/pins (degree mismatch)";
  if (err & kErrPartRange) return "a partition value is outside [0, k)";
  if (err & kErrMapRange) return "a hierarchy map value is outside the coarser level's vertex range";
  return "data error";
}

// Copy the counters to the host and wait; report device-detected data errors.
int sync_counters(jet_ctx *c) {
  CK(cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream), "counters");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  if (c->cnt_host->err) {
    int err = c->cnt_host->err;
    cudaMemsetAsync(&c->cnt->err, 0, sizeof(int), c->stream);
    return fail(c, JET_ERR_DATA, "%s", data_error_text(err));
  }
  return JET_OK;
}

// zero every counter before `err`
cudaError_t reset_counters(jet_ctx *c) {
  return cudaMemsetAsync(c->cnt, 0, offsetof(Counters, err), c->stream);
}

cudaError_t ensure_masks(jet_ctx *c, const int32_t *phi) {
  if (c->graph_path || c->phi_owner == phi) return cudaSuccess;
  return launch_masks_from_phi(c, phi);
}

// ---- profiling: events around kernel families
enum Fam { F_PIN = 0, F_CAND, F_AB, F_APPROVE, F_APPLY, F_RB_TGT, F_RB_SEL, F_RB_CTL, F_OBJ, F_OTHER };

void prof_flush(jet_ctx *c) {
  if (!c->prof_n) return;
  cudaEventSynchronize(c->prof_ev[2 * c->prof_n - 1]);
  for (int i = 0; i < c->prof_n; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) == cudaSuccess) c->fam_ms[c->prof_fam[i]] += ms;
  }
  c->prof_n = 0;
}

struct ProfScope {
  jet_ctx *c;
  int fam;
  long long l0;
  int slot = -1;
  ProfScope(jet_ctx *c_, int f) : c(c_), fam(f), l0(c_->kernel_launches) {
    if (c->prof_on && c->prof_ev && !c->capturing) {
      if (c->prof_n == jet_ctx::kProfPairs) prof_flush(c);
      slot = c->prof_n++;
      c->prof_fam[slot] = fam;
      cudaEventRecord(c->prof_ev[2 * slot], c->stream);
    }
  }
  ~ProfScope() {
    if (c->capturing) return;  // a graph's kernels are counted when the eager path runs them
    c->fam_launches[fam] += c->kernel_launches - l0;
    c->fam_calls[fam] += 1;
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
  }
};

#define CKP(fam, call, where)     \
  do {                            \
    ProfScope _ps(c, fam);        \
    CK(call, where);              \
  } while (0)

int check_ctx(jet_ctx *c) {
  if (!c) return fail(nullptr, JET_ERR_INVALID_ARG, "context is NULL");
  return JET_OK;
}

// Rebalancing rounds (Section 4.3) until balanced, nothing moved or the cap.
int rebalance_loop(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w) {
  CKP(F_RB_CTL, launch_rb_check(c, block_w), "rebalance check");  // eager form; the graph form is below
  int rc = sync_counters(c);
  if (rc) return rc;
  if (!c->cnt_host->rb_any || c->params.max_rebalance_rounds <= 0) return JET_OK;
  for (;;) {
    CKP(F_RB_TGT, launch_rebalance_candidates(c, part, phi), "rebalance targets");
    CKP(F_RB_SEL, launch_rb_select(c, part), "rebalance select");
    CKP(F_APPLY, launch_rb_apply(c, part, phi, block_w), "rebalance apply");
    CKP(F_RB_CTL, launch_rb_post(c, block_w), "rebalance post");
    rc = sync_counters(c);
    if (rc) return rc;
    if (c->cnt_host->rb_done) break;
  }
  return JET_OK;
}

int check_tau(jet_ctx *c, int32_t tau_num, int32_t tau_den) {
  if (tau_den <= 0 || tau_num < 0 || tau_num >= tau_den)
    return fail(c, JET_ERR_INVALID_ARG, "temperature %d/%d is outside [0, 1)", tau_num, tau_den);
  return JET_OK;
}

// Streams and events used while capturing this context's graphs (created once).
cudaError_t ensure_capture_streams(jet_ctx *c) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    if (!c->cap_stream[i]) e = cudaStreamCreateWithFlags(&c->cap_stream[i], cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!c->graph_ev[i]) e = cudaEventCreate(&c->graph_ev[i]);
  return e;
}

// ---- CUDA-graph form of jet_refine_round
// The kernels of one iteration are captured once per argument set: the
// candidate, afterburner, approval and apply kernels, then a WHILE node whose
// body is one rebalancing round (its condition is set on the device by the
// check kernel before the node and by the post kernel at the end of each
// round), then the objective and statistics.  One launch, no host
// synchronization.  Event-record nodes (ev0/ev1, optional) bracket the
// candidate kernels so the profiler can time them inside the graph.
// s_main must be capturing (into a top-level graph or into the body of an
// enclosing conditional node); the rebalancing body is captured on s_body.
cudaError_t capture_iteration(jet_ctx *c, cudaStream_t s_main, cudaStream_t s_body, int32_t tn, int32_t td,
                              int32_t *part, int32_t *phi, int64_t *bw, uint8_t *locked, jet_round_stats *stats,
                              cudaEvent_t ev0, cudaEvent_t ev1) {
  cudaStream_t saved = c->stream;
  c->stream = s_main;
  cudaError_t e = [&]() -> cudaError_t {
    cudaError_t e;
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(s_main, &st, nullptr, &cg, &deps, &ed, &nd)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    if ((e = reset_counters(c)) != cudaSuccess) return e;
    // external records become event-record nodes (a plain record in capture only orders streams)
    if (ev0 && (e = cudaEventRecordWithFlags(ev0, s_main, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = launch_candidates(c, tn, td, part, phi, locked)) != cudaSuccess) return e;
    if (ev1 && (e = cudaEventRecordWithFlags(ev1, s_main, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = launch_afterburner(c, part, phi)) != cudaSuccess) return e;
    if ((e = launch_approve(c, locked, nullptr, nullptr, true)) != cudaSuccess) return e;
    if ((e = launch_apply(c, part, phi, bw)) != cudaSuccess) return e;
    if ((e = launch_rb_check(c, bw, h, 1)) != cudaSuccess) return e;
    // WHILE node: rebalancing rounds
    if ((e = cudaStreamGetCaptureInfo(s_main, &st, nullptr, &cg, &deps, &ed, &nd)) != cudaSuccess) return e;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    if ((e = cudaGraphAddNode(&cn, cg, deps, ed, nd, &cp)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s_main, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
      return e;
    c->stream = s_body;
    cudaError_t eb = launch_rebalance_candidates(c, part, phi);
    if (eb == cudaSuccess) eb = launch_rb_select(c, part);
    if (eb == cudaSuccess) eb = launch_rb_apply(c, part, phi, bw);
    if (eb == cudaSuccess) eb = launch_rb_post(c, bw, h, 1);
    cudaGraph_t tmp = nullptr;
    e = cudaStreamEndCapture(s_body, &tmp);
    c->stream = s_main;
    if (eb != cudaSuccess) return eb;
    if (e != cudaSuccess) return e;
    if ((e = launch_objective(c, part)) != cudaSuccess) return e;
    return launch_stats(c, bw, stats, 0);
  }();
  c->stream = saved;
  return e;
}

int round_graph(jet_ctx *c, int32_t tn, int32_t td, int32_t *part, int32_t *phi, int64_t *bw, uint8_t *locked,
                jet_round_stats *stats) {
  jet_ctx::RoundGraph *G = nullptr;
  for (auto &g : c->graphs)
    if (g.exec && g.tau_num == tn && g.tau_den == td && g.part == part && g.phi == phi && g.bw == bw &&
        g.locked == locked && g.stats == stats)
      G = &g;
  if (!G) {
    CK(ensure_capture_streams(c), "capture streams");
    G = &c->graphs[c->graph_next];
    c->graph_next = (c->graph_next + 1) % jet_ctx::kGraphCache;
    if (G->exec) {
      cudaGraphExecDestroy(G->exec);
      G->exec = nullptr;
    }
    if (G->graph) {
      cudaGraphDestroy(G->graph);
      G->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "graph");
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap_stream[0], g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      c->capturing = 1;
      cudaError_t ec = capture_iteration(c, c->cap_stream[0], c->cap_stream[1], tn, td, part, phi, bw, locked, stats,
                                         c->graph_ev[0], c->graph_ev[1]);
      c->capturing = 0;
      cudaGraph_t done = nullptr;
      e = cudaStreamEndCapture(c->cap_stream[0], &done);
      if (ec != cudaSuccess) e = ec;
    }
    G->ev_nodes[0] = G->ev_nodes[1] = nullptr;
    if (e == cudaSuccess) {  // the event-record nodes around the candidate kernels
      size_t nn = 0;
      e = cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
      for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
        if (ev == c->graph_ev[0]) G->ev_nodes[0] = nodes[i];
        if (ev == c->graph_ev[1]) G->ev_nodes[1] = nodes[i];
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      G->exec = nullptr;
      return cuda_fail(c, e, "round graph");
    }
    G->graph = g;
    G->tau_num = tn;
    G->tau_den = td;
    G->part = part;
    G->phi = phi;
    G->bw = bw;
    G->locked = locked;
    G->stats = stats;
  }
  // the candidate kernels' event pair: a profiler slot while profiling, else the idle pair
  cudaEvent_t e0 = c->graph_ev[0], e1 = c->graph_ev[1];
  if (c->prof_on && c->prof_ev) {
    if (c->prof_n == jet_ctx::kProfPairs) prof_flush(c);
    const int slot = c->prof_n++;
    c->prof_fam[slot] = F_CAND;
    e0 = c->prof_ev[2 * slot];
    e1 = c->prof_ev[2 * slot + 1];
    c->fam_calls[F_CAND] += 1;
  }
  if (G->ev_nodes[0] && G->ev_nodes[1]) {
    CK(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_nodes[0], e0), "graph event");
    CK(cudaGraphExecEventRecordNodeSetEvent(G->exec, G->ev_nodes[1], e1), "graph event");
  }
  CK(cudaGraphLaunch(G->exec, c->stream), "graph launch");
  return JET_OK;
}

}  // namespace jet

void jet::set_global_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" {

const char *jet_last_error(const jet_ctx *ctx) { return ctx ? ctx->err : g_err; }

int jet_release_memory(void) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (int d = 0; d < kMaxDevices; ++d) {
    if (!g_pools[d]) continue;
    const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
    if (e != cudaSuccess) return fail(nullptr, JET_ERR_CUDA, "memory pool of device %d: %s", d, cudaGetErrorString(e));
  }
  return JET_OK;
}

int jet_ctx_create(jet_ctx **out, const jet_hypergraph *hg, const jet_params *p, void *stream) {
  if (!out) return fail(nullptr, JET_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!hg || !p) return fail(nullptr, JET_ERR_INVALID_ARG, "hypergraph or params is NULL");
  if (hg->n < 0 || hg->m < 0 || hg->P < 0) return fail(nullptr, JET_ERR_INVALID_ARG, "negative size");
  if (p->k < 2 || p->k > kMaxK) return fail(nullptr, JET_ERR_INVALID_ARG, "k = %d is outside [2, %d]", p->k, kMaxK);
  if (p->eps_den <= 0 || p->eps_num < 0 || p->d_den <= 0 || p->d_num < 0 || p->max_rebalance_rounds < 0)
    return fail(nullptr, JET_ERR_INVALID_ARG, "eps/d must be non-negative fractions with positive denominators");
  if (!hg->eptr || !hg->vptr || (hg->P > 0 && (!hg->pins || !hg->inc)) || (hg->n > 0 && !hg->vwgt) ||
      (hg->m > 0 && !hg->ewgt))
    return fail(nullptr, JET_ERR_INVALID_ARG, "a hypergraph array is NULL");
  jet_ctx *c = new (std::nothrow) jet_ctx();
  if (!c) return fail(nullptr, JET_ERR_OOM, "host allocation failed");
  c->n = hg->n;
  c->m = hg->m;
  c->P = hg->P;
  c->eptr = hg->eptr;
  c->vptr = hg->vptr;
  c->pins = hg->pins;
  c->inc = hg->inc;
  c->vwgt = hg->vwgt;
  c->ewgt = hg->ewgt;
  c->params = *p;
  c->k = p->k;
  const int kw = (p->k + 31) / 32;
  c->kwp = kw <= 1 ? 1 : kw <= 2 ? 2 : kw <= 4 ? 4 : 8;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  int rc = JET_OK;
  int64_t *wdeg = nullptr;
  int32_t *degc = nullptr;
  unsigned long long *scal = nullptr;
  unsigned long long hscal[4] = {0, 0, 0, 0};
  do {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { rc = cuda_fail(c, e, "device query"); break; }
    c->launch_sms = c->num_sms;
    if ((e = dalloc(c, &c->cnt, 1)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void **>(&c->cnt_host), sizeof(Counters))) != cudaSuccess ||
        (e = dalloc(c, &wdeg, c->n)) != cudaSuccess || (e = dalloc(c, &degc, c->n)) != cudaSuccess ||
        (e = dalloc(c, &scal, 4)) != cudaSuccess) {
      rc = cuda_fail(c, e, "context allocation");
      break;
    }
    memset(c->cnt_host, 0, sizeof(Counters));
    if ((e = cudaMemsetAsync(c->cnt, 0, sizeof(Counters), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(degc, 0, sizeof(int32_t) * (c->n > 0 ? c->n : 1), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(scal, 0, sizeof(unsigned long long) * 4, c->stream)) != cudaSuccess) {
      rc = cuda_fail(c, e, "context init");
      break;
    }
    if ((e = launch_validate(c, wdeg, degc, scal)) != cudaSuccess) { rc = cuda_fail(c, e, "validation"); break; }
    if ((e = cudaMemcpyAsync(hscal, scal, sizeof(hscal), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) {
      rc = cuda_fail(c, e, "validation");
      break;
    }
    if ((rc = sync_counters(c)) != JET_OK) break;
    c->W = (int64_t)hscal[0];
    c->max_wdeg = (int64_t)hscal[1];
    c->cmax = (int32_t)hscal[2];
    c->unit_ewgt = hscal[3] <= 1 ? 1 : 0;
    if ((e = prepare_candidate_kernels(c)) != cudaSuccess || (e = prepare_move_kernels(c)) != cudaSuccess ||
        (e = prepare_afterburner_kernels(c)) != cudaSuccess) {
      rc = cuda_fail(c, e, "kernel set-up");
      break;
    }
    if (c->max_wdeg >= (1ll << 31) - 1) {
      rc = fail(c, JET_ERR_OVERFLOW, "a sum of omega over I(v) (%lld) does not fit the int32 gains",
                (long long)c->max_wdeg);
      break;
    }
    if (c->cmax > kMaxVertexWeight) {
      rc = fail(c, JET_ERR_OVERFLOW, "c(v) = %d exceeds %d (exact rebalancing priorities)", c->cmax, kMaxVertexWeight);
      break;
    }
    if (c->W >= (1ll << 50)) { rc = fail(c, JET_ERR_OVERFLOW, "c(V) too large"); break; }
    // balance constants (Section 2) and the deadzone bound (Section 4.3)
    const __int128 A = ((__int128)c->W + c->k - 1) / c->k;
    c->A = (int64_t)A;
    c->Lmax = (int64_t)(((__int128)(p->eps_den + (int64_t)p->eps_num) * A) / p->eps_den);
    const __int128 R = (__int128)p->d_den * ((int64_t)p->eps_den + p->eps_num) * A - (__int128)p->d_num * p->eps_num * A;
    const __int128 D = (__int128)p->eps_den * p->d_den;
    c->dz_min = (int64_t)ceil_div(R, D);
    {  // exact 32-bit rebalancing priorities when lcm(1..cmax) keeps them small
      __int128 L = 1;
      for (int x = 2; x <= c->cmax && L < ((__int128)1 << 40); ++x) {
        __int128 a = L, b = x;
        while (b) { __int128 t = a % b; a = b; b = t; }
        L = L / a * x;
      }
      const __int128 span = (__int128)c->max_wdeg * (c->cmax + L);
      c->rb_compact = (L < ((__int128)1 << 40) && span < ((__int128)1 << 32)) ? 1 : 0;
      c->rb_L = c->rb_compact ? (int64_t)L : 1;
      c->rb_Pmax = (int64_t)c->max_wdeg * c->cmax;
      int hb = 0;
      while (hb < 64 && (((__int128)1 << hb) <= span)) ++hb;  // bit length of the largest priority part
      c->rb_hbits = c->rb_compact ? hb : 64;
      int vb = 1;
      while (vb < 31 && (1ll << vb) < (long long)c->n) ++vb;  // vertex ids need vb bits
      c->rb_vbits = vb;
      // fewest levels of <= kRbMaxDigit bits, histograms (k rows of 2^digit) no larger than max(4n, 2048k) bins
      const int tb = c->rb_hbits + c->rb_vbits;
      int levels = (tb + kRbMaxDigit - 1) / kRbMaxDigit;
      int digit = (tb + levels - 1) / levels;
      const long long cap = std::max(4ll * c->n, 2048ll * c->k);
      while (digit > 11 && ((long long)c->k << digit) > cap) {
        ++levels;
        digit = (tb + levels - 1) / levels;
      }
      c->rb_digit = digit;
    }
    // class lists, workspace
    if ((e = dalloc(c, &c->v_light, c->n)) != cudaSuccess || (e = dalloc(c, &c->e_tiny, (size_t)c->m)) != cudaSuccess ||
        (e = dalloc(c, &c->mask, (size_t)c->m * 2 * c->kwp)) != cudaSuccess || (e = dalloc(c, &c->cand, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->rg, c->n)) != cudaSuccess || (e = dalloc(c, &c->mv_v, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->mv_st, c->n)) != cudaSuccess || (e = dalloc(c, &c->vcount, c->k)) != cudaSuccess ||
        (e = dalloc(c, &c->rbb, c->k)) != cudaSuccess || (e = dalloc(c, &c->rb_hi, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->rb_v, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->rb_hist, (size_t)c->k << c->rb_digit)) != cudaSuccess ||
        (e = dalloc(c, &c->rb_ct, c->n)) != cudaSuccess || (e = dalloc(c, &c->best_part, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->locked_ws, c->n)) != cudaSuccess || (e = dalloc(c, &c->vheavy, c->n)) != cudaSuccess ||
        (e = dalloc(c, &c->stats_scratch, 1)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void **>(&c->stats_host), sizeof(jet_round_stats))) != cudaSuccess) {
      rc = cuda_fail(c, e, "workspace allocation");
      break;
    }
    if ((e = cudaMemsetAsync(c->rg, 0, sizeof(int32_t) * (c->n > 0 ? c->n : 1), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->cand, 0, sizeof(uint64_t) * (c->n > 0 ? c->n : 1), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->vcount, 0, sizeof(int32_t) * c->k, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->rb_hist, 0, sizeof(unsigned long long) * ((size_t)c->k << c->rb_digit), c->stream)) !=
            cudaSuccess) {
      rc = cuda_fail(c, e, "workspace init");
      break;
    }
    if ((e = launch_classify(c, wdeg)) != cudaSuccess) { rc = cuda_fail(c, e, "size classes"); break; }
    if ((e = prepare_afterburner(c)) != cudaSuccess) { rc = cuda_fail(c, e, "edge segments"); break; }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) { rc = cuda_fail(c, e, "context setup"); break; }
  } while (0);
  dfree(c, wdeg);
  dfree(c, degc);
  dfree(c, scal);
  if (rc != JET_OK) {
    snprintf(g_err, sizeof(g_err), "%s", c->err);
    jet_ctx_destroy(c);
    return rc;
  }
  *out = c;
  return JET_OK;
}

void jet_ctx_destroy(jet_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  void *dev[] = {c->cnt, c->v_light, c->e_tiny, c->mask, c->cand, c->rg, c->mv_v, c->mv_st, c->vcount, c->rbb,
                 c->rb_hi, c->rb_v, c->rb_hist, c->rb_ct, c->best_part, c->locked_ws, c->vheavy, c->stats_scratch,
                 c->ab_seg, c->ab_slot_edge, c->ab_tab, c->ab_nm, c->sched_q, c->sched_counts, c->adj};
  for (void *p : dev) dfree(c, p);
  cudaStreamSynchronize(c->stream);
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (int i = 0; i < 3; ++i)
    if (c->cap_stream[i]) cudaStreamDestroy(c->cap_stream[i]);
  for (int i = 0; i < 2; ++i)
    if (c->graph_ev[i]) cudaEventDestroy(c->graph_ev[i]);
  destroy_refine_graph(c);
  if (c->prof_ev) {
    for (int i = 0; i < 2 * jet_ctx::kProfPairs; ++i) cudaEventDestroy(c->prof_ev[i]);
    delete[] c->prof_ev;
    delete[] c->prof_fam;
  }
  if (c->cnt_host) cudaFreeHost(c->cnt_host);
  if (c->stats_host) cudaFreeHost(c->stats_host);
  delete c;
}

int jet_build_pincounts(jet_ctx *c, const int32_t *part, int32_t *phi, int64_t *block_w) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((c->n > 0 && !part) || (c->m > 0 && !phi && !c->graph_path) || !block_w)
    return fail(c, JET_ERR_INVALID_ARG, "part, phi or block_w is NULL");
  CKP(F_PIN, launch_pincounts(c, part, phi, block_w), "pin counts");
  return JET_OK;
}

int jet_connectivity(jet_ctx *c, const int32_t *phi, int64_t *objective_out) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((c->m > 0 && !phi) || !objective_out) return fail(c, JET_ERR_INVALID_ARG, "phi or objective_out is NULL");
  CKP(F_OTHER, launch_connectivity_dense(c, phi, objective_out), "connectivity");
  return JET_OK;
}

int jet_candidates(jet_ctx *c, int32_t tau_num, int32_t tau_den, const int32_t *part, const int32_t *phi,
                   const uint8_t *locked, int32_t *target, int32_t *gain, uint8_t *in_m) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = check_tau(c, tau_num, tau_den))) return rc;
  if (c->n > 0 && (!part || !locked || !target || !gain || !in_m)) return fail(c, JET_ERR_INVALID_ARG, "NULL array");
  if (c->m > 0 && !phi && !c->graph_path) return fail(c, JET_ERR_INVALID_ARG, "phi is NULL");
  CKP(F_PIN, ensure_masks(c, phi), "bitmasks");
  CKP(F_CAND, launch_candidates(c, tau_num, tau_den, part, phi, locked), "candidates");
  CKP(F_OTHER, launch_export_candidates(c, target, gain, in_m), "candidates export");
  return JET_OK;
}

int jet_afterburner(jet_ctx *c, const int32_t *part, const int32_t *phi, int32_t *rg, uint8_t *approved) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (c->n > 0 && (!part || !rg || !approved)) return fail(c, JET_ERR_INVALID_ARG, "NULL array");
  if (c->m > 0 && !phi && !c->graph_path) return fail(c, JET_ERR_INVALID_ARG, "phi is NULL");
  CKP(F_PIN, ensure_masks(c, phi), "bitmasks");
  CK(reset_counters(c), "counters");
  CKP(F_AB, launch_afterburner(c, part, phi), "afterburner");
  CKP(F_APPROVE, launch_approve(c, nullptr, rg, approved, false), "approve");
  return JET_OK;
}

int jet_rebalance(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w, jet_round_stats *stats) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((c->n > 0 && !part) || (c->m > 0 && !phi && !c->graph_path) || !block_w)
    return fail(c, JET_ERR_INVALID_ARG, "part, phi or block_w is NULL");
  CKP(F_PIN, ensure_masks(c, phi), "bitmasks");
  CK(reset_counters(c), "counters");
  if ((rc = rebalance_loop(c, part, phi, block_w))) return rc;
  CKP(F_OBJ, launch_objective(c, part), "objective");
  CKP(F_OBJ, launch_stats(c, block_w, stats ? stats : c->stats_scratch, 1), "stats");
  return JET_OK;
}

int jet_refine_round(jet_ctx *c, int32_t tau_num, int32_t tau_den, int32_t *part, int32_t *phi, int64_t *block_w,
                     uint8_t *locked, jet_round_stats *stats) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if ((rc = check_tau(c, tau_num, tau_den))) return rc;
  if ((c->n > 0 && (!part || !locked)) || (c->m > 0 && !phi && !c->graph_path) || !block_w)
    return fail(c, JET_ERR_INVALID_ARG, "part, phi, block_w or locked is NULL");
  CKP(F_PIN, ensure_masks(c, phi), "bitmasks");
  if (!stats) stats = c->stats_scratch;
  if (c->use_graphs) return round_graph(c, tau_num, tau_den, part, phi, block_w, locked, stats);
  CK(reset_counters(c), "counters");
  CKP(F_CAND, launch_candidates(c, tau_num, tau_den, part, phi, locked), "candidates");
  CKP(F_AB, launch_afterburner(c, part, phi), "afterburner");
  CKP(F_APPROVE, launch_approve(c, locked, nullptr, nullptr, true), "approve");
  CKP(F_APPLY, launch_apply(c, part, phi, block_w), "apply");
  if ((rc = rebalance_loop(c, part, phi, block_w))) return rc;
  CKP(F_OBJ, launch_objective(c, part), "objective");
  CKP(F_OBJ, launch_stats(c, block_w, stats, 0), "stats");
  return JET_OK;
}

int jet_set_graph_mode(jet_ctx *c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->use_graphs = enable ? 1 : 0;
  return JET_OK;
}

int jet_set_graph_path(jet_ctx *c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  enable = enable ? 1 : 0;
  if (enable == c->graph_path) return JET_OK;
  if (enable) {
    if (!c->adj) CK(dalloc(c, &c->adj, (size_t)c->P), "adjacency");
    int32_t *bad = nullptr;
    int32_t h_bad = 0;
    CK(dalloc(c, &bad, 1), "scratch");
    cudaError_t e = launch_build_adj(c, bad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    dfree(c, bad);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph path set-up");
    if (h_bad) return fail(c, JET_ERR_INVALID_ARG, "the graph path needs every edge to have two distinct pins (%d do not)",
                           h_bad);
  } else {
    CK(cudaStreamSynchronize(c->stream), "synchronize");
  }
  // captured graphs bake in the path: drop them
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = jet_ctx::RoundGraph{};
  }
  destroy_refine_graph(c);
  c->graph_path = enable;
  c->phi_owner = nullptr;  // the bitmasks are stale after the graph path ran
  return JET_OK;
}

int jet_refine(jet_ctx *c, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part, int32_t *phi,
               int64_t *block_w, jet_refine_result *result) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n_tau < 0 || (n_tau > 0 && !tau_pairs) || limit < 1)
    return fail(c, JET_ERR_INVALID_ARG, "bad schedule (n_tau %d, limit %d)", n_tau, limit);
  for (int i = 0; i < n_tau; ++i)
    if ((rc = check_tau(c, tau_pairs[2 * i], tau_pairs[2 * i + 1]))) return rc;
  if ((c->n > 0 && !part) || (c->m > 0 && !phi && !c->graph_path) || !block_w || !result)
    return fail(c, JET_ERR_INVALID_ARG, "part, phi, block_w or result is NULL");
  memset(result, 0, sizeof(*result));
  if (c->use_graphs) return refine_graph(c, tau_pairs, n_tau, limit, part, phi, block_w, result);
  jet_round_stats *st = c->stats_host;
  auto read_stats = [&]() -> int {
    CK(cudaMemcpyAsync(st, c->stats_scratch, sizeof(jet_round_stats), cudaMemcpyDeviceToHost, c->stream), "stats");
    return sync_counters(c);
  };
  CKP(F_PIN, launch_pincounts(c, part, phi, block_w), "pin counts");
  CK(reset_counters(c), "counters");
  CKP(F_OBJ, launch_objective(c, part), "objective");
  CKP(F_OBJ, launch_stats(c, block_w, c->stats_scratch, 1), "stats");
  if ((rc = read_stats())) return rc;
  result->initial_objective = st->objective;
  bool have_best = !st->imbalanced;
  int64_t best_obj = st->objective;
  if (have_best && c->n > 0)
    CK(cudaMemcpyAsync(c->best_part, part, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
  for (int ti = 0; ti < n_tau; ++ti) {
    if (c->n > 0) CK(cudaMemsetAsync(c->locked_ws, 0, c->n, c->stream), "locks");
    int it = 0;
    int64_t in_phase = 0;
    while (it < limit) {
      if ((rc = jet_refine_round(c, tau_pairs[2 * ti], tau_pairs[2 * ti + 1], part, phi, block_w, c->locked_ws,
                                 c->stats_scratch)))
        return rc;
      if ((rc = read_stats())) return rc;
      result->iterations += 1;
      in_phase += 1;
      it += 1;
      if (!st->imbalanced && (!have_best || st->objective < best_obj)) {
        have_best = true;
        best_obj = st->objective;
        if (c->n > 0)
          CK(cudaMemcpyAsync(c->best_part, part, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->stream),
             "snapshot");
        it = 0;
      }
    }
    if (ti < 8) result->phase_iterations[ti] = in_phase;
    if (have_best) {  // rollback to the best balanced partition
      CKP(F_OTHER, launch_rollback_moves(c, part, c->best_part), "rollback");
      CKP(F_APPLY, launch_apply(c, part, phi, block_w), "rollback apply");
    }
  }
  if (c->graph_path && phi) CKP(F_PIN, launch_pincounts(c, part, phi, block_w), "final pin counts");
  CK(reset_counters(c), "counters");
  CKP(F_OBJ, launch_objective(c, part), "objective");
  CKP(F_OBJ, launch_stats(c, block_w, c->stats_scratch, 1), "stats");
  if ((rc = read_stats())) return rc;
  result->objective = st->objective;
  result->balanced = !st->imbalanced;
  return JET_OK;
}

int jet_profile_enable(jet_ctx *c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (enable && !c->prof_ev) {
    c->prof_ev = new (std::nothrow) cudaEvent_t[2 * jet_ctx::kProfPairs];
    c->prof_fam = new (std::nothrow) int[jet_ctx::kProfPairs];
    if (!c->prof_ev || !c->prof_fam) return fail(c, JET_ERR_OOM, "profiler allocation");
    for (int i = 0; i < 2 * jet_ctx::kProfPairs; ++i) CK(cudaEventCreate(&c->prof_ev[i]), "profiler events");
  }
  c->prof_on = enable ? 1 : 0;
  return JET_OK;
}

int jet_profile_read(jet_ctx *c, double *ms_out, int64_t *calls_out, int64_t *launches_out, int reset) {
  int rc = check_ctx(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  if (c->prof_ev) prof_flush(c);
  for (int f = 0; f < JET_PROF_FAMILIES; ++f) {
    if (ms_out) ms_out[f] = c->fam_ms[f];
    if (calls_out) calls_out[f] = c->fam_calls[f];
    if (launches_out) launches_out[f] = c->fam_launches[f];
    if (reset) {
      c->fam_ms[f] = 0;
      c->fam_calls[f] = 0;
      c->fam_launches[f] = 0;
    }
  }
  return JET_OK;
}

int jet_quotient_schedule(jet_ctx *c, const int32_t *phi, int32_t *pairs, int32_t *round_of, int32_t *n_pairs,
                          int32_t *n_rounds) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (c->graph_path) return fail(c, JET_ERR_INVALID_ARG, "the matching schedule reads phi: turn the graph path off");
  if (c->m > 0 && !phi) return fail(c, JET_ERR_INVALID_ARG, "phi is NULL");
  if (!pairs || !round_of || !n_pairs || !n_rounds) return fail(c, JET_ERR_INVALID_ARG, "NULL output");
  if (!c->sched_q) {
    CK(dalloc(c, &c->sched_q, (size_t)c->k * c->kwp), "schedule workspace");
    CK(dalloc(c, &c->sched_counts, 2), "schedule workspace");
  }
  CKP(F_PIN, ensure_masks(c, phi), "bitmasks");
  CKP(F_OTHER, launch_quotient_schedule(c, c->sched_q, pairs, round_of, c->sched_counts), "matching schedule");
  int32_t cnt[2];
  CK(cudaMemcpyAsync(cnt, c->sched_counts, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream), "schedule counts");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  *n_pairs = cnt[0];
  *n_rounds = cnt[1];
  return JET_OK;
}

int jet_profile_work(jet_ctx *c, int64_t *out, int32_t n) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (n < 0 || n > 5 || (n > 0 && !out)) return fail(c, JET_ERR_INVALID_ARG, "n must be in [0, 5]");
  unsigned long long w[5];
  CK(cudaMemcpyAsync(w, &c->cnt->w_over, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
     "work counts");
  CK(cudaStreamSynchronize(c->stream), "synchronize");
  const int tb = c->rb_hbits + c->rb_vbits;
  w[4] = (unsigned long long)((tb + c->rb_digit - 1) / c->rb_digit);  // radix-select levels per round
  for (int i = 0; i < n; ++i) out[i] = (int64_t)w[i];
  return JET_OK;
}

int jet_refine_host(const jet_hypergraph *hh, const jet_params *p, const int32_t *tau_pairs, int32_t n_tau,
                    int32_t limit, int32_t *part, jet_refine_result *result) {
  if (!hh || !p || !part) return fail(nullptr, JET_ERR_INVALID_ARG, "NULL argument");
  if (hh->n < 0 || hh->m < 0 || hh->P < 0 || p->k < 2 || p->k > kMaxK)
    return fail(nullptr, JET_ERR_INVALID_ARG, "bad sizes or k");
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(nullptr, JET_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
  const int rc = jet::refine_host_on(hh, p, tau_pairs, n_tau, limit, part, result, s, nullptr, nullptr);
  cudaStreamDestroy(s);
  return rc;
}

}  // extern "C"

namespace {

// A job on host buffers: uploads the hypergraph and part to device buffers of
// its own (stream-ordered on s), creates a context, runs body(ctx, part, phi,
// block_w), downloads part, and frees everything.  ev_start / ev_end (may be
// NULL) are recorded before the first upload and after the download.
template <class Body>
int host_job(const jet_hypergraph *hh, const jet_params *p, int32_t *part, cudaStream_t s, cudaEvent_t ev_start,
             cudaEvent_t ev_end, Body body) {
  if (!hh || !p || !part) return fail(nullptr, JET_ERR_INVALID_ARG, "NULL argument");
  if (hh->n < 0 || hh->m < 0 || hh->P < 0 || p->k < 2 || p->k > kMaxK)
    return fail(nullptr, JET_ERR_INVALID_ARG, "bad sizes or k");
  cudaError_t e = ev_start ? cudaEventRecord(ev_start, s) : cudaSuccess;
  const size_t n = (size_t)hh->n, m = (size_t)hh->m, P = (size_t)hh->P, k = (size_t)p->k;
  int64_t *eptr = nullptr, *vptr = nullptr, *bw = nullptr;
  int32_t *pins = nullptr, *inc = nullptr, *vw = nullptr, *ew = nullptr, *pt = nullptr, *phi = nullptr;
  void **bufs[] = {(void **)&eptr, (void **)&vptr, (void **)&bw, (void **)&pins, (void **)&inc,
                   (void **)&vw, (void **)&ew, (void **)&pt, (void **)&phi};
  size_t sizes[] = {8 * (m + 1), 8 * (n + 1), 8 * k, 4 * (P ? P : 1), 4 * (P ? P : 1),
                    4 * (n ? n : 1), 4 * (m ? m : 1), 4 * (n ? n : 1), 4 * (m * k > 0 ? m * k : 1)};
  int rc = JET_OK;
  for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = jet::pool_alloc(bufs[i], sizes[i], s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eptr, hh->eptr, 8 * (m + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vptr, hh->vptr, 8 * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && P) e = cudaMemcpyAsync(pins, hh->pins, 4 * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && P) e = cudaMemcpyAsync(inc, hh->inc, 4 * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(vw, hh->vwgt, 4 * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(ew, hh->ewgt, 4 * m, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(pt, part, 4 * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) rc = fail(nullptr, e == cudaErrorMemoryAllocation ? JET_ERR_OOM : JET_ERR_CUDA, "upload: %s",
                                  cudaGetErrorString(e));
  jet_ctx *c = nullptr;
  if (rc == JET_OK) {
    jet_hypergraph dh{hh->n, hh->m, hh->P, eptr, pins, vptr, inc, vw, ew};
    rc = jet_ctx_create(&c, &dh, p, s);
  }
  if (rc == JET_OK) {
    rc = body(c, pt, phi, bw);
    if (rc != JET_OK) snprintf(g_err, sizeof(g_err), "%s", c->err);
  }
  if (rc == JET_OK && n) {
    e = cudaMemcpyAsync(part, pt, 4 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && ev_end) e = cudaEventRecord(ev_end, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(nullptr, JET_ERR_CUDA, "download: %s", cudaGetErrorString(e));
  } else if (rc == JET_OK && ev_end) {
    cudaEventRecord(ev_end, s);
  }
  if (c) jet_ctx_destroy(c);
  for (int i = 0; i < 9; ++i)
    if (*bufs[i]) cudaFreeAsync(*bufs[i], s);
  cudaStreamSynchronize(s);
  return rc;
}

}  // namespace

// jet_refine_host on a caller's stream; ev_start / ev_end (may be NULL) are
// recorded before the first upload and after the partition's download.
int jet::refine_host_on(const jet_hypergraph *hh, const jet_params *p, const int32_t *tau_pairs, int32_t n_tau,
                        int32_t limit, int32_t *part, jet_refine_result *result, cudaStream_t s, cudaEvent_t ev_start,
                        cudaEvent_t ev_end) {
  jet_refine_result local;
  return host_job(hh, p, part, s, ev_start, ev_end, [&](jet_ctx *c, int32_t *pt, int32_t *phi, int64_t *bw) {
    return jet_refine(c, tau_pairs, n_tau, limit, pt, phi, bw, result ? result : &local);
  });
}

extern "C" int jet_rounds_host(const jet_hypergraph *hh, const jet_params *p, int32_t tau_num, int32_t tau_den,
                               int32_t n_rounds, int32_t *part, jet_round_stats *stats) {
  if (n_rounds < 0) return fail(nullptr, JET_ERR_INVALID_ARG, "n_rounds = %d is negative", n_rounds);
  if (tau_den <= 0 || tau_num < 0 || tau_num >= tau_den)
    return fail(nullptr, JET_ERR_INVALID_ARG, "temperature %d/%d is outside [0, 1)", tau_num, tau_den);
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(nullptr, JET_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
  const int rc = host_job(hh, p, part, s, nullptr, nullptr, [&](jet_ctx *c, int32_t *pt, int32_t *phi, int64_t *bw) {
    int r = jet_build_pincounts(c, pt, phi, bw);
    if (r) return r;
    if (c->n > 0) CK(cudaMemsetAsync(c->locked_ws, 0, c->n, c->stream), "locks");
    for (int32_t i = 0; i < n_rounds && r == JET_OK; ++i)
      r = jet_refine_round(c, tau_num, tau_den, pt, phi, bw, c->locked_ws, c->stats_scratch);
    if (r) return r;
    if (stats) {
      CK(cudaMemcpyAsync(stats, c->stats_scratch, sizeof(jet_round_stats), cudaMemcpyDeviceToHost, c->stream),
         "stats");
    }
    return sync_counters(c);
  });
  cudaStreamDestroy(s);
  return rc;
}
