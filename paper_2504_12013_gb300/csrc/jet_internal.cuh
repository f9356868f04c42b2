// Internal declarations of libjet (deterministic Jet refinement on sm_103a).
//
// Device data layout (all int32 unless noted):
//   caller-owned: eptr/vptr (int64 CSR offsets), pins, inc, vwgt, ewgt,
//                 part[n], phi[m*k] (row-major by edge), block_w[k] (int64),
//                 locked[n] (uint8)
//   context-owned (workspace):
//     mask[m*2*KWP]  per edge KWP uint32 words of Lambda(e) = {i : phi_e[i] > 0}
//                    then KWP words of {i : phi_e[i] > 1} (KWP = ceil(k/32)
//                    rounded up to 1,2,4,8, so a row is aligned vector loads)
//     cand[n]        uint64 move-candidate record (0 = not in M), see below
//     rg[n]          recomputed gain of Algorithm 2 (zeroed after use)
//     mv_v/mv_st[n]  move list: vertex, (source | target << 16)
//     vcount[k]      vertices per block (segment sizes for rebalancing)
//     rb_*           rebalancing records and per-block state
//     class lists    vertex / edge ids by size class (built once)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "jet.h"

namespace jet {

constexpr int kMaxK = 256;
constexpr int kLightPlanes = 6;      // thread-per-vertex gain path: weighted degree < 2^6
constexpr int kTinyEdge = 8;         // thread-per-edge afterburner: |e| <= 8
constexpr int kWarpEdge = 128;       // warp-per-edge afterburner: 8 < |e| <= 128
constexpr int kSegPins = 2048;       // block-class edges are cut into segments of at most this many pins
constexpr int kHalfMidEdge = 16;     // warp-class edges of at most 16 pins: a half warp per edge
constexpr int kSmallMidEdge = 32;    // warp-class edges of at most 32 pins: one pin per lane, pipelined
constexpr int kPrioShift = 30;       // exact rebalancing priority encoding (needs c(v) <= 2^15)
constexpr int kMaxVertexWeight = 32767;

// Candidate record: bits 63..32 = INT32_MAX - gain (so smaller = earlier in
// the order "gain desc"), bits 23..16 = t(v), bits 15..8 = Pi(v), bit 0 = 1.
// The afterburner order key of v is (record & ~0xffffffff) | v.
__host__ __device__ inline uint64_t pack_cand(int32_t g, int s, int t) {
  uint32_t hi = (uint32_t)((int64_t)INT32_MAX - (int64_t)g);
  return ((uint64_t)hi << 32) | ((uint64_t)(uint32_t)t << 16) | ((uint64_t)(uint32_t)s << 8) | 1ull;
}
__host__ __device__ inline int cand_s(uint64_t r) { return (int)((r >> 8) & 0xff); }
__host__ __device__ inline int cand_t(uint64_t r) { return (int)((r >> 16) & 0xff); }
__host__ __device__ inline int32_t cand_gain(uint64_t r) { return (int32_t)((int64_t)INT32_MAX - (int64_t)(r >> 32)); }
__host__ __device__ inline uint64_t cand_key(uint64_t r, int32_t v) { return (r & 0xffffffff00000000ull) | (uint32_t)v; }

// Device-side counters of one call (one cache line each group).
struct Counters {
  unsigned long long n_moves;     // entries in the move list
  unsigned long long n_cand;      // |M|
  unsigned long long approved;    // afterburner-approved moves
  unsigned long long unused0;
  long long objective;            // (lambda-1), accumulated
  long long rb_rounds;
  long long rb_moves;
  // work counts of the current call (jet_profile_work): vertices of overloaded blocks met by the
  // rebalancing target passes, vertices they evaluated, the incidences of those, incidences moved
  unsigned long long w_over, w_eval, w_eval_pins, w_apply_pins;
  unsigned long long n_rec;       // rebalancing records of the current round
  int rb_done;                    // rebalancing loop may stop
  int rb_any;                     // an overloaded block exists
  int err;                        // bit flags of data errors found on the device
  int pad[5];
};

enum : int { kErrPartRange = 1, kErrPinRange = 2, kErrIncRange = 4, kErrOffsets = 8, kErrWeight = 16,
             kErrTranspose = 32, kErrMapRange = 64 };

// Per-block state of one rebalancing round (Section 4.3).
struct RbBlock {
  long long bw;                  // c(V_b) at the start of the round
  long long cap;                 // max c(v) that may still enter b (-1: overloaded or in the deadzone)
  long long excess;              // c(V_b) - L_max if overloaded
  long long before;              // selection: weight of b's records below the fixed key prefix
  unsigned long long pre_hi;     // selection: fixed prefix of the threshold key (high word)
  unsigned long long pre_lo;     //   ... (low word)
  int over;                      // 1 if c(V_b) > L_max
  int all;                       // selection: every record of b moves
};

// Device-side state of jet_refine's loop control (Algorithm 1).
struct RefineState {
  long long best;         // (lambda-1) of the best balanced partition so far
  int have_best;          // a balanced partition has been seen
  int snap;               // the last iteration improved: snapshot the partition
  int it;                 // iterations since the last improvement (Algorithm 1's counter)
  int in_phase;           // iterations of the current temperature
  jet_refine_result res;  // the summary returned to the caller
};

constexpr int kRbMaxDigit = 11;  // widest radix-select digit (bins per block row <= 2048)

}  // namespace jet

struct jet_ctx {
  // problem (caller-owned device arrays)
  int32_t n = 0, m = 0;
  int64_t P = 0;
  const int64_t *eptr = nullptr, *vptr = nullptr;
  const int32_t *pins = nullptr, *inc = nullptr, *vwgt = nullptr, *ewgt = nullptr;
  jet_params params{};
  int32_t k = 0, kwp = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int launch_sms = 0;  // SMs the grids are sized for (num_sms, or a share of it inside a batch)

  // balance constants (Section 2, Section 4.3)
  int64_t W = 0, A = 0, Lmax = 0, dz_min = 0;
  int64_t max_wdeg = 0;
  int32_t cmax = 0;
  int unit_ewgt = 0;  // every edge with pins has omega(e) = 1
  int stage_bps[2] = {1, 1};  // resident blocks per SM: staged candidate / rebalancing-target kernels
  // resident blocks per SM of the grid-stride kernels, so that each grid is whole waves:
  // k_apply, k_rb_apply (64-bit, 128-bit keys) | k_ab_tiny, k_ab_warp_small<16>, k_ab_warp_small<32>,
  // k_ab_warp<4>, k_ab_block, k_ab_warp<2> | k_cand_heavy, k_rbcand_heavy
  int move_bps[3] = {1, 1, 1};
  int ab_bps[6] = {1, 1, 1, 1, 1, 1};
  int heavy_bps[2] = {1, 1};
  // compact rebalancing keys: priority gain*c (gain >= 0) or gain*(L/c) (gain < 0), L = lcm(1..cmax),
  // stored as (Pmax - P) << 32 | v when max_wdeg*(cmax + L) < 2^32
  int rb_compact = 0;
  int64_t rb_L = 1, rb_Pmax = 0;

  // size classes
  int32_t *v_light = nullptr, *v_heavy = nullptr;
  int32_t n_light = 0, n_heavy = 0;
  uint8_t *vheavy = nullptr;  // per vertex: 1 if heavy (weighted degree >= 2^kLightPlanes)
  // one array of m edge ids: [tiny by size | mid <= 32 pins | mid > 32 pins, largest first | big]
  int32_t *e_tiny = nullptr, *e_mid_half = nullptr, *e_mid_small = nullptr, *e_mid = nullptr, *e_big = nullptr;
  int32_t n_tiny = 0, n_mid_half = 0, n_mid_small = 0, n_mid = 0, n_big = 0;
  int32_t n_mid_hi = 0;  // the first n_mid_hi edges of e_mid have 65..128 pins, the rest 33..64
  // block-class edges as segments (largest first): edge, first pin, pins, table slot (-1: the whole edge)
  int4 *ab_seg = nullptr;
  int32_t n_seg = 0;
  int32_t n_slots = 0;                       // edges longer than one segment
  int32_t *ab_slot_edge = nullptr;           // edge of each slot
  unsigned long long *ab_tab = nullptr;      // per slot and block: max departure key, min arrival key
  uint32_t *ab_nm = nullptr;                 // per slot: blocks holding a non-candidate pin (8 words)

  // workspace
  uint32_t *mask = nullptr;
  uint64_t *cand = nullptr;
  int32_t *rg = nullptr;
  int32_t *mv_v = nullptr;
  uint32_t *mv_st = nullptr;
  int32_t *vcount = nullptr;
  jet::Counters *cnt = nullptr;
  jet::Counters *cnt_host = nullptr;  // pinned mirror
  jet::RbBlock *rbb = nullptr;
  uint64_t *rb_hi = nullptr;          // per record: priority part of the rebalancing key
  int32_t *rb_v = nullptr;            // per record: vertex
  int32_t *rb_ct = nullptr;           // per record: c(v) << 16 | block << 8 | target
  unsigned long long *rb_hist = nullptr;  // k x 2^rb_digit weighted digit histograms (zero between uses)
  int rb_hbits = 0, rb_vbits = 1;     // key = rb_hi << rb_vbits | v, rb_hbits + rb_vbits significant bits
  int rb_digit = 1;                   // radix-select digit width: the key in as few levels of <= 16 bits
  int32_t *best_part = nullptr;       // best balanced partition of jet_refine
  uint8_t *locked_ws = nullptr;       // locks of jet_refine
  jet_round_stats *stats_scratch = nullptr;
  jet_round_stats *stats_host = nullptr;  // pinned

  const int32_t *phi_owner = nullptr;  // phi whose bitmasks `mask` holds
  char err[256] = {0};

  // CUDA graphs of jet_refine_round (one per argument set, small cache)
  struct RoundGraph {
    int32_t tau_num = 0, tau_den = 0;
    const void *part = nullptr, *phi = nullptr, *bw = nullptr, *locked = nullptr, *stats = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;                       // template, kept for the event-node updates
    cudaGraphNode_t ev_nodes[2] = {nullptr, nullptr};  // event records around the candidate kernels
  };
  static constexpr int kGraphCache = 6;
  RoundGraph graphs[kGraphCache];
  int graph_next = 0;
  int use_graphs = 1;
  // graph path (every edge two distinct pins): adj[j] = the other pin of incidence j; phi and the
  // bitmasks are then not kept up to date (jet_set_graph_path)
  int graph_path = 0;
  int32_t *adj = nullptr;
  int capturing = 0;
  cudaStream_t cap_stream[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t graph_ev[2] = {nullptr, nullptr};  // idle targets of the graphs' event-record nodes

  // CUDA graph of jet_refine (Algorithm 1 on the device), one cached argument set
  struct RefineGraph {
    std::vector<int32_t> tau;
    int32_t limit = 0;
    const void *part = nullptr, *phi = nullptr, *bw = nullptr, *res = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  RefineGraph refine_graph;
  jet::RefineState *rstate = nullptr;      // device: loop state and summary of jet_refine
  uint32_t *sched_q = nullptr;             // quotient graph bits (k x KWP) of jet_quotient_schedule
  int32_t *sched_counts = nullptr;         // its pair and round counts (device)
  jet_refine_result *res_host = nullptr;   // pinned copy of the summary

  // profiling: kernel launches (always counted) and event pairs per family
  long long kernel_launches = 0;
  long long fam_launches[JET_PROF_FAMILIES] = {0};
  long long fam_calls[JET_PROF_FAMILIES] = {0};
  double fam_ms[JET_PROF_FAMILIES] = {0};
  int prof_on = 0;
  static constexpr int kProfPairs = 2048;
  cudaEvent_t *prof_ev = nullptr;  // 2 * kProfPairs events
  int *prof_fam = nullptr;
  int prof_n = 0;                  // pairs recorded and not yet read
};

namespace jet {

// ---- shared host helpers (jet_abi.cu) ----
int fail(jet_ctx *c, int code, const char *fmt, ...);
int cuda_fail(jet_ctx *c, cudaError_t e, const char *where);
int sync_counters(jet_ctx *c);
cudaError_t reset_counters(jet_ctx *c);
int check_ctx(jet_ctx *c);
int check_tau(jet_ctx *c, int32_t tau_num, int32_t tau_den);
cudaError_t ensure_capture_streams(jet_ctx *c);
cudaError_t capture_iteration(jet_ctx *c, cudaStream_t s_main, cudaStream_t s_body, int32_t tn, int32_t td,
                              int32_t *part, int32_t *phi, int64_t *bw, uint8_t *locked, jet_round_stats *stats,
                              cudaEvent_t ev0, cudaEvent_t ev1);
// ---- device-side Algorithm 1 and batches (jet_graph.cu) ----
int refine_graph(jet_ctx *c, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part, int32_t *phi,
                 int64_t *block_w, jet_refine_result *result);
cudaError_t capture_refine(jet_ctx *c, const int32_t *tau_pairs, int32_t n_tau, int32_t limit, int32_t *part,
                           int32_t *phi, int64_t *block_w, jet_refine_result *result_dst);
void destroy_refine_graph(jet_ctx *c);

// ---- launchers (one per kernel family); all enqueue on ctx->stream ----
// state kernels (k_state.cu)
cudaError_t launch_validate(jet_ctx *c, int64_t *wdeg_tmp, int32_t *degcount_tmp, unsigned long long *scal);
cudaError_t launch_classify(jet_ctx *c, const int64_t *wdeg);
cudaError_t launch_pincounts(jet_ctx *c, const int32_t *part, int32_t *phi, int64_t *block_w);
cudaError_t launch_masks_from_phi(jet_ctx *c, const int32_t *phi);
cudaError_t launch_connectivity_dense(jet_ctx *c, const int32_t *phi, int64_t *out);
cudaError_t launch_objective(jet_ctx *c, const int32_t *part);  // (lambda-1) into cnt->objective
cudaError_t launch_build_adj(jet_ctx *c, int32_t *bad_edges);       // graph path set-up
// candidates (k_cand.cu)
cudaError_t prepare_candidate_kernels(jet_ctx *c);
cudaError_t launch_candidates(jet_ctx *c, int32_t tau_num, int32_t tau_den, const int32_t *part, const int32_t *phi,
                              const uint8_t *locked);
cudaError_t launch_rebalance_candidates(jet_ctx *c, const int32_t *part, const int32_t *phi);
// afterburner (k_ab.cu)
cudaError_t prepare_afterburner(jet_ctx *c);
cudaError_t prepare_afterburner_kernels(jet_ctx *c);  // ab_bps
cudaError_t launch_afterburner(jet_ctx *c, const int32_t *part, const int32_t *phi);
cudaError_t launch_approve(jet_ctx *c, uint8_t *locked, int32_t *rg_out, uint8_t *approved_out, bool build_moves);
cudaError_t launch_export_candidates(jet_ctx *c, int32_t *target, int32_t *gain, uint8_t *in_m);
// moves, rebalancing, loop control (k_moves.cu)
cudaError_t prepare_move_kernels(jet_ctx *c);  // move_bps
cudaError_t launch_apply(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w);  // applies the move list
cudaError_t launch_rb_check(jet_ctx *c, const int64_t *block_w, cudaGraphConditionalHandle cond = 0,
                            int use_cond = 0);
cudaError_t launch_rb_select(jet_ctx *c, const int32_t *part);
cudaError_t launch_rb_apply(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w);  // applies the selection
cudaError_t launch_rb_post(jet_ctx *c, const int64_t *block_w, cudaGraphConditionalHandle cond = 0,
                           int use_cond = 0);
cudaError_t launch_stats(jet_ctx *c, const int64_t *block_w, jet_round_stats *stats, int rebalance_only);
cudaError_t launch_rollback_moves(jet_ctx *c, const int32_t *part, const int32_t *best, const int *enable = nullptr);
// matching schedule of k-way refinement (k_sched.cu)
cudaError_t launch_quotient_schedule(jet_ctx *c, uint32_t *qbits, int32_t *pairs, int32_t *round_of, int32_t *counts);

// Block-wide append to a global list: every thread of the block calls it (same
// iteration); each thread with `sel` gets a distinct slot.  One atomicAdd per
// block instead of one per warp keeps the list counter from serializing.
// s_wc: blockDim.x/32 unsigned, s_base: one unsigned long long, both shared.
__device__ __forceinline__ unsigned long long block_append(bool sel, unsigned long long *counter, unsigned *s_wc,
                                                           unsigned long long *s_base) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, sel);
  if (lane == 0) s_wc[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int i = 0; i < nw; ++i) {
      const unsigned x = s_wc[i];
      s_wc[i] = tot;
      tot += x;
    }
    *s_base = tot ? atomicAdd(counter, (unsigned long long)tot) : 0ull;
  }
  __syncthreads();
  const unsigned long long pos = *s_base + s_wc[wid] + __popc(bal & ((1u << lane) - 1));
  __syncthreads();
  return pos;
}

// jet_refine_host on the caller's stream s (not destroyed); ev_start / ev_end (may be NULL) are recorded on s
// before the first upload and after the partition's download (the job's interval on the GPU timeline).
int refine_host_on(const jet_hypergraph *hh, const jet_params *p, const int32_t *tau_pairs, int32_t n_tau,
                   int32_t limit, int32_t *part, jet_refine_result *result, cudaStream_t s, cudaEvent_t ev_start,
                   cudaEvent_t ev_end);

// ---- batched form as one persistent kernel (k_batch.cu)
struct TeamPlan;  // device descriptors of a batch's instances, their queue order and summaries
int team_plan_build(TeamPlan **out, jet_ctx *const *ctxs, int32_t count, int32_t *const *part, int32_t *const *phi,
                    int64_t *const *block_w, const int32_t *tau_pairs, int32_t n_tau, cudaStream_t s);
void team_plan_destroy(TeamPlan *p, cudaStream_t s);
cudaError_t team_launch(TeamPlan *p, int ctas, int threads, long long split_pins, int32_t limit, int32_t iter_cap,
                        cudaStream_t s, const int32_t *sub_order, int32_t n_sub);
cudaError_t team_results(TeamPlan *p, jet_refine_result *dst, cudaStream_t s);
int team_first_error(TeamPlan *p, cudaStream_t s);
std::vector<int32_t> team_sample(TeamPlan *p, int32_t n);
long long team_pins(TeamPlan *p, int32_t i);

// Sets the message returned by jet_last_error(NULL) (for entry points without a context).
void set_global_error(const char *fmt, ...);

// The lanes of the warp whose value equals this lane's (what __match_any_sync
// returns) for values below 2^BITS, from BITS ballots: every lane calls it.
// For a few bits the ballots are cheaper than the general match.
template <int BITS>
__device__ __forceinline__ unsigned match_bits(unsigned x) {
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (x >> b) & 1u;
    const unsigned v = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? v : ~v;
  }
  return peers;
}

// Device memory of the library: stream-ordered allocations from a pool of its
// own, one per device, which keeps the memory the library frees for its next
// calls instead of returning it to the driver at each synchronization (a
// call on host buffers maps gigabytes afresh otherwise).  jet_release_memory
// returns it.
cudaError_t pool_alloc_bytes(void **p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t pool_alloc(T **p, size_t bytes, cudaStream_t s) {
  return pool_alloc_bytes(reinterpret_cast<void **>(p), bytes, s);
}

// Resident blocks per SM of `kernel` at this block size and dynamic shared
// memory (at least 1), for grids sized in whole waves.
template <class K>
inline cudaError_t resident_blocks(K kernel, int threads, size_t smem, int *out) {
  int b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
  *out = b > 0 ? b : 1;
  return e;
}

inline int grid_for(int64_t items, int per_block, int num_sms, int blocks_per_sm = 8) {
  int64_t g = (items + per_block - 1) / per_block;
  int64_t cap = (int64_t)num_sms * blocks_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace jet
