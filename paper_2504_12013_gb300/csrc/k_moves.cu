// ApplyMoves (Algorithm 1), deterministic rebalancing rounds (Section 4.3),
// statistics and rollback moves.
//
// All updates are integer atomics whose final values do not depend on their
// order: phi row entries +-1, block weights and counts aggregated per thread
// block, and XOR toggles of the edge bitmasks at the phi crossings.
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void add_i64(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

struct MoveArgs {
  const int64_t *vptr;
  const int32_t *inc, *vwgt;
  int32_t *part, *phi;
  int64_t *bw;
  int32_t *vcount;
  uint32_t *mask;
  const int32_t *mv_v;
  const uint32_t *mv_st;
  int32_t k, kwp;
  int graph;  // graph path: phi and the bitmasks are not kept, a move changes Pi and c(V_i) only
  Counters *cnt;
};

// A group of kMoveLanes lanes per move, the lanes striding over I(v): more
// loads and atomics in flight than one thread per move when the move list is
// short (rebalancing rounds).
constexpr int kMoveLanes = 8;

// The phi and bitmask updates of one move s -> t over the incidences j,
// j + kMoveLanes, ... below j1 (one lane's share of I(v)).  kMoveIlp
// incidences are loaded first and their atomics issued together, so that
// several atomics with return are in flight per lane before the first result
// is needed.
constexpr int kMoveIlp = 4;
// Grids of the apply kernels: this many waves of resident blocks.  The moves
// are dealt to blocks round-robin but their costs differ (degree, hub rows
// shared with other moves), and blocks that finish early take the next wave.
// A block with no move (or record) to take returns at once, so short move
// lists (late rebalancing rounds) do not pay for the large grid.
constexpr int kMoveWaves = 4;
constexpr int kRbMoveWaves = 4;  // the same for the rebalancing apply

__device__ __forceinline__ void move_incidences(const MoveArgs &a, int64_t j, int64_t j1, int s, int t) {
  const uint32_t sbit = 1u << (s & 31), tbit = 1u << (t & 31);
  for (; j < j1; j += kMoveIlp * kMoveLanes) {
    int64_t e[kMoveIlp];
#pragma unroll
    for (int q = 0; q < kMoveIlp; ++q) {
      const int64_t jj = j + q * kMoveLanes;
      e[q] = jj < j1 ? a.inc[jj] : -1;
    }
    int os[kMoveIlp], ot[kMoveIlp];
#pragma unroll
    for (int q = 0; q < kMoveIlp; ++q) {
      os[q] = 0;  // no crossing for an absent incidence
      ot[q] = 2;
      if (e[q] >= 0) {
        os[q] = atomicSub(&a.phi[e[q] * a.k + s], 1);  // os -> os - 1
        ot[q] = atomicAdd(&a.phi[e[q] * a.k + t], 1);  // ot -> ot + 1
      }
    }
#pragma unroll
    for (int q = 0; q < kMoveIlp; ++q) {
      if (e[q] < 0) continue;
      uint32_t *row = a.mask + e[q] * 2 * a.kwp;
      if (os[q] == 1) atomicXor(&row[s >> 5], sbit);           // 1 -> 0
      if (os[q] == 2) atomicXor(&row[a.kwp + (s >> 5)], sbit);  // 2 -> 1
      if (ot[q] == 0) atomicXor(&row[t >> 5], tbit);           // 0 -> 1
      if (ot[q] == 1) atomicXor(&row[a.kwp + (t >> 5)], tbit);  // 1 -> 2
    }
  }
}

// Pi(v) <- t and phi_e[s]--, phi_e[t]++ for every e in I(v); c(V_s), c(V_t)
// and |V_s|, |V_t| through shared-memory partial sums; and both bitmasks of
// every touched edge, exactly, without a second pass: the atomic updates of
// one phi entry are serialized in some order, so its 0 <-> 1 crossings (and
// 1 <-> 2 crossings) alternate, and the final bit is the initial bit XOR the
// parity of the crossings.  Each thread whose own atomic crosses toggles the
// bit with atomicXor; XOR commutes, so the order of the toggles is irrelevant.
__global__ void __launch_bounds__(256) k_apply(MoveArgs a) {
  __shared__ long long s_dw[kMaxK];
  __shared__ int s_dc[kMaxK];
  const long long nm = (long long)a.cnt->n_moves;
  if ((long long)blockIdx.x * (blockDim.x / kMoveLanes) >= nm) return;  // no move for this block
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) { s_dw[b] = 0; s_dc[b] = 0; }
  __syncthreads();
  unsigned long long pins = 0;  // incidences moved by this thread's moves (work count)
  const int sub = threadIdx.x % kMoveLanes;
  const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kMoveLanes;
  const long long ng = ((long long)gridDim.x * blockDim.x) / kMoveLanes;
  for (long long i = g0; i < nm; i += ng) {
    const int v = a.mv_v[i];
    const uint32_t st = a.mv_st[i];
    const int s = st & 0xffff, t = st >> 16;
    if (sub == 0) {
      a.part[v] = t;
      const int c = a.vwgt[v];
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)(-(long long)c));
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[t]), (unsigned long long)c);
      atomicSub(&s_dc[s], 1);
      atomicAdd(&s_dc[t], 1);
    }
    const int64_t j1 = a.vptr[v + 1];
    if (sub == 0) pins += (unsigned long long)(j1 - a.vptr[v]);
    if (a.graph) continue;
    move_incidences(a, a.vptr[v] + sub, j1, s, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pins += __shfl_xor_sync(kFull, pins, o);
  __shared__ unsigned long long s_pins;
  if (threadIdx.x == 0) s_pins = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && pins) atomicAdd(&s_pins, pins);
  __syncthreads();
  if (threadIdx.x == 0 && s_pins) atomicAdd(&a.cnt->w_apply_pins, s_pins);
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    if (s_dw[b]) add_i64(reinterpret_cast<long long *>(&a.bw[b]), s_dw[b]);
    if (s_dc[b]) atomicAdd(&a.vcount[b], s_dc[b]);
  }
}

// ---------------------------------------------------------------- rebalancing
// Selection of the minimal prefix per overloaded block (Section 4.3) as a
// radix select over all records at once.  Every vertex v of an overloaded
// block with a valid target has a record with the key
// K(v) = hi(v) << vb | v  (priority descending, then id ascending, as one
// ascending number of hb + vb bits; 64-bit when it fits, else 128-bit).
// Per level (rb_digit <= kRbMaxDigit = 11 bits, from the top, so a pick scans
// at most 2048 bins per block; three levels cover keys of up to 33 bits) a
// grid-wide pass adds c(v) of every record that matches its
// block's fixed prefix into the (block, digit) histogram -- for the first
// level the target kernels do this while they write the records -- and one
// small kernel per overloaded block picks the digit at which the cumulative
// weight reaches the excess.  After the last level the prefix is the
// threshold key, and every record up to it moves.
typedef unsigned __int128 u128;
constexpr int kPickThreads = 1024;

struct RbArgs {
  const int64_t *bw;
  RbBlock *rbb;
  const uint64_t *rb_hi;
  const int32_t *rb_v, *rb_ct;  // record: vertex; c << 16 | block << 8 | target
  unsigned long long *hist;
  int32_t *mv_v;
  uint32_t *mv_st;
  int32_t n, k;
  int vbits, tbits;
  int digit, bins;               // radix-select digit width and bins per block row
  long long Lmax, dz_min;
  int32_t max_rounds;
  Counters *cnt;
};

// Per-block state of the next round: overloaded flag, excess, target
// capacity (deadzone and L_max), cleared selection state and counters.  One
// block of kMaxK threads, thread b for block b.
__device__ __forceinline__ void rb_prep_blocks(const RbArgs &a) {
  const int b = threadIdx.x;
  if (b < a.k) {
    const long long bwb = a.bw[b];
    RbBlock r;
    r.bw = bwb;
    r.over = bwb > a.Lmax ? 1 : 0;
    r.excess = r.over ? bwb - a.Lmax : 0;
    r.cap = (r.over || bwb >= a.dz_min) ? -1 : a.Lmax - bwb;
    r.before = 0;
    r.pre_hi = 0;
    r.pre_lo = 0;
    r.all = 0;
    a.rbb[b] = r;
  }
  if (b == 0) {
    a.cnt->n_moves = 0;
    a.cnt->n_rec = 0;
  }
}

// Any block above L_max?  If so, the state of the first round.  In a CUDA
// graph (use_cond) it also sets the condition of the rebalancing WHILE node.
__global__ void k_rb_check(RbArgs a, cudaGraphConditionalHandle cond, int use_cond) {
  const int b = threadIdx.x;
  const bool over = b < a.k && a.bw[b] > a.Lmax;
  const int any = __syncthreads_or(over);
  if (b == 0) {
    a.cnt->rb_any = any;
    a.cnt->rb_done = !any;
    if (use_cond) cudaGraphSetConditional(cond, (any && a.max_rounds > 0) ? 1u : 0u);
  }
  if (any) rb_prep_blocks(a);
}

template <class KT>
__device__ __forceinline__ KT rb_full_key(uint64_t hi, int v, int vbits) {
  return ((KT)hi << vbits) | (KT)(uint32_t)v;
}

template <class KT>
__device__ __forceinline__ KT rb_prefix(const RbBlock &r) {
  if constexpr (sizeof(KT) > 8) return ((KT)r.pre_hi << 64) | (KT)r.pre_lo;
  else return (KT)r.pre_lo;
}

// One level: digit = bits [lo, lo + w) of K(v) for the records whose higher bits
// equal their block's prefix; one atomic per matching record.
template <class KT>
__global__ void __launch_bounds__(256) k_rb_level(RbArgs a, int lo, int w) {
  const int up = lo + w;
  const KT dmask = ((KT)1 << w) - 1;
  const long long nrec = (long long)a.cnt->n_rec;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nrec; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    bool m = false;
    int b = 0, d = 0;
    unsigned c = 0;
    if (i < nrec) {
      const int32_t ct = a.rb_ct[i];
      b = (ct >> 8) & 255;
      const RbBlock &r = a.rbb[b];
      if (!r.all) {
        const KT K = rb_full_key<KT>(a.rb_hi[i], a.rb_v[i], a.vbits);
        m = up >= a.tbits || (K >> up) == (rb_prefix<KT>(r) >> up);
        d = (int)((K >> lo) & dmask);
        c = (unsigned)(ct >> 16);
      }
    }
    if (m) atomicAdd(&a.hist[(int64_t)b * a.bins + d], (unsigned long long)c);
  }
}

// Per overloaded block: the digit at which the cumulative weight first reaches
// the excess; at the first level a total below the excess selects everything.
// Warp w owns a contiguous segment of bins and reads it 32 bins at a time
// (coalesced); the warp whose segment holds the threshold walks it again.
// Leaves the histogram row zeroed.
__global__ void __launch_bounds__(kPickThreads) k_rb_pick(RbArgs a, int lo, int first) {
  constexpr int kWarps = kPickThreads / 32;
  const int b = blockIdx.x;
  RbBlock *r = &a.rbb[b];
  if (!r->over || r->all) return;
  __shared__ long long s_warp[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int seg = (a.bins + kWarps - 1) / kWarps;
  const int x0 = wid * seg < a.bins ? wid * seg : a.bins;
  const int x1 = x0 + seg < a.bins ? x0 + seg : a.bins;
  unsigned long long *row = a.hist + (int64_t)b * a.bins;
  long long part = 0;
#pragma unroll 8
  for (int x = x0 + lane; x < x1; x += 32) part += (long long)row[x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
  if (lane == 0) s_warp[wid] = part;
  // read before the barrier: the threshold warp rewrites r->before below
  const long long before = r->before, need = r->excess;
  __syncthreads();
  long long excl = 0, total = 0;
  for (int i = 0; i < kWarps; ++i) {
    if (i < wid) excl += s_warp[i];
    total += s_warp[i];
  }
  if (first && total < need) {
    if (threadIdx.x == 0) r->all = 1;
  } else if (before + excl < need && before + excl + part >= need) {  // warp-uniform
    long long run = before + excl;
    for (int x = x0; x < x1; x += 32) {
      const long long w = x + lane < x1 ? (long long)row[x + lane] : 0;
      long long incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned hit = __ballot_sync(kFull, run + incl >= need);
      if (hit) {
        const int l = __ffs(hit) - 1;
        const long long prev = __shfl_sync(kFull, incl - w, l);
        if (lane == 0) {
          r->before = run + prev;
          const u128 pre = (((u128)r->pre_hi << 64) | r->pre_lo) | ((u128)(unsigned)(x + l) << lo);
          r->pre_hi = (unsigned long long)(pre >> 64);
          r->pre_lo = (unsigned long long)pre;
        }
        break;
      }
      run += __shfl_sync(kFull, incl, 31);
    }
  }
  __syncthreads();  // the threshold walk above reads the row
  for (int x = x0 + lane; x < x1; x += 32) row[x] = 0ull;
}

// Apply the selection: every record with K(v) <= its block's threshold (or of
// an `all` block) moves v to its target.  A warp tests 32 records (one per
// lane) and then applies the selected ones four at a time, kMoveLanes lanes
// per move striding over I(v) as k_apply does; the moves are counted for the
// round's statistics.
template <class KT>
__global__ void __launch_bounds__(256) k_rb_apply(RbArgs r, MoveArgs a) {
  __shared__ long long s_dw[kMaxK];
  __shared__ int s_dc[kMaxK];
  __shared__ unsigned long long s_moves, s_pins;
  const long long nrec = (long long)r.cnt->n_rec;
  if ((long long)blockIdx.x * blockDim.x >= nrec) return;  // no record for this block
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) { s_dw[b] = 0; s_dc[b] = 0; }
  if (threadIdx.x == 0) { s_moves = 0; s_pins = 0; }
  __syncthreads();
  unsigned long long moves = 0, pins = 0;
  const int lane = threadIdx.x & 31, grp = lane / kMoveLanes, sub = lane % kMoveLanes;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = w0 * 32; base < nrec; base += nw * 32) {
    const long long i = base + lane;
    bool sel = false;
    int v = 0;
    int32_t ct = 0;
    if (i < nrec) {
      ct = r.rb_ct[i];
      v = r.rb_v[i];
      const RbBlock &rb = r.rbb[(ct >> 8) & 255];
      KT pre;
      if constexpr (sizeof(KT) > 8) pre = ((KT)rb.pre_hi << 64) | (KT)rb.pre_lo;
      else pre = (KT)rb.pre_lo;
      sel = rb.all || rb_full_key<KT>(r.rb_hi[i], v, r.vbits) <= pre;
    }
    unsigned bal = __ballot_sync(kFull, sel);
    while (bal) {
      const int nsel = __popc(bal);
      const int src = grp < nsel ? (int)__fns(bal, 0, grp + 1) : -1;  // this group's record lane
      const int mv = __shfl_sync(kFull, v, src < 0 ? 0 : src);
      const int32_t mct = __shfl_sync(kFull, ct, src < 0 ? 0 : src);
      if (src >= 0) {
        const int s = (mct >> 8) & 255, t = mct & 255;
        const int64_t j0 = a.vptr[mv], j1 = a.vptr[mv + 1];
        if (sub == 0) {
          a.part[mv] = t;
          const int c = (mct >> 16) & 0xffff;
          atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)(-(long long)c));
          atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[t]), (unsigned long long)c);
          atomicSub(&s_dc[s], 1);
          atomicAdd(&s_dc[t], 1);
          ++moves;
          pins += (unsigned long long)(j1 - j0);
        }
        if (!a.graph) move_incidences(a, j0 + sub, j1, s, t);
      }
      // drop the (up to) 32 / kMoveLanes records just applied
      for (int q = 0; q < 32 / kMoveLanes && bal; ++q) bal &= bal - 1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    moves += __shfl_xor_sync(kFull, moves, o);
    pins += __shfl_xor_sync(kFull, pins, o);
  }
  if (lane == 0) {
    if (moves) atomicAdd(&s_moves, moves);
    if (pins) atomicAdd(&s_pins, pins);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_moves) atomicAdd(&r.cnt->n_moves, s_moves);
    if (s_pins) atomicAdd(&r.cnt->w_apply_pins, s_pins);
  }
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    if (s_dw[b]) add_i64(reinterpret_cast<long long *>(&a.bw[b]), s_dw[b]);
    if (s_dc[b]) atomicAdd(&a.vcount[b], s_dc[b]);
  }
}

// End of a round: count it, and stop if nothing moved, nothing is overloaded
// any more, or the round cap is reached; otherwise the state of the next round.
__global__ void k_rb_post(RbArgs a, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ int s_done;
  const int b = threadIdx.x;
  const bool over = b < a.k && a.bw[b] > a.Lmax;
  const int any = __syncthreads_or(over);
  if (b == 0) {
    const long long moved = (long long)a.cnt->n_moves;
    a.cnt->rb_rounds += 1;
    a.cnt->rb_moves += moved;
    a.cnt->rb_any = any;
    const int done = (moved == 0) || !any || (a.cnt->rb_rounds >= a.max_rounds);
    a.cnt->rb_done = done;
    s_done = done;
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
  __syncthreads();
  if (!s_done) rb_prep_blocks(a);
}

__global__ void k_stats(const int64_t *bw, int32_t k, long long Lmax, const Counters *cnt, jet_round_stats *out,
                        int rebalance_only) {
  __shared__ long long s_mx[256];
  const int b = threadIdx.x;
  s_mx[b] = b < k ? bw[b] : 0;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (b < o && s_mx[b + o] > s_mx[b]) s_mx[b] = s_mx[b + o];
    __syncthreads();
  }
  if (b == 0) {
    jet_round_stats st;
    st.candidates = rebalance_only ? 0 : (long long)cnt->n_cand;
    st.approved = rebalance_only ? 0 : (long long)cnt->approved;
    st.rebalance_rounds = cnt->rb_rounds;
    st.rebalance_moves = cnt->rb_moves;
    st.objective = cnt->objective;
    st.max_block_weight = s_mx[0];
    st.imbalanced = s_mx[0] > Lmax ? 1 : 0;
    st.reserved = 0;
    *out = st;
  }
}

// Moves that take part back to best (rollback at the end of a phase).
__global__ void __launch_bounds__(256) k_rollback_moves(const int32_t *part, const int32_t *best, int32_t n,
                                                        int32_t *mv_v, uint32_t *mv_st, Counters *cnt,
                                                        const int *enable) {
  __shared__ unsigned s_wc[8];
  __shared__ unsigned long long s_base;
  if (enable && !*enable) return;  // uniform: no snapshot to roll back to
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int s = 0, t = 0;
    bool mv = false;
    if (v < n) {
      s = part[v];
      t = best[v];
      mv = s != t && (unsigned)s < kMaxK && (unsigned)t < kMaxK;
    }
    const unsigned long long pos = block_append(mv, &cnt->n_moves, s_wc, &s_base);
    if (mv) {
      mv_v[pos] = (int32_t)v;
      mv_st[pos] = (uint32_t)s | ((uint32_t)t << 16);
    }
  }
}

MoveArgs move_args(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w) {
  MoveArgs a{};
  a.vptr = c->vptr;
  a.inc = c->inc;
  a.vwgt = c->vwgt;
  a.part = part;
  a.phi = phi;
  a.bw = block_w;
  a.vcount = c->vcount;
  a.mask = c->mask;
  a.graph = c->graph_path;
  a.mv_v = c->mv_v;
  a.mv_st = c->mv_st;
  a.k = c->k;
  a.kwp = c->kwp;
  a.cnt = c->cnt;
  return a;
}

RbArgs rb_args(jet_ctx *c, const int64_t *block_w, const int32_t *part) {
  RbArgs a{};
  a.bw = block_w;
  a.rbb = c->rbb;
  a.rb_hi = c->rb_hi;
  a.rb_v = c->rb_v;
  a.rb_ct = c->rb_ct;
  (void)part;
  a.hist = c->rb_hist;
  a.mv_v = c->mv_v;
  a.mv_st = c->mv_st;
  a.n = c->n;
  a.k = c->k;
  a.vbits = c->rb_vbits;
  a.tbits = c->rb_hbits + c->rb_vbits;
  a.digit = c->rb_digit;
  a.bins = 1 << c->rb_digit;
  a.Lmax = c->Lmax;
  a.dz_min = c->dz_min;
  a.max_rounds = c->params.max_rebalance_rounds;
  a.cnt = c->cnt;
  return a;
}

}  // namespace

cudaError_t prepare_move_kernels(jet_ctx *c) {
  cudaError_t e = resident_blocks(k_apply, 256, 0, &c->move_bps[0]);
  if (e == cudaSuccess) e = resident_blocks(k_rb_apply<unsigned long long>, 256, 0, &c->move_bps[1]);
  if (e == cudaSuccess) e = resident_blocks(k_rb_apply<u128>, 256, 0, &c->move_bps[2]);
  return e;
}

cudaError_t launch_apply(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w) {
  if (c->n == 0) return cudaSuccess;
  const MoveArgs a = move_args(c, part, phi, block_w);
  k_apply<<<grid_for((int64_t)c->n * kMoveLanes, 256, c->launch_sms, kMoveWaves * c->move_bps[0]), 256, 0,
            c->stream>>>(a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_check(jet_ctx *c, const int64_t *block_w, cudaGraphConditionalHandle cond, int use_cond) {
  k_rb_check<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w, nullptr), cond, use_cond);
  ++c->kernel_launches;
  return cudaGetLastError();
}

template <class KT>
void rb_select_levels(jet_ctx *c, const RbArgs &a) {
  const int g = grid_for(c->n, 256, c->launch_sms);
  int first = 1;
  for (int hi = a.tbits; hi > 0; first = 0) {
    const int lo = hi - a.digit > 0 ? hi - a.digit : 0;
    if (!first) {  // the first level's histogram comes from the target kernels
      k_rb_level<KT><<<g, 256, 0, c->stream>>>(a, lo, hi - lo);
      ++c->kernel_launches;
    }
    k_rb_pick<<<c->k, kPickThreads, 0, c->stream>>>(a, lo, first);
    ++c->kernel_launches;
    hi = lo;
  }
}

cudaError_t launch_rb_select(jet_ctx *c, const int32_t *part) {
  if (c->n == 0) return cudaSuccess;
  const RbArgs a = rb_args(c, nullptr, part);
  if (a.tbits <= 64) rb_select_levels<unsigned long long>(c, a);
  else rb_select_levels<u128>(c, a);
  return cudaGetLastError();
}

cudaError_t launch_rb_apply(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w) {
  if (c->n == 0) return cudaSuccess;
  const RbArgs r = rb_args(c, block_w, part);
  const MoveArgs a = move_args(c, part, phi, block_w);
  if (r.tbits <= 64)
    k_rb_apply<unsigned long long><<<grid_for(c->n, 256, c->launch_sms, kRbMoveWaves * c->move_bps[1]), 256, 0,
                                     c->stream>>>(r, a);
  else
    k_rb_apply<u128><<<grid_for(c->n, 256, c->launch_sms, kRbMoveWaves * c->move_bps[2]), 256, 0, c->stream>>>(r, a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_post(jet_ctx *c, const int64_t *block_w, cudaGraphConditionalHandle cond, int use_cond) {
  k_rb_post<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w, nullptr), cond, use_cond);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_stats(jet_ctx *c, const int64_t *block_w, jet_round_stats *stats, int rebalance_only) {
  k_stats<<<1, 256, 0, c->stream>>>(block_w, c->k, c->Lmax, c->cnt, stats, rebalance_only);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rollback_moves(jet_ctx *c, const int32_t *part, const int32_t *best, const int *enable) {
  cudaError_t e = cudaMemsetAsync(&c->cnt->n_moves, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess || c->n == 0) return e;
  k_rollback_moves<<<grid_for(c->n, 256, c->launch_sms), 256, 0, c->stream>>>(part, best, c->n, c->mv_v, c->mv_st,
                                                                         c->cnt, enable);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
