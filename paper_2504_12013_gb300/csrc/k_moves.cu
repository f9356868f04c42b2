// ApplyMoves (Algorithm 1), deterministic rebalancing rounds (Section 4.3),
// statistics and rollback moves.
//
// All updates are integer atomics whose final values do not depend on their
// order: phi row entries +-1, block weights and counts aggregated per thread
// block, and the Lambda(e) bitmasks (set the target bit during the move, then
// clear the source bit only if the final phi entry is 0).
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
  Counters *cnt;
};

// Thread per move: Pi(v) <- t, phi_e[s]--, phi_e[t]++ and the bit of t in
// Lambda(e) for every e in I(v); c(V_s), c(V_t) and |V_s|, |V_t| through
// shared-memory partial sums.
__global__ void __launch_bounds__(256) k_apply(MoveArgs a) {
  __shared__ long long s_dw[kMaxK];
  __shared__ int s_dc[kMaxK];
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) { s_dw[b] = 0; s_dc[b] = 0; }
  __syncthreads();
  const long long nm = (long long)a.cnt->n_moves;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm; i += (long long)gridDim.x * blockDim.x) {
    const int v = a.mv_v[i];
    const uint32_t st = a.mv_st[i];
    const int s = st & 0xffff, t = st >> 16;
    a.part[v] = t;
    const int c = a.vwgt[v];
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)(-(long long)c));
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[t]), (unsigned long long)c);
    atomicSub(&s_dc[s], 1);
    atomicAdd(&s_dc[t], 1);
    const int64_t j1 = a.vptr[v + 1];
    const uint32_t tbit = 1u << (t & 31);
    for (int64_t j = a.vptr[v]; j < j1; ++j) {
      const int64_t e = a.inc[j];
      atomicSub(&a.phi[e * a.k + s], 1);
      atomicAdd(&a.phi[e * a.k + t], 1);
      atomicOr(&a.mask[e * a.kwp + (t >> 5)], tbit);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    if (s_dw[b]) add_i64(reinterpret_cast<long long *>(&a.bw[b]), s_dw[b]);
    if (s_dc[b]) atomicAdd(&a.vcount[b], s_dc[b]);
  }
}

// After all moves: clear the source bit of Lambda(e) where phi_e[s] reached 0.
__global__ void __launch_bounds__(256) k_fix_masks(MoveArgs a) {
  const long long nm = (long long)a.cnt->n_moves;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm; i += (long long)gridDim.x * blockDim.x) {
    const int v = a.mv_v[i];
    const int s = a.mv_st[i] & 0xffff;
    const int64_t j1 = a.vptr[v + 1];
    for (int64_t j = a.vptr[v]; j < j1; ++j) {
      const int64_t e = a.inc[j];
      if (a.phi[e * a.k + s] == 0) atomicAnd(&a.mask[e * a.kwp + (s >> 5)], ~(1u << (s & 31)));
    }
  }
}

// ---------------------------------------------------------------- rebalancing
struct RbArgs {
  const int64_t *bw;
  const int32_t *vcount;
  RbBlock *rbb;
  int32_t *rb_cursor;
  const uint64_t *rb_key;
  const int32_t *rb_v, *rb_ct;
  int32_t *mv_v;
  uint32_t *mv_st;
  int32_t k;
  long long Lmax, dz_min;
  int32_t max_rounds;
  Counters *cnt;
};

// Any block above L_max?  One block of 256 threads (k <= 256).
__global__ void k_rb_check(RbArgs a) {
  const int b = threadIdx.x;
  const bool over = b < a.k && a.bw[b] > a.Lmax;
  const int any = __syncthreads_or(over);
  if (b == 0) {
    a.cnt->rb_any = any;
    a.cnt->rb_done = !any;
  }
}

// Per-block state of the round: overloaded flag, excess, target capacity
// (deadzone and L_max), record segment offsets (exclusive scan of |V_b|).
__global__ void k_rb_prep(RbArgs a) {
  __shared__ int s_scan[kMaxK];
  const int b = threadIdx.x;
  long long bwb = 0;
  int cntb = 0;
  if (b < a.k) {
    bwb = a.bw[b];
    cntb = a.vcount[b];
  }
  s_scan[b] = cntb;
  __syncthreads();
  for (int o = 1; o < kMaxK; o <<= 1) {  // inclusive Hillis-Steele scan over 256 entries
    int x = b >= o ? s_scan[b - o] : 0;
    __syncthreads();
    s_scan[b] += x;
    __syncthreads();
  }
  if (b < a.k) {
    RbBlock r;
    r.bw = bwb;
    r.over = bwb > a.Lmax ? 1 : 0;
    r.excess = r.over ? bwb - a.Lmax : 0;
    r.cap = (r.over || bwb >= a.dz_min) ? -1 : a.Lmax - bwb;
    r.off = s_scan[b] - cntb;
    a.rbb[b] = r;
    a.rb_cursor[b] = 0;
  }
  if (b == 0) a.cnt->n_moves = 0;
}

// One block per overloaded block b: the minimal prefix of b's records in the
// order (U asc, v asc) whose weight reaches the excess, found by an MSD radix
// select over the 96-bit key (U, v) with 8-bit digits; then every record up to
// that threshold joins the move list.
constexpr int kSelThreads = 512;

__global__ void __launch_bounds__(kSelThreads) k_rb_select(RbArgs a) {
  const int b = blockIdx.x;
  const RbBlock bb = a.rbb[b];
  if (!bb.over) return;
  const int len = a.rb_cursor[b];
  const uint64_t *key = a.rb_key + bb.off;
  const int32_t *vv = a.rb_v + bb.off;
  const int32_t *ct = a.rb_ct + bb.off;
  __shared__ long long s_hist[256];
  __shared__ long long s_part[kSelThreads / 32];
  __shared__ unsigned long long s_pu;
  __shared__ unsigned s_pv;
  __shared__ long long s_before;
  __shared__ int s_all;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  long long tw = 0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) tw += ct[i] >> 8;
  for (int o = 16; o > 0; o >>= 1) tw += __shfl_xor_sync(kFull, tw, o);
  if (lane == 0) s_part[wid] = tw;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < kSelThreads / 32; ++i) t += s_part[i];
    s_all = t < bb.excess;
    s_pu = 0;
    s_pv = 0;
    s_before = 0;
  }
  __syncthreads();
  if (!s_all) {
    for (int level = 0; level < 12; ++level) {
      for (int d = threadIdx.x; d < 256; d += blockDim.x) s_hist[d] = 0;
      __syncthreads();
      const unsigned long long pu = s_pu;
      const unsigned pv = s_pv;
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const unsigned long long U = key[i];
        const unsigned v = (unsigned)vv[i];
        bool match;
        int digit;
        if (level < 8) {
          match = level == 0 || (U >> (64 - 8 * level)) == (pu >> (64 - 8 * level));
          digit = (int)((U >> (56 - 8 * level)) & 255u);
        } else {
          const int lv = level - 8;
          match = U == pu && (lv == 0 || (v >> (32 - 8 * lv)) == (pv >> (32 - 8 * lv)));
          digit = (int)((v >> (24 - 8 * lv)) & 255u);
        }
        if (match) atomicAdd(reinterpret_cast<unsigned long long *>(&s_hist[digit]), (unsigned long long)(ct[i] >> 8));
      }
      __syncthreads();
      if (wid == 0) {
        // lane l owns digits 8l .. 8l+7
        long long loc[8];
        long long sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { loc[q] = s_hist[8 * lane + q]; sum += loc[q]; }
        long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          long long y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const long long before = s_before;
        const long long need = bb.excess;
        const long long excl = incl - sum;
        // the digit where before + cumulative weight first reaches the excess
        const bool here = before + excl < need && before + incl >= need;
        const unsigned who = __ballot_sync(kFull, here);
        if (here && lane == __ffs(who) - 1) {
          long long run = before + excl;
          int d = 8 * lane;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (run + loc[q] >= need) { d = 8 * lane + q; break; }
            run += loc[q];
          }
          s_before = run;
          if (level < 8) s_pu = pu | ((unsigned long long)d << (56 - 8 * level));
          else s_pv = pv | ((unsigned)d << (24 - 8 * (level - 8)));
        }
      }
      __syncthreads();
    }
  }
  const unsigned long long pu = s_pu;
  const unsigned pv = s_pv;
  const bool all = s_all;
  for (int base = 0; base < len; base += blockDim.x) {
    const int i = base + threadIdx.x;
    bool sel = false;
    int v = 0, t = 0;
    if (i < len) {
      const unsigned long long U = key[i];
      v = vv[i];
      t = ct[i] & 255;
      sel = all || U < pu || (U == pu && (unsigned)v <= pv);
    }
    const unsigned bal = __ballot_sync(kFull, sel);
    unsigned long long pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(&a.cnt->n_moves, (unsigned long long)__popc(bal));
    pos0 = __shfl_sync(kFull, pos0, 0);
    if (sel) {
      const unsigned long long pos = pos0 + __popc(bal & ((1u << lane) - 1));
      a.mv_v[pos] = v;
      a.mv_st[pos] = (uint32_t)b | ((uint32_t)t << 16);
    }
  }
}

// End of a round: count it, and stop if nothing moved, nothing is overloaded
// any more, or the round cap is reached.
__global__ void k_rb_post(RbArgs a) {
  const int b = threadIdx.x;
  const bool over = b < a.k && a.bw[b] > a.Lmax;
  const int any = __syncthreads_or(over);
  if (b == 0) {
    const long long moved = (long long)a.cnt->n_moves;
    a.cnt->rb_rounds += 1;
    a.cnt->rb_moves += moved;
    a.cnt->rb_any = any;
    a.cnt->rb_done = (moved == 0) || !any || (a.cnt->rb_rounds >= a.max_rounds);
  }
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
                                                        int32_t *mv_v, uint32_t *mv_st, Counters *cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int s = 0, t = 0;
    bool mv = false;
    if (v < n) {
      s = part[v];
      t = best[v];
      mv = s != t && (unsigned)s < kMaxK && (unsigned)t < kMaxK;
    }
    const unsigned bal = __ballot_sync(kFull, mv);
    unsigned long long pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(&cnt->n_moves, (unsigned long long)__popc(bal));
    pos0 = __shfl_sync(kFull, pos0, 0);
    if (mv) {
      const unsigned long long pos = pos0 + __popc(bal & ((1u << lane) - 1));
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
  a.mv_v = c->mv_v;
  a.mv_st = c->mv_st;
  a.k = c->k;
  a.kwp = c->kwp;
  a.cnt = c->cnt;
  return a;
}

RbArgs rb_args(jet_ctx *c, const int64_t *block_w) {
  RbArgs a{};
  a.bw = block_w;
  a.vcount = c->vcount;
  a.rbb = c->rbb;
  a.rb_cursor = c->rb_cursor;
  a.rb_key = c->rb_key;
  a.rb_v = c->rb_v;
  a.rb_ct = c->rb_ct;
  a.mv_v = c->mv_v;
  a.mv_st = c->mv_st;
  a.k = c->k;
  a.Lmax = c->Lmax;
  a.dz_min = c->dz_min;
  a.max_rounds = c->params.max_rebalance_rounds;
  a.cnt = c->cnt;
  return a;
}

}  // namespace

cudaError_t launch_apply(jet_ctx *c, int32_t *part, int32_t *phi, int64_t *block_w) {
  if (c->n == 0) return cudaSuccess;
  MoveArgs a = move_args(c, part, phi, block_w);
  const int g = grid_for(c->n, 256, c->num_sms, 4);
  k_apply<<<g, 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  k_fix_masks<<<g, 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_check(jet_ctx *c, const int64_t *block_w) {
  k_rb_check<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w));
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_prep(jet_ctx *c, const int64_t *block_w) {
  k_rb_prep<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w));
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_select(jet_ctx *c) {
  k_rb_select<<<c->k, kSelThreads, 0, c->stream>>>(rb_args(c, nullptr));
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_post(jet_ctx *c, const int64_t *block_w) {
  k_rb_post<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w));
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_stats(jet_ctx *c, const int64_t *block_w, jet_round_stats *stats, int rebalance_only) {
  k_stats<<<1, 256, 0, c->stream>>>(block_w, c->k, c->Lmax, c->cnt, stats, rebalance_only);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rollback_moves(jet_ctx *c, const int32_t *part, const int32_t *best) {
  cudaError_t e = cudaMemsetAsync(&c->cnt->n_moves, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess || c->n == 0) return e;
  k_rollback_moves<<<grid_for(c->n, 256, c->num_sms), 256, 0, c->stream>>>(part, best, c->n, c->mv_v, c->mv_st,
                                                                         c->cnt);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
