// ApplyMoves (Algorithm 1), deterministic rebalancing rounds (Section 4.3),
// statistics and rollback moves.
//
// All updates are integer atomics whose final values do not depend on their
// order: phi row entries +-1, block weights and counts aggregated per thread
// block; after all moves a second pass sets the bits of the source and target
// blocks in both edge bitmasks from the final phi entries.
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void add_i64(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

struct MoveArgs {
  const int64_t *vptr, *eptr;
  const int32_t *inc, *vwgt, *pins;
  int32_t *mtag;
  const int32_t *elist;
  int32_t nlist;
  long long P;
  int32_t *part, *phi;
  int64_t *bw;
  int32_t *vcount;
  uint32_t *mask;
  const int32_t *mv_v;
  const uint32_t *mv_st;
  int32_t k, kwp;
  Counters *cnt;
};

// A group of kMoveLanes lanes per move, the lanes striding over I(v): more
// loads and atomics in flight than one thread per move when the move list is
// short (rebalancing rounds).
constexpr int kMoveLanes = 8;

// Large move lists are applied edge by edge: every edge's owner (a thread, a
// warp or a block) adds the net +-1 of its moved pins to its own phi row and
// rewrites its own mask words, with no atomics and no fix-up pass.  Small
// lists are applied move by move with atomics plus the mask fix-up.  The
// choice is made on the device from the moved incidences: edge by edge when
// more than half of all incidences move (the phi row traffic is the same
// either way; the edge pass saves the atomics and the fix-up pass but has to
// read every pin).
__device__ __forceinline__ bool edge_centric(const MoveArgs &a) { return (long long)a.cnt->mv_inc * 2 > a.P; }

// Tags every moved vertex (source | target << 8) and sums the moved incidences.
__global__ void __launch_bounds__(256) k_apply_prep(MoveArgs a) {
  const long long nm = (long long)a.cnt->n_moves;
  unsigned long long inc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm; i += (long long)gridDim.x * blockDim.x) {
    const int v = a.mv_v[i];
    const uint32_t st = a.mv_st[i];
    a.mtag[v] = (int32_t)((st & 0xffff) | ((st >> 16) << 8));
    inc += (unsigned long long)(a.vptr[v + 1] - a.vptr[v]);
  }
  for (int o = 16; o > 0; o >>= 1) inc += __shfl_xor_sync(kFull, inc, o);
  if ((threadIdx.x & 31) == 0 && inc) atomicAdd(&a.cnt->mv_inc, inc);
}

// Owner of row e: one bit of both mask words of block b from its count `val`.
__device__ __forceinline__ void owner_set_bits(uint32_t *mrow, int kwp, int b, int val) {
  const uint32_t bit = 1u << (b & 31);
  uint32_t *w1 = &mrow[b >> 5], *w2 = &mrow[kwp + (b >> 5)];
  *w1 = (*w1 & ~bit) | (val > 0 ? bit : 0u);
  *w2 = (*w2 & ~bit) | (val > 1 ? bit : 0u);
}

// Edges of at most kTinyEdge pins, one thread each.
__global__ void __launch_bounds__(256) k_apply_edges_tiny(MoveArgs a) {
  if (!edge_centric(a)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nlist; i += gridDim.x * blockDim.x) {
    const int64_t e = a.elist[i];
    const int64_t p0 = a.eptr[e];
    const int sz = (int)(a.eptr[e + 1] - p0);
    int tg[kTinyEdge];
    bool any = false;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      tg[q] = q < sz ? a.mtag[a.pins[p0 + q]] : -1;
      any |= tg[q] >= 0;
    }
    if (!any) continue;
    int32_t *row = a.phi + e * a.k;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q)
      if (tg[q] >= 0) {
        row[tg[q] & 255] -= 1;
        row[tg[q] >> 8] += 1;
      }
    uint32_t *mrow = a.mask + e * 2 * a.kwp;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q)
      if (tg[q] >= 0) {
        const int s = tg[q] & 255, t = tg[q] >> 8;
        owner_set_bits(mrow, a.kwp, s, row[s]);
        owner_set_bits(mrow, a.kwp, t, row[t]);
      }
  }
}

// Edges of 9..2048 pins, one warp each: net deltas per block in shared memory,
// then only the changed entries of the row and their mask bits are written.
constexpr int kApplyWarps = 8;

__global__ void __launch_bounds__(kApplyWarps * 32) k_apply_edges_warp(MoveArgs a) {
  if (!edge_centric(a)) return;
  __shared__ int s_delta[kApplyWarps][kMaxK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *delta = s_delta[w];
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < a.nlist; i += nw) {
    const int64_t e = a.elist[i];
    const int64_t p1 = a.eptr[e + 1];
    for (int b = lane; b < a.k; b += 32) delta[b] = 0;
    __syncwarp();
    bool any = false;
    for (int64_t p = a.eptr[e] + lane; p < p1; p += 32) {
      const int tg = a.mtag[a.pins[p]];
      if (tg >= 0) {
        any = true;
        atomicSub(&delta[tg & 255], 1);
        atomicAdd(&delta[tg >> 8], 1);
      }
    }
    any = __any_sync(kFull, any);
    __syncwarp();
    if (any) {
      int32_t *row = a.phi + e * a.k;
      uint32_t *mrow = a.mask + e * 2 * a.kwp;
      for (int q = 0; q < a.kwp; ++q) {
        const int b = q * 32 + lane;
        const int d = b < a.k ? delta[b] : 0;
        int val = 0;
        if (d) {  // only the changed entries of the row are read and written
          val = row[b] + d;
          row[b] = val;
        }
        const unsigned chg = __ballot_sync(kFull, d != 0);
        if (!chg) continue;
        const unsigned one = __ballot_sync(kFull, val > 0), two = __ballot_sync(kFull, val > 1);
        if (lane == 0) {
          mrow[q] = (mrow[q] & ~chg) | (one & chg);
          mrow[a.kwp + q] = (mrow[a.kwp + q] & ~chg) | (two & chg);
        }
      }
    }
    __syncwarp();
  }
}

// Edges of more than 2048 pins, one block each.
__global__ void __launch_bounds__(512) k_apply_edges_block(MoveArgs a) {
  if (!edge_centric(a)) return;
  __shared__ int s_delta[kMaxK];
  __shared__ int s_any;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < a.nlist; i += gridDim.x) {
    const int64_t e = a.elist[i];
    const int64_t p1 = a.eptr[e + 1];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) s_delta[b] = 0;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    bool any = false;
    for (int64_t p = a.eptr[e] + threadIdx.x; p < p1; p += blockDim.x) {
      const int tg = a.mtag[a.pins[p]];
      if (tg >= 0) {
        any = true;
        atomicSub(&s_delta[tg & 255], 1);
        atomicAdd(&s_delta[tg >> 8], 1);
      }
    }
    if (__any_sync(kFull, any) && lane == 0) s_any = 1;
    __syncthreads();
    if (s_any) {
      int32_t *row = a.phi + e * a.k;
      uint32_t *mrow = a.mask + e * 2 * a.kwp;
      for (int q = w; q < a.kwp; q += blockDim.x / 32) {  // warp q owns mask word q
        const int b = q * 32 + lane;
        const int d = b < a.k ? s_delta[b] : 0;
        int val = 0;
        if (d) {
          val = row[b] + d;
          row[b] = val;
        }
        const unsigned chg = __ballot_sync(kFull, d != 0);
        if (!chg) continue;
        const unsigned one = __ballot_sync(kFull, val > 0), two = __ballot_sync(kFull, val > 1);
        if (lane == 0) {
          mrow[q] = (mrow[q] & ~chg) | (one & chg);
          mrow[a.kwp + q] = (mrow[a.kwp + q] & ~chg) | (two & chg);
        }
      }
    }
    __syncthreads();
  }
}

// Pi(v) <- t and phi_e[s]--, phi_e[t]++ for every e in I(v); c(V_s), c(V_t)
// and |V_s|, |V_t| through shared-memory partial sums.
__global__ void __launch_bounds__(256) k_apply(MoveArgs a) {
  __shared__ long long s_dw[kMaxK];
  __shared__ int s_dc[kMaxK];
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) { s_dw[b] = 0; s_dc[b] = 0; }
  __syncthreads();
  const long long nm = (long long)a.cnt->n_moves;
  const bool edge_mode = edge_centric(a);
  const int sub = threadIdx.x % kMoveLanes;
  const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kMoveLanes;
  const long long ng = ((long long)gridDim.x * blockDim.x) / kMoveLanes;
  for (long long i = g0; i < nm; i += ng) {
    const int v = a.mv_v[i];
    const uint32_t st = a.mv_st[i];
    const int s = st & 0xffff, t = st >> 16;
    if (sub == 0) {
      a.part[v] = t;
      a.mtag[v] = -1;
      const int c = a.vwgt[v];
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)(-(long long)c));
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[t]), (unsigned long long)c);
      atomicSub(&s_dc[s], 1);
      atomicAdd(&s_dc[t], 1);
    }
    if (edge_mode) continue;  // the edge owners updated phi and the masks
    const int64_t j1 = a.vptr[v + 1];
    for (int64_t j = a.vptr[v] + sub; j < j1; j += kMoveLanes) {
      const int64_t e = a.inc[j];
      atomicSub(&a.phi[e * a.k + s], 1);
      atomicAdd(&a.phi[e * a.k + t], 1);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    if (s_dw[b]) add_i64(reinterpret_cast<long long *>(&a.bw[b]), s_dw[b]);
    if (s_dc[b]) atomicAdd(&a.vcount[b], s_dc[b]);
  }
}

// After all moves: bring the bits of s and t in both masks of every e in I(v)
// (phi_e[.] >= 1 and >= 2) to their final values, read from the final phi.
// Each word of the row is read once and changed by at most one atomicOr and
// one atomicAnd, only where it differs.  Every writer of a bit writes its
// final value, so a stale read that already shows that value can never hide
// a needed change.
__global__ void __launch_bounds__(256) k_fix_masks(MoveArgs a) {
  if (edge_centric(a)) return;
  const long long nm = (long long)a.cnt->n_moves;
  const int sub = threadIdx.x % kMoveLanes;
  const long long g0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kMoveLanes;
  const long long ng = ((long long)gridDim.x * blockDim.x) / kMoveLanes;
  for (long long i = g0; i < nm; i += ng) {
    const int v = a.mv_v[i];
    const uint32_t st = a.mv_st[i];
    const int s = st & 0xffff, t = st >> 16;
    const int ws = s >> 5, wt = t >> 5;
    const uint32_t sbit = 1u << (s & 31), tbit = 1u << (t & 31);
    const int64_t j1 = a.vptr[v + 1];
    for (int64_t j = a.vptr[v] + sub; j < j1; j += kMoveLanes) {
      const int64_t e = a.inc[j];
      const int ps = __ldcg(&a.phi[e * a.k + s]), pt = __ldcg(&a.phi[e * a.k + t]);
      uint32_t *row = a.mask + e * 2 * a.kwp;
      // words: Lambda at [0, kwp), ">= 2" at [kwp, 2 kwp)
      const int w1s = ws, w2s = a.kwp + ws, w1t = wt, w2t = a.kwp + wt;
      uint32_t set1s = ps > 0 ? sbit : 0, set2s = ps > 1 ? sbit : 0, set1t = tbit, set2t = pt > 1 ? tbit : 0;
      const uint32_t cur1s = __ldcg(&row[w1s]), cur2s = __ldcg(&row[w2s]);
      const uint32_t cur1t = w1t == w1s ? cur1s : __ldcg(&row[w1t]);
      const uint32_t cur2t = w2t == w2s ? cur2s : __ldcg(&row[w2t]);
      if (w1t == w1s) {  // s and t share the words: one update per word
        const uint32_t want1 = (cur1s & ~(sbit | tbit)) | set1s | set1t;
        const uint32_t want2 = (cur2s & ~(sbit | tbit)) | set2s | set2t;
        if (want1 != cur1s) {
          if (want1 & ~cur1s) atomicOr(&row[w1s], want1 & ~cur1s);
          if (cur1s & ~want1) atomicAnd(&row[w1s], ~(cur1s & ~want1));
        }
        if (want2 != cur2s) {
          if (want2 & ~cur2s) atomicOr(&row[w2s], want2 & ~cur2s);
          if (cur2s & ~want2) atomicAnd(&row[w2s], ~(cur2s & ~want2));
        }
      } else {
        if ((cur1s & sbit) != set1s) { if (set1s) atomicOr(&row[w1s], sbit); else atomicAnd(&row[w1s], ~sbit); }
        if ((cur2s & sbit) != set2s) { if (set2s) atomicOr(&row[w2s], sbit); else atomicAnd(&row[w2s], ~sbit); }
        if ((cur1t & tbit) != set1t) { if (set1t) atomicOr(&row[w1t], tbit); else atomicAnd(&row[w1t], ~tbit); }
        if ((cur2t & tbit) != set2t) { if (set2t) atomicOr(&row[w2t], tbit); else atomicAnd(&row[w2t], ~tbit); }
      }
    }
  }
}

// ---------------------------------------------------------------- rebalancing
// Selection of the minimal prefix per overloaded block (Section 4.3) as a
// radix select over all records at once.  Every vertex v of an overloaded
// block with a valid target has a record with the key
// K(v) = hi(v) << vb | v  (priority descending, then id ascending, as one
// ascending number of hb + vb bits; 64-bit when it fits, else 128-bit).
// Per level (kRbDigitBits bits, from the top) one grid-wide kernel adds c(v)
// of every record that matches its block's fixed prefix into the (block,
// digit) histogram, and one small kernel per overloaded block picks the
// digit at which the cumulative weight reaches the excess.  After the last
// level the prefix is the threshold key, and every record up to it moves.
typedef unsigned __int128 u128;

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
  long long Lmax, dz_min;
  int32_t max_rounds;
  Counters *cnt;
};

// Any block above L_max?  One block of 256 threads (k <= 256).  In a CUDA
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
}

// Per-block state of the round: overloaded flag, excess, target capacity
// (deadzone and L_max), cleared selection state.
__global__ void k_rb_prep(RbArgs a) {
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
    a.cnt->mv_inc = 0;
  }
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
// equal their block's prefix; weights aggregated per warp and (block, digit).
template <class KT>
__global__ void __launch_bounds__(256) k_rb_level(RbArgs a, int lo, int w) {
  const int lane = threadIdx.x & 31;
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
    const int code = m ? (b << kRbDigitBits) | d : -1 - lane;
    const unsigned grp = __match_any_sync(kFull, code);
    const unsigned sum = __reduce_add_sync(grp, c);
    if (m && lane == __ffs(grp) - 1) atomicAdd(&a.hist[(int64_t)b * kRbBins + d], (unsigned long long)sum);
  }
}

// Per overloaded block: the digit at which the cumulative weight first reaches
// the excess; at the first level a total below the excess selects everything.
// Leaves the histogram row zeroed.
__global__ void __launch_bounds__(256) k_rb_pick(RbArgs a, int lo, int first) {
  const int b = blockIdx.x;
  RbBlock *r = &a.rbb[b];
  if (!r->over || r->all) return;
  constexpr int kPer = kRbBins / 256;
  unsigned long long *row = a.hist + (int64_t)b * kRbBins;
  __shared__ long long s_warp[8];
  __shared__ long long s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long loc[kPer];
  long long sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    loc[q] = (long long)row[threadIdx.x * kPer + q];
    sum += loc[q];
  }
  long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  long long wbase = 0;
  for (int i = 0; i < wid; ++i) wbase += s_warp[i];
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < 8; ++i) t += s_warp[i];
    s_total = t;
  }
  const long long excl = wbase + incl - sum;
  const long long before = r->before, need = r->excess;
  __syncthreads();
  if (first && s_total < need) {
    if (threadIdx.x == 0) r->all = 1;
  } else if (before + excl < need && before + excl + sum >= need) {
    long long run = before + excl;
    int d = threadIdx.x * kPer;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (run + loc[q] >= need) { d = threadIdx.x * kPer + q; break; }
      run += loc[q];
    }
    r->before = run;
    const u128 pre = (((u128)r->pre_hi << 64) | r->pre_lo) | ((u128)(unsigned)d << lo);
    r->pre_hi = (unsigned long long)(pre >> 64);
    r->pre_lo = (unsigned long long)pre;
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) row[threadIdx.x * kPer + q] = 0ull;
}

// Every record with K(v) <= its block's threshold (or of an `all` block) moves.
template <class KT>
__global__ void __launch_bounds__(256) k_rb_mark(RbArgs a) {
  __shared__ unsigned s_wc[8];
  __shared__ unsigned long long s_base;
  const long long nrec = (long long)a.cnt->n_rec;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nrec; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    bool sel = false;
    int v = 0, b = 0, t = 0;
    if (i < nrec) {
      const int32_t ct = a.rb_ct[i];
      b = (ct >> 8) & 255;
      t = ct & 255;
      v = a.rb_v[i];
      const RbBlock &r = a.rbb[b];
      sel = r.all || rb_full_key<KT>(a.rb_hi[i], v, a.vbits) <= rb_prefix<KT>(r);
    }
    const unsigned long long pos = block_append(sel, &a.cnt->n_moves, s_wc, &s_base);
    if (sel) {
      a.mv_v[pos] = v;
      a.mv_st[pos] = (uint32_t)b | ((uint32_t)t << 16);
    }
  }
}

// End of a round: count it, and stop if nothing moved, nothing is overloaded
// any more, or the round cap is reached.
__global__ void k_rb_post(RbArgs a, cudaGraphConditionalHandle cond, int use_cond) {
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
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
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
  __shared__ unsigned s_wc[8];
  __shared__ unsigned long long s_base;
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
  a.eptr = c->eptr;
  a.inc = c->inc;
  a.vwgt = c->vwgt;
  a.pins = c->pins;
  a.mtag = c->mtag;
  a.P = c->P;
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
  const int g = grid_for((int64_t)c->n * kMoveLanes, 256, c->num_sms, 8);
  k_apply_prep<<<grid_for(c->n, 256, c->num_sms), 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  if (c->n_tiny > 0) {
    a.elist = c->e_tiny;
    a.nlist = c->n_tiny;
    k_apply_edges_tiny<<<grid_for(c->n_tiny, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid > 0) {
    a.elist = c->e_mid;
    a.nlist = c->n_mid;
    k_apply_edges_warp<<<grid_for((int64_t)c->n_mid * 32, kApplyWarps * 32, c->num_sms), kApplyWarps * 32, 0,
                         c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_big > 0) {
    a.elist = c->e_big;
    a.nlist = c->n_big;
    k_apply_edges_block<<<c->num_sms * 2, 512, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  k_apply<<<g, 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  k_fix_masks<<<g, 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_check(jet_ctx *c, const int64_t *block_w, cudaGraphConditionalHandle cond, int use_cond) {
  k_rb_check<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w, nullptr), cond, use_cond);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rb_prep(jet_ctx *c, const int64_t *block_w) {
  k_rb_prep<<<1, kMaxK, 0, c->stream>>>(rb_args(c, block_w, nullptr));
  ++c->kernel_launches;
  return cudaGetLastError();
}

template <class KT>
void rb_select_levels(jet_ctx *c, const RbArgs &a) {
  const int g = grid_for(c->n, 256, c->num_sms);
  int first = 1;
  for (int hi = a.tbits; hi > 0; first = 0) {
    const int lo = hi - kRbDigitBits > 0 ? hi - kRbDigitBits : 0;
    k_rb_level<KT><<<g, 256, 0, c->stream>>>(a, lo, hi - lo);
    ++c->kernel_launches;
    k_rb_pick<<<c->k, 256, 0, c->stream>>>(a, lo, first);
    ++c->kernel_launches;
    hi = lo;
  }
  k_rb_mark<KT><<<g, 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
}

cudaError_t launch_rb_select(jet_ctx *c, const int32_t *part) {
  if (c->n == 0) return cudaSuccess;
  const RbArgs a = rb_args(c, nullptr, part);
  if (a.tbits <= 64) rb_select_levels<unsigned long long>(c, a);
  else rb_select_levels<u128>(c, a);
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

cudaError_t launch_rollback_moves(jet_ctx *c, const int32_t *part, const int32_t *best) {
  cudaError_t e = cudaMemsetAsync(&c->cnt->n_moves, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->cnt->mv_inc, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess || c->n == 0) return e;
  k_rollback_moves<<<grid_for(c->n, 256, c->num_sms), 256, 0, c->stream>>>(part, best, c->n, c->mv_v, c->mv_st,
                                                                         c->cnt);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
