// Hypergraph afterburner (Algorithm 2), without sorting.
//
// Algorithm 2 replays, per edge e, the pins of e cap M in the order
// (gain desc, id asc) on a copy of phi_e and credits +omega(e) to a pin whose
// departure empties its source block in e and -omega(e) to a pin whose
// arrival makes its target block nonempty.  Every pin moves once, so for a
// block b of e, with D_b the departing pins (source b) and R_b the arriving
// pins (target b) among e cap M:
//   * the count of b after a departure i is (#D_b after i) + (#R_b before i)
//     + (pins of e in b outside M); it is 0 iff every pin of e in b is in M
//     (phi_e[b] = |D_b|), i is the last departure of D_b and no arrival
//     precedes i;
//   * the count of b before an arrival i is (#D_b after i) + (#R_b before i)
//     + (pins outside M); it is 0 iff phi_e[b] = |D_b|, every departure of
//     D_b precedes i and i is the first arrival of R_b.
// So per (e, b) at most one pin gains +omega(e) (the last departure) and at
// most one pays -omega(e) (the first arrival), and both need
// phi_e[b] = |D_b| and max(D_b) < min(R_b) in the order.  This is the same
// result as the replay, computed with counts and a max/min per block.
// phi_e[b] = |D_b| holds exactly when no pin of e outside M lies in b, which
// the kernels test with a bitmask of the blocks of e's non-candidate pins
// (gathered from the partition), so the afterburner reads no phi entry.
//
// Size classes: |e| <= 8 one thread per edge (pairwise tests in registers);
// 8 < |e| <= 2048 one warp per edge and > 2048 one thread block per edge,
// both with a per-block max / min table and a non-candidate bitmask in
// shared memory.
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct AbArgs {
  const int64_t *eptr;
  const int32_t *pins, *ewgt, *part;
  const uint64_t *cand;
  int32_t *rg;
  int32_t k;
  const int32_t *elist;
  int32_t nlist;
  Counters *cnt;
};

__global__ void __launch_bounds__(256) k_ab_tiny(AbArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nlist; i += gridDim.x * blockDim.x) {
    const int e = a.elist[i];
    const int64_t p0 = a.eptr[e];
    const int sz = (int)(a.eptr[e + 1] - p0);
    uint64_t key[kTinyEdge];
    uint32_t st[kTinyEdge];  // s | t << 8 | 1 << 16 for a candidate; block | 1 << 17 for another pin
    int vid[kTinyEdge];
    int nin = 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      key[q] = 0;
      st[q] = 0;
      vid[q] = 0;
      if (q < sz) {
        const int v = a.pins[p0 + q];
        const uint64_t r = a.cand[v];
        vid[q] = v;
        if (r) {
          ++nin;
          key[q] = cand_key(r, v);
          st[q] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 8) | 0x10000u;
        } else {
          st[q] = 0x20000u;
        }
      }
    }
    if (nin == 0) continue;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q)
      if (st[q] & 0x20000u) st[q] |= (uint32_t)(a.part[vid[q]] & 255);  // block of a non-candidate pin
    const int w = a.ewgt[e];
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      if (!(st[q] & 0x10000u)) continue;
      const int s = st[q] & 255, t = (st[q] >> 8) & 255;
      const uint64_t K = key[q];
      bool last_dep = true, no_arr_before = true, first_arr = true, no_dep_after = true, nm_s = false, nm_t = false;
#pragma unroll
      for (int r = 0; r < kTinyEdge; ++r) {
        if (st[r] & 0x20000u) {
          const int br = st[r] & 255;
          nm_s |= br == s;
          nm_t |= br == t;
        }
        if (!(st[r] & 0x10000u)) continue;
        const int sr = st[r] & 255, tr = (st[r] >> 8) & 255;
        const uint64_t Kr = key[r];
        if (sr == s && Kr > K) last_dep = false;
        if (tr == s && Kr < K) no_arr_before = false;
        if (tr == t && Kr < K) first_arr = false;
        if (sr == t && Kr > K) no_dep_after = false;
      }
      int delta = 0;
      if (last_dep && no_arr_before && !nm_s) delta += w;
      if (first_arr && no_dep_after && !nm_t) delta -= w;
      if (delta) atomicAdd(&a.rg[(int)(K & 0xffffffffu)], delta);
    }
  }
}

constexpr int kAbWarps = 8;

// Warp per edge (8 < |e| <= 2048): the per-block form of the replay in
// shared memory, one table per warp: max key of the departures and min key
// of the arrivals of every block, and the blocks holding a non-candidate pin.
// A key is never 0 (its high word is INT32_MAX - gain >= 1), so max = 0 means
// "no departure" and min = ~0 "no arrival".  Only the entries (and mask
// words) of blocks some candidate of the edge leaves or enters are reset and
// read, so the cost is O(|e|) and not O(k) per edge: pass 1 resets them,
// pass 2 adds the departures, arrivals and non-candidate blocks, pass 3 lets
// the last departure and the first arrival of each block decide.
__global__ void __launch_bounds__(kAbWarps * 32) k_ab_warp(AbArgs a) {
  extern __shared__ unsigned long long s_tab[];  // per warp: maxd[k], mina[k]
  __shared__ uint32_t s_nm[kAbWarps][kMaxK / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long *maxd = s_tab + (size_t)w * 2 * a.k;
  unsigned long long *mina = maxd + a.k;
  uint32_t *nm = s_nm[w];
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < a.nlist; i += nw) {
    const int e = a.elist[i];
    const int64_t p0 = a.eptr[e], p1 = a.eptr[e + 1];
    if (p1 - p0 <= 32) {  // one pin per lane: the pin's data stays in registers for the three passes
      const bool has = lane < p1 - p0;
      const int v = has ? a.pins[p0 + lane] : 0;
      const uint64_t r = has ? a.cand[v] : 0ull;
      const int b = (has && !r) ? (a.part[v] & 255) : -1;
      const int s = cand_s(r), t = cand_t(r);
      if (r) {
        maxd[s] = 0ull;
        mina[s] = ~0ull;
        maxd[t] = 0ull;
        mina[t] = ~0ull;
        nm[s >> 5] = 0u;
        nm[t >> 5] = 0u;
      }
      if (!__any_sync(kFull, r != 0)) continue;
      __syncwarp();
      const uint64_t K = cand_key(r, v);
      if (r) {
        atomicMax(&maxd[s], (unsigned long long)K);
        atomicMin(&mina[t], (unsigned long long)K);
      } else if (b >= 0) {
        atomicOr(&nm[b >> 5], 1u << (b & 31));
      }
      __syncwarp();
      if (r) {
        const int wt = a.ewgt[e];
        int delta = 0;
        if (maxd[s] == K && !((nm[s >> 5] >> (s & 31)) & 1u) && (mina[s] == ~0ull || K < mina[s])) delta += wt;
        if (mina[t] == K && !((nm[t >> 5] >> (t & 31)) & 1u) && maxd[t] < K) delta -= wt;
        if (delta) atomicAdd(&a.rg[v], delta);
      }
      __syncwarp();
      continue;
    }
    bool any = false;
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const uint64_t r = a.cand[a.pins[p]];
      if (r) {
        any = true;
        const int s = cand_s(r), t = cand_t(r);
        maxd[s] = 0ull;
        mina[s] = ~0ull;
        maxd[t] = 0ull;
        mina[t] = ~0ull;
        nm[s >> 5] = 0u;
        nm[t >> 5] = 0u;
      }
    }
    if (!__any_sync(kFull, any)) continue;
    __syncwarp();
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const int v = a.pins[p];
      const uint64_t r = a.cand[v];
      if (r) {
        const uint64_t K = cand_key(r, v);
        atomicMax(&maxd[cand_s(r)], (unsigned long long)K);
        atomicMin(&mina[cand_t(r)], (unsigned long long)K);
      } else {
        const int b = a.part[v] & 255;
        atomicOr(&nm[b >> 5], 1u << (b & 31));
      }
    }
    __syncwarp();
    const int wt = a.ewgt[e];
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const int v = a.pins[p];
      const uint64_t r = a.cand[v];
      if (!r) continue;
      const uint64_t K = cand_key(r, v);
      const int s = cand_s(r), t = cand_t(r);
      int delta = 0;
      // last departure from s, no arrival to s before it, no pin of e staying in s
      if (maxd[s] == K && !((nm[s >> 5] >> (s & 31)) & 1u) && (mina[s] == ~0ull || K < mina[s])) delta += wt;
      // first arrival to t, every departure from t before it, no pin of e staying in t
      if (mina[t] == K && !((nm[t >> 5] >> (t & 31)) & 1u) && maxd[t] < K) delta -= wt;
      if (delta) atomicAdd(&a.rg[v], delta);
    }
    __syncwarp();
  }
}

// Block per edge: the big class (|e| > 2048).
__global__ void __launch_bounds__(512) k_ab_block(AbArgs a) {
  extern __shared__ unsigned long long s_mem[];
  unsigned long long *s_maxd = s_mem;            // k: max key among departures
  unsigned long long *s_mina = s_mem + a.k;      // k: min key among arrivals
  int *s_cntd = reinterpret_cast<int *>(s_mem + 2 * a.k);  // k: number of departures
  __shared__ uint32_t s_nm[kMaxK / 32];          // blocks holding a non-candidate pin
  for (int i = blockIdx.x; i < a.nlist; i += gridDim.x) {
    const int e = a.elist[i];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
      s_maxd[b] = 0ull;
      s_mina[b] = ~0ull;
      s_cntd[b] = 0;
    }
    if (threadIdx.x < kMaxK / 32) s_nm[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p1 = a.eptr[e + 1];
    for (int64_t p = a.eptr[e] + threadIdx.x; p < p1; p += blockDim.x) {
      const int v = a.pins[p];
      const uint64_t r = a.cand[v];
      if (r) {
        const uint64_t K = cand_key(r, v);
        const int s = cand_s(r), t = cand_t(r);
        atomicAdd(&s_cntd[s], 1);
        atomicMax(&s_maxd[s], (unsigned long long)K);
        atomicMin(&s_mina[t], (unsigned long long)K);
      } else {
        const int b = a.part[v] & 255;
        const uint32_t bit = 1u << (b & 31);
        if (!(s_nm[b >> 5] & bit)) atomicOr(&s_nm[b >> 5], bit);
      }
    }
    __syncthreads();
    const int w = a.ewgt[e];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
      const int nd = s_cntd[b];
      const bool has_a = s_mina[b] != ~0ull;
      if (nd == 0 && !has_a) continue;
      if ((s_nm[b >> 5] >> (b & 31)) & 1u) continue;  // a pin of e in b stays
      if (nd > 0 && has_a && !(s_maxd[b] < s_mina[b])) continue;
      if (nd > 0) atomicAdd(&a.rg[(int)(s_maxd[b] & 0xffffffffu)], w);
      if (has_a) atomicAdd(&a.rg[(int)(s_mina[b] & 0xffffffffu)], -w);
    }
    __syncthreads();
  }
}

// Approval: v in M and recomputed gain > 0.  Resets rg, counts |M|; with
// build_moves writes the move list and locked[v] := approved.
struct ApArgs {
  int32_t n;
  const uint64_t *cand;
  int32_t *rg;
  uint8_t *locked;
  int32_t *rg_out;
  uint8_t *approved_out;
  int build_moves;
  int32_t *mv_v;
  uint32_t *mv_st;
  Counters *cnt;
};

// Counters and move-list slots are aggregated per thread block (one atomic
// per block and iteration) rather than per warp, which would serialize on
// the few counter addresses.
__global__ void __launch_bounds__(256) k_approve(ApArgs a) {
  constexpr int kWarps = 256 / 32;
  __shared__ unsigned s_wc[kWarps];
  __shared__ unsigned long long s_base;
  __shared__ unsigned long long s_cand[kWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long ncand = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const bool valid = v < a.n;
    const uint64_t r = valid ? a.cand[v] : 0;
    const int32_t g = valid ? a.rg[v] : 0;
    const bool in = r != 0;
    const bool ap = in && g > 0;
    if (valid) {
      a.rg[v] = 0;
      if (a.locked) a.locked[v] = ap ? 1 : 0;
      if (a.rg_out) a.rg_out[v] = g;
      if (a.approved_out) a.approved_out[v] = ap ? 1 : 0;
    }
    ncand += __popc(__ballot_sync(kFull, in));
    if (a.build_moves) {
      const unsigned bap = __ballot_sync(kFull, ap);
      if (lane == 0) s_wc[wid] = __popc(bap);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int i = 0; i < kWarps; ++i) {
          const unsigned x = s_wc[i];
          s_wc[i] = tot;
          tot += x;
        }
        s_base = tot ? atomicAdd(&a.cnt->n_moves, (unsigned long long)tot) : 0ull;
        if (tot) atomicAdd(&a.cnt->approved, (unsigned long long)tot);
      }
      __syncthreads();
      if (ap) {
        const unsigned long long pos = s_base + s_wc[wid] + __popc(bap & ((1u << lane) - 1));
        a.mv_v[pos] = (int32_t)v;
        a.mv_st[pos] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 16);
      }
      __syncthreads();
    }
  }
  if (lane == 0) s_cand[wid] = ncand;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < kWarps; ++i) t += s_cand[i];
    if (t) atomicAdd(&a.cnt->n_cand, t);
  }
}

__global__ void k_export_cand(const uint64_t *cand, int32_t n, int32_t *target, int32_t *gain, uint8_t *in_m) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = cand[v];
    in_m[v] = r ? 1 : 0;
    target[v] = r ? cand_t(r) : -1;
    gain[v] = r ? cand_gain(r) : 0;
  }
}

}  // namespace

cudaError_t launch_afterburner(jet_ctx *c, const int32_t *part, const int32_t *phi) {
  (void)phi;  // phi_e[b] = |D_b| is tested through the non-candidate pins' blocks
  AbArgs a{};
  a.eptr = c->eptr;
  a.pins = c->pins;
  a.ewgt = c->ewgt;
  a.part = part;
  a.cand = c->cand;
  a.rg = c->rg;
  a.k = c->k;
  a.cnt = c->cnt;
  if (c->n_tiny > 0) {
    a.elist = c->e_tiny;
    a.nlist = c->n_tiny;
    k_ab_tiny<<<grid_for(c->n_tiny, 256, c->launch_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid > 0) {
    a.elist = c->e_mid;
    a.nlist = c->n_mid;
    const size_t smem = (size_t)kAbWarps * 2 * c->k * sizeof(unsigned long long);
    k_ab_warp<<<grid_for((int64_t)c->n_mid * 32, kAbWarps * 32, c->launch_sms), kAbWarps * 32, smem, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_big > 0) {
    a.elist = c->e_big;
    a.nlist = c->n_big;
    const size_t smem = (size_t)c->k * (2 * sizeof(unsigned long long) + sizeof(int));
    k_ab_block<<<c->launch_sms * 2, 512, smem, c->stream>>>(a);
    ++c->kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_approve(jet_ctx *c, uint8_t *locked, int32_t *rg_out, uint8_t *approved_out, bool build_moves) {
  if (c->n == 0) return cudaSuccess;
  ApArgs a{};
  a.n = c->n;
  a.cand = c->cand;
  a.rg = c->rg;
  a.locked = locked;
  a.rg_out = rg_out;
  a.approved_out = approved_out;
  a.build_moves = build_moves ? 1 : 0;
  a.mv_v = c->mv_v;
  a.mv_st = c->mv_st;
  a.cnt = c->cnt;
  k_approve<<<grid_for(c->n, 256, c->launch_sms), 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_export_candidates(jet_ctx *c, int32_t *target, int32_t *gain, uint8_t *in_m) {
  if (c->n == 0) return cudaSuccess;
  k_export_cand<<<grid_for(c->n, 256, c->launch_sms), 256, 0, c->stream>>>(c->cand, c->n, target, gain, in_m);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
