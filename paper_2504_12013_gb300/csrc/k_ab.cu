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
//
// Size classes: |e| <= 8 one thread per edge (pairwise tests in registers);
// 8 < |e| <= 2048 one warp per edge, candidates gathered in shared memory,
// pairwise tests over at most 32 candidates; larger edges and warp-class
// edges with more than 32 candidates: one block per edge with per-block
// counters / max / min in shared memory.
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct AbArgs {
  const int64_t *eptr;
  const int32_t *pins, *ewgt, *phi;
  const uint64_t *cand;
  int32_t *rg;
  int32_t k;
  const int32_t *elist;
  int32_t nlist;
  int32_t *deferred;  // append area for warp-class edges with > 32 candidates
  int32_t n_big;
  Counters *cnt;
};

// Contribution of candidate i (key K, source s, target t) of edge e given the
// other candidates' (key, s|t<<8) through `get(j)`, j < cnt.
template <class Get>
__device__ __forceinline__ int pin_delta(const AbArgs &a, int64_t e, int w, uint64_t K, int s, int t, int cnt,
                                         Get get) {
  bool last_dep = true, no_arr_before = true, first_arr = true, no_dep_after = true;
  int n_src_s = 0, n_src_t = 0;
  for (int j = 0; j < cnt; ++j) {
    uint64_t Kj;
    uint32_t stj;
    get(j, Kj, stj);
    const int sj = stj & 255, tj = stj >> 8;
    if (sj == s) { ++n_src_s; if (Kj > K) last_dep = false; }
    if (tj == s && Kj < K) no_arr_before = false;
    if (tj == t && Kj < K) first_arr = false;
    if (sj == t) { ++n_src_t; if (Kj > K) no_dep_after = false; }
  }
  int delta = 0;
  if (last_dep && no_arr_before && a.phi[e * a.k + s] == n_src_s) delta += w;
  if (first_arr && no_dep_after && a.phi[e * a.k + t] == n_src_t) delta -= w;
  return delta;
}

__global__ void __launch_bounds__(256) k_ab_tiny(AbArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nlist; i += gridDim.x * blockDim.x) {
    const int e = a.elist[i];
    const int64_t p0 = a.eptr[e];
    const int sz = (int)(a.eptr[e + 1] - p0);
    uint64_t key[kTinyEdge];
    uint32_t st[kTinyEdge];
    int nin = 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      key[q] = 0;
      st[q] = 0;
      if (q < sz) {
        const int v = a.pins[p0 + q];
        const uint64_t r = a.cand[v];
        if (r) {
          ++nin;
          key[q] = cand_key(r, v);
          st[q] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 8) | 0x10000u;  // bit 16: in M
        }
      }
    }
    if (nin == 0) continue;
    const int w = a.ewgt[e];
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      if (!(st[q] & 0x10000u)) continue;
      const int s = st[q] & 255, t = (st[q] >> 8) & 255;
      const uint64_t K = key[q];
      bool last_dep = true, no_arr_before = true, first_arr = true, no_dep_after = true;
      int n_src_s = 0, n_src_t = 0;
#pragma unroll
      for (int r = 0; r < kTinyEdge; ++r) {
        if (!(st[r] & 0x10000u)) continue;
        const int sr = st[r] & 255, tr = (st[r] >> 8) & 255;
        const uint64_t Kr = key[r];
        if (sr == s) { ++n_src_s; if (Kr > K) last_dep = false; }
        if (tr == s && Kr < K) no_arr_before = false;
        if (tr == t && Kr < K) first_arr = false;
        if (sr == t) { ++n_src_t; if (Kr > K) no_dep_after = false; }
      }
      int delta = 0;
      if (last_dep && no_arr_before && a.phi[(int64_t)e * a.k + s] == n_src_s) delta += w;
      if (first_arr && no_dep_after && a.phi[(int64_t)e * a.k + t] == n_src_t) delta -= w;
      if (delta) atomicAdd(&a.rg[(int)(K & 0xffffffffu)], delta);
    }
  }
}

constexpr int kAbWarps = 8;

__global__ void __launch_bounds__(kAbWarps * 32) k_ab_warp(AbArgs a) {
  __shared__ uint64_t s_key[kAbWarps][kWarpEdgeSlots];
  __shared__ uint32_t s_st[kAbWarps][kWarpEdgeSlots];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < a.nlist; i += nw) {
    const int e = a.elist[i];
    const int64_t p0 = a.eptr[e], p1 = a.eptr[e + 1];
    int cnt = 0;
    bool overflow = false;
    for (int64_t base = p0; base < p1; base += 32) {
      const int64_t p = base + lane;
      uint64_t r = 0;
      int v = 0;
      if (p < p1) {
        v = a.pins[p];
        r = a.cand[v];
      }
      const unsigned bal = __ballot_sync(kFull, r != 0);
      const int pos = cnt + __popc(bal & ((1u << lane) - 1));
      if (r != 0 && pos < kWarpEdgeSlots) {
        s_key[w][pos] = cand_key(r, v);
        s_st[w][pos] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 8);
      }
      cnt += __popc(bal);
      if (cnt > kWarpEdgeSlots) { overflow = true; break; }
    }
    __syncwarp();
    if (overflow) {
      if (lane == 0) {
        const unsigned long long slot = atomicAdd(&a.cnt->n_deferred, 1ull);
        a.deferred[slot] = e;
      }
      __syncwarp();
      continue;
    }
    if (lane < cnt) {
      const uint64_t K = s_key[w][lane];
      const int s = s_st[w][lane] & 255, t = s_st[w][lane] >> 8;
      const int delta = pin_delta(a, e, a.ewgt[e], K, s, t, cnt, [&](int j, uint64_t &Kj, uint32_t &stj) {
        Kj = s_key[w][j];
        stj = s_st[w][j];
      });
      if (delta) atomicAdd(&a.rg[(int)(K & 0xffffffffu)], delta);
    }
    __syncwarp();
  }
}

// Block per edge: the big class (a.elist[0..n_big)) and the deferred
// warp-class edges (a.deferred[0..n_deferred)).
__global__ void __launch_bounds__(512) k_ab_block(AbArgs a) {
  extern __shared__ unsigned long long s_mem[];
  unsigned long long *s_maxd = s_mem;            // k: max key among departures
  unsigned long long *s_mina = s_mem + a.k;      // k: min key among arrivals
  int *s_cntd = reinterpret_cast<int *>(s_mem + 2 * a.k);  // k: number of departures
  const int total = a.n_big + (int)a.cnt->n_deferred;
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const int e = i < a.n_big ? a.elist[i] : a.deferred[i - a.n_big];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
      s_maxd[b] = 0ull;
      s_mina[b] = ~0ull;
      s_cntd[b] = 0;
    }
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
      }
    }
    __syncthreads();
    const int w = a.ewgt[e];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
      const int nd = s_cntd[b];
      const bool has_a = s_mina[b] != ~0ull;
      if (nd == 0 && !has_a) continue;
      if (a.phi[(int64_t)e * a.k + b] != nd) continue;  // a pin of e in b stays
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

__global__ void __launch_bounds__(256) k_approve(ApArgs a) {
  const int lane = threadIdx.x & 31;
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
    const unsigned bin = __ballot_sync(kFull, in);
    const unsigned bap = __ballot_sync(kFull, ap);
    if (lane == 0 && bin) atomicAdd(&a.cnt->n_cand, (unsigned long long)__popc(bin));
    if (a.build_moves) {
      unsigned long long pos0 = 0;
      if (lane == 0 && bap) {
        pos0 = atomicAdd(&a.cnt->n_moves, (unsigned long long)__popc(bap));
        atomicAdd(&a.cnt->approved, (unsigned long long)__popc(bap));
      }
      pos0 = __shfl_sync(kFull, pos0, 0);
      if (ap) {
        const unsigned long long pos = pos0 + __popc(bap & ((1u << lane) - 1));
        a.mv_v[pos] = (int32_t)v;
        a.mv_st[pos] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 16);
      }
    }
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
  (void)part;
  AbArgs a{};
  a.eptr = c->eptr;
  a.pins = c->pins;
  a.ewgt = c->ewgt;
  a.phi = phi;
  a.cand = c->cand;
  a.rg = c->rg;
  a.k = c->k;
  a.cnt = c->cnt;
  a.deferred = c->e_big + c->n_big;
  a.n_big = c->n_big;
  cudaError_t e = cudaMemsetAsync(&c->cnt->n_deferred, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return e;
  if (c->n_tiny > 0) {
    a.elist = c->e_tiny;
    a.nlist = c->n_tiny;
    k_ab_tiny<<<grid_for(c->n_tiny, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid > 0) {
    a.elist = c->e_mid;
    a.nlist = c->n_mid;
    k_ab_warp<<<grid_for((int64_t)c->n_mid * 32, kAbWarps * 32, c->num_sms), kAbWarps * 32, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid > 0 || c->n_big > 0) {
    a.elist = c->e_big;
    a.nlist = c->n_big;
    size_t smem = (size_t)c->k * (2 * sizeof(unsigned long long) + sizeof(int));
    k_ab_block<<<c->num_sms * 2, 512, smem, c->stream>>>(a);
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
  k_approve<<<grid_for(c->n, 256, c->num_sms), 256, 0, c->stream>>>(a);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_export_candidates(jet_ctx *c, int32_t *target, int32_t *gain, uint8_t *in_m) {
  if (c->n == 0) return cudaSuccess;
  k_export_cand<<<grid_for(c->n, 256, c->num_sms), 256, 0, c->stream>>>(c->cand, c->n, target, gain, in_m);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
