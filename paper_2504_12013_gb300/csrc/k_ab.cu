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
// 8 < |e| <= 16 a half warp per edge and 16 < |e| <= 128 one warp per edge
// (<= 32 pins: software-pipelined over the group's edges; larger: up to four
// pins per lane in registers, largest edges first) and > 128 one thread block per segment of <= 2048 pins, each
// with a per-block max / min table and a non-candidate bitmask in shared
// memory.
#include <algorithm>
#include <vector>

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

// Thread per edge (|e| <= 8), software-pipelined over the thread's edges:
// while edge j is decided, the pins of edge j+1, the offsets of edge j+2 and
// the id of edge j+3 are in flight.
__global__ void __launch_bounds__(256) k_ab_tiny(AbArgs a) {
  const int stride = gridDim.x * blockDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  auto edge_at = [&](long long i) -> int { return i < a.nlist ? a.elist[i] : -1; };
  int e3 = edge_at(i0 + 2ll * stride);
  int e2 = edge_at(i0 + (long long)stride);
  int64_t p2 = e2 >= 0 ? a.eptr[e2] : 0;
  int sz2 = e2 >= 0 ? (int)(a.eptr[e2 + 1] - p2) : 0;
  int e1 = edge_at(i0), sz1 = 0;
  int pins1[kTinyEdge];
  {
    const int64_t p1 = e1 >= 0 ? a.eptr[e1] : 0;
    sz1 = e1 >= 0 ? (int)(a.eptr[e1 + 1] - p1) : 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pins1[q] = q < sz1 ? a.pins[p1 + q] : 0;
  }
  for (long long i = i0; i < a.nlist; i += stride) {
    const int e = e1, sz = sz1;
    int pin[kTinyEdge];
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pin[q] = pins1[q];
    // advance the pipeline: first used in the next iteration
    const int e4 = edge_at(i + 3ll * stride);
    const int64_t p3 = e3 >= 0 ? a.eptr[e3] : 0;
    const int sz3 = e3 >= 0 ? (int)(a.eptr[e3 + 1] - p3) : 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pins1[q] = q < sz2 ? a.pins[p2 + q] : 0;
    e1 = e2; sz1 = sz2;
    e2 = e3; p2 = p3; sz2 = sz3;
    e3 = e4;
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
        const int v = pin[q];
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

// Warp per edge (32 < |e| <= 32 PPL): the per-block form of the replay in
// shared memory, one table per warp: max key of the departures and min key
// of the arrivals of every block, and the blocks holding a non-candidate pin.
// A 64-bit key is kept as two 32-bit words, found in two rounds of 32-bit
// shared-memory atomics (the high words, then the low words of the keys
// whose high word is the extreme one): cheaper than 64-bit atomic max / min.
// A key is never 0 (its high word is INT32_MAX - gain >= 1), so max = 0 means
// "no departure" and min = ~0 "no arrival".  Only the entries (and mask
// words) of blocks some candidate of the edge leaves or enters are reset and
// read, so the cost is O(|e|) and not O(k) per edge: pass 1 resets them,
// pass 2 adds the departures, arrivals and non-candidate blocks, pass 3 lets
// the last departure and the first arrival of each block decide.  Each lane
// holds PPL pins (their records and blocks) in registers for the three
// passes, loaded together, and the next edge's offsets are loaded while the
// current edge is decided.
template <int PPL>
__global__ void __launch_bounds__(kAbWarps * 32) k_ab_warp(AbArgs a) {
  extern __shared__ unsigned long long s_tab[];  // per warp: the high and low words of maxd[k], mina[k]
  __shared__ uint32_t s_nm[kAbWarps][kMaxK / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t *dh = reinterpret_cast<uint32_t *>(s_tab + (size_t)w * 2 * a.k);
  uint32_t *dl = dh + a.k, *ah = dl + a.k, *al = ah + a.k;
  uint32_t *nm = s_nm[w];
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int en = gw < a.nlist ? a.elist[gw] : -1;
  int64_t p0n = en >= 0 ? a.eptr[en] : 0, p1n = en >= 0 ? a.eptr[en + 1] : 0;
  for (int i = gw; i < a.nlist; i += nw) {
    const int e = en;
    const int64_t p0 = p0n, p1 = p1n;
    en = i + nw < a.nlist ? a.elist[i + nw] : -1;  // first used in the next iteration
    if (en >= 0) {
      p0n = a.eptr[en];
      p1n = a.eptr[en + 1];
    }
    int v[PPL], b[PPL];
    uint64_t r[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      const int64_t p = p0 + lane + 32 * q;
      v[q] = p < p1 ? a.pins[p] : -1;
    }
#pragma unroll
    for (int q = 0; q < PPL; ++q) r[q] = v[q] >= 0 ? a.cand[v[q]] : 0ull;
    bool any = false;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      b[q] = (v[q] >= 0 && !r[q]) ? (a.part[v[q]] & 255) : -1;  // block of a non-candidate pin
      if (r[q]) {
        any = true;
        const int s = cand_s(r[q]), t = cand_t(r[q]);
        dh[s] = 0u; dl[s] = 0u; ah[s] = ~0u; al[s] = ~0u;
        dh[t] = 0u; dl[t] = 0u; ah[t] = ~0u; al[t] = ~0u;
        nm[s >> 5] = 0u;
        nm[t >> 5] = 0u;
      }
    }
    if (!__any_sync(kFull, any)) continue;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      if (r[q]) {
        const uint32_t kh = (uint32_t)(cand_key(r[q], v[q]) >> 32);
        atomicMax(&dh[cand_s(r[q])], kh);
        atomicMin(&ah[cand_t(r[q])], kh);
      } else if (b[q] >= 0) {
        atomicOr(&nm[b[q] >> 5], 1u << (b[q] & 31));
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < PPL; ++q) {  // the low words among the keys with the extreme high word
      if (!r[q]) continue;
      const uint32_t kh = (uint32_t)(cand_key(r[q], v[q]) >> 32);
      const int s = cand_s(r[q]), t = cand_t(r[q]);
      if (dh[s] == kh) atomicMax(&dl[s], (uint32_t)v[q]);
      if (ah[t] == kh) atomicMin(&al[t], (uint32_t)v[q]);
    }
    __syncwarp();
    const int wt = a.ewgt[e];
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
      if (!r[q]) continue;
      const uint64_t K = cand_key(r[q], v[q]);
      const int s = cand_s(r[q]), t = cand_t(r[q]);
      const uint64_t maxd_s = ((uint64_t)dh[s] << 32) | dl[s], mina_s = ((uint64_t)ah[s] << 32) | al[s];
      const uint64_t maxd_t = ((uint64_t)dh[t] << 32) | dl[t], mina_t = ((uint64_t)ah[t] << 32) | al[t];
      int delta = 0;
      // last departure from s, no arrival to s before it, no pin of e staying in s
      if (maxd_s == K && !((nm[s >> 5] >> (s & 31)) & 1u) && (mina_s == ~0ull || K < mina_s)) delta += wt;
      // first arrival to t, every departure from t before it, no pin of e staying in t
      if (mina_t == K && !((nm[t >> 5] >> (t & 31)) & 1u) && maxd_t < K) delta -= wt;
      if (delta) atomicAdd(&a.rg[v[q]], delta);
    }
    __syncwarp();
  }
}

// G lanes per edge (G = 16 for 8 < |e| <= 16, two edges per warp; G = 32 for
// 16 < |e| <= 32), one pin per lane, software-pipelined over the group's
// edges: while edge j is evaluated, the candidate records and blocks of edge
// j+1, the pins of edge j+2, the offsets of edge j+3 and the id of edge j+4
// are in flight, so the chain list -> offsets -> pins -> records costs one
// memory latency per edge instead of four.  The evaluation is the same three
// passes as in k_ab_warp, on one table per group.
template <int G>
__global__ void __launch_bounds__(kAbWarps * 32) k_ab_warp_small(AbArgs a) {
  static_assert(G == 16 || G == 32, "a group is a half warp or a warp");
  constexpr int kGroups = kAbWarps * (32 / G);
  extern __shared__ unsigned long long s_tab[];  // per group: the high and low words of maxd[k], mina[k]
  __shared__ uint32_t s_nm[kGroups][kMaxK / 32];
  const int li = threadIdx.x % G, grp = threadIdx.x / G;
  uint32_t *dh = reinterpret_cast<uint32_t *>(s_tab + (size_t)grp * 2 * a.k);
  uint32_t *dl = dh + a.k, *ah = dl + a.k, *al = ah + a.k;
  uint32_t *nm = s_nm[grp];
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const long long nw = (gridDim.x * (long long)blockDim.x) / G;
  auto edge_at = [&](long long i) -> int { return i < a.nlist ? a.elist[i] : -1; };
  // stage registers, named by how many edges ahead of the evaluated one they are
  int e4 = edge_at(gw + 4 * nw);
  int e3 = edge_at(gw + 3 * nw);
  int64_t p3 = e3 >= 0 ? a.eptr[e3] : 0;
  int sz3 = e3 >= 0 ? (int)(a.eptr[e3 + 1] - p3) : 0;
  int e2 = edge_at(gw + 2 * nw);
  int v2 = -1;
  if (e2 >= 0) {
    const int64_t q = a.eptr[e2];
    if (li < a.eptr[e2 + 1] - q) v2 = a.pins[q + li];
  }
  int e1 = edge_at(gw + nw), v1 = -1;
  uint64_t r1 = 0;
  int b1 = 0;
  if (e1 >= 0) {
    const int64_t q = a.eptr[e1];
    if (li < a.eptr[e1 + 1] - q) {
      v1 = a.pins[q + li];
      r1 = a.cand[v1];
      b1 = a.part[v1];
    }
  }
  int e0 = edge_at(gw), v0 = -1;
  uint64_t r0 = 0;
  int b0 = 0;
  if (e0 >= 0) {
    const int64_t q = a.eptr[e0];
    if (li < a.eptr[e0 + 1] - q) {
      v0 = a.pins[q + li];
      r0 = a.cand[v0];
      b0 = a.part[v0];
    }
  }
  // The groups of a warp run in lockstep: the loop bound is the warp's first
  // group (a group past the end of the list has e0 = -1 and no pins), so the
  // warp-wide votes and barriers below see every lane.
  const long long wfirst = (blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31)) / G;
  for (long long i = gw, iw = wfirst; iw < a.nlist; i += nw, iw += nw) {
    // advance the pipeline: every load below is first used one iteration later
    const int e5 = edge_at(i + 5 * nw);
    const int64_t p4 = e4 >= 0 ? a.eptr[e4] : 0;
    const int sz4 = e4 >= 0 ? (int)(a.eptr[e4 + 1] - p4) : 0;
    const int v3 = li < sz3 ? a.pins[p3 + li] : -1;
    const uint64_t r2 = v2 >= 0 ? a.cand[v2] : 0ull;
    const int b2 = v2 >= 0 ? a.part[v2] : 0;
    // evaluate edge e0 with v0 / r0 / b0
    const uint64_t r = r0;
    const int s = cand_s(r), t = cand_t(r);
    if (r) {
      dh[s] = 0u; dl[s] = 0u; ah[s] = ~0u; al[s] = ~0u;
      dh[t] = 0u; dl[t] = 0u; ah[t] = ~0u; al[t] = ~0u;
      nm[s >> 5] = 0u;
      nm[t >> 5] = 0u;
    }
    if (__any_sync(kFull, r != 0)) {
      __syncwarp();
      const uint64_t K = cand_key(r, v0);
      const uint32_t kh = (uint32_t)(K >> 32), kl = (uint32_t)K;
      if (r) {
        atomicMax(&dh[s], kh);
        atomicMin(&ah[t], kh);
      } else if (v0 >= 0) {
        const int b = b0 & 255;
        atomicOr(&nm[b >> 5], 1u << (b & 31));
      }
      __syncwarp();
      if (r) {  // the low words among the keys with the extreme high word
        if (dh[s] == kh) atomicMax(&dl[s], kl);
        if (ah[t] == kh) atomicMin(&al[t], kl);
      }
      __syncwarp();
      if (r) {
        const int wt = a.ewgt[e0];
        const uint64_t maxd_s = ((uint64_t)dh[s] << 32) | dl[s], mina_s = ((uint64_t)ah[s] << 32) | al[s];
        const uint64_t maxd_t = ((uint64_t)dh[t] << 32) | dl[t], mina_t = ((uint64_t)ah[t] << 32) | al[t];
        int delta = 0;
        if (maxd_s == K && !((nm[s >> 5] >> (s & 31)) & 1u) && (mina_s == ~0ull || K < mina_s)) delta += wt;
        if (mina_t == K && !((nm[t >> 5] >> (t & 31)) & 1u) && maxd_t < K) delta -= wt;
        if (delta) atomicAdd(&a.rg[v0], delta);
      }
      __syncwarp();
    }
    e0 = e1; v0 = v1; r0 = r1; b0 = b1;
    e1 = e2; v1 = v2; r1 = r2; b1 = b2;
    e2 = e3; v2 = v3;
    e3 = e4; p3 = p4; sz3 = sz4;
    e4 = e5;
  }
}

// Block-class edges (|e| > kWarpEdge) in segments of at most kSegPins pins,
// one thread block per segment, so a hub edge of 200,000 pins is spread over
// ~100 blocks instead of serialising one.  A block builds the per-block
// max-departure / min-arrival table and the non-candidate mask of its
// segment in shared memory.  An edge that is a single segment is decided
// right there; the segments of a longer edge merge their tables into the
// edge's slot of a global table (atomic max / min / or), and k_ab_slots
// decides those edges afterwards and resets the slots.
constexpr int kSegThreads = 256;

struct SegArgs {
  AbArgs ab;
  const int4 *seg;                 // edge, first pin (offset in pins), pins, slot or -1
  int32_t nseg;
  const int32_t *slot_edge;
  unsigned long long *tab;         // slot * 2k: maxd[k] then mina[k]
  uint32_t *nmw;                   // slot * 8 words
  int32_t nslots;
};

__device__ __forceinline__ void ab_decide(const AbArgs &a, int b, unsigned long long md, unsigned long long ma,
                                          bool nm, int w) {
  const bool has_d = md != 0ull, has_a = ma != ~0ull;
  if ((!has_d && !has_a) || nm) return;        // nothing moves here, or a pin of e in b stays
  if (has_d && has_a && !(md < ma)) return;     // an arrival precedes the last departure
  if (has_d) atomicAdd(&a.rg[(int)(md & 0xffffffffu)], w);
  if (has_a) atomicAdd(&a.rg[(int)(ma & 0xffffffffu)], -w);
  (void)b;
}

__global__ void __launch_bounds__(kSegThreads) k_ab_block(SegArgs sa) {
  const AbArgs &a = sa.ab;
  extern __shared__ unsigned long long s_mem[];
  // high and low words of the max key among departures (dh, dl) and of the min key among arrivals (ah, al)
  uint32_t *dh = reinterpret_cast<uint32_t *>(s_mem), *dl = dh + a.k, *ah = dl + a.k, *al = ah + a.k;
  __shared__ uint32_t s_nm[kMaxK / 32];      // blocks holding a non-candidate pin
  constexpr int kPer = kSegPins / kSegThreads;
  for (int i = blockIdx.x; i < sa.nseg; i += gridDim.x) {
    const int4 sg = sa.seg[i];
    for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
      dh[b] = 0u;
      dl[b] = 0u;
      ah[b] = ~0u;
      al[b] = ~0u;
    }
    if (threadIdx.x < kMaxK / 32) s_nm[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p0 = a.eptr[sg.x] + sg.y;
    int v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int j = q * kSegThreads + threadIdx.x;
      v[q] = j < sg.z ? a.pins[p0 + j] : -1;
    }
    uint64_t r[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) r[q] = v[q] >= 0 ? a.cand[v[q]] : 0ull;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (v[q] < 0) continue;
      if (r[q]) {
        const uint32_t kh = (uint32_t)(cand_key(r[q], v[q]) >> 32);
        atomicMax(&dh[cand_s(r[q])], kh);
        atomicMin(&ah[cand_t(r[q])], kh);
      } else {
        const int b = a.part[v[q]] & 255;
        const uint32_t bit = 1u << (b & 31);
        if (!(s_nm[b >> 5] & bit)) atomicOr(&s_nm[b >> 5], bit);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {  // the low words among the keys with the extreme high word
      if (!r[q]) continue;
      const uint32_t kh = (uint32_t)(cand_key(r[q], v[q]) >> 32), kl = (uint32_t)v[q];
      const int s = cand_s(r[q]), t = cand_t(r[q]);
      if (dh[s] == kh) atomicMax(&dl[s], kl);
      if (ah[t] == kh) atomicMin(&al[t], kl);
    }
    __syncthreads();
    if (sg.w < 0) {  // the whole edge: decide here
      const int w = a.ewgt[sg.x];
      for (int b = threadIdx.x; b < a.k; b += blockDim.x)
        ab_decide(a, b, ((unsigned long long)dh[b] << 32) | dl[b], ((unsigned long long)ah[b] << 32) | al[b],
                  (s_nm[b >> 5] >> (b & 31)) & 1u, w);
    } else {  // one segment of a longer edge: merge into its slot
      unsigned long long *tmax = sa.tab + (size_t)sg.w * 2 * a.k, *tmin = tmax + a.k;
      for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
        const unsigned long long md = ((unsigned long long)dh[b] << 32) | dl[b];
        const unsigned long long ma = ((unsigned long long)ah[b] << 32) | al[b];
        if (md != 0ull) atomicMax(&tmax[b], md);
        if (ma != ~0ull) atomicMin(&tmin[b], ma);
      }
      if (threadIdx.x < kMaxK / 32 && s_nm[threadIdx.x]) atomicOr(&sa.nmw[sg.w * 8 + threadIdx.x], s_nm[threadIdx.x]);
    }
    __syncthreads();
  }
}

// The edges longer than one segment: decide every (edge, block) from the
// merged tables, then reset the slot for the next call.
__global__ void __launch_bounds__(256) k_ab_slots(SegArgs sa) {
  const AbArgs &a = sa.ab;
  const int64_t total = (int64_t)sa.nslots * a.k;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(x / a.k), b = (int)(x % a.k);
    unsigned long long *tmax = sa.tab + (size_t)slot * 2 * a.k, *tmin = tmax + a.k;
    const bool nm = (sa.nmw[slot * 8 + (b >> 5)] >> (b & 31)) & 1u;
    ab_decide(a, b, tmax[b], tmin[b], nm, a.ewgt[sa.slot_edge[slot]]);
    tmax[b] = 0ull;
    tmin[b] = ~0ull;
  }
}

__global__ void k_ab_slots_clear_nm(uint32_t *nmw, int32_t words) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < words; x += gridDim.x * blockDim.x) nmw[x] = 0u;
}

__global__ void k_edge_sizes(const int64_t *eptr, const int32_t *ids, int32_t n, int64_t *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = eptr[ids[i] + 1] - eptr[ids[i]];
}

__global__ void k_ab_slots_init(unsigned long long *tab, int32_t nslots, int32_t k) {
  const int64_t total = (int64_t)nslots * 2 * k;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x)
    tab[x] = ((x / k) & 1) ? ~0ull : 0ull;
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

// Graph path: for a two-pin edge e = {v, u} the replay of Algorithm 2 gives v
// +omega(e) when u's block at v's turn differs from s (the last departure) and
// -omega(e) when it differs from t (the first arrival); u's block at v's turn
// is t(u) if u is a candidate ordered before v, else Pi(u).  So rg(v) is a
// sum over v's neighbours, computed per candidate with no atomics: a lane per
// vertex of degree <= 64 (four neighbours in flight), the whole warp for
// larger degrees.
struct AbGraphArgs {
  const int64_t *vptr;
  const int32_t *adj, *inc, *ewgt, *part;
  const uint64_t *cand;
  int32_t *rg;
  int32_t n;
  int unit;
};

__device__ __forceinline__ int32_t ab_graph_term(const AbGraphArgs &a, uint64_t kv, int s, int t, int64_t j) {
  const int u = a.adj[j];
  const uint64_t ru = a.cand[u];
  const int bu = ru ? (cand_key(ru, u) < kv ? cand_t(ru) : cand_s(ru)) : a.part[u];
  const int32_t w = a.unit ? 1 : a.ewgt[a.inc[j]];
  return w * ((int)(bu != s) - (int)(bu != t));
}

__global__ void __launch_bounds__(256) k_ab_graph(AbGraphArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; base < a.n; base += stride) {
    const int64_t v = base + lane;
    const uint64_t rec = v < a.n ? a.cand[v] : 0ull;
    int64_t j0 = 0, j1 = 0;
    if (rec) {
      j0 = a.vptr[v];
      j1 = a.vptr[v + 1];
    }
    const bool heavy = rec && j1 - j0 > 64;
    if (rec && !heavy) {
      const uint64_t kv = cand_key(rec, (int32_t)v);
      const int s = cand_s(rec), t = cand_t(rec);
      int32_t acc = 0;
      int64_t j = j0;
      for (; j + 4 <= j1; j += 4) {
        int32_t x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = ab_graph_term(a, kv, s, t, j + q);
        acc += x[0] + x[1] + x[2] + x[3];
      }
      for (; j < j1; ++j) acc += ab_graph_term(a, kv, s, t, j);
      a.rg[v] = acc;
    }
    unsigned bal = __ballot_sync(0xffffffffu, heavy);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const int64_t hv = base + src;
      const uint64_t hrec = __shfl_sync(0xffffffffu, rec, src);
      const int64_t h0 = __shfl_sync(0xffffffffu, j0, src), h1 = __shfl_sync(0xffffffffu, j1, src);
      const uint64_t kv = cand_key(hrec, (int32_t)hv);
      const int s = cand_s(hrec), t = cand_t(hrec);
      int32_t acc = 0;
      for (int64_t j = h0 + lane; j < h1; j += 32) acc += ab_graph_term(a, kv, s, t, j);
      acc = __reduce_add_sync(0xffffffffu, acc);
      if (lane == 0) a.rg[hv] = acc;
    }
  }
}

}  // namespace

cudaError_t launch_afterburner(jet_ctx *c, const int32_t *part, const int32_t *phi) {
  (void)phi;  // phi_e[b] = |D_b| is tested through the non-candidate pins' blocks
  if (c->graph_path) {
    if (c->n == 0) return cudaSuccess;
    AbGraphArgs g{c->vptr, c->adj, c->inc, c->ewgt, part, c->cand, c->rg, c->n, c->unit_ewgt};
    k_ab_graph<<<grid_for(c->n, 256, c->launch_sms, 8), 256, 0, c->stream>>>(g);
    ++c->kernel_launches;
    return cudaGetLastError();
  }
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
    k_ab_tiny<<<grid_for(c->n_tiny, 256, c->launch_sms, c->ab_bps[0]), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid_half > 0) {
    a.elist = c->e_mid_half;
    a.nlist = c->n_mid_half;
    const size_t smem = (size_t)kAbWarps * 2 * 2 * c->k * sizeof(unsigned long long);
    k_ab_warp_small<16><<<grid_for((int64_t)c->n_mid_half * 16, kAbWarps * 32, c->launch_sms, c->ab_bps[1]),
                          kAbWarps * 32, smem, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid_small > 0) {
    a.elist = c->e_mid_small;
    a.nlist = c->n_mid_small;
    const size_t smem = (size_t)kAbWarps * 2 * c->k * sizeof(unsigned long long);
    k_ab_warp_small<32><<<grid_for((int64_t)c->n_mid_small * 32, kAbWarps * 32, c->launch_sms, c->ab_bps[2]),
                          kAbWarps * 32, smem, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_mid > 0) {  // 65..128 pins first, then 33..64
    const size_t smem = (size_t)kAbWarps * 2 * c->k * sizeof(unsigned long long);
    if (c->n_mid_hi > 0) {
      a.elist = c->e_mid;
      a.nlist = c->n_mid_hi;
      k_ab_warp<4><<<grid_for((int64_t)c->n_mid_hi * 32, kAbWarps * 32, c->launch_sms, c->ab_bps[3]), kAbWarps * 32,
                     smem, c->stream>>>(a);
      ++c->kernel_launches;
    }
    if (c->n_mid > c->n_mid_hi) {
      a.elist = c->e_mid + c->n_mid_hi;
      a.nlist = c->n_mid - c->n_mid_hi;
      k_ab_warp<2><<<grid_for((int64_t)a.nlist * 32, kAbWarps * 32, c->launch_sms, c->ab_bps[5]), kAbWarps * 32, smem,
                     c->stream>>>(a);
      ++c->kernel_launches;
    }
  }
  if (c->n_seg > 0) {
    SegArgs sa{};
    sa.ab = a;
    sa.seg = c->ab_seg;
    sa.nseg = c->n_seg;
    sa.slot_edge = c->ab_slot_edge;
    sa.tab = c->ab_tab;
    sa.nmw = c->ab_nm;
    sa.nslots = c->n_slots;
    const size_t smem = (size_t)c->k * 2 * sizeof(unsigned long long);
    k_ab_block<<<grid_for(c->n_seg, 1, c->launch_sms, c->ab_bps[4]), kSegThreads, smem, c->stream>>>(sa);
    ++c->kernel_launches;
    if (c->n_slots > 0) {
      k_ab_slots<<<grid_for((int64_t)c->n_slots * c->k, 256, c->launch_sms), 256, 0, c->stream>>>(sa);
      k_ab_slots_clear_nm<<<grid_for((int64_t)c->n_slots * 8, 256, c->launch_sms), 256, 0, c->stream>>>(
          c->ab_nm, c->n_slots * 8);
      c->kernel_launches += 2;
    }
  }
  return cudaGetLastError();
}

// Resident blocks per SM of the afterburner kernels at this context's k.
cudaError_t prepare_afterburner_kernels(jet_ctx *c) {
  const size_t warp_tab = (size_t)kAbWarps * 2 * c->k * sizeof(unsigned long long);
  // The half-warp kernel holds two tables per warp: above 48 KB for k > 192.  The limit is a property
  // of the kernel, shared by every context, so it is set for the largest k, not for this context's.
  cudaError_t e = cudaFuncSetAttribute(k_ab_warp_small<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)kAbWarps * 2 * 2 * kMaxK * sizeof(unsigned long long)));
  if (e == cudaSuccess) e = resident_blocks(k_ab_tiny, 256, 0, &c->ab_bps[0]);
  if (e == cudaSuccess) e = resident_blocks(k_ab_warp_small<16>, kAbWarps * 32, 2 * warp_tab, &c->ab_bps[1]);
  if (e == cudaSuccess) e = resident_blocks(k_ab_warp_small<32>, kAbWarps * 32, warp_tab, &c->ab_bps[2]);
  if (e == cudaSuccess) e = resident_blocks(k_ab_warp<4>, kAbWarps * 32, warp_tab, &c->ab_bps[3]);
  if (e == cudaSuccess) e = resident_blocks(k_ab_warp<2>, kAbWarps * 32, warp_tab, &c->ab_bps[5]);
  if (e == cudaSuccess)
    e = resident_blocks(k_ab_block, kSegThreads, (size_t)c->k * 2 * sizeof(unsigned long long), &c->ab_bps[4]);
  return e;
}

// Cuts the block-class edges into segments (largest first) and sets up the
// merge table of the edges longer than one segment.  Host work, once per
// context (synchronizes the stream).
cudaError_t prepare_afterburner(jet_ctx *c) {
  if (c->n_big == 0) return cudaSuccess;
  std::vector<int32_t> ids(c->n_big);
  cudaError_t e = cudaMemcpyAsync(ids.data(), c->e_big, sizeof(int32_t) * c->n_big, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
  std::vector<int64_t> sz(c->n_big);
  int64_t *dsz = nullptr;
  if ((e = jet::pool_alloc(reinterpret_cast<void **>(&dsz), sizeof(int64_t) * c->n_big, c->stream)) != cudaSuccess)
    return e;
  k_edge_sizes<<<grid_for(c->n_big, 256, c->launch_sms), 256, 0, c->stream>>>(c->eptr, c->e_big, c->n_big, dsz);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sz.data(), dsz, sizeof(int64_t) * c->n_big, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFreeAsync(dsz, c->stream);
  if (e != cudaSuccess) return e;
  std::vector<int4> seg;
  std::vector<int32_t> slot_edge;
  for (int32_t i = 0; i < c->n_big; ++i) {
    const int slot = sz[i] > kSegPins ? (int)slot_edge.size() : -1;
    if (slot >= 0) slot_edge.push_back(ids[i]);
    for (int64_t off = 0; off < sz[i]; off += kSegPins)
      seg.push_back(make_int4(ids[i], (int)off, (int)std::min<int64_t>(kSegPins, sz[i] - off), slot));
  }
  std::stable_sort(seg.begin(), seg.end(), [](const int4 &x, const int4 &y) { return x.z > y.z; });
  c->n_seg = (int32_t)seg.size();
  c->n_slots = (int32_t)slot_edge.size();
  if ((e = jet::pool_alloc(reinterpret_cast<void **>(&c->ab_seg), sizeof(int4) * seg.size(), c->stream)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(c->ab_seg, seg.data(), sizeof(int4) * seg.size(), cudaMemcpyHostToDevice, c->stream)) !=
      cudaSuccess)
    return e;
  if (c->n_slots > 0) {
    const size_t ns = (size_t)c->n_slots;
    if ((e = jet::pool_alloc(reinterpret_cast<void **>(&c->ab_slot_edge), sizeof(int32_t) * ns, c->stream)) !=
            cudaSuccess ||
        (e = jet::pool_alloc(reinterpret_cast<void **>(&c->ab_tab), sizeof(unsigned long long) * ns * 2 * c->k,
                             c->stream)) != cudaSuccess ||
        (e = jet::pool_alloc(reinterpret_cast<void **>(&c->ab_nm), sizeof(uint32_t) * ns * 8, c->stream)) !=
            cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(c->ab_slot_edge, slot_edge.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return e;
    k_ab_slots_init<<<grid_for((int64_t)ns * 2 * c->k, 256, c->launch_sms), 256, 0, c->stream>>>(c->ab_tab,
                                                                                                   c->n_slots, c->k);
    k_ab_slots_clear_nm<<<grid_for((int64_t)ns * 8, 256, c->launch_sms), 256, 0, c->stream>>>(c->ab_nm,
                                                                                              c->n_slots * 8);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(c->stream);
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
