// Move candidates (Section 4.1) and rebalancing targets (Section 4.3).
//
// gain(v, b) = conn(v, b) - A(v) for v in V_s, where conn(v, b) = sum of
// omega(e) over e in I(v) with phi_e[b] >= 1 and A(v) = sum of omega(e) over
// e in I(v) with phi_e[s] >= 2.  Both come from the two bitmasks of each
// edge (phi_e[.] >= 1 and >= 2), so this pass reads no phi entry.  (Per edge, [phi_e[s] = 1] - [phi_e[b] = 0]
// = [phi_e[b] >= 1] - [phi_e[s] >= 2], which is the +-omega rule of
// Algorithm 2 summed over I(v).)
//
// Light vertices (weighted degree < 2^kLightPlanes): one thread per vertex
// keeps conn(v, .) for all k blocks as kLightPlanes bit planes of k-bit
// words and adds each incident edge's Lambda(e) bitmask with a ripple-carry
// over the planes.  The argmax over a candidate block set C is then a
// bit-serial maximum: from the top plane down, keep the blocks of C whose
// bit is set if any is; the lowest remaining block id is the smallest-id
// maximiser.  Heavy vertices: one warp per vertex, lane l owning blocks
// l, l+32, ..., exact int32 counters, and a warp argmax.
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct CandArgs {
  const int64_t *vptr;
  const int32_t *inc, *ewgt, *vwgt, *part, *phi;
  const uint32_t *mask;
  const uint8_t *locked;
  const int32_t *vlist;
  int32_t nlist, k;
  int32_t tau_num, tau_den;
  uint64_t *cand;
  // rebalancing
  const RbBlock *rbb;
  uint64_t *rb_hi;
  int32_t *rb_v, *rb_ct;
  long long A;
  int32_t n;
  Counters *cnt;
  int rb_compact;
  long long rb_L, rb_Pmax;
};

// One edge's mask row: KWP words of Lambda(e) then KWP words of the blocks
// with >= 2 pins of e (aligned vector loads, 2*KWP*4 bytes).
template <int KWP>
__device__ __forceinline__ void load_rows(const uint32_t *row, uint32_t (&M)[KWP], uint32_t (&M2)[KWP]) {
  if constexpr (KWP == 1) {
    const uint2 x = __ldg(reinterpret_cast<const uint2 *>(row));
    M[0] = x.x; M2[0] = x.y;
  } else if constexpr (KWP == 2) {
    const uint4 x = __ldg(reinterpret_cast<const uint4 *>(row));
    M[0] = x.x; M[1] = x.y; M2[0] = x.z; M2[1] = x.w;
  } else {
#pragma unroll
    for (int h = 0; h < KWP / 4; ++h) {
      const uint4 x = __ldg(reinterpret_cast<const uint4 *>(row) + h);
      const uint4 y = __ldg(reinterpret_cast<const uint4 *>(row + KWP) + h);
      M[4 * h] = x.x; M[4 * h + 1] = x.y; M[4 * h + 2] = x.z; M[4 * h + 3] = x.w;
      M2[4 * h] = y.x; M2[4 * h + 1] = y.y; M2[4 * h + 2] = y.z; M2[4 * h + 3] = y.w;
    }
  }
}

// bit b of a KWP-word mask (word chosen without dynamic register indexing)
template <int KWP>
__device__ __forceinline__ bool mask_bit(const uint32_t (&M)[KWP], int b) {
  uint32_t x = 0;
#pragma unroll
  for (int q = 0; q < KWP; ++q) x |= (q == (b >> 5)) ? M[q] : 0u;
  return (x >> (b & 31)) & 1u;
}

// planes += w * M  (w < 2^NP, no overflow past the top plane by construction)
template <int KWP, int NP>
__device__ __forceinline__ void add_weighted(uint32_t (&pl)[NP][KWP], const uint32_t (&M)[KWP], uint32_t w) {
  while (w) {
    const int p0 = __ffs(w) - 1;
    w &= w - 1;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      uint32_t carry = M[q];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p >= p0) {
          uint32_t c2 = pl[p][q] & carry;
          pl[p][q] ^= carry;
          carry = c2;
        }
      }
    }
  }
}

// planes += M (unit weight): ripple carry that stops as soon as no carry is left
template <int KWP, int NP>
__device__ __forceinline__ void add_one(uint32_t (&pl)[NP][KWP], const uint32_t (&M)[KWP]) {
  uint32_t carry[KWP];
#pragma unroll
  for (int q = 0; q < KWP; ++q) carry[q] = M[q];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    uint32_t nz = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      const uint32_t c2 = pl[p][q] & carry[q];
      pl[p][q] ^= carry[q];
      carry[q] = c2;
      nz |= c2;
    }
    if (!nz) break;
  }
}

// smallest block id maximising conn over the nonempty set C; returns the id and conn
template <int KWP, int NP>
__device__ __forceinline__ int argmax_planes(const uint32_t (&pl)[NP][KWP], uint32_t (&C)[KWP], int32_t &conn) {
#pragma unroll
  for (int p = NP - 1; p >= 0; --p) {
    uint32_t X[KWP];
    uint32_t nz = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) { X[q] = C[q] & pl[p][q]; nz |= X[q]; }
    if (nz) {
#pragma unroll
      for (int q = 0; q < KWP; ++q) C[q] = X[q];
    }
  }
  int t = -1;
#pragma unroll
  for (int q = KWP - 1; q >= 0; --q)
    if (C[q]) t = q * 32 + __ffs(C[q]) - 1;
  conn = 0;
  const int tq = t >> 5, tb = t & 31;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    uint32_t bit = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) bit |= (q == tq) ? ((pl[p][q] >> tb) & 1u) : 0u;
    conn |= (int32_t)bit << p;
  }
  return t;
}

// conn planes, union of Lambda(e) and A(v) over I(v) for a light vertex.
// UNIT: every omega(e) is 1 (no weight gathers, increments instead of adds).
template <int KWP, int NP, bool UNIT>
__device__ __forceinline__ int32_t accumulate_light(const CandArgs &a, int v, int s, uint32_t (&pl)[NP][KWP],
                                                    uint32_t (&any)[KWP]) {
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    any[q] = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) pl[p][q] = 0;
  }
  int32_t A = 0;
  const int64_t j1 = a.vptr[v + 1];
  int64_t j = a.vptr[v];
  // B incidences at a time: their gathers are issued before any is used
  // (fewer for wide masks, to keep registers and occupancy in balance)
  constexpr int B = KWP >= 4 ? 2 : 4;
  for (; j + B <= j1; j += B) {
    int e[B], w[B];
    uint32_t M[B][KWP], M2[B][KWP];
#pragma unroll
    for (int u = 0; u < B; ++u) e[u] = a.inc[j + u];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      w[u] = UNIT ? 1 : a.ewgt[e[u]];
      load_rows<KWP>(a.mask + (int64_t)e[u] * 2 * KWP, M[u], M2[u]);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      uint32_t Mu[KWP], M2u[KWP];
#pragma unroll
      for (int q = 0; q < KWP; ++q) { Mu[q] = M[u][q]; M2u[q] = M2[u][q]; }
      A += mask_bit<KWP>(M2u, s) ? w[u] : 0;  // phi_e[s] >= 2
#pragma unroll
      for (int q = 0; q < KWP; ++q) any[q] |= Mu[q];
      if (UNIT) add_one<KWP, NP>(pl, Mu);
      else add_weighted<KWP, NP>(pl, Mu, (uint32_t)w[u]);
    }
  }
  for (; j < j1; ++j) {
    const int e = a.inc[j];
    const int w = UNIT ? 1 : a.ewgt[e];
    uint32_t M[KWP], M2[KWP];
    load_rows<KWP>(a.mask + (int64_t)e * 2 * KWP, M, M2);
    A += mask_bit<KWP>(M2, s) ? w : 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) any[q] |= M[q];
    if (UNIT) add_one<KWP, NP>(pl, M);
    else add_weighted<KWP, NP>(pl, M, (uint32_t)w);
  }
  return A;
}

template <int KWP, bool UNIT>
__global__ void __launch_bounds__(256) k_cand_light(CandArgs a) {
  constexpr int NP = kLightPlanes;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nlist; i += gridDim.x * blockDim.x) {
    const int v = a.vlist[i];
    uint64_t rec = 0;
    const int s = a.part[v];
    if ((unsigned)s >= (unsigned)a.k) {  // invalid block id: report, never index with it
      atomicOr(&a.cnt->err, kErrPartRange);
    } else if (!a.locked[v]) {
      uint32_t pl[NP][KWP], any[KWP];
      const int32_t A = accumulate_light<KWP, NP, UNIT>(a, v, s, pl, any);
      uint32_t C[KWP];
      uint32_t nz = 0;
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        C[q] = any[q] & ~((s >> 5) == q ? (1u << (s & 31)) : 0u);
        nz |= C[q];
      }
      if (nz) {
        int32_t conn;
        const int t = argmax_planes<KWP, NP>(pl, C, conn);
        const int32_t g = conn - A;
        if ((long long)a.tau_den * g >= -(long long)a.tau_num * A) rec = pack_cand(g, s, t);
      }
    }
    a.cand[v] = rec;
  }
}

// Warp argmax of (conn desc, block asc); block -1 = none.  Result on all lanes.
__device__ __forceinline__ void warp_argmax(int32_t &c, int &b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int32_t c2 = __shfl_xor_sync(kFull, c, o);
    int b2 = __shfl_xor_sync(kFull, b, o);
    bool take = b2 >= 0 && (b < 0 || c2 > c || (c2 == c && b2 < b));
    if (take) { c = c2; b = b2; }
  }
}

// conn(v, b) for the lane's blocks b = lane + 32q, Lambda-adjacency bits and A(v)
template <int KWP>
__device__ __forceinline__ int32_t accumulate_heavy(const CandArgs &a, int v, int s, int32_t (&conn)[KWP],
                                                    uint32_t &adj) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < KWP; ++q) conn[q] = 0;
  adj = 0;
  int32_t Ap = 0;
  const int64_t j0 = a.vptr[v], j1 = a.vptr[v + 1];
  for (int64_t base = j0; base < j1; base += 32) {
    const int64_t j = base + lane;
    const bool ok = j < j1;
    int e = 0, w = 0;
    uint32_t M[KWP], M2[KWP];
#pragma unroll
    for (int q = 0; q < KWP; ++q) M[q] = M2[q] = 0;
    if (ok) {
      e = a.inc[j];
      w = a.ewgt[e];
      load_rows<KWP>(a.mask + (int64_t)e * 2 * KWP, M, M2);
      if (mask_bit<KWP>(M2, s)) Ap += w;  // phi_e[s] >= 2
    }
    const int cntc = (int)((j1 - base) < 32 ? (j1 - base) : 32);
    for (int l = 0; l < cntc; ++l) {
      const int wl = __shfl_sync(kFull, w, l);
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        const uint32_t Mq = __shfl_sync(kFull, M[q], l);
        if ((Mq >> lane) & 1u) { conn[q] += wl; adj |= 1u << q; }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Ap += __shfl_xor_sync(kFull, Ap, o);
  return Ap;
}

template <int KWP>
__global__ void __launch_bounds__(256) k_cand_heavy(CandArgs a) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < a.nlist; i += nw) {
    const int v = a.vlist[i];
    const int s = a.part[v];
    if (a.locked[v] || (unsigned)s >= (unsigned)a.k) {
      if (lane == 0) {
        a.cand[v] = 0;
        if ((unsigned)s >= (unsigned)a.k) atomicOr(&a.cnt->err, kErrPartRange);
      }
      continue;
    }
    int32_t conn[KWP];
    uint32_t adj;
    const int32_t A = accumulate_heavy<KWP>(a, v, s, conn, adj);
    int bb = -1;
    int32_t bc = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      const int b = q * 32 + lane;
      if (b < a.k && b != s && ((adj >> q) & 1u) && (bb < 0 || conn[q] > bc)) { bb = b; bc = conn[q]; }
    }
    warp_argmax(bc, bb);
    if (lane == 0) {
      uint64_t rec = 0;
      if (bb >= 0) {
        const int32_t g = bc - A;
        if ((long long)a.tau_den * g >= -(long long)a.tau_num * A) rec = pack_cand(g, s, bb);
      }
      a.cand[v] = rec;
    }
  }
}

// ------------------------------------------------------------ rebalancing
// Exact priority (Section 4.3): gain * c for gain >= 0; for gain < 0 the
// ratio gain / c scaled by 2^30 and truncated.  With c <= 2^15 two distinct
// ratios differ by >= 2^-30, so the scaled values differ by >= 1 and the
// truncation keeps their order; equal ratios stay equal.  All gain < 0 keys
// are <= -2^15 < 0 <= every gain >= 0 key, so the classes keep their order.
// U = INT64_MAX - P (mod 2^64) turns "priority desc" into "U asc".
// Compact form (rb_compact): with L = lcm(1..cmax), gain/c = gain*(L/c) / L,
// so gain*(L/c) orders the gain < 0 class exactly (equal ratios stay equal)
// and stays <= -1 < 0 <= gain*c of the gain >= 0 class; Pmax - P is then
// below 2^32 (checked by the context) and needs far fewer key bits.
__device__ __forceinline__ uint64_t rb_order_key(int32_t g, int32_t c) {
  long long P = g >= 0 ? (long long)g * c : ((long long)g * (1ll << kPrioShift)) / c;
  return (uint64_t)0x7fffffffffffffffull - (uint64_t)P;
}

// Record of v for the selection: the priority part of its key and (c, target).
__device__ __forceinline__ uint64_t rb_hi_of(const CandArgs &a, int32_t g, int32_t c) {
  if (a.rb_compact) {
    const long long P = g >= 0 ? (long long)g * c : (long long)g * (a.rb_L / c);
    return (uint64_t)(a.rb_Pmax - P);
  }
  return rb_order_key(g, c);
}

template <int KWP>
__device__ __forceinline__ void eligible_words(const long long *s_cap, int k, int32_t c, uint32_t (&E)[KWP]) {
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    uint32_t w = 0;
    for (int bit = 0; bit < 32; ++bit) {
      const int b = q * 32 + bit;
      if (b < k && s_cap[b] >= c) w |= 1u << bit;
    }
    E[q] = w;
  }
}

template <int KWP, bool UNIT>
__global__ void __launch_bounds__(256) k_rbcand_light(CandArgs a) {
  constexpr int NP = kLightPlanes;
  constexpr int kTab = 32;  // eligibility words tabulated for c(v) <= 32
  __shared__ long long s_cap[kMaxK], s_bw[kMaxK];
  __shared__ int s_over[kMaxK];
  __shared__ uint32_t s_elig[kTab][KWP];
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    s_cap[b] = a.rbb[b].cap;
    s_bw[b] = a.rbb[b].bw;
    s_over[b] = a.rbb[b].over;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < kTab * KWP; x += blockDim.x) {
    const int c = x / KWP + 1, q = x % KWP;
    uint32_t w = 0;
    for (int bit = 0; bit < 32; ++bit) {
      const int b = q * 32 + bit;
      if (b < a.k && s_cap[b] >= c) w |= 1u << bit;
    }
    s_elig[c - 1][q] = w;
  }
  __syncthreads();
  for (int base = blockIdx.x * blockDim.x; base < a.nlist; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    bool rec = false;
    int v = 0, s = 0;
    uint64_t hi = 0;
    int32_t ct = 0;
    if (i < a.nlist) {
      v = a.vlist[i];
      s = a.part[v];
      if ((unsigned)s < (unsigned)a.k && s_over[s]) {
        const int32_t c = a.vwgt[v];
        if (2ll * c <= 3ll * (s_bw[s] - a.A)) {  // heavy vertices are never moved
          uint32_t C[KWP];
          if (c <= kTab) {
#pragma unroll
            for (int q = 0; q < KWP; ++q) C[q] = s_elig[c - 1][q];
          } else {
            eligible_words<KWP>(s_cap, a.k, c, C);
          }
          uint32_t nz = 0;
#pragma unroll
          for (int q = 0; q < KWP; ++q) nz |= C[q];
          if (nz) {
            uint32_t pl[NP][KWP], any[KWP];
            const int32_t A = accumulate_light<KWP, NP, UNIT>(a, v, s, pl, any);
            int32_t conn;
            const int t = argmax_planes<KWP, NP>(pl, C, conn);
            hi = rb_hi_of(a, conn - A, c);
            ct = (c << 16) | (s << 8) | t;
            rec = true;
          }
        }
      }
    }
    // warp-level append: the gain work between appends spreads these atomics out in time
    const unsigned bal = __ballot_sync(kFull, rec);
    unsigned long long pos0 = 0;
    if ((threadIdx.x & 31) == 0 && bal) pos0 = atomicAdd(&a.cnt->n_rec, (unsigned long long)__popc(bal));
    pos0 = __shfl_sync(kFull, pos0, 0);
    if (rec) {
      const unsigned long long pos = pos0 + __popc(bal & ((1u << (threadIdx.x & 31)) - 1));
      a.rb_hi[pos] = hi;
      a.rb_v[pos] = v;
      a.rb_ct[pos] = ct;
    }
  }
}

template <int KWP>
__global__ void __launch_bounds__(256) k_rbcand_heavy(CandArgs a) {
  __shared__ long long s_cap[kMaxK], s_bw[kMaxK];
  __shared__ int s_over[kMaxK];
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    s_cap[b] = a.rbb[b].cap;
    s_bw[b] = a.rbb[b].bw;
    s_over[b] = a.rbb[b].over;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < a.nlist; i += nw) {
    const int v = a.vlist[i];
    const int s = a.part[v];
    const int32_t c = a.vwgt[v];
    bool any_elig = false;
    if ((unsigned)s < (unsigned)a.k && s_over[s] && 2ll * c <= 3ll * (s_bw[s] - a.A)) {
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        const int b = q * 32 + lane;
        any_elig |= b < a.k && s_cap[b] >= c;
      }
    }
    if (!__any_sync(kFull, any_elig)) continue;  // no record (warp-uniform: one vertex per warp)
    int32_t conn[KWP];
    uint32_t adj;
    const int32_t A = accumulate_heavy<KWP>(a, v, s, conn, adj);
    int bb = -1;
    int32_t bc = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      const int b = q * 32 + lane;
      if (b < a.k && s_cap[b] >= c && (bb < 0 || conn[q] > bc)) { bb = b; bc = conn[q]; }
    }
    warp_argmax(bc, bb);
    if (lane == 0) {
      const unsigned long long pos = atomicAdd(&a.cnt->n_rec, 1ull);
      a.rb_hi[pos] = rb_hi_of(a, bc - A, c);
      a.rb_v[pos] = v;
      a.rb_ct[pos] = (c << 16) | (s << 8) | bb;
    }
  }
}

template <int KWP>
cudaError_t launch_cand_kwp(jet_ctx *c, const CandArgs &base) {
  CandArgs a = base;
  if (c->n_light > 0) {
    a.vlist = c->v_light;
    a.nlist = c->n_light;
    if (c->unit_ewgt) k_cand_light<KWP, true><<<grid_for(c->n_light, 256, c->num_sms), 256, 0, c->stream>>>(a);
    else k_cand_light<KWP, false><<<grid_for(c->n_light, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_heavy > 0) {
    a.vlist = c->v_heavy;
    a.nlist = c->n_heavy;
    k_cand_heavy<KWP><<<grid_for((int64_t)c->n_heavy * 32, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  return cudaGetLastError();
}

template <int KWP>
cudaError_t launch_rbcand_kwp(jet_ctx *c, const CandArgs &base) {
  CandArgs a = base;
  if (c->n_light > 0) {
    a.vlist = c->v_light;
    a.nlist = c->n_light;
    if (c->unit_ewgt) k_rbcand_light<KWP, true><<<grid_for(c->n_light, 256, c->num_sms), 256, 0, c->stream>>>(a);
    else k_rbcand_light<KWP, false><<<grid_for(c->n_light, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_heavy > 0) {
    a.vlist = c->v_heavy;
    a.nlist = c->n_heavy;
    k_rbcand_heavy<KWP><<<grid_for((int64_t)c->n_heavy * 32, 256, c->num_sms), 256, 0, c->stream>>>(a);
    ++c->kernel_launches;
  }
  return cudaGetLastError();
}

CandArgs make_args(jet_ctx *c, const int32_t *part, const int32_t *phi) {
  CandArgs a{};
  a.vptr = c->vptr;
  a.inc = c->inc;
  a.ewgt = c->ewgt;
  a.vwgt = c->vwgt;
  a.part = part;
  a.phi = phi;
  a.mask = c->mask;
  a.k = c->k;
  a.cand = c->cand;
  a.rbb = c->rbb;
  a.rb_hi = c->rb_hi;
  a.rb_v = c->rb_v;
  a.rb_ct = c->rb_ct;
  a.A = c->A;
  a.n = c->n;
  a.cnt = c->cnt;
  a.rb_compact = c->rb_compact;
  a.rb_L = c->rb_L;
  a.rb_Pmax = c->rb_Pmax;
  return a;
}

}  // namespace

cudaError_t launch_candidates(jet_ctx *c, int32_t tau_num, int32_t tau_den, const int32_t *part, const int32_t *phi,
                              const uint8_t *locked) {
  CandArgs a = make_args(c, part, phi);
  a.locked = locked;
  a.tau_num = tau_num;
  a.tau_den = tau_den;
  switch (c->kwp) {
    case 1: return launch_cand_kwp<1>(c, a);
    case 2: return launch_cand_kwp<2>(c, a);
    case 4: return launch_cand_kwp<4>(c, a);
    default: return launch_cand_kwp<8>(c, a);
  }
}

cudaError_t launch_rebalance_candidates(jet_ctx *c, const int32_t *part, const int32_t *phi) {
  CandArgs a = make_args(c, part, phi);
  switch (c->kwp) {
    case 1: return launch_rbcand_kwp<1>(c, a);
    case 2: return launch_rbcand_kwp<2>(c, a);
    case 4: return launch_rbcand_kwp<4>(c, a);
    default: return launch_rbcand_kwp<8>(c, a);
  }
}

}  // namespace jet
