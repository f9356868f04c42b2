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
#include "jet_gain.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct CandArgs {
  const int64_t *vptr;
  const int32_t *inc, *ewgt, *vwgt, *part, *phi;
  const uint32_t *mask;
  const int32_t *adj;  // graph path: the other pin of every incidence (NULL: hypergraph rows)
  const uint8_t *locked;
  const uint8_t *vheavy;
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
  unsigned long long *rb_hist;  // first-level histogram of the rebalancing selection
  int rb_vbits, rb_tbits, rb_digit;
};

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
      if (a.adj) {  // e = {v, u}: Lambda(e) = {s, Pi(u)}, and phi_e[s] >= 2 iff Pi(u) = s
        const int pu = a.part[a.adj[j]];
#pragma unroll
        for (int q = 0; q < KWP; ++q)
          M[q] = ((s >> 5) == q ? 1u << (s & 31) : 0u) | ((pu >> 5) == q ? 1u << (pu & 31) : 0u);
        if (pu == s) Ap += w;
      } else {
        load_rows<KWP>(a.mask + (int64_t)e * 2 * KWP, M, M2);
        if (mask_bit<KWP>(M2, s)) Ap += w;  // phi_e[s] >= 2
      }
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
// Record of v for the selection: the priority part of its key (Section 4.3;
// the exact integer encodings are in jet_gain.cuh) and (c, target).
__device__ __forceinline__ uint64_t rb_hi_of(const CandArgs &a, int32_t g, int32_t c) {
  return rb_priority_key(a.rb_compact, a.rb_L, a.rb_Pmax, g, c);
}

// Adds the thread's work counts to the call's totals: one atomic per thread
// block and counter (every thread of the block calls it).
__device__ __forceinline__ void count_work(Counters *cnt, unsigned long long over, unsigned long long eval,
                                           unsigned long long pins) {
  __shared__ unsigned long long s_w[3];
  if (threadIdx.x < 3) s_w[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    over += __shfl_xor_sync(kFull, over, o);
    eval += __shfl_xor_sync(kFull, eval, o);
    pins += __shfl_xor_sync(kFull, pins, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (over) atomicAdd(&s_w[0], over);
    if (eval) atomicAdd(&s_w[1], eval);
    if (pins) atomicAdd(&s_w[2], pins);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_w[0]) atomicAdd(&cnt->w_over, s_w[0]);
    if (s_w[1]) atomicAdd(&cnt->w_eval, s_w[1]);
    if (s_w[2]) atomicAdd(&cnt->w_eval_pins, s_w[2]);
  }
}

// Top digit of the selection key K(v) = hi << vbits | v (the first radix
// level), added with c(v) into the (block, digit) histogram: one atomic per
// record.  (Grouping the warp's records by (block, digit) with
// __match_any_sync first, one atomic per group, made the rebalancing rounds
// slower: the vote costs more than the atomics it saves.)
__device__ __forceinline__ void rb_first_level(const CandArgs &a, bool rec, int s, uint64_t hi, int v, int32_t c) {
  const int lo = a.rb_tbits - a.rb_digit > 0 ? a.rb_tbits - a.rb_digit : 0;
  int d = 0;
  if (rec) {
    if (a.rb_tbits <= 64) {
      const uint64_t K = (hi << a.rb_vbits) | (uint32_t)v;
      d = (int)((K >> lo) & ((1ull << (a.rb_tbits - lo)) - 1));
    } else {
      const unsigned __int128 K = ((unsigned __int128)hi << a.rb_vbits) | (uint32_t)v;
      d = (int)((K >> lo) & ((1ull << (a.rb_tbits - lo)) - 1));
    }
  }
  if (rec) atomicAdd(&a.rb_hist[((int64_t)s << a.rb_digit) + d], (unsigned long long)c);
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

// ------------------------------------------------------------ light vertices
// A warp takes 32 consecutive vertex ids; each lane evaluates one light
// vertex.  Its incidences I(v) are processed in batches of kBatch: the mask
// rows of a batch are copied into the lane's slots of a double-buffered
// shared-memory stage with cp.async, so batch b+1's gathers (and batch b+2's
// incidence loads) are in flight while batch b is added into the bit planes.
// Slot t of lane l is row t*32 + l of a buffer, so the lanes' reads of the
// stage are bank-conflict free.  Lanes never read each other's slots.

// Minimum resident blocks per SM of the staged light kernels: the register
// budget per thread is 65,536 / (256 x blocks).  At k <= 128 (KWP = 4) three
// blocks leave 85 registers, so the rebalancing-target kernel does not spill
// (at four blocks, 64 registers, it did, and its rounds took 9 % longer).
template <int KWP>
constexpr int kLightBlocks = KWP >= 8 ? 2 : (KWP == 4 ? 3 : 4);

template <int KWP>
struct Stage {
  static constexpr int kRow = 2 * KWP;                          // words of one mask row
  static constexpr int kBatch = KWP <= 2 ? 4 : 2;  // rows per lane per batch
  // per-warp stage: 2 buffers x kBatch x 32 rows | the same for omega (weighted only)
  template <bool UNIT>
  static constexpr int bytes() {
    return 2 * kBatch * 32 * (kRow + (UNIT ? 0 : 1)) * 4;
  }
};

__device__ __forceinline__ void cp_async_16(uint32_t *dst, const uint32_t *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t *dst, const uint32_t *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(int32_t *dst, const int32_t *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every committed group but the most recent one has completed
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int KWP>
__device__ __forceinline__ void smem_row(const uint32_t *r, uint32_t (&M)[KWP]) {
  if constexpr (KWP == 1) {
    M[0] = r[0];
  } else if constexpr (KWP == 2) {
    const uint2 x = *reinterpret_cast<const uint2 *>(r);
    M[0] = x.x; M[1] = x.y;
  } else {
#pragma unroll
    for (int h = 0; h < KWP / 4; ++h) {
      const uint4 x = reinterpret_cast<const uint4 *>(r)[h];
      M[4 * h] = x.x; M[4 * h + 1] = x.y; M[4 * h + 2] = x.z; M[4 * h + 3] = x.w;
    }
  }
}

// conn(v, .) bit planes, the union of Lambda(e) and A(v) over I(v) for this
// lane's vertex: deg incidences starting at inc[j0] (deg = 0 on a lane with
// no vertex to evaluate; s is read only when deg > 0).  UNIT: every omega(e)
// is 1 (no weight gathers).
template <int KWP, int NP, bool UNIT>
__device__ __forceinline__ int32_t stage_accumulate(const CandArgs &a, uint8_t *stage, int64_t j0, int deg, int s,
                                                    uint32_t (&pl)[NP][KWP], uint32_t (&any)[KWP]) {
  using S = Stage<KWP>;
  constexpr int R = S::kBatch;
  const int lane = threadIdx.x & 31;
  uint32_t *rows = reinterpret_cast<uint32_t *>(stage);
  int32_t *wts = reinterpret_cast<int32_t *>(rows + 2 * R * 32 * S::kRow);
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    any[q] = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) pl[p][q] = 0;
  }
  int32_t A = 0;
  if (a.adj) {  // graph path: e = {v, u} gives Lambda(e) = {s, Pi(u)}; four neighbours in flight
    for (int j = 0; j < deg; j += 4) {
      int pu[4], w[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) pu[t] = j + t < deg ? a.adj[j0 + j + t] : -1;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        w[t] = UNIT || pu[t] < 0 ? 1 : a.ewgt[a.inc[j0 + j + t]];
        pu[t] = pu[t] >= 0 ? a.part[pu[t]] : -1;
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (pu[t] < 0) continue;
        uint32_t M[KWP];
#pragma unroll
        for (int qq = 0; qq < KWP; ++qq)
          M[qq] = ((s >> 5) == qq ? 1u << (s & 31) : 0u) | ((pu[t] >> 5) == qq ? 1u << (pu[t] & 31) : 0u);
        if (pu[t] == s) A += w[t];
#pragma unroll
        for (int qq = 0; qq < KWP; ++qq) any[qq] |= M[qq];
        if (UNIT) add_one<KWP, NP>(pl, M);
        else add_weighted<KWP, NP>(pl, M, (uint32_t)w[t]);
      }
    }
    return A;
  }
  const int nb = (deg + R - 1) / R;
  int e[R];
  auto load_inc = [&](int b) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int j = b * R + t;
      e[t] = j < deg ? a.inc[j0 + j] : -1;
    }
  };
  auto issue_rows = [&](int b) {
    const int q = b & 1;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (e[t] >= 0) {
        const int slot = (q * R + t) * 32 + lane;
        const uint32_t *src = a.mask + (int64_t)e[t] * S::kRow;
        uint32_t *dst = rows + slot * S::kRow;
        if constexpr (KWP == 1) {
          cp_async_8(dst, src);
        } else {
#pragma unroll
          for (int h = 0; h < S::kRow / 4; ++h) cp_async_16(dst + 4 * h, src + 4 * h);
        }
        if constexpr (!UNIT) cp_async_4(wts + slot, a.ewgt + e[t]);
      }
    }
    cp_async_commit();
  };
  if (nb > 0) {
    load_inc(0);
    issue_rows(0);
    if (nb > 1) load_inc(1);
  }
  for (int b = 0; b < nb; ++b) {
    if (b + 1 < nb) {
      issue_rows(b + 1);
      if (b + 2 < nb) load_inc(b + 2);
      cp_async_wait_prior();  // batch b has landed, batch b+1 may be in flight
    } else {
      cp_async_wait_all();
    }
    const int q = b & 1;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (b * R + t < deg) {
        const int slot = (q * R + t) * 32 + lane;
        const uint32_t *r = rows + slot * S::kRow;
        uint32_t M[KWP];
        smem_row<KWP>(r, M);
        const int w = UNIT ? 1 : wts[slot];
        if ((r[KWP + (s >> 5)] >> (s & 31)) & 1u) A += w;  // phi_e[s] >= 2
#pragma unroll
        for (int qq = 0; qq < KWP; ++qq) any[qq] |= M[qq];
        if (UNIT) add_one<KWP, NP>(pl, M);
        else add_weighted<KWP, NP>(pl, M, (uint32_t)w);
      }
    }
  }
  return A;
}

// Light vertices are scanned in groups of 32 consecutive ids per warp.  The
// ones to evaluate (unlocked for move candidates; in an overloaded block with
// an eligible target for rebalancing) are appended to a per-warp queue, and
// the warp evaluates them 32 at a time, so lanes are not left idle by the
// vertices a pass skips (locked ones, or blocks that are not overloaded).
// Heavy vertices are skipped here and handled by the warp-per-vertex kernels.
struct WarpQueue {
  static constexpr int kCap = 64;
  int v[kCap], s[kCap], c[kCap], deg[kCap];
  long long j0[kCap];
};

// Raw inputs of a scan group, loaded one group ahead so that their latency
// overlaps the previous group's work (first used in the next iteration).
struct GroupRaw {
  int s, hv, lk;
};

__device__ __forceinline__ GroupRaw fetch_group(const CandArgs &a, int64_t v, bool want_lock) {
  GroupRaw r{0, 1, 1};
  if (v < a.n) {
    r.s = a.part[v];
    r.hv = a.vheavy[v];
    r.lk = want_lock ? a.locked[v] : 0;
  }
  return r;
}

// Appends this lane's vertex (if `act`) to the warp queue; returns the new
// (warp-uniform) queue length.
__device__ __forceinline__ int enqueue(WarpQueue *q, int qn, bool act, int v, int s, int c, int64_t j0, int deg) {
  const int lane = threadIdx.x & 31;
  const unsigned bal = __ballot_sync(kFull, act);
  if (act) {
    const int pos = qn + __popc(bal & ((1u << lane) - 1));
    q->v[pos] = v;
    q->s[pos] = s;
    q->c[pos] = c;
    q->deg[pos] = deg;
    q->j0[pos] = j0;
  }
  __syncwarp();
  return qn + __popc(bal);
}

// Removes the first 32 entries of the queue (qn >= 32).
__device__ __forceinline__ int dequeue32(WarpQueue *q, int qn) {
  const int lane = threadIdx.x & 31;
  const int rest = qn - 32;
  int v = 0, s = 0, c = 0, deg = 0;
  long long j0 = 0;
  if (lane < rest) {
    v = q->v[32 + lane]; s = q->s[32 + lane]; c = q->c[32 + lane]; deg = q->deg[32 + lane]; j0 = q->j0[32 + lane];
  }
  __syncwarp();
  if (lane < rest) {
    q->v[lane] = v; q->s[lane] = s; q->c[lane] = c; q->deg[lane] = deg; q->j0[lane] = j0;
  }
  __syncwarp();
  return rest;
}

// Evaluates queue entries 0..cnt-1 (lane l takes entry l) for move candidates.
template <int KWP, bool UNIT>
__device__ __forceinline__ void cand_batch(const CandArgs &a, uint8_t *stage, const WarpQueue *q, int cnt) {
  constexpr int NP = kLightPlanes;
  const int lane = threadIdx.x & 31;
  const bool mine = lane < cnt;
  const int v = mine ? q->v[lane] : 0, s = mine ? q->s[lane] : 0, deg = mine ? q->deg[lane] : 0;
  const int64_t j0 = mine ? q->j0[lane] : 0;
  uint32_t pl[NP][KWP], any[KWP];
  const int32_t A = stage_accumulate<KWP, NP, UNIT>(a, stage, j0, deg, s, pl, any);
  if (!mine) return;
  uint64_t rec = 0;
  uint32_t C[KWP];
  uint32_t nz = 0;
#pragma unroll
  for (int qq = 0; qq < KWP; ++qq) {
    C[qq] = any[qq] & ~((s >> 5) == qq ? (1u << (s & 31)) : 0u);
    nz |= C[qq];
  }
  if (nz) {
    int32_t conn;
    const int t = argmax_planes<KWP, NP>(pl, C, conn);
    const int32_t g = conn - A;
    if ((long long)a.tau_den * g >= -(long long)a.tau_num * A) rec = pack_cand(g, s, t);
  }
  a.cand[v] = rec;
}

template <int KWP, bool UNIT>
__global__ void __launch_bounds__(256, kLightBlocks<KWP>) k_cand_light(CandArgs a) {
  extern __shared__ __align__(16) uint8_t dyn_smem[];
  __shared__ WarpQueue s_q[8];
  const int w = threadIdx.x >> 5;
  uint8_t *stage = dyn_smem + w * Stage<KWP>::template bytes<UNIT>();
  WarpQueue *q = &s_q[w];
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * warps * 32;
  int64_t base = ((int64_t)blockIdx.x * warps + w) * 32;
  GroupRaw cur = fetch_group(a, base + lane, true);
  int qn = 0;
  for (; base < a.n; base += stride) {
    const GroupRaw nxt = fetch_group(a, base + stride + lane, true);
    const int64_t v = base + lane;
    bool act = false;
    int64_t j0 = 0;
    int deg = 0;
    if (v < a.n && !cur.hv) {
      if ((unsigned)cur.s >= (unsigned)a.k) {  // invalid block id: report, never index with it
        atomicOr(&a.cnt->err, kErrPartRange);
        a.cand[v] = 0;
      } else if (cur.lk) {
        a.cand[v] = 0;
      } else {
        act = true;
        j0 = a.vptr[v];
        deg = (int)(a.vptr[v + 1] - j0);
      }
    }
    qn = enqueue(q, qn, act, (int)v, cur.s, 0, j0, deg);
    if (qn >= 32) {
      cand_batch<KWP, UNIT>(a, stage, q, 32);
      qn = dequeue32(q, qn);
    }
    cur = nxt;
  }
  if (qn > 0) cand_batch<KWP, UNIT>(a, stage, q, qn);
}

// Evaluates queue entries 0..cnt-1 for rebalancing and appends their records.
template <int KWP, bool UNIT, int kTab>
__device__ __forceinline__ void rb_batch(const CandArgs &a, uint8_t *stage, const WarpQueue *q, int cnt,
                                         const long long *s_cap, const uint32_t (*s_elig)[KWP]) {
  constexpr int NP = kLightPlanes;
  const int lane = threadIdx.x & 31;
  const bool mine = lane < cnt;
  const int v = mine ? q->v[lane] : 0, s = mine ? q->s[lane] : 0, deg = mine ? q->deg[lane] : 0;
  const int32_t c = mine ? q->c[lane] : 0;
  const int64_t j0 = mine ? q->j0[lane] : 0;
  uint32_t pl[NP][KWP], any[KWP];
  const int32_t A = stage_accumulate<KWP, NP, UNIT>(a, stage, j0, deg, s, pl, any);
  uint64_t hi = 0;
  int32_t ct = 0;
  if (mine) {
    uint32_t C[KWP];
    if (c <= kTab) {
#pragma unroll
      for (int qq = 0; qq < KWP; ++qq) C[qq] = s_elig[c - 1][qq];
    } else {
      eligible_words<KWP>(s_cap, a.k, c, C);
    }
    int32_t conn;
    const int t = argmax_planes<KWP, NP>(pl, C, conn);
    hi = rb_hi_of(a, conn - A, c);
    ct = (c << 16) | (s << 8) | t;
  }
  rb_first_level(a, mine, s, hi, v, c);
  const unsigned bal = __ballot_sync(kFull, mine);
  unsigned long long pos0 = 0;
  if (lane == 0) pos0 = atomicAdd(&a.cnt->n_rec, (unsigned long long)__popc(bal));
  pos0 = __shfl_sync(kFull, pos0, 0);
  if (mine) {
    const unsigned long long pos = pos0 + lane;
    a.rb_hi[pos] = hi;
    a.rb_v[pos] = v;
    a.rb_ct[pos] = ct;
  }
}

template <int KWP, bool UNIT>
__global__ void __launch_bounds__(256, kLightBlocks<KWP>) k_rbcand_light(CandArgs a) {
  constexpr int kTab = 32;  // eligibility words tabulated for c(v) <= 32
  __shared__ long long s_cap[kMaxK], s_bw[kMaxK];
  __shared__ int s_over[kMaxK];
  __shared__ uint32_t s_elig[kTab][KWP];
  __shared__ WarpQueue s_q[8];
  extern __shared__ __align__(16) uint8_t dyn_smem[];
  const int w = threadIdx.x >> 5;
  uint8_t *stage = dyn_smem + w * Stage<KWP>::template bytes<UNIT>();
  WarpQueue *q = &s_q[w];
  for (int b = threadIdx.x; b < a.k; b += blockDim.x) {
    s_cap[b] = a.rbb[b].cap;
    s_bw[b] = a.rbb[b].bw;
    s_over[b] = a.rbb[b].over;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < kTab * KWP; x += blockDim.x) {
    const int c = x / KWP + 1, qq = x % KWP;
    uint32_t wd = 0;
    for (int bit = 0; bit < 32; ++bit) {
      const int b = qq * 32 + bit;
      if (b < a.k && s_cap[b] >= c) wd |= 1u << bit;
    }
    s_elig[c - 1][qq] = wd;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * warps * 32;
  int64_t base = ((int64_t)blockIdx.x * warps + w) * 32;
  GroupRaw cur = fetch_group(a, base + lane, false);
  int qn = 0;
  unsigned long long w_over = 0, w_eval = 0, w_pins = 0;
  for (; base < a.n; base += stride) {
    const GroupRaw nxt = fetch_group(a, base + stride + lane, false);
    const int64_t v = base + lane;
    const int s = cur.s;
    bool act = false;
    int32_t c = 0;
    int64_t j0 = 0;
    int deg = 0;
    if (v < a.n && !cur.hv && (unsigned)s < (unsigned)a.k && s_over[s]) {
      ++w_over;
      c = a.vwgt[v];
      if (2ll * c <= 3ll * (s_bw[s] - a.A)) {  // heavy vertices (Section 4.3) are never moved
        uint32_t nz = 0;
        if (c <= kTab) {
#pragma unroll
          for (int qq = 0; qq < KWP; ++qq) nz |= s_elig[c - 1][qq];
        } else {
          uint32_t C[KWP];
          eligible_words<KWP>(s_cap, a.k, c, C);
#pragma unroll
          for (int qq = 0; qq < KWP; ++qq) nz |= C[qq];
        }
        if (nz) {
          act = true;
          j0 = a.vptr[v];
          deg = (int)(a.vptr[v + 1] - j0);
          ++w_eval;
          w_pins += deg;
        }
      }
    }
    qn = enqueue(q, qn, act, (int)v, s, c, j0, deg);
    if (qn >= 32) {
      rb_batch<KWP, UNIT, kTab>(a, stage, q, 32, s_cap, s_elig);
      qn = dequeue32(q, qn);
    }
    cur = nxt;
  }
  if (qn > 0) rb_batch<KWP, UNIT, kTab>(a, stage, q, qn, s_cap, s_elig);
  count_work(a.cnt, w_over, w_eval, w_pins);
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
  unsigned long long w_over = 0, w_eval = 0, w_pins = 0;
  for (int i = gw; i < a.nlist; i += nw) {
    const int v = a.vlist[i];
    const int s = a.part[v];
    const int32_t c = a.vwgt[v];
    bool any_elig = false;
    if (lane == 0 && (unsigned)s < (unsigned)a.k && s_over[s]) ++w_over;
    if ((unsigned)s < (unsigned)a.k && s_over[s] && 2ll * c <= 3ll * (s_bw[s] - a.A)) {
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        const int b = q * 32 + lane;
        any_elig |= b < a.k && s_cap[b] >= c;
      }
    }
    if (!__any_sync(kFull, any_elig)) continue;  // no record (warp-uniform: one vertex per warp)
    if (lane == 0) {
      ++w_eval;
      w_pins += (unsigned long long)(a.vptr[v + 1] - a.vptr[v]);
    }
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
    const uint64_t hi = rb_hi_of(a, bc - A, c);
    rb_first_level(a, lane == 0, s, hi, v, c);
    if (lane == 0) {
      const unsigned long long pos = atomicAdd(&a.cnt->n_rec, 1ull);
      a.rb_hi[pos] = hi;
      a.rb_v[pos] = v;
      a.rb_ct[pos] = (c << 16) | (s << 8) | bb;
    }
  }
  count_work(a.cnt, w_over, w_eval, w_pins);
}

template <int KWP>
cudaError_t launch_cand_kwp(jet_ctx *c, const CandArgs &base) {
  CandArgs a = base;
  if (c->n_light > 0) {
    a.vlist = c->v_light;
    a.nlist = c->n_light;
    const int g = grid_for(c->n, 256, c->launch_sms, c->stage_bps[0]);
    if (c->unit_ewgt) k_cand_light<KWP, true><<<g, 256, 8 * Stage<KWP>::template bytes<true>(), c->stream>>>(a);
    else k_cand_light<KWP, false><<<g, 256, 8 * Stage<KWP>::template bytes<false>(), c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_heavy > 0) {
    a.vlist = c->v_heavy;
    a.nlist = c->n_heavy;
    k_cand_heavy<KWP><<<grid_for((int64_t)c->n_heavy * 32, 256, c->launch_sms, c->heavy_bps[0]), 256, 0,
                            c->stream>>>(a);
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
    const int g = grid_for(c->n, 256, c->launch_sms, c->stage_bps[1]);
    if (c->unit_ewgt) k_rbcand_light<KWP, true><<<g, 256, 8 * Stage<KWP>::template bytes<true>(), c->stream>>>(a);
    else k_rbcand_light<KWP, false><<<g, 256, 8 * Stage<KWP>::template bytes<false>(), c->stream>>>(a);
    ++c->kernel_launches;
  }
  if (c->n_heavy > 0) {
    a.vlist = c->v_heavy;
    a.nlist = c->n_heavy;
    k_rbcand_heavy<KWP><<<grid_for((int64_t)c->n_heavy * 32, 256, c->launch_sms, c->heavy_bps[1]), 256, 0,
                              c->stream>>>(a);
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
  a.vheavy = c->vheavy;
  a.part = part;
  a.phi = phi;
  a.mask = c->mask;
  a.adj = c->graph_path ? c->adj : nullptr;
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
  a.rb_hist = c->rb_hist;
  a.rb_vbits = c->rb_vbits;
  a.rb_tbits = c->rb_hbits + c->rb_vbits;
  a.rb_digit = c->rb_digit;
  return a;
}

// Dynamic shared memory limits and resident blocks per SM of the staged light
// kernels this context launches (grids are sized to one resident wave).
template <int KWP, bool UNIT>
cudaError_t prepare_stage(jet_ctx *c) {
  const int bytes = 8 * Stage<KWP>::template bytes<UNIT>();
  cudaError_t e = cudaFuncSetAttribute(k_cand_light<KWP, UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rbcand_light<KWP, UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->stage_bps[0], k_cand_light<KWP, UNIT>, 256, bytes);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->stage_bps[1], k_rbcand_light<KWP, UNIT>, 256, bytes);
  for (int i = 0; i < 2; ++i)
    if (c->stage_bps[i] < 1) c->stage_bps[i] = 1;
  if (e == cudaSuccess) e = resident_blocks(k_cand_heavy<KWP>, 256, 0, &c->heavy_bps[0]);
  if (e == cudaSuccess) e = resident_blocks(k_rbcand_heavy<KWP>, 256, 0, &c->heavy_bps[1]);
  return e;
}

template <int KWP>
cudaError_t prepare_stage_kwp(jet_ctx *c) {
  return c->unit_ewgt ? prepare_stage<KWP, true>(c) : prepare_stage<KWP, false>(c);
}

}  // namespace

cudaError_t prepare_candidate_kernels(jet_ctx *c) {
  switch (c->kwp) {
    case 1: return prepare_stage_kwp<1>(c);
    case 2: return prepare_stage_kwp<2>(c);
    case 4: return prepare_stage_kwp<4>(c);
    default: return prepare_stage_kwp<8>(c);
  }
}

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
