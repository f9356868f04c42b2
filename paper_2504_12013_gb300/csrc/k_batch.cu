// Batched form as ONE persistent kernel: many independent instances refined
// to convergence (Algorithm 1 with the temperature schedule of Section 7.2).
//
// A team of `ctas` thread blocks (a thread-block cluster; one block when
// ctas = 1) takes the next instance from a device work queue (largest first)
// and runs all of Algorithm 1 on it: pin counts, every Jet iteration
// (candidates of Section 4.1, the afterburner of Algorithm 2, ApplyMoves and
// the rebalancing rounds of Section 4.3), the objective, the improvement
// counter, the snapshot of the best balanced partition and the rollback.
// The phases of one instance are separated by the team's barrier (the
// cluster barrier, in hardware: nothing spins), so every instance advances at
// its own pace and no barrier spans the grid.  The arithmetic is the integer,
// order-independent arithmetic of the per-instance kernels (bit planes for
// gains, the closed form of Algorithm 2, exact priority keys, +-1 atomics on
// phi with XOR-maintained bitmasks), so every instance ends bit-identical to
// jet_refine on it alone.
//
// Memory written by one block of a team and read by another is read with
// ld.global.cg (L2, not the non-coherent L1), ordered by the release/acquire
// cluster barrier.  The state of an instance lives in its context's
// workspace and the caller's part/phi/block_w arrays; the kernel allocates
// nothing.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <new>
#include <vector>

#include "jet_gain.cuh"
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTeamMaxThreads = 1024;

// Per-instance counters of the team kernel (device, one per instance).
struct TeamCount {
  unsigned long long n_moves;  // entries of the move list (Jet moves, a round's selection, rollback)
  unsigned long long n_rec;    // rebalancing records of the current round
  unsigned long long n_cand;   // |M| of the current iteration
  unsigned long long moved;    // rebalancing moves of the current round
  long long obj;               // (lambda-1) accumulator
  int err;                     // a partition value outside [0, k) (the instance is not refined)
  int pad[5];
};

// One instance as the team kernel sees it.
struct TeamInst {
  int32_t n, m, k, unit_ewgt;
  int64_t P;
  const int64_t *eptr, *vptr;
  const int32_t *pins, *inc, *vwgt, *ewgt;
  long long A, Lmax, dz_min;
  int32_t max_rounds;
  int rb_compact, rb_vbits, rb_tbits;
  long long rb_L, rb_Pmax;
  const int32_t *v_light, *v_heavy;
  int32_t n_light, n_heavy;
  const int32_t *e_tiny, *e_rest;  // edges of <= 8 pins; the others (e_rest = e_tiny + n_tiny)
  int32_t n_tiny, n_rest;
  int32_t *part, *phi;
  int64_t *bw;
  uint32_t *mask;
  uint64_t *cand;
  int32_t *rg, *mv_v;
  uint32_t *mv_st;
  uint8_t *locked;
  int32_t *best;
  uint64_t *rb_hi;
  int32_t *rb_v, *rb_ct;
  unsigned long long *hist;  // k x 256 weighted digit histograms (the plan's; zero between uses)
  RbBlock *rbb;
  TeamCount *tc;
  jet_refine_result *res;  // device: the summary
};

struct TeamArgs {
  const TeamInst *inst;
  const int32_t *order;  // instances, largest first
  int32_t count;
  unsigned *queue;        // next index into order (zeroed before the launch)
  int32_t *team_inst;     // per team: the instance it is working on (broadcast slot)
  const int32_t *tau;     // schedule pairs
  int32_t n_tau, limit;
  int32_t iter_cap;       // > 0: stop each instance after this many iterations (autotuner trials)
  long long split_pins;   // multi-block teams: instances with fewer pins run on single blocks of the cluster
};

struct Team {
  unsigned rank, size;  // block rank within the team, blocks per team
  long long tid, nthr;  // thread index within the team, threads per team
  long long wid, nwarps;
  int lane;
};

// Loads of state that another block of the team may have written: L2 (cg) for
// multi-block teams; ordinary loads when the team is one block (one L1).
template <bool MULTI, class T>
__device__ __forceinline__ T ldm(const T *p) {
  if constexpr (MULTI) return __ldcg(p);
  else return *p;
}

// The team barrier.  For a cluster, arrive has release and wait has acquire semantics at cluster scope, which
// orders every thread's earlier global and shared writes before the other blocks' later reads.
template <bool MULTI>
__device__ __forceinline__ void team_sync() {
  if constexpr (MULTI) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ bool leader(const Team &tm) { return tm.tid == 0; }

// Sum of a per-thread value over the block, added to *dst by one atomic per block.
__device__ __forceinline__ void block_add(long long x, long long *dst, long long *s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_red[i];
    if (t) atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)t);
  }
  __syncthreads();
}

template <bool MULTI, int KWP>
__device__ __forceinline__ void load_rows_m(const uint32_t *row, uint32_t (&M)[KWP], uint32_t (&M2)[KWP]) {
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    M[q] = ldm<MULTI>(row + q);
    M2[q] = ldm<MULTI>(row + KWP + q);
  }
}

// Adds the block's shared-memory block-weight deltas to c(V_i) and clears them (every thread of the block).
__device__ __forceinline__ void flush_bw(const TeamInst &I, long long *s_dw) {
  __syncthreads();
  for (int b = threadIdx.x; b < I.k; b += blockDim.x) {
    if (s_dw[b]) atomicAdd(reinterpret_cast<unsigned long long *>(&I.bw[b]), (unsigned long long)s_dw[b]);
    s_dw[b] = 0;
  }
  __syncthreads();
}

// ------------------------------------------------------------ pin counts, objective
// phi and block weights from part (Section 2), then both bitmasks per edge.
template <bool MULTI, int KWP>
__device__ void team_pincounts(const TeamInst &I, const Team &tm, long long *s_dw) {
  for (long long i = tm.tid; i < (long long)I.m * I.k; i += tm.nthr) I.phi[i] = 0;
  for (int b = threadIdx.x; b < I.k; b += blockDim.x) s_dw[b] = 0;
  if (leader(tm))
    for (int b = 0; b < I.k; ++b) I.bw[b] = 0;
  team_sync<MULTI>();
  for (long long v = tm.tid; v < I.n; v += tm.nthr) {
    const int s = ldm<MULTI>(I.part + v);
    if ((unsigned)s >= (unsigned)I.k) {  // never index with it: report, and the instance is not refined
      atomicOr(&I.tc->err, kErrPartRange);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)I.vwgt[v]);
    for (int64_t j = I.vptr[v]; j < I.vptr[v + 1]; ++j) atomicAdd(&I.phi[(int64_t)I.inc[j] * I.k + s], 1);
  }
  flush_bw(I, s_dw);
  team_sync<MULTI>();
  for (long long e = tm.tid; e < I.m; e += tm.nthr) {
    const int32_t *row = I.phi + e * I.k;
    uint32_t *mrow = I.mask + e * 2 * KWP;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      uint32_t one = 0, two = 0;
      for (int bit = 0; bit < 32; ++bit) {
        const int b = 32 * q + bit;
        if (b >= I.k) break;
        const int x = ldm<MULTI>(row + b);
        one |= (x >= 1 ? 1u : 0u) << bit;
        two |= (x >= 2 ? 1u : 0u) << bit;
      }
      mrow[q] = one;
      mrow[KWP + q] = two;
    }
  }
  team_sync<MULTI>();
}

// (lambda-1) = sum over edges of omega(e) * (|Lambda(e)| - 1) (empty edges: 0), and max_i c(V_i).
template <bool MULTI, int KWP>
__device__ void team_objective(const TeamInst &I, const Team &tm, long long *s_red, long long &obj, long long &maxbw) {
  if (leader(tm)) I.tc->obj = 0;
  team_sync<MULTI>();
  long long part = 0;
  for (long long base = (long long)tm.rank * blockDim.x; base < I.m; base += tm.nthr) {
    const long long e = base + threadIdx.x;
    if (e < I.m) {
      int lam = 0;
#pragma unroll
      for (int q = 0; q < KWP; ++q) lam += __popc(ldm<MULTI>(I.mask + e * 2 * KWP + q));
      if (lam > 1) part += (long long)(lam - 1) * (I.unit_ewgt ? 1 : I.ewgt[e]);
    }
  }
  block_add(part, &I.tc->obj, s_red);
  team_sync<MULTI>();
  obj = ldm<MULTI>(&I.tc->obj);
  maxbw = 0;
  for (int b = 0; b < I.k; ++b) {
    const long long w = ldm<MULTI>(I.bw + b);
    maxbw = w > maxbw ? w : maxbw;
  }
}

// ------------------------------------------------------------ gains (Section 4.1, 4.3)
// Bit planes of conn(v, .) over I(v), the union of Lambda(e), and A(v) for a light vertex in block s.  The
// incidences go four at a time: their edge ids, then their bitmask rows and weights, are loaded together.
template <bool MULTI, int KWP>
__device__ __forceinline__ int32_t light_planes(const TeamInst &I, int v, int s, uint32_t (&pl)[kLightPlanes][KWP],
                                                uint32_t (&any)[KWP]) {
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    any[q] = 0;
#pragma unroll
    for (int p = 0; p < kLightPlanes; ++p) pl[p][q] = 0;
  }
  int32_t A = 0;
  const int64_t j0 = I.vptr[v], j1 = I.vptr[v + 1];
  for (int64_t jb = j0; jb < j1; jb += 4) {
    int e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = jb + u < j1 ? I.inc[jb + u] : -1;
    uint32_t M[4][KWP], M2[4][KWP];
    int w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e[u] >= 0) {
        load_rows_m<MULTI, KWP>(I.mask + (int64_t)e[u] * 2 * KWP, M[u], M2[u]);
        w[u] = I.unit_ewgt ? 1 : I.ewgt[e[u]];
      } else {
#pragma unroll
        for (int q = 0; q < KWP; ++q) M[u][q] = M2[u][q] = 0u;
        w[u] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (e[u] < 0) continue;
      if (mask_bit<KWP>(M2[u], s)) A += w[u];  // phi_e[s] >= 2
#pragma unroll
      for (int q = 0; q < KWP; ++q) any[q] |= M[u][q];
      if (I.unit_ewgt) add_one<KWP, kLightPlanes>(pl, M[u]);
      else add_weighted<KWP, kLightPlanes>(pl, M[u], (uint32_t)w[u]);
    }
  }
  return A;
}

// conn(v, b) exact for the lane's blocks b = lane + 32q (one warp per heavy vertex), their adjacency bits, A(v).
template <bool MULTI, int KWP>
__device__ __forceinline__ int32_t heavy_conn(const TeamInst &I, int v, int s, int32_t (&conn)[KWP], uint32_t &adj) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < KWP; ++q) conn[q] = 0;
  adj = 0;
  int32_t Ap = 0;
  const int64_t j0 = I.vptr[v], j1 = I.vptr[v + 1];
  for (int64_t base = j0; base < j1; base += 32) {
    const int64_t j = base + lane;
    int w = 0;
    uint32_t M[KWP], M2[KWP];
#pragma unroll
    for (int q = 0; q < KWP; ++q) M[q] = M2[q] = 0;
    if (j < j1) {
      const int e = I.inc[j];
      w = I.unit_ewgt ? 1 : I.ewgt[e];
      load_rows_m<MULTI, KWP>(I.mask + (int64_t)e * 2 * KWP, M, M2);
      if (mask_bit<KWP>(M2, s)) Ap += w;
    }
    const int cnt = (int)((j1 - base) < 32 ? (j1 - base) : 32);
    for (int l = 0; l < cnt; ++l) {
      const int wl = __shfl_sync(kFull, w, l);
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        const uint32_t Mq = __shfl_sync(kFull, M[q], l);
        if ((Mq >> lane) & 1u) {
          conn[q] += wl;
          adj |= 1u << q;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Ap += __shfl_xor_sync(kFull, Ap, o);
  return Ap;
}

// ------------------------------------------------------------ one Jet iteration
// Move candidates (Section 4.1): cand[v] for every vertex (0 = not in M).
template <bool MULTI, int KWP>
__device__ void team_candidates(const TeamInst &I, const Team &tm, int32_t tn, int32_t td, long long *s_red) {
  long long cnt = 0;
  // the next vertex's id, lock and block are loaded while the current one is evaluated
  int nv = tm.tid < I.n_light ? I.v_light[tm.tid] : -1;
  int nlk = nv >= 0 ? ldm<MULTI>(I.locked + nv) : 1, ns = nv >= 0 ? ldm<MULTI>(I.part + nv) : 0;
  for (long long i = tm.tid; i < I.n_light; i += tm.nthr) {
    const int v = nv, lk = nlk, sv = ns;
    nv = i + tm.nthr < I.n_light ? I.v_light[i + tm.nthr] : -1;
    nlk = nv >= 0 ? ldm<MULTI>(I.locked + nv) : 1;
    ns = nv >= 0 ? ldm<MULTI>(I.part + nv) : 0;
    uint64_t rec = 0;
    if (!lk) {
      const int s = sv;
      uint32_t pl[kLightPlanes][KWP], any[KWP];
      const int32_t A = light_planes<MULTI, KWP>(I, v, s, pl, any);
      uint32_t C[KWP], nz = 0;
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        C[q] = any[q] & ~((s >> 5) == q ? (1u << (s & 31)) : 0u);
        nz |= C[q];
      }
      if (nz) {
        int32_t conn;
        const int t = argmax_planes<KWP, kLightPlanes>(pl, C, conn);
        const int32_t g = conn - A;
        if ((long long)td * g >= -(long long)tn * A) rec = pack_cand(g, s, t);
      }
    }
    I.cand[v] = rec;
    cnt += rec ? 1 : 0;
  }
  const int lane = threadIdx.x & 31;
  for (long long i = tm.wid; i < I.n_heavy; i += tm.nwarps) {
    const int v = I.v_heavy[i];
    uint64_t rec = 0;
    if (!ldm<MULTI>(I.locked + v)) {
      const int s = ldm<MULTI>(I.part + v);
      int32_t conn[KWP];
      uint32_t adj;
      const int32_t A = heavy_conn<MULTI, KWP>(I, v, s, conn, adj);
      int bb = -1;
      int32_t bc = 0;
#pragma unroll
      for (int q = 0; q < KWP; ++q) {
        const int b = 32 * q + lane;
        if (b < I.k && b != s && ((adj >> q) & 1u) && (bb < 0 || conn[q] > bc)) {
          bb = b;
          bc = conn[q];
        }
      }
      warp_argmax(bc, bb);
      if (bb >= 0) {
        const int32_t g = bc - A;
        if ((long long)td * g >= -(long long)tn * A) rec = pack_cand(g, s, bb);
      }
    }
    if (lane == 0) {
      I.cand[v] = rec;
      cnt += rec ? 1 : 0;
    }
  }
  block_add(cnt, reinterpret_cast<long long *>(&I.tc->n_cand), s_red);
}

// Afterburner (Algorithm 2) in closed form: per (e, b) only the last departure
// from b can earn +omega(e) and only the first arrival into b can pay
// -omega(e), both only when no non-candidate pin of e lies in b and every
// departure from b precedes every arrival into b (in the order gain desc, id
// asc, i.e. ascending candidate key).  Edges of <= 8 pins: one thread,
// pairwise tests; larger edges: one warp with per-block max/min tables in
// shared memory (only the entries of blocks the candidates touch are used).
template <bool MULTI, int KWP>
__device__ void team_afterburner(const TeamInst &I, const Team &tm, unsigned long long *s_tab) {
  // software pipeline over the thread's edges: while edge i is decided, the pins of edge i+1, the offsets
  // of edge i+2 and the id of edge i+3 are in flight
  auto edge_at = [&](long long i) -> int { return i < I.n_tiny ? I.e_tiny[i] : -1; };
  const long long st0 = tm.tid, stride = tm.nthr;
  int e3 = edge_at(st0 + 2 * stride);
  int e2 = edge_at(st0 + stride);
  int64_t p2 = e2 >= 0 ? I.eptr[e2] : 0;
  int sz2 = e2 >= 0 ? (int)(I.eptr[e2 + 1] - p2) : 0;
  int e1 = edge_at(st0), sz1 = 0;
  int pins1[kTinyEdge];
  {
    const int64_t p1 = e1 >= 0 ? I.eptr[e1] : 0;
    sz1 = e1 >= 0 ? (int)(I.eptr[e1 + 1] - p1) : 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pins1[q] = q < sz1 ? I.pins[p1 + q] : 0;
  }
  for (long long i = st0; i < I.n_tiny; i += stride) {
    const int e = e1, sz = sz1;
    int pin[kTinyEdge];
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pin[q] = pins1[q];
    const int e4 = edge_at(i + 3 * stride);
    const int64_t p3 = e3 >= 0 ? I.eptr[e3] : 0;
    const int sz3 = e3 >= 0 ? (int)(I.eptr[e3 + 1] - p3) : 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) pins1[q] = q < sz2 ? I.pins[p2 + q] : 0;
    e1 = e2;
    sz1 = sz2;
    e2 = e3;
    p2 = p3;
    sz2 = sz3;
    e3 = e4;
    uint64_t key[kTinyEdge];
    uint32_t st[kTinyEdge];  // s | t << 8 | 1 << 16 for a candidate; block | 1 << 17 for another pin
    int nin = 0;
#pragma unroll
    for (int q = 0; q < kTinyEdge; ++q) {
      key[q] = 0;
      st[q] = 0;
      if (q < sz) {
        const int v = pin[q];
        const uint64_t r = ldm<MULTI>(I.cand + v);
        if (r) {
          ++nin;
          key[q] = cand_key(r, v);
          st[q] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 8) | 0x10000u;
        } else {
          st[q] = 0x20000u | (uint32_t)(ldm<MULTI>(I.part + v) & 255);
        }
      }
    }
    if (nin == 0) continue;
    const int w = I.unit_ewgt ? 1 : I.ewgt[e];
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
      if (delta) atomicAdd(&I.rg[(int)(K & 0xffffffffu)], delta);
    }
  }
  const int lane = threadIdx.x & 31;
  unsigned long long *maxd = s_tab + (size_t)(threadIdx.x >> 5) * (2 * I.k + (KWP + 1) / 2);
  unsigned long long *mina = maxd + I.k;
  uint32_t *nm = reinterpret_cast<uint32_t *>(mina + I.k);
  for (long long i = tm.wid; i < I.n_rest; i += tm.nwarps) {
    const int e = I.e_rest[i];
    const int64_t p0 = I.eptr[e], p1 = I.eptr[e + 1];
    bool any = false;
    for (int64_t p = p0 + lane; p < p1; p += 32) {  // reset the entries of the candidates' blocks
      const uint64_t r = ldm<MULTI>(I.cand + I.pins[p]);
      if (r) {
        any = true;
        maxd[cand_s(r)] = 0ull;
        mina[cand_s(r)] = ~0ull;
        maxd[cand_t(r)] = 0ull;
        mina[cand_t(r)] = ~0ull;
      }
    }
    if (!__any_sync(kFull, any)) continue;
    if (lane < KWP) nm[lane] = 0u;
    __syncwarp();
    for (int64_t p = p0 + lane; p < p1; p += 32) {  // departures, arrivals, blocks of non-candidate pins
      const int v = I.pins[p];
      const uint64_t r = ldm<MULTI>(I.cand + v);
      if (r) {
        const uint64_t K = cand_key(r, v);
        atomicMax(&maxd[cand_s(r)], (unsigned long long)K);
        atomicMin(&mina[cand_t(r)], (unsigned long long)K);
      } else {
        const int b = ldm<MULTI>(I.part + v);
        atomicOr(&nm[b >> 5], 1u << (b & 31));
      }
    }
    __syncwarp();
    const int wt = I.unit_ewgt ? 1 : I.ewgt[e];
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const int v = I.pins[p];
      const uint64_t r = ldm<MULTI>(I.cand + v);
      if (!r) continue;
      const int s = cand_s(r), t = cand_t(r);
      const uint64_t K = cand_key(r, v);
      int delta = 0;
      if (maxd[s] == K && !((nm[s >> 5] >> (s & 31)) & 1u) && (mina[s] == ~0ull || K < mina[s])) delta += wt;
      if (mina[t] == K && !((nm[t >> 5] >> (t & 31)) & 1u) && maxd[t] < K) delta -= wt;
      if (delta) atomicAdd(&I.rg[v], delta);
    }
    __syncwarp();
  }
}

// Approval (recomputed gain > 0), locks, and the move list; clears rg.  The loop is uniform over the block.
template <bool MULTI>
__device__ void team_approve(const TeamInst &I, const Team &tm, unsigned *s_wc, unsigned long long *s_base) {
  for (long long base = (long long)tm.rank * blockDim.x; base < I.n; base += tm.nthr) {
    const long long v = base + threadIdx.x;
    bool ok = false;
    uint64_t r = 0;
    if (v < I.n) {
      r = ldm<MULTI>(I.cand + v);
      const int32_t g = ldm<MULTI>(I.rg + v);
      if (g) I.rg[v] = 0;
      ok = r != 0 && g > 0;
      I.locked[v] = ok ? 1 : 0;
    }
    const unsigned long long pos = block_append(ok, &I.tc->n_moves, s_wc, s_base);
    if (ok) {
      I.mv_v[pos] = (int32_t)v;
      I.mv_st[pos] = (uint32_t)cand_s(r) | ((uint32_t)cand_t(r) << 16);
    }
  }
}

// One move v: s -> t: Pi(v), the block-weight deltas (shared memory), phi_e[s]--, phi_e[t]++ for e in I(v) with
// the bitmask toggles at the crossings (the atomic updates of one entry are serialized, so its 0 <-> 1 and
// 1 <-> 2 crossings alternate; each thread whose own update crosses toggles the bit, XOR commutes).
template <int KWP>
__device__ __forceinline__ void move_vertex(const TeamInst &I, int v, int s, int t, int32_t c, long long *s_dw) {
  I.part[v] = t;
  atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[s]), (unsigned long long)(-(long long)c));
  atomicAdd(reinterpret_cast<unsigned long long *>(&s_dw[t]), (unsigned long long)c);
  const uint32_t sbit = 1u << (s & 31), tbit = 1u << (t & 31);
  const int64_t j1 = I.vptr[v + 1];
  for (int64_t j = I.vptr[v]; j < j1; ++j) {
    const int64_t e = I.inc[j];
    const int os = atomicSub(&I.phi[e * I.k + s], 1);
    const int ot = atomicAdd(&I.phi[e * I.k + t], 1);
    uint32_t *row = I.mask + e * 2 * KWP;
    if (os == 1) atomicXor(&row[s >> 5], sbit);
    if (os == 2) atomicXor(&row[KWP + (s >> 5)], sbit);
    if (ot == 0) atomicXor(&row[t >> 5], tbit);
    if (ot == 1) atomicXor(&row[KWP + (t >> 5)], tbit);
  }
}

// ApplyMoves of the move list (nm entries).
template <bool MULTI, int KWP>
__device__ void team_apply_list(const TeamInst &I, const Team &tm, long long nm, long long *s_dw) {
  for (long long i = tm.tid; i < nm; i += tm.nthr) {
    const int v = ldm<MULTI>(I.mv_v + i);
    const uint32_t st = ldm<MULTI>(I.mv_st + i);
    move_vertex<KWP>(I, v, st & 0xffff, st >> 16, I.vwgt[v], s_dw);
  }
  flush_bw(I, s_dw);
}

// ------------------------------------------------------------ rebalancing (Section 4.3)
typedef unsigned __int128 u128;

// Per-block state of a round in shared memory, from c(V_i) at its start: overloaded, cap (the largest c(v)
// that may enter: L_max - c(V_b) outside the deadzone and below L_max, else -1), excess.  Returns whether a
// block is overloaded (the same answer in every thread of the team).
template <bool MULTI>
__device__ bool round_state(const TeamInst &I, long long *s_cap, long long *s_bw, int *s_over) {
  bool any = false;
  for (int b = 0; b < I.k; ++b) any |= ldm<MULTI>(I.bw + b) > I.Lmax;
  for (int b = threadIdx.x; b < I.k; b += blockDim.x) {
    const long long w = ldm<MULTI>(I.bw + b);
    s_bw[b] = w;
    s_over[b] = w > I.Lmax ? 1 : 0;
    s_cap[b] = (w > I.Lmax || w >= I.dz_min) ? -1 : I.Lmax - w;
  }
  __syncthreads();
  return any;
}

template <int KWP>
__device__ __forceinline__ void eligible_set(const long long *s_cap, int k, int32_t c, uint32_t (&E)[KWP]) {
#pragma unroll
  for (int q = 0; q < KWP; ++q) {
    uint32_t w = 0;
    for (int bit = 0; bit < 32; ++bit) {
      const int b = 32 * q + bit;
      if (b < k && s_cap[b] >= c) w |= 1u << bit;
    }
    E[q] = w;
  }
}

// Records of the round: every vertex v of an overloaded block s with 2c(v) <= 3(c(V_s) - ceil(c(V)/k)) and an
// eligible target gets its best eligible target (ties to the smaller block) and its priority key.
template <bool MULTI, int KWP>
__device__ void team_targets(const TeamInst &I, const Team &tm, const long long *s_cap, const long long *s_bw,
                             const int *s_over, unsigned *s_wc, unsigned long long *s_base) {
  // the next vertex's id, block and weight are loaded while the current one is evaluated
  const long long i0 = (long long)tm.rank * blockDim.x + threadIdx.x;
  int nv = i0 < I.n_light ? I.v_light[i0] : -1;
  int ns = nv >= 0 ? ldm<MULTI>(I.part + nv) : 0;
  int32_t nc = nv >= 0 ? I.vwgt[nv] : 0;
  for (long long base = (long long)tm.rank * blockDim.x; base < I.n_light; base += tm.nthr) {
    const long long i = base + threadIdx.x;
    bool rec = false;
    int v = nv, s = ns, t = 0;
    int32_t c = nc;
    uint64_t hi = 0;
    nv = i + tm.nthr < I.n_light ? I.v_light[i + tm.nthr] : -1;
    ns = nv >= 0 ? ldm<MULTI>(I.part + nv) : 0;
    nc = nv >= 0 ? I.vwgt[nv] : 0;
    if (i < I.n_light) {
      if (s_over[s] && 2ll * c <= 3ll * (s_bw[s] - I.A)) {
        uint32_t C[KWP], nz = 0;
        eligible_set<KWP>(s_cap, I.k, c, C);
#pragma unroll
        for (int q = 0; q < KWP; ++q) nz |= C[q];
        if (nz) {
          uint32_t pl[kLightPlanes][KWP], any[KWP];
          const int32_t A = light_planes<MULTI, KWP>(I, v, s, pl, any);
          int32_t conn;
          t = argmax_planes<KWP, kLightPlanes>(pl, C, conn);
          hi = rb_priority_key(I.rb_compact, I.rb_L, I.rb_Pmax, conn - A, c);
          rec = true;
        }
      }
    }
    const unsigned long long pos = block_append(rec, &I.tc->n_rec, s_wc, s_base);
    if (rec) {
      I.rb_hi[pos] = hi;
      I.rb_v[pos] = v;
      I.rb_ct[pos] = (c << 16) | (s << 8) | t;
    }
  }
  const int lane = threadIdx.x & 31;
  for (long long i = tm.wid; i < I.n_heavy; i += tm.nwarps) {
    const int v = I.v_heavy[i];
    const int s = ldm<MULTI>(I.part + v);
    const int32_t c = I.vwgt[v];
    if (!s_over[s] || 2ll * c > 3ll * (s_bw[s] - I.A)) continue;  // warp-uniform
    bool elig = false;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      const int b = 32 * q + lane;
      elig |= b < I.k && s_cap[b] >= c;
    }
    if (!__any_sync(kFull, elig)) continue;
    int32_t conn[KWP];
    uint32_t adj;
    const int32_t A = heavy_conn<MULTI, KWP>(I, v, s, conn, adj);
    int bb = -1;
    int32_t bc = 0;
#pragma unroll
    for (int q = 0; q < KWP; ++q) {
      const int b = 32 * q + lane;
      if (b < I.k && s_cap[b] >= c && (bb < 0 || conn[q] > bc)) {
        bb = b;
        bc = conn[q];
      }
    }
    warp_argmax(bc, bb);
    if (lane == 0) {
      const unsigned long long pos = atomicAdd(&I.tc->n_rec, 1ull);
      I.rb_hi[pos] = rb_priority_key(I.rb_compact, I.rb_L, I.rb_Pmax, bc - A, c);
      I.rb_v[pos] = v;
      I.rb_ct[pos] = (c << 16) | (s << 8) | bb;
    }
  }
}

// Selection: per overloaded block the minimal prefix of its records in key order whose weight reaches the
// excess (all records if they never do), by a radix select over 8-bit digits of the key from the top.  The
// per-block threshold (prefix), the weight below the fixed prefix (before) and the all-flag live in rbb.
template <bool MULTI>
__device__ void team_select(const TeamInst &I, const Team &tm, long long nrec, const int *s_over) {
  const int tb = I.rb_tbits;
  const int lane = threadIdx.x & 31;
  for (int hi_bit = tb, level = 0; hi_bit > 0; ++level) {
    const int lo = hi_bit > 8 ? hi_bit - 8 : 0;
    const int up = hi_bit;
    for (long long i = tm.tid; i < nrec; i += tm.nthr) {  // histogram of this digit
      const int32_t ct = ldm<MULTI>(I.rb_ct + i);
      const int b = (ct >> 8) & 255;
      if (ldm<MULTI>(&I.rbb[b].all)) continue;
      const u128 K = ((u128)ldm<MULTI>(I.rb_hi + i) << I.rb_vbits) | (u128)(uint32_t)ldm<MULTI>(I.rb_v + i);
      const u128 pre = ((u128)ldm<MULTI>(&I.rbb[b].pre_hi) << 64) | (u128)ldm<MULTI>(&I.rbb[b].pre_lo);
      if (up < tb && (K >> up) != (pre >> up)) continue;
      const int d = (int)((K >> lo) & (u128)255);
      atomicAdd(&I.hist[(int64_t)b * 256 + d], (unsigned long long)(ct >> 16));
    }
    team_sync<MULTI>();
    for (long long b = tm.wid; b < I.k; b += tm.nwarps) {  // one warp per overloaded block picks the digit
      if (!s_over[b]) continue;
      RbBlock *r = &I.rbb[b];
      if (ldm<MULTI>(&r->all)) continue;
      unsigned long long *row = I.hist + b * 256;
      long long w[8], tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        w[q] = (long long)ldm<MULTI>(row + lane * 8 + q);
        tot += w[q];
      }
      long long incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const long long total = __shfl_sync(kFull, incl, 31);
      const long long before = ldm<MULTI>(&r->before), need = ldm<MULTI>(&r->excess);
      __syncwarp();
      if (level == 0 && total < need) {
        if (lane == 0) r->all = 1;
      } else {
        const long long run0 = before + incl - tot;  // weight below this lane's 8 bins
        const unsigned hit = __ballot_sync(kFull, run0 < need && run0 + tot >= need);
        if (lane == __ffs(hit) - 1) {
          long long run = run0;
          int q = 0;
          for (; q < 8; ++q) {
            if (run + w[q] >= need) break;
            run += w[q];
          }
          r->before = run;
          const u128 pre = (((u128)ldm<MULTI>(&r->pre_hi) << 64) | ldm<MULTI>(&r->pre_lo)) |
                           ((u128)(unsigned)(lane * 8 + q) << lo);
          r->pre_hi = (unsigned long long)(pre >> 64);
          r->pre_lo = (unsigned long long)pre;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) row[lane * 8 + q] = 0ull;
    }
    team_sync<MULTI>();
    hi_bit = lo;
  }
}

// Every record up to its block's threshold (or of an `all` block) moves.
template <bool MULTI, int KWP>
__device__ void team_apply_selection(const TeamInst &I, const Team &tm, long long nrec, long long *s_dw,
                                     long long *s_red) {
  long long moved = 0;
  for (long long i = tm.tid; i < nrec; i += tm.nthr) {
    const int32_t ct = ldm<MULTI>(I.rb_ct + i);
    const int b = (ct >> 8) & 255;
    const int v = ldm<MULTI>(I.rb_v + i);
    bool sel = ldm<MULTI>(&I.rbb[b].all) != 0;
    if (!sel) {
      const u128 K = ((u128)ldm<MULTI>(I.rb_hi + i) << I.rb_vbits) | (u128)(uint32_t)v;
      const u128 pre = ((u128)ldm<MULTI>(&I.rbb[b].pre_hi) << 64) | (u128)ldm<MULTI>(&I.rbb[b].pre_lo);
      sel = K <= pre;
    }
    if (sel) {
      move_vertex<KWP>(I, v, b, ct & 255, (ct >> 16) & 0xffff, s_dw);
      ++moved;
    }
  }
  flush_bw(I, s_dw);
  block_add(moved, reinterpret_cast<long long *>(&I.tc->moved), s_red);
}

struct SmemPtrs {
  long long *s_dw, *s_cap, *s_bw, *s_red;
  int *s_over;
  unsigned *s_wc;
  unsigned long long *s_base, *s_tab;
};

// Rebalancing rounds until balanced, a round moves nothing, or the round cap.  Returns the rounds; moves in *mv.
template <bool MULTI, int KWP>
__device__ long long team_rebalance(const TeamInst &I, const Team &tm, const SmemPtrs &sm, long long *mv) {
  long long rounds = 0, moves = 0;
  for (;;) {
    const bool any = round_state<MULTI>(I, sm.s_cap, sm.s_bw, sm.s_over);
    if (!any || rounds >= I.max_rounds) break;
    if (leader(tm)) {
      I.tc->n_rec = 0;
      I.tc->moved = 0;
    }
    for (long long b = tm.tid; b < I.k; b += tm.nthr) {
      const long long w = sm.s_bw[b];
      RbBlock r;
      r.bw = w;
      r.over = w > I.Lmax ? 1 : 0;
      r.excess = r.over ? w - I.Lmax : 0;
      r.cap = sm.s_cap[b];
      r.before = 0;
      r.pre_hi = 0;
      r.pre_lo = 0;
      r.all = 0;
      I.rbb[b] = r;
    }
    team_sync<MULTI>();
    team_targets<MULTI, KWP>(I, tm, sm.s_cap, sm.s_bw, sm.s_over, sm.s_wc, sm.s_base);
    team_sync<MULTI>();
    const long long nrec = (long long)ldm<MULTI>(&I.tc->n_rec);
    team_select<MULTI>(I, tm, nrec, sm.s_over);
    team_apply_selection<MULTI, KWP>(I, tm, nrec, sm.s_dw, sm.s_red);
    team_sync<MULTI>();
    const long long moved = (long long)ldm<MULTI>(&I.tc->moved);
    rounds += 1;
    moves += moved;
    team_sync<MULTI>();  // every thread has read `moved` before the next round resets it
    if (moved == 0) break;
  }
  *mv = moves;
  return rounds;
}

// Algorithm 1 on one instance.
template <bool MULTI, int KWP>
__device__ void team_refine(const TeamInst &I, const Team &tm, const TeamArgs &a, const SmemPtrs &sm) {
  if (leader(tm)) I.tc->err = 0;
  team_sync<MULTI>();
  team_pincounts<MULTI, KWP>(I, tm, sm.s_dw);
  if (ldm<MULTI>(&I.tc->err)) {  // the same answer in every thread: nothing was written but err
    team_sync<MULTI>();
    return;
  }
  long long obj = 0, maxbw = 0;
  team_objective<MULTI, KWP>(I, tm, sm.s_red, obj, maxbw);
  jet_refine_result res;
  memset(&res, 0, sizeof(res));
  res.initial_objective = obj;
  bool have_best = maxbw <= I.Lmax;
  long long best_obj = obj;
  if (have_best)
    for (long long v = tm.tid; v < I.n; v += tm.nthr) I.best[v] = ldm<MULTI>(I.part + v);
  long long iters = 0;
  bool capped = false;
  for (int ti = 0; ti < a.n_tau && !capped; ++ti) {
    const int32_t tn = a.tau[2 * ti], td = a.tau[2 * ti + 1];
    for (long long v = tm.tid; v < I.n; v += tm.nthr) I.locked[v] = 0;
    int it = 0;
    long long in_phase = 0;
    while (it < a.limit) {
      if (a.iter_cap > 0 && iters >= a.iter_cap) {
        capped = true;
        break;
      }
      if (leader(tm)) {
        I.tc->n_cand = 0;
        I.tc->n_moves = 0;
      }
      team_sync<MULTI>();
      team_candidates<MULTI, KWP>(I, tm, tn, td, sm.s_red);
      team_sync<MULTI>();
      team_afterburner<MULTI, KWP>(I, tm, sm.s_tab);
      team_sync<MULTI>();
      team_approve<MULTI>(I, tm, sm.s_wc, sm.s_base);
      team_sync<MULTI>();
      team_apply_list<MULTI, KWP>(I, tm, (long long)ldm<MULTI>(&I.tc->n_moves), sm.s_dw);
      team_sync<MULTI>();
      long long rb_moves = 0;
      team_rebalance<MULTI, KWP>(I, tm, sm, &rb_moves);
      team_objective<MULTI, KWP>(I, tm, sm.s_red, obj, maxbw);
      iters += 1;
      in_phase += 1;
      it += 1;
      if (maxbw <= I.Lmax && (!have_best || obj < best_obj)) {  // Algorithm 1: a balanced improvement
        have_best = true;
        best_obj = obj;
        it = 0;
        for (long long v = tm.tid; v < I.n; v += tm.nthr) I.best[v] = ldm<MULTI>(I.part + v);
      }
      team_sync<MULTI>();
    }
    if (ti < 8) res.phase_iterations[ti] = in_phase;
    if (have_best) {  // rollback to the best balanced partition, by moves
      if (leader(tm)) I.tc->n_moves = 0;
      team_sync<MULTI>();
      for (long long base = (long long)tm.rank * blockDim.x; base < I.n; base += tm.nthr) {
        const long long v = base + threadIdx.x;
        int s = 0, t = 0;
        bool mvd = false;
        if (v < I.n) {
          s = ldm<MULTI>(I.part + v);
          t = ldm<MULTI>(I.best + v);
          mvd = s != t;
        }
        const unsigned long long pos = block_append(mvd, &I.tc->n_moves, sm.s_wc, sm.s_base);
        if (mvd) {
          I.mv_v[pos] = (int32_t)v;
          I.mv_st[pos] = (uint32_t)s | ((uint32_t)t << 16);
        }
      }
      team_sync<MULTI>();
      team_apply_list<MULTI, KWP>(I, tm, (long long)ldm<MULTI>(&I.tc->n_moves), sm.s_dw);
      team_sync<MULTI>();
    }
  }
  team_objective<MULTI, KWP>(I, tm, sm.s_red, obj, maxbw);
  res.iterations = iters;
  res.objective = obj;
  res.balanced = maxbw <= I.Lmax ? 1 : 0;
  if (leader(tm)) *I.res = res;
  team_sync<MULTI>();
}

// The persistent kernel: teams of gridDim.x / clusterDim blocks loop over the work queue.
template <bool MULTI, int KWP>
__global__ void __launch_bounds__(kTeamMaxThreads) k_batch_teams(TeamArgs a, int kmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_wc[kTeamMaxThreads / 32];
  __shared__ unsigned long long s_base;
  __shared__ long long s_red[kTeamMaxThreads / 32];
  SmemPtrs sm;
  sm.s_dw = reinterpret_cast<long long *>(smem);
  sm.s_cap = sm.s_dw + kmax;
  sm.s_bw = sm.s_cap + kmax;
  sm.s_over = reinterpret_cast<int *>(sm.s_bw + kmax);
  sm.s_tab = reinterpret_cast<unsigned long long *>(sm.s_over + kmax + (kmax & 1));
  sm.s_wc = s_wc;
  sm.s_base = &s_base;
  sm.s_red = s_red;
  Team tm;
  if constexpr (MULTI) {
    unsigned r, sz;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(sz));
    tm.rank = r;
    tm.size = sz;
  } else {
    tm.rank = 0;
    tm.size = 1;
  }
  tm.tid = (long long)tm.rank * blockDim.x + threadIdx.x;
  tm.nthr = (long long)tm.size * blockDim.x;
  tm.lane = threadIdx.x & 31;
  tm.wid = tm.tid >> 5;
  tm.nwarps = tm.nthr >> 5;
  for (int b = threadIdx.x; b < kmax; b += blockDim.x) sm.s_dw[b] = 0;
  const long long team = blockIdx.x / tm.size;
  int idx = -1;
  for (;;) {
    if (leader(tm)) {
      const unsigned q = atomicAdd(a.queue, 1u);
      a.team_inst[team] = q < (unsigned)a.count ? a.order[q] : -1;
    }
    team_sync<MULTI>();
    idx = ldm<MULTI>(a.team_inst + team);
    team_sync<MULTI>();  // every thread has the index before the leader overwrites the slot
    if (idx < 0) return;
    if (MULTI && a.inst[idx].P < a.split_pins) break;  // the queue is largest first: the rest are smaller
    team_refine<MULTI, KWP>(a.inst[idx], tm, a, sm);
  }
  if constexpr (MULTI) {
    // Split: from the first instance below split_pins on, every block of the cluster is a team of its
    // own (no cluster barrier from here on).  Block 0 takes the instance the cluster just drew; every
    // block then draws instances on its own until the queue is empty.
    Team one;
    one.rank = 0;
    one.size = 1;
    one.tid = threadIdx.x;
    one.nthr = blockDim.x;
    one.lane = threadIdx.x & 31;
    one.wid = threadIdx.x >> 5;
    one.nwarps = blockDim.x >> 5;
    __shared__ int s_idx;
    if (tm.rank == 0) team_refine<false, KWP>(a.inst[idx], one, a, sm);
    for (;;) {
      if (threadIdx.x == 0) {
        const unsigned q = atomicAdd(a.queue, 1u);
        s_idx = q < (unsigned)a.count ? a.order[q] : -1;
      }
      __syncthreads();
      const int j = s_idx;
      __syncthreads();
      if (j < 0) return;
      team_refine<false, KWP>(a.inst[j], one, a, sm);
    }
  }
}

}  // namespace

// ------------------------------------------------------------ host side
struct TeamPlan {
  std::vector<TeamInst> host;   // descriptors (device pointers)
  std::vector<int32_t> kwp;     // per instance
  std::vector<long long> pins;  // per instance
  TeamInst *dev = nullptr;
  TeamCount *counts = nullptr;
  jet_refine_result *res = nullptr;  // device, per instance
  int32_t *order = nullptr;          // device: instances grouped by mask width, largest first within a group
  std::vector<int32_t> group_start, group_kwp, group_kmax;  // groups of `order`
  int32_t *tau = nullptr;            // device schedule
  int32_t n_tau = 0;
  unsigned *queue = nullptr;         // one counter per group
  int32_t *sample = nullptr;         // device: the instances of a tuning trial
  int32_t *team_inst = nullptr;
  unsigned long long *hist = nullptr;  // device: k x 256 digit histograms per instance
  int32_t team_slots = 0;
  int num_sms = 0;
};

namespace {

template <bool MULTI, int KWP>
cudaError_t launch_group(const TeamArgs &a, int kmax, int ctas, int threads, int num_sms, cudaStream_t s,
                         int max_teams) {
  auto kern = k_batch_teams<MULTI, KWP>;
  const size_t smem = (size_t)kmax * (8 + 8 + 8 + 4) + 8 * (size_t)(kmax & 1) +
                      (size_t)(threads / 32) * (2 * kmax + (KWP + 1) / 2) * 8;
  // The limit is a property of the kernel, shared by every batch and graph that launches it: set it for
  // the largest instance this mask width allows (k = 32 KWP) and 1,024 threads, so it never shrinks
  // under an earlier launch.
  constexpr size_t kSmemMax =
      (size_t)(32 * KWP) * (8 + 8 + 8 + 4) + 8 + (size_t)32 * (2 * 32 * KWP + (KWP + 1) / 2) * 8;
  static_assert(kSmemMax <= 227 * 1024, "the team kernel's shared memory must fit one block");
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
  if (e != cudaSuccess) return e;
  if (MULTI && ctas > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  int teams = 0;
  if (MULTI) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(ctas * num_sms);
    e = cudaOccupancyMaxActiveClusters(&teams, kern, &cfg);
    if (e != cudaSuccess) return e;
  } else {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    teams = per_sm * num_sms;
  }
  if (teams < 1) return cudaErrorInvalidConfiguration;
  if (teams > max_teams) teams = max_teams;
  cfg.gridDim = dim3(teams * ctas);
  return cudaLaunchKernelEx(&cfg, kern, a, kmax);
}

template <int KWP>
cudaError_t launch_kwp(const TeamArgs &a, int kmax, int ctas, int threads, int num_sms, cudaStream_t s, int max_teams) {
  if (ctas > 1) return launch_group<true, KWP>(a, kmax, ctas, threads, num_sms, s, max_teams);
  return launch_group<false, KWP>(a, kmax, ctas, threads, num_sms, s, max_teams);
}

}  // namespace

void team_plan_destroy(TeamPlan *p, cudaStream_t s);

int team_plan_build(TeamPlan **out, jet_ctx *const *ctxs, int32_t count, int32_t *const *part, int32_t *const *phi,
                    int64_t *const *block_w, const int32_t *tau_pairs, int32_t n_tau, cudaStream_t s) {
  *out = nullptr;
  TeamPlan *p = new (std::nothrow) TeamPlan;
  if (!p) return fail(nullptr, JET_ERR_OOM, "host allocation failed");
  p->n_tau = n_tau;
  p->num_sms = ctxs[0]->num_sms;
  for (int i = 0; i < count; ++i) {
    jet_ctx *c = ctxs[i];
    TeamInst t{};
    t.n = c->n;
    t.m = c->m;
    t.k = c->k;
    t.unit_ewgt = c->unit_ewgt;
    t.P = c->P;
    t.eptr = c->eptr;
    t.vptr = c->vptr;
    t.pins = c->pins;
    t.inc = c->inc;
    t.vwgt = c->vwgt;
    t.ewgt = c->ewgt;
    t.A = c->A;
    t.Lmax = c->Lmax;
    t.dz_min = c->dz_min;
    t.max_rounds = c->params.max_rebalance_rounds;
    t.rb_compact = c->rb_compact;
    t.rb_vbits = c->rb_vbits;
    t.rb_tbits = c->rb_hbits + c->rb_vbits;
    t.rb_L = c->rb_L;
    t.rb_Pmax = c->rb_Pmax;
    t.v_light = c->v_light;
    t.v_heavy = c->v_heavy;
    t.n_light = c->n_light;
    t.n_heavy = c->n_heavy;
    t.e_tiny = c->e_tiny;
    t.n_tiny = c->n_tiny;
    t.e_rest = c->e_tiny + c->n_tiny;
    t.n_rest = c->m - c->n_tiny;
    t.part = part[i];
    t.phi = phi[i];
    t.bw = block_w[i];
    t.mask = c->mask;
    t.cand = c->cand;
    t.rg = c->rg;
    t.mv_v = c->mv_v;
    t.mv_st = c->mv_st;
    t.locked = c->locked_ws;
    t.best = c->best_part;
    t.rb_hi = c->rb_hi;
    t.rb_v = c->rb_v;
    t.rb_ct = c->rb_ct;
    t.hist = nullptr;  // set below, in the plan's histogram buffer
    t.rbb = c->rbb;
    p->host.push_back(t);
    p->kwp.push_back(c->kwp);
    p->pins.push_back(c->P);
  }
  // queue order: grouped by mask width, largest instance first within a group
  std::vector<int32_t> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (p->kwp[a] != p->kwp[b]) return p->kwp[a] < p->kwp[b];
    return p->pins[a] > p->pins[b];
  });
  for (int i = 0; i < count; ++i) {
    if (i == 0 || p->kwp[ord[i]] != p->kwp[ord[i - 1]]) {
      p->group_start.push_back(i);
      p->group_kwp.push_back(p->kwp[ord[i]]);
      p->group_kmax.push_back(0);
    }
    p->group_kmax.back() = std::max(p->group_kmax.back(), (int32_t)p->host[ord[i]].k);
  }
  p->group_start.push_back(count);
  const size_t ng = p->group_kwp.size();
  p->team_slots = 4096;
  cudaError_t e = jet::pool_alloc(reinterpret_cast<void **>(&p->dev), sizeof(TeamInst) * count, s);
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->counts), sizeof(TeamCount) * count, s);
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->res), sizeof(jet_refine_result) * count, s);
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->order), sizeof(int32_t) * count, s);
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->sample), sizeof(int32_t) * count, s);
  if (e == cudaSuccess)
    e = jet::pool_alloc(reinterpret_cast<void **>(&p->tau), sizeof(int32_t) * (2 * n_tau > 0 ? 2 * n_tau : 1), s);
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->queue), sizeof(unsigned) * ng, s);
  if (e == cudaSuccess)
    e = jet::pool_alloc(reinterpret_cast<void **>(&p->team_inst), sizeof(int32_t) * p->team_slots, s);
  size_t nbins = 0;
  for (int i = 0; i < count; ++i) nbins += (size_t)p->host[i].k * 256;
  if (e == cudaSuccess) e = jet::pool_alloc(reinterpret_cast<void **>(&p->hist), sizeof(unsigned long long) * nbins, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->hist, 0, sizeof(unsigned long long) * nbins, s);
  if (e == cudaSuccess) {
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
      p->host[i].tc = p->counts + i;
      p->host[i].res = p->res + i;
      p->host[i].hist = p->hist + off;
      off += (size_t)p->host[i].k * 256;
    }
    e = cudaMemcpyAsync(p->dev, p->host.data(), sizeof(TeamInst) * count, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->order, ord.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_tau > 0)
    e = cudaMemcpyAsync(p->tau, tau_pairs, sizeof(int32_t) * 2 * n_tau, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->counts, 0, sizeof(TeamCount) * count, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors above are sources of the copies
  if (e != cudaSuccess) {
    team_plan_destroy(p, s);
    return cuda_fail(nullptr, e, "batch team plan");
  }
  *out = p;
  return JET_OK;
}

void team_plan_destroy(TeamPlan *p, cudaStream_t s) {
  if (!p) return;
  void *bufs[] = {p->dev, p->counts, p->res, p->order, p->sample, p->tau, p->queue, p->team_inst, p->hist};
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  cudaStreamSynchronize(s);
  delete p;
}

// The persistent launches of a plan (one per mask-width group), each over its group's instances (or over the
// n_sub instances of sub_order, a HOST list of instances of the first group, for tuning trials).  iter_cap > 0
// stops each instance after that many Jet iterations; with ctas > 1, instances of fewer than split_pins pins
// run on single blocks.  Results land in the plan's device summaries.
cudaError_t team_launch(TeamPlan *p, int ctas, int threads, long long split_pins, int32_t limit, int32_t iter_cap,
                        cudaStream_t s, const int32_t *sub_order, int32_t n_sub) {
  const size_t ng = p->group_kwp.size();
  cudaError_t e = cudaMemsetAsync(p->queue, 0, sizeof(unsigned) * ng, s);
  if (e == cudaSuccess && sub_order) {
    e = cudaMemcpyAsync(p->sample, sub_order, sizeof(int32_t) * n_sub, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // sub_order is pageable host memory
    sub_order = p->sample;
  }
  for (size_t g = 0; g < ng && e == cudaSuccess; ++g) {
    TeamArgs a{};
    a.inst = p->dev;
    a.order = sub_order ? sub_order : p->order + p->group_start[g];
    a.count = sub_order ? (g == 0 ? n_sub : 0) : p->group_start[g + 1] - p->group_start[g];
    if (a.count == 0) continue;
    a.queue = p->queue + g;
    a.team_inst = p->team_inst;
    a.tau = p->tau;
    a.n_tau = p->n_tau;
    a.limit = limit;
    a.iter_cap = iter_cap;
    a.split_pins = split_pins;
    const int kwp = sub_order ? p->group_kwp[0] : p->group_kwp[g];
    const int kmax = p->group_kmax[sub_order ? 0 : g];
    const int max_teams = std::min(p->team_slots, a.count);
    switch (kwp) {
      case 1: e = launch_kwp<1>(a, kmax, ctas, threads, p->num_sms, s, max_teams); break;
      case 2: e = launch_kwp<2>(a, kmax, ctas, threads, p->num_sms, s, max_teams); break;
      case 4: e = launch_kwp<4>(a, kmax, ctas, threads, p->num_sms, s, max_teams); break;
      default: e = launch_kwp<8>(a, kmax, ctas, threads, p->num_sms, s, max_teams); break;
    }
  }
  return e;
}

cudaError_t team_results(TeamPlan *p, jet_refine_result *dst, cudaStream_t s) {
  return cudaMemcpyAsync(dst, p->res, sizeof(jet_refine_result) * p->host.size(), cudaMemcpyDeviceToHost, s);
}

// Index of the first instance whose partition held a block id outside [0, k) in the last launch, or -1.
// Synchronizes the stream.
int team_first_error(TeamPlan *p, cudaStream_t s) {
  std::vector<TeamCount> h(p->host.size());
  if (cudaMemcpyAsync(h.data(), p->counts, sizeof(TeamCount) * h.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -2;
  for (size_t i = 0; i < h.size(); ++i)
    if (h[i].err) return (int)i;
  return -1;
}

// The plan's instances of the first mask-width group, spread over its sizes (for tuning trials): n of them.
std::vector<int32_t> team_sample(TeamPlan *p, int32_t n) {
  std::vector<int32_t> ord(p->host.size());
  cudaMemcpy(ord.data(), p->order, sizeof(int32_t) * ord.size(), cudaMemcpyDeviceToHost);
  const int32_t cnt = p->group_start[1] - p->group_start[0];
  std::vector<int32_t> out;
  if (n >= cnt) {
    out.assign(ord.begin(), ord.begin() + cnt);
  } else {
    for (int32_t i = 0; i < n; ++i) out.push_back(ord[(int64_t)i * cnt / n]);
  }
  return out;
}

long long team_pins(TeamPlan *p, int32_t i) { return p->pins[i]; }

}  // namespace jet
