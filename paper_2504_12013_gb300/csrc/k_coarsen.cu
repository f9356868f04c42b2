// Deterministic synchronous coarsening (Section 6, Algorithm 4) and the
// contraction of its clusters.
//
// Clustering.  Clusters are label classes (label[v] starts as v).  The
// vertices are visited in sub-rounds of a caller-given order (the random
// split of Algorithm 4): `single` sub-rounds of one vertex, then sizes 2, 4,
// 8, ... up to floor(n / cap_div) (prefix doubling).  Within a sub-round,
// from the state at its start, every vertex still in a singleton cluster
// rates the clusters of its neighbours with the corrected heavy-edge rating
// (an edge adds omega(e)/(|e|-1) once per cluster it touches; 32.32 fixed
// point, each term rounded down; edges of more than rmax pins add nothing)
// and proposes the best one that stays within the weight bound (ties to the
// smaller label).  Mutual proposals u <-> v are resolved towards the heavier
// would-be cluster (swap prevention), then every target accepts the longest
// prefix of its proposers in (weight, id) order that fits, and the accepted
// vertices move together.
//
//   k_cl_serial   the leading one-vertex sub-rounds, one block, in order
//   k_cl_rate     hash table of the neighbour clusters per vertex, a warp
//                 per vertex (table in shared memory, else a slice of a
//                 global pool sized per sub-round)
//   k_cl_rate_heavy  a 16-warp block per vertex whose table exceeds 2048
//                 entries: the warps take its edges from a shared counter
//                 (edges above 64 pins first), each edge's clusters
//                 deduplicated in a per-warp set, the sums integer atomics
//   k_cl_swap     swap prevention, group lists of the proposals
//   k_cl_approve  weight-ordered prefix per target (fast path: all fit)
//   k_cl_apply    moves, resets the per-sub-round state
//
// Contraction.  Non-empty label classes become coarse vertices in label
// order; each edge keeps its distinct coarse pins (ascending), is dropped
// below two, and edges with equal pin sets merge into the smallest id with
// summed weights; incidences are listed in coarse-edge order.  Uses an
// exclusive scan and a stable LSD radix sort of 64-bit keys written here.
#include <algorithm>
#include <vector>

#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTile = 2048;        // scan / radix tile: 256 threads x 8 items
constexpr int kSmemTab = 128;      // hash-table entries per warp held in shared memory
constexpr int kWarpTab = 2048;     // larger tables: the whole block rates the vertex (heavy vertices)
constexpr int kBlockTab = 4096;    // a heavy vertex's table in shared memory up to this size
constexpr int kHeavyWarps = 16;    // warps of a block that rates one heavy vertex
constexpr int kFirstEdge = 64;     // a heavy vertex's edges above this size are rated first
constexpr int kSetCap = 2048;      // per-warp set of the distinct clusters of one edge (heavy vertices)
constexpr int kSetEdge = kSetCap / 2;  // edges up to this size are deduplicated in that set
constexpr size_t kHeavySmem = sizeof(int32_t) * kHeavyWarps * kSetCap + 16 * kBlockTab;
constexpr int64_t kMaxTab = 1 << 28;

struct Tab {
  int32_t key;   // cluster label, -1 = empty
  int32_t last;  // last edge that added to this entry
  unsigned long long val;
};

__device__ __forceinline__ uint32_t mix32(uint32_t x) {  // integer hash (xor-shift-multiply)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {  // splitmix64 finaliser
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// ------------------------------------------------------------------ scan

__device__ __forceinline__ long long warp_incl(long long x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__global__ void __launch_bounds__(256) k_scan_tiles(const int64_t *in, int64_t n, int64_t *tile_sums) {
  __shared__ long long s_w[8];
  const int64_t base = blockIdx.x * (int64_t)kTile;
  long long s = 0;
  for (int i = threadIdx.x; i < kTile; i += 256)
    if (base + i < n) s += in[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    tile_sums[blockIdx.x] = t;
  }
}

// Exclusive scan of v[0..nt) in place by one block; *total gets the sum.
__global__ void __launch_bounds__(1024) k_scan_top(int64_t *v, int64_t nt, int64_t *total) {
  __shared__ long long s_w[32];
  __shared__ long long s_carry;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) s_carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nt; c0 += 1024) {
    const int64_t i = c0 + t;
    const long long x = i < nt ? v[i] : 0;
    const long long incl = warp_incl(x, lane);
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const long long w = s_w[lane];
      s_w[lane] = warp_incl(w, lane) - w;
    }
    __syncthreads();
    const long long excl = s_carry + s_w[wid] + incl - x;
    if (i < nt) v[i] = excl;
    __syncthreads();
    if (t == 1023) s_carry = excl + x;
    __syncthreads();
  }
  if (t == 0 && total) *total = s_carry;
}

__global__ void __launch_bounds__(256) k_scan_apply(const int64_t *in, int64_t n, const int64_t *tile_offs,
                                                     int64_t *out) {
  __shared__ long long s_w[8];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t base = blockIdx.x * (int64_t)kTile + (int64_t)t * 8;
  long long vals[8];
  long long s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    vals[j] = base + j < n ? in[base + j] : 0;
    s += vals[j];
  }
  const long long incl = warp_incl(s, lane);
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  long long wo = 0;
  for (int w = 0; w < wid; ++w) wo += s_w[w];
  long long run = tile_offs[blockIdx.x] + wo + incl - s;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (base + j < n) out[base + j] = run;
    run += vals[j];
  }
}

int64_t scan_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// Exclusive scan of in[0..n) into out (may alias in); tmp holds scan_tiles(n) + 1 entries;
// *total_dev (device, may be NULL) gets the sum.
cudaError_t scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, int64_t *total_dev,
                           cudaStream_t s) {
  if (n <= 0) return total_dev ? cudaMemsetAsync(total_dev, 0, sizeof(int64_t), s) : cudaSuccess;
  const int64_t nt = scan_tiles(n);
  k_scan_tiles<<<(unsigned)nt, 256, 0, s>>>(in, n, tmp);
  k_scan_top<<<1, 1024, 0, s>>>(tmp, nt, total_dev);
  k_scan_apply<<<(unsigned)nt, 256, 0, s>>>(in, n, tmp, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort

__global__ void __launch_bounds__(256) k_radix_hist(const unsigned long long *keys, int64_t n, int shift,
                                                     int64_t *hist, int64_t nb) {
  __shared__ int s_h[256];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kTile;
  for (int r = 0; r < 8; ++r) {
    const int64_t i = base + r * 256 + threadIdx.x;
    if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one tile: items are ranked in index order (round, warp, lane).
__global__ void __launch_bounds__(256) k_radix_scatter(const unsigned long long *in, unsigned long long *out,
                                                        int64_t n, int shift, const int64_t *offs, int64_t nb) {
  __shared__ long long s_base[256];
  __shared__ long long s_wo[8][256];
  __shared__ int s_wc[8][256];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  s_base[t] = offs[(int64_t)t * nb + blockIdx.x];
  const int64_t base = blockIdx.x * (int64_t)kTile;
  for (int r = 0; r < 8; ++r) {
#pragma unroll
    for (int w = 0; w < 8; ++w) s_wc[w][t] = 0;
    __syncthreads();
    const int64_t i = base + r * 256 + t;
    const bool have = i < n;
    const unsigned long long key = have ? in[i] : 0ull;
    const int d = have ? (int)((key >> shift) & 255) : 256;
    const unsigned peers = match_bits<9>((unsigned)d);  // d <= 256
    const int rank = __popc(peers & ((1u << lane) - 1));
    if (have && rank == 0) s_wc[wid][d] = __popc(peers);
    __syncthreads();
    long long run = s_base[t];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      s_wo[w][t] = run;
      run += s_wc[w][t];
    }
    s_base[t] = run;
    __syncthreads();
    if (have) out[s_wo[wid][d] + rank] = key;
    __syncthreads();
  }
}

struct SortBufs {
  unsigned long long *tmp = nullptr;  // n keys
  int64_t *hist = nullptr;            // 256 * tiles
  int64_t *scan_tmp = nullptr;        // scan_tiles(256 * tiles) + 1
};

int64_t sort_hist_entries(int64_t n) { return 256 * std::max<int64_t>(scan_tiles(n), 1); }

// Sorts keys[0..n) (values below 2^bits) ascending and stably; the result is in keys.
cudaError_t radix_sort(unsigned long long *keys, int64_t n, int bits, const SortBufs &b, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t nb = scan_tiles(n);
  unsigned long long *src = keys, *dst = b.tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<(unsigned)nb, 256, 0, s>>>(src, n, shift, b.hist, nb);
    cudaError_t e = scan_exclusive(b.hist, b.hist, 256 * nb, b.scan_tmp, nullptr, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<(unsigned)nb, 256, 0, s>>>(src, dst, n, shift, b.hist, nb);
    std::swap(src, dst);
  }
  if (src != keys) return cudaMemcpyAsync(keys, src, sizeof(unsigned long long) * (size_t)n,
                                          cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

int bits_for(unsigned long long max_value) {
  int b = 0;
  while (b < 64 && (max_value >> b) != 0) ++b;
  return b;
}

// ------------------------------------------------------------------ validation

// Error flags: bit 0 = bad CSR / index, bit 1 = order is not a permutation, bit 2 = rating overflow,
// bit 3 = a rated neighbourhood beyond kMaxTab, bit 4 = label out of range, bit 5 = coarse weight overflow.
__global__ void k_check_hg(jet_hypergraph g, int *err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.P; i += stride) {
    if ((unsigned)g.pins[i] >= (unsigned)g.n || (unsigned)g.inc[i] >= (unsigned)g.m) atomicOr(err, 1);
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.m; e += stride) {
    if (g.eptr[e] > g.eptr[e + 1] || g.ewgt[e] < 1) atomicOr(err, 1);
  }
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += stride) {
    if (g.vptr[v] > g.vptr[v + 1] || g.vwgt[v] < 1) atomicOr(err, 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (g.eptr[0] != 0 || g.eptr[g.m] != g.P || g.vptr[0] != 0 || g.vptr[g.n] != g.P) atomicOr(err, 1);
  }
}

__global__ void k_check_order(const int32_t *order, int32_t n, int32_t *seen, int *err) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[x];
    if ((unsigned)v >= (unsigned)n) atomicOr(err, 2);
    else if (atomicExch(&seen[v], 1) == 1) atomicOr(err, 2);
  }
}

// ------------------------------------------------------------------ clustering state

struct Cl {
  int32_t *label;  // caller's output
  long long *cw;   // cluster weights by label
  int32_t *csize;  // cluster sizes by label
  int32_t *T, *T2; // proposals before / after swap prevention (-1 = none)
  long long *pw, *pw2;  // proposal weight per target label (before / after)
  int32_t *head, *next; // proposers of each target (linked lists)
  uint8_t *acc;         // approved
  int32_t *cap;         // hash-table entries per vertex
};

__global__ void k_cl_setup(jet_hypergraph g, int32_t rmax, Cl cl, int *err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    cl.label[v] = (int32_t)v;
    cl.cw[v] = g.vwgt[v];
    cl.csize[v] = 1;
    cl.T[v] = cl.T2[v] = -1;
    cl.pw[v] = cl.pw2[v] = 0;
    cl.head[v] = -1;
    cl.acc[v] = 0;
    unsigned long long sum = 0;
    int64_t bound = 0;
    for (int64_t i = g.vptr[v]; i < g.vptr[v + 1]; ++i) {
      const int32_t e = g.inc[i];
      const int64_t size = g.eptr[e + 1] - g.eptr[e];
      if (size < 2 || size > rmax) continue;
      sum += ((unsigned long long)(uint32_t)g.ewgt[e] << 32) / (unsigned long long)(size - 1);
      if (sum >= (1ull << 63)) {
        atomicOr(err, 4);
        sum = 0;
      }
      bound += size - 1;
    }
    int64_t cap = 0;
    if (bound > 0) {
      cap = 32;
      while (cap < 2 * bound) cap <<= 1;
    }
    if (cap > kMaxTab) {
      atomicOr(err, 8);
      cap = 0;
    }
    cl.cap[v] = (int32_t)cap;
  }
}

// The sub-round of each position x (bounds[r] <= x < bounds[r+1]).
__device__ __forceinline__ int round_of(const int32_t *bounds, int32_t rounds, int64_t x) {
  int lo = 0, hi = rounds - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bounds[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per sub-round: heavy vertices (tables beyond kWarpTab) and the global-pool entries of the tables that
// fit neither a warp's shared slice nor a block's shared memory.
__global__ void k_cl_need(const int32_t *order, int32_t n, const int32_t *bounds, int32_t rounds, const int32_t *cap,
                          unsigned long long *need, unsigned long long *heavy) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cap[order[x]];
    if (c <= kSmemTab) continue;
    const int r = round_of(bounds, rounds, x);
    if (c > kWarpTab) atomicAdd(&heavy[r], 1ull);
    if (c <= kWarpTab || c > kBlockTab) atomicAdd(&need[r], (unsigned long long)c);
  }
}

// The heavy positions of every sub-round, at hoff[r] onwards (any order within a sub-round).
__global__ void k_cl_heavy_list(const int32_t *order, int32_t n, const int32_t *bounds, int32_t rounds,
                                const int32_t *cap, const int64_t *hoff, unsigned long long *hcur, int32_t *hpos) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    if (cap[order[x]] <= kWarpTab) continue;
    const int r = round_of(bounds, rounds, x);
    hpos[hoff[r] + (int64_t)atomicAdd(&hcur[r], 1ull)] = (int32_t)x;
  }
}

// Slot of cluster C in a table of cap entries (a power of two above the number of keys), inserted if new.
__device__ __forceinline__ uint32_t tab_slot(Tab *tab, int32_t cap, int32_t C) {
  uint32_t h = mix32((uint32_t)C) & (uint32_t)(cap - 1);
  for (;;) {
    int32_t k = *(volatile int32_t *)&tab[h].key;
    if (k == -1) {
      k = atomicCAS(&tab[h].key, -1, C);
      if (k == -1) k = C;
    }
    if (k == C) return h;
    h = (h + 1) & (uint32_t)(cap - 1);
  }
}


// The rating of u over the clusters of its neighbours, accumulated in tab (cap entries, a power of
// two above twice the rated pins), and the best cluster within the weight bound (-1 if none).
// Called by a whole warp.
__device__ int32_t rate_vertex(const jet_hypergraph &g, int32_t u, const int32_t *label, const long long *cw,
                               long long cmax, int32_t rmax, Tab *tab, int32_t cap, int lane) {
  for (int i = lane; i < cap; i += 32) {
    tab[i].key = -1;
    tab[i].last = -1;
    tab[i].val = 0;
  }
  __syncwarp();
  const int64_t i1 = g.vptr[u + 1];
  for (int64_t i = g.vptr[u]; i < i1; ++i) {
    const int32_t e = g.inc[i];
    const int64_t p0 = g.eptr[e], p1 = g.eptr[e + 1];
    const int64_t size = p1 - p0;
    if (size < 2 || size > rmax) continue;
    const unsigned long long term = ((unsigned long long)(uint32_t)g.ewgt[e] << 32) / (unsigned long long)(size - 1);
    for (int64_t p = p0; p < p1; p += 128) {  // four chunks of 32 pins in flight, applied in order
      int32_t C[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t pp = p + q * 32 + lane;
        C[q] = pp < p1 ? g.pins[pp] : u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) C[q] = C[q] != u ? label[C[q]] : -1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned peers = __match_any_sync(kFull, C[q]);
        if (C[q] >= 0 && C[q] != u && lane == __ffs(peers) - 1) {  // one lane per distinct cluster of this chunk
          const uint32_t h = tab_slot(tab, cap, C[q]);
          if (tab[h].last != e) {  // once per edge and cluster
            tab[h].last = e;
            tab[h].val += term;
          }
        }
        __syncwarp();
      }
    }
  }
  const long long cu = g.vwgt[u];
  unsigned long long bv = 0;
  int32_t bk = -1;
  for (int i = lane; i < cap; i += 32) {
    const int32_t k = tab[i].key;
    if (k < 0 || cw[k] + cu > cmax) continue;
    const unsigned long long v = tab[i].val;
    if (bk < 0 || v > bv || (v == bv && k < bk)) {
      bv = v;
      bk = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(kFull, bv, o);
    const int32_t ok = __shfl_xor_sync(kFull, bk, o);
    if (ok >= 0 && (bk < 0 || ov > bv || (ov == bv && ok < bk))) {
      bv = ov;
      bk = ok;
    }
  }
  __syncwarp();
  return bk;
}

// Inserts C into a warp's set of the clusters of one edge (scap slots, cleared to -1 before the edge);
// true if it was not there.
__device__ __forceinline__ bool set_insert(int32_t *set, int32_t scap, int32_t C) {
  uint32_t h = mix32((uint32_t)C) & (uint32_t)(scap - 1);
  for (;;) {
    int32_t k = *(volatile int32_t *)&set[h];
    if (k == -1) {
      k = atomicCAS(&set[h], -1, C);
      if (k == -1) return true;
    }
    if (k == C) return false;
    h = (h + 1) & (uint32_t)(scap - 1);
  }
}

// The rating of a heavy vertex by the whole block (same result as rate_vertex).  Its edges are spread
// over the warps and the sums are atomic (integer, order-free); a cluster counts once per edge through
// match_any within a chunk and, for edges of 33 to kSetEdge pins, the warp's set of the edge's
// clusters.  Larger edges follow, by warp 0 alone, counted once per edge and cluster through the
// entry's last edge.  s_set: kHeavyWarps x kSetCap words; s_bk/s_bv: per-warp reduction scratch;
// s_next: the shared edge counters of the two passes.
// Chunks of an edge are taken four at a time, so that their loads overlap.
__device__ int32_t rate_block(const jet_hypergraph &g, int32_t u, const int32_t *label, const long long *cw,
                              long long cmax, int32_t rmax, Tab *tab, int32_t cap, int32_t *s_set,
                              int32_t *s_bk, unsigned long long *s_bv, int *s_next) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  for (int i = t; i < cap; i += blockDim.x) {
    tab[i].key = -1;
    tab[i].last = -1;
    tab[i].val = 0;
  }
  if (t < 2) s_next[t] = 0;
  __syncthreads();
  int32_t *set = s_set + wid * kSetCap;
  const int64_t i0 = g.vptr[u], i1 = g.vptr[u + 1];
  bool big = false;
  // edges are taken one at a time from a shared counter, so that warps that drew small edges take more;
  // edges of more than kFirstEdge pins in a first pass, the rest in a second (largest work first)
  for (int pass = 0; pass < 2; ++pass)
  for (;;) {
    int64_t i = 0;
    if (lane == 0) i = i0 + atomicAdd(&s_next[pass], 1);
    i = __shfl_sync(kFull, i, 0);
    if (i >= i1) break;
    const int32_t e = g.inc[i];
    const int64_t p0 = g.eptr[e], p1 = g.eptr[e + 1], size = p1 - p0;
    if (size < 2 || size > rmax || (size > kFirstEdge) != (pass == 0)) continue;
    if (size > kSetEdge) {
      big = true;
      continue;
    }
    const unsigned long long term = ((unsigned long long)(uint32_t)g.ewgt[e] << 32) / (unsigned long long)(size - 1);
    if (size <= 32) {
      int32_t C = -1;
      if (lane < size) {
        const int32_t v = g.pins[p0 + lane];
        if (v != u) C = label[v];
      }
      const unsigned peers = __match_any_sync(kFull, C);
      if (C >= 0 && C != u && lane == __ffs(peers) - 1) atomicAdd(&tab[tab_slot(tab, cap, C)].val, term);
      continue;
    }
    int32_t scap = 64;
    while (scap < 2 * size) scap <<= 1;
    for (int q = lane; q < scap; q += 32) set[q] = -1;
    __syncwarp();
    for (int64_t p = p0; p < p1; p += 128) {
      int32_t C[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t pp = p + q * 32 + lane;
        C[q] = pp < p1 ? g.pins[pp] : u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) C[q] = C[q] != u ? label[C[q]] : -1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned peers = __match_any_sync(kFull, C[q]);
        if (C[q] >= 0 && C[q] != u && lane == __ffs(peers) - 1 && set_insert(set, scap, C[q]))
          atomicAdd(&tab[tab_slot(tab, cap, C[q])].val, term);
      }
    }
    __syncwarp();
  }
  if (lane == 0) s_bk[wid] = big ? 1 : 0;
  __syncthreads();
  int any_big = 0;
  for (int w = 0; w < nw; ++w) any_big |= s_bk[w];
  if (any_big && wid == 0) {
    for (int64_t i = i0; i < i1; ++i) {
      const int32_t e = g.inc[i];
      const int64_t p0 = g.eptr[e], p1 = g.eptr[e + 1], size = p1 - p0;
      if (size <= kSetEdge || size > rmax) continue;
      const unsigned long long term = ((unsigned long long)(uint32_t)g.ewgt[e] << 32) / (unsigned long long)(size - 1);
      for (int64_t p = p0; p < p1; p += 32) {
        int32_t C = -1;
        if (p + lane < p1) {
          const int32_t v = g.pins[p + lane];
          if (v != u) C = label[v];
        }
        const unsigned peers = __match_any_sync(kFull, C);
        if (C >= 0 && C != u && lane == __ffs(peers) - 1) {
          const uint32_t h = tab_slot(tab, cap, C);
          if (tab[h].last != e) {
            tab[h].last = e;
            tab[h].val += term;
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  const long long cu = g.vwgt[u];
  unsigned long long bv = 0;
  int32_t bk = -1;
  for (int i = t; i < cap; i += blockDim.x) {
    const int32_t k = tab[i].key;
    if (k < 0 || cw[k] + cu > cmax) continue;
    const unsigned long long v = tab[i].val;
    if (bk < 0 || v > bv || (v == bv && k < bk)) {
      bv = v;
      bk = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(kFull, bv, o);
    const int32_t ok = __shfl_xor_sync(kFull, bk, o);
    if (ok >= 0 && (bk < 0 || ov > bv || (ov == bv && ok < bk))) {
      bv = ov;
      bk = ok;
    }
  }
  __syncthreads();  // s_bk reuse
  if (lane == 0) {
    s_bk[wid] = bk;
    s_bv[wid] = bv;
  }
  __syncthreads();
  bk = -1;
  bv = 0;
  for (int w = 0; w < nw; ++w) {
    const int32_t ok = s_bk[w];
    const unsigned long long ov = s_bv[w];
    if (ok >= 0 && (bk < 0 || ov > bv || (ov == bv && ok < bk))) {
      bv = ov;
      bk = ok;
    }
  }
  __syncthreads();
  return bk;
}

// One-vertex sub-rounds x0..x1 in order, by one block: no swaps, and a proposal always fits (it was
// rated only if c(C) + c(u) <= cmax), so the vertex moves at once.  Dynamic shared memory: kHeavySmem.
__global__ void __launch_bounds__(kHeavyWarps * 32) k_cl_serial(jet_hypergraph g, const int32_t *order, int32_t x0, int32_t x1,
                                                   long long cmax, int32_t rmax, Cl cl, Tab *pool) {
  extern __shared__ unsigned long long s_dyn[];
  __shared__ int32_t s_bk[kHeavyWarps];
  __shared__ unsigned long long s_bv[kHeavyWarps];
  __shared__ int s_next[2];
  Tab *s_tab = reinterpret_cast<Tab *>(s_dyn);
  int32_t *s_set = reinterpret_cast<int32_t *>(s_tab + kBlockTab);
  for (int32_t x = x0; x < x1; ++x) {
    const int32_t u = order[x];
    if (cl.csize[u] != 1 || cl.label[u] != u) continue;
    const int32_t cap = cl.cap[u];
    const int32_t j = rate_block(g, u, cl.label, cl.cw, cmax, rmax, cap <= kBlockTab ? s_tab : pool, cap, s_set,
                                 s_bk, s_bv, s_next);
    if (j >= 0 && threadIdx.x == 0) {
      const long long c = g.vwgt[u];
      cl.label[u] = j;
      cl.cw[j] += c;
      cl.cw[u] -= c;
      cl.csize[j] += 1;
      cl.csize[u] -= 1;
    }
    __syncthreads();
  }
}

// Warp per position of the sub-round: the vertices of tables up to kWarpTab entries (in the warp's
// shared slice, else a slice of the global pool).
__global__ void __launch_bounds__(256) k_cl_rate(jet_hypergraph g, const int32_t *order, int32_t a, int32_t b,
                                                 long long cmax, int32_t rmax, Cl cl, Tab *pool,
                                                 unsigned long long *ctr) {
  __shared__ Tab s_tab[8][kSmemTab];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t x = a + blockIdx.x * 8ll + wid;
  if (x >= b) return;
  const int32_t u = order[x];
  const int32_t cap = cl.cap[u];
  if (cap > kWarpTab || cl.csize[u] != 1 || cl.label[u] != u) return;
  Tab *tab = s_tab[wid];
  if (cap > kSmemTab) {
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(ctr, (unsigned long long)cap);
    tab = pool + __shfl_sync(kFull, off, 0);
  }
  const int32_t j = rate_vertex(g, u, cl.label, cl.cw, cmax, rmax, tab, cap, lane);
  if (lane == 0 && j >= 0) {
    cl.T[u] = j;
    atomicAdd(reinterpret_cast<unsigned long long *>(&cl.pw[j]), (unsigned long long)g.vwgt[u]);
  }
}

// Block per heavy position of the sub-round (hpos).  Dynamic shared memory: kHeavySmem.
__global__ void __launch_bounds__(kHeavyWarps * 32) k_cl_rate_heavy(jet_hypergraph g, const int32_t *order, const int32_t *hpos,
                                                       long long cmax, int32_t rmax, Cl cl, Tab *pool,
                                                       unsigned long long *ctr) {
  extern __shared__ unsigned long long s_dyn[];
  __shared__ int32_t s_bk[kHeavyWarps];
  __shared__ unsigned long long s_bv[kHeavyWarps];
  __shared__ unsigned long long s_off;
  __shared__ int s_next[2];
  const int32_t u = order[hpos[blockIdx.x]];
  if (cl.csize[u] != 1 || cl.label[u] != u) return;
  const int32_t cap = cl.cap[u];
  Tab *tab = reinterpret_cast<Tab *>(s_dyn);
  int32_t *s_set = reinterpret_cast<int32_t *>(tab + kBlockTab);
  if (cap > kBlockTab) {
    if (threadIdx.x == 0) s_off = atomicAdd(ctr, (unsigned long long)cap);
    __syncthreads();
    tab = pool + s_off;
  }
  const int32_t j = rate_block(g, u, cl.label, cl.cw, cmax, rmax, tab, cap, s_set, s_bk, s_bv, s_next);
  if (threadIdx.x == 0 && j >= 0) {
    cl.T[u] = j;
    atomicAdd(reinterpret_cast<unsigned long long *>(&cl.pw[j]), (unsigned long long)g.vwgt[u]);
  }
}

__global__ void k_cl_swap(const int32_t *vwgt, const int32_t *order, int32_t a, int32_t b, Cl cl) {
  const int64_t x = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= b) return;
  const int32_t u = order[x];
  const int32_t v = cl.T[u];
  int32_t t2 = v;
  if (v >= 0 && cl.T[v] == u) {
    const long long wu = vwgt[u] + cl.pw[u] - vwgt[v];
    const long long wv = vwgt[v] + cl.pw[v] - vwgt[u];
    if (wu > wv || (wu == wv && u < v)) t2 = -1;  // u stays, v joins u
  }
  cl.T2[u] = t2;
  if (t2 >= 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&cl.pw2[t2]), (unsigned long long)vwgt[u]);
    cl.next[u] = atomicExch(&cl.head[t2], u);
  }
}

__global__ void k_cl_approve(const int32_t *vwgt, const int32_t *order, int32_t a, int32_t b, long long cmax, Cl cl) {
  const int64_t x = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= b) return;
  const int32_t u = order[x];
  const int32_t j = cl.T2[u];
  if (j < 0) return;
  const long long room = cmax - cl.cw[j];
  bool ok = cl.pw2[j] <= room;
  if (!ok) {  // the proposers before u in (weight, id) order, and u itself, must fit
    const int32_t cu = vwgt[u];
    long long s = cu;
    for (int32_t w = cl.head[j]; w >= 0 && s <= room; w = cl.next[w]) {
      const int32_t c = vwgt[w];
      if (c < cu || (c == cu && w < u)) s += c;
    }
    ok = s <= room;
  }
  cl.acc[u] = ok ? 1 : 0;
}

__global__ void k_cl_apply(const int32_t *vwgt, const int32_t *order, int32_t a, int32_t b, Cl cl) {
  const int64_t x = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= b) return;
  const int32_t u = order[x];
  const int32_t t = cl.T[u], j = cl.T2[u];
  if (j >= 0 && cl.acc[u]) {
    const long long c = vwgt[u];
    cl.label[u] = j;
    atomicAdd(reinterpret_cast<unsigned long long *>(&cl.cw[j]), (unsigned long long)c);
    atomicAdd(reinterpret_cast<unsigned long long *>(&cl.cw[u]), (unsigned long long)(-c));
    atomicAdd(&cl.csize[j], 1);
    atomicAdd(&cl.csize[u], -1);
  }
  if (t >= 0) cl.pw[t] = 0;
  if (j >= 0) {
    cl.pw2[j] = 0;
    cl.head[j] = -1;
  }
  cl.T[u] = cl.T2[u] = -1;
  cl.acc[u] = 0;
}

// ------------------------------------------------------------------ contraction

__global__ void k_check_labels(const int32_t *label, int32_t n, int64_t *used, int *err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = label[v];
    if ((unsigned)l >= (unsigned)n) atomicOr(err, 16);
    else used[l] = 1;
  }
}

__global__ void k_ct_map(const int32_t *label, const int32_t *vwgt, int32_t n, const int64_t *cid, int32_t *map,
                         long long *cvw) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)cid[label[v]];
    map[v] = c;
    atomicAdd(reinterpret_cast<unsigned long long *>(&cvw[c]), (unsigned long long)vwgt[v]);
  }
}

__global__ void k_ct_vwgt(const long long *cvw, int32_t nc, int32_t *out, int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const long long w = cvw[c];
    if (w > INT32_MAX) atomicOr(err, 32);
    out[c] = (int32_t)w;
  }
}

// keys[p] = e * nc + map[pin] for every pin p of edge e (warp per edge).
__global__ void k_ct_keys(jet_hypergraph g, const int32_t *map, int32_t nc, unsigned long long *keys) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += warps) {
    const unsigned long long base = (unsigned long long)e * (unsigned long long)nc;
    for (int64_t p = g.eptr[e] + lane; p < g.eptr[e + 1]; p += 32) keys[p] = base + (unsigned)map[g.pins[p]];
  }
}

// Per edge (warp), from its sorted keys: the distinct coarse pins written ascending at the front of
// the edge's range in tpins, their number, and an order-independent hash of the set.
__global__ void k_ct_distinct(jet_hypergraph g, int32_t nc, const unsigned long long *keys, int32_t *tpins,
                              int32_t *cnt, unsigned long long *hash) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += warps) {
    const int64_t p0 = g.eptr[e], p1 = g.eptr[e + 1];
    const unsigned long long base = (unsigned long long)e * (unsigned long long)nc;
    int32_t run = 0;
    unsigned long long h = 0;
    for (int64_t p = p0; p < p1; p += 32) {
      const int64_t q = p + lane;
      bool fresh = false;
      int32_t c = 0;
      if (q < p1) {
        const unsigned long long k = keys[q];
        c = (int32_t)(k - base);
        fresh = q == p0 || keys[q - 1] != k;
      }
      const unsigned bal = __ballot_sync(kFull, fresh);
      if (fresh) {
        tpins[p0 + run + __popc(bal & ((1u << lane) - 1))] = c;
        h += mix64((unsigned long long)(uint32_t)c + 0x9e3779b97f4a7c15ull);
      }
      run += __popc(bal);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(kFull, h, o);
    if (lane == 0) {
      cnt[e] = run;
      hash[e] = h;
    }
  }
}

// Sort key of an edge for finding equal pin sets: 63 - ebits bits of hash, then the edge id;
// edges with fewer than two coarse pins get ~0 and sort last.
__global__ void k_ct_hkeys(int32_t m, int ebits, const int32_t *cnt, const unsigned long long *hash,
                           unsigned long long *hkeys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    if (cnt[e] < 2) {
      hkeys[e] = ~0ull;
      continue;
    }
    const unsigned long long hv = mix64(hash[e] ^ ((unsigned long long)cnt[e] << 40)) & 0x7fffffffffffffffull;
    hkeys[e] = ((hv >> ebits) << ebits) | (unsigned long long)e;
  }
}

__device__ bool same_pins(const int64_t *eptr, const int32_t *tpins, const int32_t *cnt, int32_t a, int32_t b) {
  if (cnt[a] != cnt[b]) return false;
  const int32_t *pa = tpins + eptr[a], *pb = tpins + eptr[b];
  for (int32_t i = 0; i < cnt[a]; ++i)
    if (pa[i] != pb[i]) return false;
  return true;
}

// Runs of equal hash (edge ids ascending within a run): the first thread of a run walks it and maps
// every edge to the first earlier edge of the run with the same pin set (itself if none), adding
// its weight there.
__global__ void k_ct_runs(int32_t m, int ebits, const unsigned long long *hkeys, const int64_t *eptr,
                          const int32_t *tpins, const int32_t *cnt, const int32_t *ewgt, int32_t *rep,
                          long long *ew) {
  const unsigned long long emask = (1ull << ebits) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = hkeys[i];
    if (k == ~0ull) continue;
    if (i > 0 && (hkeys[i - 1] >> ebits) == (k >> ebits)) continue;  // not the first of its run
    for (int64_t j = i; j < m && hkeys[j] != ~0ull && (hkeys[j] >> ebits) == (k >> ebits); ++j) {
      const int32_t e = (int32_t)(hkeys[j] & emask);
      int32_t r = e;
      for (int64_t q = i; q < j; ++q) {
        const int32_t f = (int32_t)(hkeys[q] & emask);
        if (rep[f] == f && same_pins(eptr, tpins, cnt, f, e)) {
          r = f;
          break;
        }
      }
      rep[e] = r;
      atomicAdd(reinterpret_cast<unsigned long long *>(&ew[r]), (unsigned long long)ewgt[e]);
    }
  }
}

__global__ void k_ct_keep(int32_t m, const int32_t *cnt, const int32_t *rep, int64_t *kf, int64_t *sz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const bool keep = cnt[e] >= 2 && rep[e] == e;
    kf[e] = keep ? 1 : 0;
    sz[e] = keep ? cnt[e] : 0;
  }
}

// Warp per kept edge: its coarse row, weight, and the (coarse vertex, coarse edge) incidence keys.
__global__ void k_ct_write(int32_t m, const int64_t *eptr, const int32_t *tpins, const int32_t *cnt,
                           const int32_t *rep, const long long *ew, const int64_t *ceid, const int64_t *cpos,
                           int32_t mc, int64_t pc, jet_hypergraph_out out, unsigned long long *ikeys, int *err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w0 == 0 && lane == 0) out.eptr[mc] = pc;
  for (int64_t e = w0; e < m; e += warps) {
    if (cnt[e] < 2 || rep[e] != e) continue;
    const int32_t f = (int32_t)ceid[e];
    const int64_t o = cpos[e];
    if (lane == 0) {
      out.eptr[f] = o;
      if (ew[e] > INT32_MAX) atomicOr(err, 32);
      out.ewgt[f] = (int32_t)ew[e];
    }
    for (int32_t i = lane; i < cnt[e]; i += 32) {
      const int32_t c = tpins[eptr[e] + i];
      out.pins[o + i] = c;
      ikeys[o + i] = (unsigned long long)c * (unsigned long long)mc + (unsigned)f;
    }
  }
}

// From the incidence keys sorted by (coarse vertex, coarse edge): inc, and vptr at the boundaries.
__global__ void k_ct_inc(const unsigned long long *ikeys, int64_t pc, int32_t mc, int32_t nc,
                         jet_hypergraph_out out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pc; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = ikeys[p];
    const int64_t c = (int64_t)(k / (unsigned long long)mc);
    out.inc[p] = (int32_t)(k - (unsigned long long)c * (unsigned long long)mc);
    const int64_t prev = p == 0 ? -1 : (int64_t)(ikeys[p - 1] / (unsigned long long)mc);
    for (int64_t x = prev + 1; x <= c; ++x) out.vptr[x] = p;
    if (p == pc - 1)
      for (int64_t x = c + 1; x <= nc; ++x) out.vptr[x] = pc;
  }
}

__global__ void k_fill_i64(int64_t *a, int64_t n, int64_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// ------------------------------------------------------------------ host side

int sms_of_current_device() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Stream-ordered scratch of one call, released at the end.
struct Scratch {
  cudaStream_t s;
  std::vector<void *> blocks;
  cudaError_t err = cudaSuccess;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  T *get(int64_t count) {
    void *p = nullptr;
    const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    const cudaError_t e = jet::pool_alloc(&p, bytes, s);
    if (e != cudaSuccess) {
      if (err == cudaSuccess) err = e;
      return nullptr;
    }
    blocks.push_back(p);
    return static_cast<T *>(p);
  }
  ~Scratch() {
    for (void *p : blocks) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  }
};

int gfail(int code, const char *fmt, const char *what) {
  set_global_error(fmt, what);
  return code;
}

int cuda_error(cudaError_t e, const char *where) {
  set_global_error("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? JET_ERR_OOM : JET_ERR_CUDA;
}

int check_hg_args(const jet_hypergraph *hg) {
  if (!hg) return gfail(JET_ERR_INVALID_ARG, "%s", "hypergraph is NULL");
  if (hg->n < 0 || hg->m < 0 || hg->P < 0) return gfail(JET_ERR_INVALID_ARG, "%s", "negative size");
  if (!hg->eptr || !hg->vptr || (hg->n > 0 && !hg->vwgt) || (hg->m > 0 && !hg->ewgt) ||
      (hg->P > 0 && (!hg->pins || !hg->inc)))
    return gfail(JET_ERR_INVALID_ARG, "%s", "NULL array");
  return JET_OK;
}

// Runs a CSR check and returns JET_ERR_DATA if the hypergraph is malformed.
int validate_hg(const jet_hypergraph *hg, int *d_err, cudaStream_t s, int sms) {
  const int64_t items = std::max<int64_t>(std::max<int64_t>(hg->P, hg->m), hg->n);
  k_check_hg<<<grid_for(items, 256, sms, 4), 256, 0, s>>>(*hg, d_err);
  int h_err = 0;
  cudaError_t e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "validation");
  if (h_err) return gfail(JET_ERR_DATA, "%s", "malformed hypergraph (CSR offsets, index or weight out of range)");
  return JET_OK;
}

std::vector<int32_t> subround_bounds(int32_t n, int32_t single, int32_t cap_div) {
  int64_t cap = n / std::max(cap_div, 1);
  if (cap < 1) cap = 1;
  std::vector<int32_t> b;
  int64_t pos = 0, size = 1, r = 0;
  while (pos < n) {
    if (r < single) size = 1;
    else if (r == single) size = 2;
    else size *= 2;
    if (size > cap) size = cap;
    b.push_back((int32_t)pos);
    pos += std::min<int64_t>(size, n - pos);
    ++r;
  }
  b.push_back(n);
  return b;
}

}  // namespace
}  // namespace jet

using namespace jet;

extern "C" {

int jet_cluster(const jet_hypergraph *hg, const jet_coarsen_params *p, const int32_t *order, int32_t *label,
                void *stream) {
  int rc = check_hg_args(hg);
  if (rc != JET_OK) return rc;
  if (!p || (hg->n > 0 && (!order || !label))) return gfail(JET_ERR_INVALID_ARG, "%s", "NULL argument");
  if (p->max_cluster_weight < 1 || p->rating_max_edge < 2 || p->single_subrounds < 0 || p->subround_cap_div < 1)
    return gfail(JET_ERR_INVALID_ARG, "%s", "bad coarsening parameters");
  const int32_t n = hg->n;
  if (n == 0) return JET_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = sms_of_current_device();
  Scratch sc(s);
  int *d_err = sc.get<int>(1);
  Cl cl;
  cl.label = label;
  cl.cw = sc.get<long long>(n);
  cl.csize = sc.get<int32_t>(n);
  cl.T = sc.get<int32_t>(n);
  cl.T2 = sc.get<int32_t>(n);
  cl.pw = sc.get<long long>(n);
  cl.pw2 = sc.get<long long>(n);
  cl.head = sc.get<int32_t>(n);
  cl.next = sc.get<int32_t>(n);
  cl.acc = sc.get<uint8_t>(n);
  cl.cap = sc.get<int32_t>(n);
  const std::vector<int32_t> bounds = subround_bounds(n, p->single_subrounds, p->subround_cap_div);
  const int32_t rounds = (int32_t)bounds.size() - 1;
  int32_t *d_bounds = sc.get<int32_t>((int64_t)bounds.size());
  // per sub-round: pool entries, pool cursor, heavy count, heavy cursor
  unsigned long long *d_need = sc.get<unsigned long long>(4 * (int64_t)rounds);
  int64_t *d_hoff = sc.get<int64_t>(rounds);
  if (sc.err != cudaSuccess) return cuda_error(sc.err, "jet_cluster: workspace");
  unsigned long long *d_ctr = d_need + rounds, *d_heavy = d_need + 2 * rounds, *d_hcur = d_need + 3 * rounds;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_need, 0, sizeof(unsigned long long) * 4 * (size_t)rounds, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_bounds, bounds.data(), sizeof(int32_t) * bounds.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cl.T, 0, sizeof(int32_t) * (size_t)n, s);  // "seen" of the order check
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cl_serial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeavySmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cl_rate_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeavySmem);
  if (e != cudaSuccess) return cuda_error(e, "jet_cluster");
  rc = validate_hg(hg, d_err, s, sms);
  if (rc != JET_OK) return rc;
  const int g = grid_for(n, 256, sms, 4);
  k_check_order<<<g, 256, 0, s>>>(order, n, cl.T, d_err);
  k_cl_setup<<<g, 256, 0, s>>>(*hg, p->rating_max_edge, cl, d_err);
  k_cl_need<<<g, 256, 0, s>>>(order, n, d_bounds, rounds, cl.cap, d_need, d_heavy);
  int h_err = 0;
  std::vector<unsigned long long> need(rounds), heavy(rounds);
  e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(need.data(), d_need, sizeof(unsigned long long) * (size_t)rounds, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(heavy.data(), d_heavy, sizeof(unsigned long long) * (size_t)rounds, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "jet_cluster: set-up");
  if (h_err & 2) return gfail(JET_ERR_DATA, "%s", "order is not a permutation of the vertices");
  if (h_err & 4) return gfail(JET_ERR_OVERFLOW, "%s", "a vertex's rating sum reaches 2^63");
  if (h_err & 8) return gfail(JET_ERR_OVERFLOW, "%s", "a vertex's rated neighbourhood exceeds 2^27 pins");
  unsigned long long pool_entries = 1;
  for (unsigned long long x : need) pool_entries = std::max(pool_entries, x);
  std::vector<int64_t> hoff(rounds);
  int64_t n_heavy = 0;
  for (int32_t q = 0; q < rounds; ++q) {
    hoff[q] = n_heavy;
    n_heavy += (int64_t)heavy[q];
  }
  Tab *pool = sc.get<Tab>((int64_t)pool_entries);
  int32_t *hpos = sc.get<int32_t>(n_heavy);
  if (sc.err != cudaSuccess) return cuda_error(sc.err, "jet_cluster: rating tables");
  e = cudaMemcpyAsync(d_hoff, hoff.data(), sizeof(int64_t) * (size_t)rounds, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "jet_cluster");
  if (n_heavy > 0) k_cl_heavy_list<<<g, 256, 0, s>>>(order, n, d_bounds, rounds, cl.cap, d_hoff, d_hcur, hpos);
  // leading one-vertex sub-rounds: one block, in order
  int32_t r = 0;
  while (r < rounds && bounds[r + 1] - bounds[r] == 1) ++r;
  if (r > 0) k_cl_serial<<<1, kHeavyWarps * 32, kHeavySmem, s>>>(*hg, order, bounds[0], bounds[r], p->max_cluster_weight,
                                                    p->rating_max_edge, cl, pool);
  for (; r < rounds; ++r) {
    const int32_t a = bounds[r], b = bounds[r + 1];
    const unsigned gw = (unsigned)((b - a + 7) / 8), gt = (unsigned)((b - a + 255) / 256);
    k_cl_rate<<<gw, 256, 0, s>>>(*hg, order, a, b, p->max_cluster_weight, p->rating_max_edge, cl, pool, d_ctr + r);
    if (heavy[r] > 0)
      k_cl_rate_heavy<<<(unsigned)heavy[r], kHeavyWarps * 32, kHeavySmem, s>>>(*hg, order, hpos + hoff[r], p->max_cluster_weight,
                                                                  p->rating_max_edge, cl, pool, d_ctr + r);
    k_cl_swap<<<gt, 256, 0, s>>>(hg->vwgt, order, a, b, cl);
    k_cl_approve<<<gt, 256, 0, s>>>(hg->vwgt, order, a, b, p->max_cluster_weight, cl);
    k_cl_apply<<<gt, 256, 0, s>>>(hg->vwgt, order, a, b, cl);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "jet_cluster");
  return JET_OK;
}

int jet_contract(const jet_hypergraph *hg, const int32_t *label, int32_t *map, const jet_hypergraph_out *out,
                 int32_t *n_out, int32_t *m_out, int64_t *P_out, void *stream) {
  int rc = check_hg_args(hg);
  if (rc != JET_OK) return rc;
  if (!out || !n_out || !m_out || !P_out || (hg->n > 0 && (!label || !map)))
    return gfail(JET_ERR_INVALID_ARG, "%s", "NULL argument");
  if (!out->eptr || !out->vptr || (hg->n > 0 && !out->vwgt) || (hg->m > 0 && !out->ewgt) ||
      (hg->P > 0 && (!out->pins || !out->inc)))
    return gfail(JET_ERR_INVALID_ARG, "%s", "NULL output array");
  *n_out = 0;
  *m_out = 0;
  *P_out = 0;
  const int32_t n = hg->n, m = hg->m;
  const int64_t P = hg->P;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sms = sms_of_current_device();
  Scratch sc(s);
  int *d_err = sc.get<int>(1);
  int64_t *d_tot = sc.get<int64_t>(2);
  int64_t *cid = sc.get<int64_t>((int64_t)n);
  const int64_t big = std::max<int64_t>(std::max<int64_t>(P, m), n);
  int64_t *scan_tmp = sc.get<int64_t>(scan_tiles(sort_hist_entries(big)) + 1);
  if (sc.err != cudaSuccess) return cuda_error(sc.err, "jet_contract: workspace");
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cid, 0, sizeof(int64_t) * (size_t)std::max(n, 1), s);
  if (e != cudaSuccess) return cuda_error(e, "jet_contract");
  rc = validate_hg(hg, d_err, s, sms);
  if (rc != JET_OK) return rc;
  if (n == 0) {
    e = cudaMemsetAsync(out->eptr, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out->vptr, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? JET_OK : cuda_error(e, "jet_contract");
  }
  // coarse vertices: the used labels, in label order
  const int gn = grid_for(n, 256, sms, 4);
  k_check_labels<<<gn, 256, 0, s>>>(label, n, cid, d_err);
  e = scan_exclusive(cid, cid, n, scan_tmp, d_tot, s);
  int h_err = 0;
  int64_t nc64 = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nc64, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "jet_contract: coarse vertices");
  if (h_err & 16) return gfail(JET_ERR_DATA, "%s", "a label is outside [0, n)");
  const int32_t nc = (int32_t)nc64;
  long long *cvw = sc.get<long long>(nc);
  unsigned long long *keys = sc.get<unsigned long long>(std::max<int64_t>(P, m));
  SortBufs sb;
  sb.tmp = sc.get<unsigned long long>(std::max<int64_t>(P, m));
  sb.hist = sc.get<int64_t>(sort_hist_entries(big));
  sb.scan_tmp = scan_tmp;
  int32_t *tpins = sc.get<int32_t>(P);
  int32_t *cnt = sc.get<int32_t>(m);
  unsigned long long *hash = sc.get<unsigned long long>(m);
  int32_t *rep = sc.get<int32_t>(m);
  long long *ew = sc.get<long long>(m);
  int64_t *kf = sc.get<int64_t>(m);
  int64_t *sz = sc.get<int64_t>(m);
  if (sc.err != cudaSuccess) return cuda_error(sc.err, "jet_contract: workspace");
  e = cudaMemsetAsync(cvw, 0, sizeof(long long) * (size_t)std::max(nc, 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ew, 0, sizeof(long long) * (size_t)std::max(m, 1), s);
  if (e != cudaSuccess) return cuda_error(e, "jet_contract");
  k_ct_map<<<gn, 256, 0, s>>>(label, hg->vwgt, n, cid, map, cvw);
  k_ct_vwgt<<<grid_for(nc, 256, sms, 4), 256, 0, s>>>(cvw, nc, out->vwgt, d_err);
  int64_t mc64 = 0, pc = 0;
  if (m > 0) {
    // distinct coarse pins of every edge: sort (edge, coarse pin) keys
    const int gw = grid_for((int64_t)m * 32, 256, sms, 8);
    k_ct_keys<<<gw, 256, 0, s>>>(*hg, map, nc, keys);
    e = radix_sort(keys, P, bits_for((unsigned long long)m * (unsigned long long)nc - 1), sb, s);
    if (e != cudaSuccess) return cuda_error(e, "jet_contract: pin sort");
    k_ct_distinct<<<gw, 256, 0, s>>>(*hg, nc, keys, tpins, cnt, hash);
    // equal pin sets: sort edges by (hash, id), walk the runs
    const int ebits = std::max(bits_for((unsigned long long)m - 1), 1);
    k_ct_hkeys<<<grid_for(m, 256, sms, 4), 256, 0, s>>>(m, ebits, cnt, hash, keys);
    e = radix_sort(keys, m, 64, sb, s);
    if (e != cudaSuccess) return cuda_error(e, "jet_contract: edge sort");
    k_ct_runs<<<grid_for(m, 256, sms, 4), 256, 0, s>>>(m, ebits, keys, hg->eptr, tpins, cnt, hg->ewgt, rep, ew);
    k_ct_keep<<<grid_for(m, 256, sms, 4), 256, 0, s>>>(m, cnt, rep, kf, sz);
    e = scan_exclusive(kf, kf, m, scan_tmp, d_tot, s);
    if (e == cudaSuccess) e = scan_exclusive(sz, sz, m, scan_tmp, d_tot + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mc64, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&pc, d_tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "jet_contract: coarse edges");
  }
  const int32_t mc = (int32_t)mc64;
  if (mc > 0) {
    // rows, weights and incidence keys; the incidences sorted by (coarse vertex, coarse edge)
    k_ct_write<<<grid_for((int64_t)m * 32, 256, sms, 8), 256, 0, s>>>(m, hg->eptr, tpins, cnt, rep, ew, kf, sz, mc,
                                                                       pc, *out, keys, d_err);
    e = radix_sort(keys, pc, bits_for((unsigned long long)nc * (unsigned long long)mc - 1), sb, s);
    if (e != cudaSuccess) return cuda_error(e, "jet_contract: incidence sort");
    k_ct_inc<<<grid_for(pc, 256, sms, 4), 256, 0, s>>>(keys, pc, mc, nc, *out);
  } else {
    e = cudaMemsetAsync(out->eptr, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_error(e, "jet_contract");
    k_fill_i64<<<grid_for((int64_t)nc + 1, 256, sms, 4), 256, 0, s>>>(out->vptr, (int64_t)nc + 1, 0);
  }
  e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "jet_contract");
  if (h_err & 32) return gfail(JET_ERR_OVERFLOW, "%s", "a coarse vertex or edge weight leaves int32");
  *n_out = nc;
  *m_out = mc;
  *P_out = pc;
  return JET_OK;
}

}  // extern "C"
