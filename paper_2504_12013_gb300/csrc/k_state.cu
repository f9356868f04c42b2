// State kernels: input validation, size classes, pin counts phi_e[i] with
// their connectivity bitmasks, block weights, and the connectivity metric
// (lambda-1) of Section 2.
#include <vector>

#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void add_i64(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Sum of a long long over the block, returned on thread 0.
__device__ long long block_sum_ll(long long x) {
  __shared__ long long s_part[32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_part[w] = x;
  __syncthreads();
  long long tot = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += s_part[i];
  __syncthreads();
  return tot;
}

// ---------------------------------------------------------------- validation
// Phase 1: offsets monotone and in range, weights positive and bounded.
__global__ void k_validate_offsets(const int64_t *eptr, const int64_t *vptr, const int32_t *vwgt,
                                   const int32_t *ewgt, int32_t n, int32_t m, int64_t P, Counters *cnt) {
  int err = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)m + n + 2;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i <= m) {  // eptr[i]
      int64_t a = eptr[i];
      if (a < 0 || a > P) err |= kErrOffsets;
      if (i == 0 && a != 0) err |= kErrOffsets;
      if (i == m && a != P) err |= kErrOffsets;
      if (i < m && eptr[i + 1] < a) err |= kErrOffsets;
      if (i < m && ewgt[i] < 1) err |= kErrWeight;
    } else {
      int64_t v = i - m - 1;  // vptr[v], v in [0, n]
      int64_t a = vptr[v];
      if (a < 0 || a > P) err |= kErrOffsets;
      if (v == 0 && a != 0) err |= kErrOffsets;
      if (v == n && a != P) err |= kErrOffsets;
      if (v < n && vptr[v + 1] < a) err |= kErrOffsets;
      if (v < n && vwgt[v] < 1) err |= kErrWeight;
    }
  }
  if (err) atomicOr(&cnt->err, err);
}

// Phase 2: pin and incidence ids in range; occurrences of every vertex among the pins.
__global__ void k_validate_ids(const int32_t *pins, const int32_t *inc, int32_t n, int32_t m, int64_t P,
                               int32_t *degcount, Counters *cnt) {
  int err = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = pins[p];
    if (v < 0 || v >= n) err |= kErrPinRange;
    else atomicAdd(&degcount[v], 1);
    int32_t e = inc[p];
    if (e < 0 || e >= m) err |= kErrIncRange;
  }
  if (err) atomicOr(&cnt->err, err);
}

// Phase 3: degree of the transpose, weighted degree sum of omega over I(v), c(V), max c(v).
// scal[0] = c(V), scal[1] = max weighted degree, scal[2] = max c(v),
// scal[3] = max omega(e) over edges with at least one pin.
__global__ void k_validate_degrees(const int64_t *vptr, const int32_t *inc, const int32_t *vwgt,
                                   const int32_t *ewgt, int32_t n, const int32_t *degcount, int64_t *wdeg,
                                   unsigned long long *scal, Counters *cnt) {
  int err = 0;
  long long wsum = 0;
  unsigned long long wmax = 0, cm = 0, om = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t j0 = vptr[v], j1 = vptr[v + 1];
    if (j1 - j0 != degcount[v]) err |= kErrTranspose;
    long long d = 0;
    for (int64_t j = j0; j < j1; ++j) {
      const int32_t w = ewgt[inc[j]];
      d += w;
      om = (unsigned long long)w > om ? (unsigned long long)w : om;
    }
    wdeg[v] = d;
    wmax = d > (long long)wmax ? (unsigned long long)d : wmax;
    int32_t c = vwgt[v];
    wsum += c;
    cm = (unsigned long long)c > cm ? (unsigned long long)c : cm;
  }
  long long tot = block_sum_ll(wsum);
  if (threadIdx.x == 0) atomicAdd(&scal[0], (unsigned long long)tot);
  atomicMax(&scal[1], wmax);
  atomicMax(&scal[2], cm);
  atomicMax(&scal[3], om);
  if (err) atomicOr(&cnt->err, err);
}

// ---------------------------------------------------------------- classes
// Stable partition of ids [0, count) by class code (0 .. kClasses-1).
constexpr int kClasses = 24;
static_assert(kClasses < 32, "class codes and the no-class code fit match_bits<5>");

__global__ void k_class_count(const uint8_t *code, int32_t count, int32_t *blk_counts) {
  __shared__ int s_c[kClasses];
  if (threadIdx.x < kClasses) s_c[threadIdx.x] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c = i < count ? code[i] : kClasses;
  const unsigned grp = match_bits<5>((unsigned)c);  // c <= kClasses < 32
  if (c < kClasses && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&s_c[c], __popc(grp));
  __syncthreads();
  if (threadIdx.x < kClasses) blk_counts[blockIdx.x * kClasses + threadIdx.x] = s_c[threadIdx.x];
}

__global__ void k_class_scatter(const uint8_t *code, int32_t count, const int32_t *blk_off, int32_t *out) {
  __shared__ int s_w[32][kClasses];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int x = threadIdx.x; x < 32 * kClasses; x += blockDim.x) s_w[x / kClasses][x % kClasses] = 0;
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c = i < count ? code[i] : kClasses;
  const unsigned grp = match_bits<5>((unsigned)c);  // c <= kClasses < 32
  const unsigned rank = __popc(grp & ((1u << lane) - 1));
  if (c < kClasses && lane == __ffs(grp) - 1) s_w[w][c] = __popc(grp);
  __syncthreads();
  if (c < kClasses) {
    int base = blk_off[blockIdx.x * kClasses + c];
    for (int ww = 0; ww < w; ++ww) base += s_w[ww][c];
    out[base + rank] = (int32_t)i;
  }
}

__global__ void k_vertex_codes(const int64_t *wdeg, int32_t n, uint8_t *code) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    code[v] = wdeg[v] < (1ll << kLightPlanes) ? 0 : 1;
}

// Edge classes: code = |e| for |e| <= kTinyEdge (so the tiny list comes out
// ordered by size and a warp's edges tend to share one size); then the warp
// class split into edges of at most kHalfMidEdge and of at most
// kSmallMidEdge pins (one code each) and larger ones by size bucket, largest
// first, so the warps that get the longest edges start first; then the block
// class.
__global__ void k_edge_codes(const int64_t *eptr, int32_t m, uint8_t *code) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sz = eptr[e + 1] - eptr[e];
    int c;
    if (sz <= kTinyEdge) c = (int)sz;
    else if (sz <= kHalfMidEdge) c = kTinyEdge + 1;
    else if (sz <= kSmallMidEdge) c = kTinyEdge + 2;
    else if (sz <= kWarpEdge) c = sz > 64 ? kTinyEdge + 3 : kTinyEdge + 4;  // 65..128 first, then 33..64
    else c = kTinyEdge + 5;
    code[e] = (uint8_t)c;
  }
}

// ---------------------------------------------------------------- pin counts
// Warp per edge: histogram of the pins' blocks in shared memory, then one
// coalesced store of the phi row and one ballot per mask word.  An edge longer
// than one segment (kSegPins pins: the hub rows of a row-net) would hold its
// warp for thousands of steps; its warp only clears the row, and
// k_pincounts_seg and k_masks_from_phi complete it.
__global__ void __launch_bounds__(256) k_pincounts(const int64_t *eptr, const int32_t *pins, const int32_t *part,
                                                   int32_t m, int32_t k, int32_t kwp, int32_t *phi, uint32_t *mask,
                                                   Counters *cnt) {
  extern __shared__ int s_hist[];
  const int lane = threadIdx.x & 31;
  int *h = s_hist + (threadIdx.x >> 5) * k;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int err = 0;
  for (int64_t e = gw; e < m; e += nw) {
    const int64_t p0 = eptr[e], p1 = eptr[e + 1];
    if (p1 - p0 > kSegPins) {  // warp-uniform
      for (int b = lane; b < k; b += 32) phi[e * k + b] = 0;
      continue;
    }
    for (int b = lane; b < k; b += 32) h[b] = 0;
    __syncwarp();
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      int b = part[pins[p]];
      if ((unsigned)b < (unsigned)k) atomicAdd(&h[b], 1);
      else err |= kErrPartRange;
    }
    __syncwarp();
    int32_t *row = phi + e * k;
    for (int q = 0; q < kwp; ++q) {
      int b = q * 32 + lane;
      int val = b < k ? h[b] : 0;
      if (b < k) row[b] = val;
      const unsigned one = __ballot_sync(kFull, val > 0), two = __ballot_sync(kFull, val > 1);
      if (lane == 0) {
        mask[e * 2 * kwp + q] = one;        // Lambda(e)
        mask[e * 2 * kwp + kwp + q] = two;  // blocks holding >= 2 pins of e
      }
    }
    __syncwarp();
  }
  if (err) atomicOr(&cnt->err, err);
}

// The edges longer than one segment: a thread block per segment of at most
// kSegPins pins (the afterburner's segment list, whose slot field is >= 0 for
// exactly these edges) counts the blocks of its pins in shared memory and adds
// the counts into the edge's row, cleared by k_pincounts: one atomic per block
// of the partition that the segment touches.
__global__ void __launch_bounds__(256) k_pincounts_seg(const int64_t *eptr, const int32_t *pins, const int32_t *part,
                                                       const int4 *seg, int32_t nseg, int32_t k, int32_t *phi,
                                                       Counters *cnt) {
  __shared__ int s_h[kMaxK];
  int err = 0;
  for (int i = blockIdx.x; i < nseg; i += gridDim.x) {
    const int4 sg = seg[i];  // edge, first pin (offset in the edge), pins, slot
    if (sg.w < 0) continue;  // a one-segment edge: counted by k_pincounts (block-uniform)
    for (int b = threadIdx.x; b < k; b += blockDim.x) s_h[b] = 0;
    __syncthreads();
    const int64_t p0 = eptr[sg.x] + sg.y;
#pragma unroll 4
    for (int j = threadIdx.x; j < sg.z; j += blockDim.x) {
      const int b = part[pins[p0 + j]];
      if ((unsigned)b < (unsigned)k) atomicAdd(&s_h[b], 1);
      else err |= kErrPartRange;
    }
    __syncthreads();
    int32_t *row = phi + (int64_t)sg.x * k;
    for (int b = threadIdx.x; b < k; b += blockDim.x)
      if (s_h[b]) atomicAdd(&row[b], s_h[b]);
    __syncthreads();
  }
  if (err) atomicOr(&cnt->err, err);
}

// c(V_i) and |V_i|, aggregated per block in shared memory.
__global__ void k_block_weights(const int32_t *part, const int32_t *vwgt, int32_t n, int32_t k, int64_t *bw,
                                int32_t *vcount, Counters *cnt) {
  __shared__ long long s_bw[kMaxK];
  __shared__ int s_cnt[kMaxK];
  for (int b = threadIdx.x; b < k; b += blockDim.x) { s_bw[b] = 0; s_cnt[b] = 0; }
  __syncthreads();
  int err = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int b = part[v];
    if ((unsigned)b < (unsigned)k) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_bw[b]), (unsigned long long)vwgt[v]);
      atomicAdd(&s_cnt[b], 1);
    } else {
      err |= kErrPartRange;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < k; b += blockDim.x) {
    if (s_bw[b]) add_i64(reinterpret_cast<long long *>(&bw[b]), s_bw[b]);
    if (s_cnt[b]) atomicAdd(&vcount[b], s_cnt[b]);
  }
  if (err) atomicOr(&cnt->err, err);
}

// Bitmasks of Lambda(e) and of the blocks with >= 2 pins from a dense phi
// (warp per edge): of every edge, or of the m edges listed in `list`.
__global__ void __launch_bounds__(256) k_masks_from_phi(const int32_t *phi, int32_t m, int32_t k, int32_t kwp,
                                                        uint32_t *mask, const int32_t *list) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < m; i += nw) {
    const int64_t e = list ? list[i] : i;
    const int32_t *row = phi + e * k;
    for (int q = 0; q < kwp; ++q) {
      int b = q * 32 + lane;
      const int val = b < k ? row[b] : 0;
      const unsigned one = __ballot_sync(kFull, val > 0), two = __ballot_sync(kFull, val > 1);
      if (lane == 0) {
        mask[e * 2 * kwp + q] = one;
        mask[e * 2 * kwp + kwp + q] = two;
      }
    }
  }
}

// (lambda-1) from a dense phi: warp per edge counts the nonzero entries of its row.
__global__ void __launch_bounds__(256) k_connectivity_dense(const int32_t *phi, const int32_t *ewgt, int32_t m,
                                                            int32_t k, long long *out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  long long acc = 0;
  for (int64_t e = gw; e < m; e += nw) {
    const int32_t *row = phi + e * k;
    int lam = 0;
    for (int b0 = 0; b0 < k; b0 += 32) lam += __popc(__ballot_sync(kFull, b0 + lane < k && row[b0 + lane] > 0));
    if (lane == 0 && lam > 0) acc += (long long)(lam - 1) * ewgt[e];
  }
  long long tot = block_sum_ll(acc);
  if (threadIdx.x == 0 && tot) add_i64(out, tot);
}

// (lambda-1) from the bitmasks: thread per edge.
__global__ void __launch_bounds__(256) k_objective_masks(const uint32_t *mask, const int32_t *ewgt, int32_t m,
                                                         int32_t kwp, Counters *cnt) {
  long long acc = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int lam = 0;
    for (int q = 0; q < kwp; ++q) lam += __popc(mask[e * 2 * kwp + q]);
    if (lam > 0) acc += (long long)(lam - 1) * ewgt[e];
  }
  long long tot = block_sum_ll(acc);
  if (threadIdx.x == 0 && tot) add_i64(&cnt->objective, tot);
}

// (lambda-1) of a graph (every edge two pins, so edge e's pins are pins[2e], pins[2e+1]): the weighted
// edge cut.  `pairs` is pins read as 8-byte pairs (NULL when pins is not 8-byte aligned); unit: all omega = 1.
__global__ void __launch_bounds__(256) k_objective_cut(const int32_t *pins, const int2 *pairs, const int32_t *part,
                                                       const int32_t *ewgt, int32_t m, int unit, Counters *cnt) {
  long long acc = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs ? pairs[e] : make_int2(pins[2 * e], pins[2 * e + 1]);
    if (part[p.x] != part[p.y]) acc += unit ? 1 : ewgt[e];
  }
  long long tot = block_sum_ll(acc);
  if (threadIdx.x == 0 && tot) add_i64(&cnt->objective, tot);
}

// Edges that are not two distinct pins (the graph path needs none).
__global__ void k_count_non_pairs(const int64_t *eptr, const int32_t *pins, int32_t m, int32_t *bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = eptr[e];
    if (eptr[e + 1] - p != 2 || pins[p] == pins[p + 1]) atomicAdd(bad, 1);
  }
}

// adj[j] = the other pin of edge inc[j], for every incidence j of every vertex.
__global__ void k_build_adj(const int64_t *vptr, const int32_t *inc, const int64_t *eptr, const int32_t *pins,
                            int32_t n, int32_t *adj) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t j = vptr[v]; j < vptr[v + 1]; ++j) {
      const int64_t p = eptr[inc[j]];
      adj[j] = pins[p] == (int32_t)v ? pins[p + 1] : pins[p];
    }
  }
}

}  // namespace

cudaError_t launch_validate(jet_ctx *c, int64_t *wdeg_tmp, int32_t *degcount_tmp, unsigned long long *scal) {
  // phases 1..3; the caller synchronizes and checks cnt->err between phases
  cudaStream_t s = c->stream;
  int g = grid_for((int64_t)c->m + c->n + 2, 256, c->launch_sms);
  k_validate_offsets<<<g, 256, 0, s>>>(c->eptr, c->vptr, c->vwgt, c->ewgt, c->n, c->m, c->P, c->cnt);
  ++c->kernel_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (c->cnt_host->err) return cudaSuccess;  // offsets unusable: stop before indexing with them
  if (c->P > 0) {
    k_validate_ids<<<grid_for(c->P, 256, c->launch_sms), 256, 0, s>>>(c->pins, c->inc, c->n, c->m, c->P, degcount_tmp,
                                                                    c->cnt);
    ++c->kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  e = cudaMemcpyAsync(c->cnt_host, c->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (c->cnt_host->err) return cudaSuccess;
  if (c->n > 0) {
    k_validate_degrees<<<grid_for(c->n, 256, c->launch_sms), 256, 0, s>>>(c->vptr, c->inc, c->vwgt, c->ewgt, c->n,
                                                                        degcount_tmp, wdeg_tmp, scal, c->cnt);
    ++c->kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Builds the class lists into one id array per kind (vertex: light, heavy;
// edge: tiny, mid, big).  Synchronizes.
static cudaError_t stable_partition(jet_ctx *c, const uint8_t *code, int32_t count, int32_t *out,
                                    int32_t totals[kClasses]) {
  for (int cl = 0; cl < kClasses; ++cl) totals[cl] = 0;
  if (count == 0) return cudaSuccess;
  const int bs = 1024;
  const int nb = (int)((count + bs - 1) / bs);
  int32_t *d_cnt = nullptr, *d_off = nullptr;
  cudaError_t e = jet::pool_alloc(&d_cnt, sizeof(int32_t) * kClasses * nb, c->stream);
  if (e != cudaSuccess) return e;
  e = jet::pool_alloc(&d_off, sizeof(int32_t) * kClasses * nb, c->stream);
  if (e != cudaSuccess) { cudaFreeAsync(d_cnt, c->stream); return e; }
  std::vector<int32_t> h((size_t)kClasses * nb);
  k_class_count<<<nb, bs, 0, c->stream>>>(code, count, d_cnt);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_cnt, sizeof(int32_t) * kClasses * nb, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) {
    int64_t tot[kClasses] = {0}, run[kClasses];
    for (int b = 0; b < nb; ++b)
      for (int cl = 0; cl < kClasses; ++cl) tot[cl] += h[(size_t)kClasses * b + cl];
    int64_t acc = 0;
    for (int cl = 0; cl < kClasses; ++cl) { run[cl] = acc; acc += tot[cl]; }
    for (int b = 0; b < nb; ++b)
      for (int cl = 0; cl < kClasses; ++cl) {
        const int32_t x = h[(size_t)kClasses * b + cl];
        h[(size_t)kClasses * b + cl] = (int32_t)run[cl];
        run[cl] += x;
      }
    for (int cl = 0; cl < kClasses; ++cl) totals[cl] = (int32_t)tot[cl];
    e = cudaMemcpyAsync(d_off, h.data(), sizeof(int32_t) * kClasses * nb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
      k_class_scatter<<<nb, bs, 0, c->stream>>>(code, count, d_off, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  cudaFreeAsync(d_cnt, c->stream);
  cudaFreeAsync(d_off, c->stream);
  return e;
}

cudaError_t launch_classify(jet_ctx *c, const int64_t *wdeg) {
  // vertex lists live in one array: [light | heavy]; edge lists in one array
  // of m + (mid count) entries: [tiny | mid | big | room for deferred mid edges]
  int64_t mx = c->n > c->m ? c->n : c->m;
  uint8_t *code = nullptr;
  cudaError_t e = jet::pool_alloc(&code, mx > 0 ? mx : 1, c->stream);
  if (e != cudaSuccess) return e;
  int32_t t[kClasses];
  if (c->n > 0) {
    k_vertex_codes<<<grid_for(c->n, 256, c->launch_sms), 256, 0, c->stream>>>(wdeg, c->n, c->vheavy);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = stable_partition(c, c->vheavy, c->n, c->v_light, t);
  if (e == cudaSuccess) {
    c->n_light = t[0];
    c->n_heavy = t[1];
    c->v_heavy = c->v_light + t[0];
    if (c->m > 0) {
      k_edge_codes<<<grid_for(c->m, 256, c->launch_sms), 256, 0, c->stream>>>(c->eptr, c->m, code);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = stable_partition(c, code, c->m, c->e_tiny, t);
  if (e == cudaSuccess) {
    c->n_tiny = 0;
    for (int cl = 0; cl <= kTinyEdge; ++cl) c->n_tiny += t[cl];
    c->n_mid_half = t[kTinyEdge + 1];
    c->n_mid_small = t[kTinyEdge + 2];
    c->n_mid = t[kTinyEdge + 3] + t[kTinyEdge + 4];
    c->n_mid_hi = t[kTinyEdge + 3];
    c->n_big = t[kTinyEdge + 5];
    c->e_mid_half = c->e_tiny + c->n_tiny;
    c->e_mid_small = c->e_mid_half + c->n_mid_half;
    c->e_mid = c->e_mid_small + c->n_mid_small;
    c->e_big = c->e_mid + c->n_mid;
  }
  cudaFreeAsync(code, c->stream);
  return e;
}

cudaError_t launch_pincounts(jet_ctx *c, const int32_t *part, int32_t *phi, int64_t *block_w) {
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemsetAsync(block_w, 0, sizeof(int64_t) * c->k, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->vcount, 0, sizeof(int32_t) * c->k, s);
  if (e != cudaSuccess) return e;
  if (c->m > 0 && phi) {
    const int threads = 256;
    size_t smem = (size_t)(threads / 32) * c->k * sizeof(int);
    k_pincounts<<<grid_for((int64_t)c->m * 32, threads, c->launch_sms), threads, smem, s>>>(
        c->eptr, c->pins, part, c->m, c->k, c->kwp, phi, c->mask, c->cnt);
    ++c->kernel_launches;
    if (c->n_slots > 0) {  // edges longer than one segment
      k_pincounts_seg<<<grid_for(c->n_seg, 1, c->launch_sms), 256, 0, s>>>(c->eptr, c->pins, part, c->ab_seg,
                                                                           c->n_seg, c->k, phi, c->cnt);
      k_masks_from_phi<<<grid_for((int64_t)c->n_slots * 32, 256, c->launch_sms), 256, 0, s>>>(
          phi, c->n_slots, c->k, c->kwp, c->mask, c->ab_slot_edge);
      c->kernel_launches += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c->n > 0) {
    k_block_weights<<<grid_for(c->n, 256, c->launch_sms, 2), 256, 0, s>>>(part, c->vwgt, c->n, c->k, block_w,
                                                                        c->vcount, c->cnt);
    ++c->kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  c->phi_owner = phi;
  return cudaSuccess;
}

cudaError_t launch_masks_from_phi(jet_ctx *c, const int32_t *phi) {
  if (c->m > 0) {
    k_masks_from_phi<<<grid_for((int64_t)c->m * 32, 256, c->launch_sms), 256, 0, c->stream>>>(phi, c->m, c->k, c->kwp,
                                                                                            c->mask, nullptr);
    ++c->kernel_launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c->phi_owner = phi;
  return cudaSuccess;
}

cudaError_t launch_connectivity_dense(jet_ctx *c, const int32_t *phi, int64_t *out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), c->stream);
  if (e != cudaSuccess || c->m == 0) return e;
  k_connectivity_dense<<<grid_for((int64_t)c->m * 32, 256, c->launch_sms), 256, 0, c->stream>>>(
      phi, c->ewgt, c->m, c->k, reinterpret_cast<long long *>(out));
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_objective(jet_ctx *c, const int32_t *part) {
  cudaError_t e = cudaMemsetAsync(&c->cnt->objective, 0, sizeof(long long), c->stream);
  if (e != cudaSuccess || c->m == 0) return e;
  if (c->graph_path) {
    const int2 *pairs = ((uintptr_t)c->pins & 7) ? nullptr : reinterpret_cast<const int2 *>(c->pins);
    k_objective_cut<<<grid_for(c->m, 256, c->launch_sms), 256, 0, c->stream>>>(c->pins, pairs, part, c->ewgt, c->m,
                                                                             c->unit_ewgt, c->cnt);
  }
  else
    k_objective_masks<<<grid_for(c->m, 256, c->launch_sms), 256, 0, c->stream>>>(c->mask, c->ewgt, c->m, c->kwp,
                                                                               c->cnt);
  ++c->kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_build_adj(jet_ctx *c, int32_t *bad_edges) {
  cudaError_t e = cudaMemsetAsync(bad_edges, 0, sizeof(int32_t), c->stream);
  if (e != cudaSuccess) return e;
  if (c->m > 0) {
    k_count_non_pairs<<<grid_for(c->m, 256, c->launch_sms), 256, 0, c->stream>>>(c->eptr, c->pins, c->m, bad_edges);
    ++c->kernel_launches;
  }
  if (c->n > 0 && c->adj) {
    k_build_adj<<<grid_for(c->n, 256, c->launch_sms), 256, 0, c->stream>>>(c->vptr, c->inc, c->eptr, c->pins, c->n,
                                                                         c->adj);
    ++c->kernel_launches;
  }
  return cudaGetLastError();
}

}  // namespace jet
