// Matching schedule of k-way refinement (Section 5, "K-Way Refinement:
// Matching Schedule").  The quotient graph Q has the blocks as vertices and
// an edge {i, j} when some hyperedge has pins in both V_i and V_j.  Block
// pairs are scheduled in rounds, each a maximal matching in the quotient
// edges not scheduled yet, the blocks of high remaining degree first, so
// that every block takes part in at most one two-way refinement at a time.
//
// k_quotient builds Q as k rows of KWP bit words from the edge bitmasks
// Lambda(e) (for every block i of Lambda(e), row i |= Lambda(e)), aggregated
// per thread block in shared memory.  k_schedule runs the rounds in one
// warp: per round the blocks are ordered by (remaining degree at the round's
// start desc, id asc); each one still unmatched in its turn takes its
// unmatched remaining neighbour of the largest such degree (ties to the
// smaller id).
#include "jet_internal.cuh"

namespace jet {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(256) k_quotient(const uint32_t *mask, int32_t m, int kwp, int32_t k, uint32_t *q) {
  __shared__ uint32_t s_q[kMaxK * 8];
  for (int x = threadIdx.x; x < k * kwp; x += blockDim.x) s_q[x] = 0u;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t *row = mask + e * 2 * kwp;  // Lambda(e): the first kwp words
    uint32_t L[8];
    int bits = 0;
    for (int w = 0; w < kwp; ++w) {
      L[w] = row[w];
      bits += __popc(L[w]);
    }
    if (bits < 2) continue;  // a hyperedge inside one block links no pair
    for (int w = 0; w < kwp; ++w) {
      uint32_t x = L[w];
      while (x) {
        const int i = w * 32 + __ffs(x) - 1;
        x &= x - 1;
        for (int u = 0; u < kwp; ++u)
          if (L[u] && (s_q[i * kwp + u] & L[u]) != L[u]) atomicOr(&s_q[i * kwp + u], L[u]);
      }
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < k * kwp; x += blockDim.x)
    if (s_q[x]) atomicOr(&q[x], s_q[x]);
}

// The schedule by one warp: lane l owns blocks l, l+32, ...  Per round the
// blocks are ordered by (remaining degree desc, id asc) with a stable
// counting sort over the degrees; each turn is one warp-wide maximum of the
// partner bids (degree + 1) << 8 | (255 - id), so no block-level barrier is
// needed anywhere.
__global__ void __launch_bounds__(32) k_schedule(const uint32_t *q, int32_t k, int kwp, int32_t *pairs,
                                                 int32_t *round_of, int32_t *out_counts) {
  __shared__ uint32_t s_rem[kMaxK * 8];
  __shared__ int s_deg[kMaxK];
  __shared__ int s_matched[kMaxK];
  __shared__ int s_order[kMaxK];
  __shared__ int s_cnt[kMaxK];
  const int lane = threadIdx.x;
  const unsigned lt = (1u << lane) - 1;
  for (int x = lane; x < k * kwp; x += 32) s_rem[x] = q[x];
  __syncwarp();
  for (int j = lane; j < k; j += 32) s_rem[j * kwp + (j >> 5)] &= ~(1u << (j & 31));  // no self pairs
  __syncwarp();
  int np = 0, round = 0;
  for (;;) {
    int left = 0;
    for (int j = lane; j < k; j += 32) {
      int d = 0;
      for (int w = 0; w < kwp; ++w) d += __popc(s_rem[j * kwp + w]);
      s_deg[j] = d;
      s_matched[j] = 0;
      left += d;
    }
    for (int x = lane; x < kMaxK; x += 32) s_cnt[x] = 0;
    left = __reduce_add_sync(kFull, left);
    if (left == 0) break;
    __syncwarp();
    // stable counting sort by key 255 - degree (degree desc), ids ascending within a key
    for (int j = lane; j < k; j += 32) atomicAdd(&s_cnt[255 - s_deg[j]], 1);
    __syncwarp();
    {
      int v[8], sum = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t] = s_cnt[lane * 8 + t];
        sum += v[t];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - sum;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        s_cnt[lane * 8 + t] = run;
        run += v[t];
      }
    }
    __syncwarp();
    for (int c0 = 0; c0 < k; c0 += 32) {
      const int j = c0 + lane;
      const int key = j < k ? 255 - s_deg[j] : 256 + lane;
      const unsigned peers = match_bits<9>((unsigned)key);  // key <= 256 + 31
      const int rank = __popc(peers & lt);
      const int base = j < k ? s_cnt[key] : 0;
      __syncwarp();
      if (j < k) {
        s_order[base + rank] = j;
        if (rank == 0) s_cnt[key] = base + __popc(peers);
      }
      __syncwarp();
    }
    for (int x = 0; x < k; ++x) {
      const int i = s_order[x];
      if (s_deg[i] == 0) break;  // the rest have no remaining edge
      if (s_matched[i]) continue;
      unsigned bid = 0;
      for (int j = lane; j < k; j += 32)
        if (!s_matched[j] && ((s_rem[i * kwp + (j >> 5)] >> (j & 31)) & 1u))
          bid = max(bid, ((unsigned)(s_deg[j] + 1) << 8) | (unsigned)(255 - j));
      bid = __reduce_max_sync(kFull, bid);
      if (bid == 0) continue;
      const int p = 255 - (int)(bid & 255u);
      if (lane == 0) {
        s_matched[i] = s_matched[p] = 1;
        s_rem[i * kwp + (p >> 5)] &= ~(1u << (p & 31));
        s_rem[p * kwp + (i >> 5)] &= ~(1u << (i & 31));
        pairs[2 * np] = i;
        pairs[2 * np + 1] = p;
        round_of[np] = round;
      }
      ++np;
      __syncwarp();
    }
    ++round;
    __syncwarp();
  }
  if (lane == 0) {
    out_counts[0] = np;
    out_counts[1] = round;
  }
}

}  // namespace

cudaError_t launch_quotient_schedule(jet_ctx *c, uint32_t *qbits, int32_t *pairs, int32_t *round_of,
                                     int32_t *counts) {
  cudaError_t e = cudaMemsetAsync(qbits, 0, sizeof(uint32_t) * c->k * c->kwp, c->stream);
  if (e != cudaSuccess) return e;
  if (c->m > 0) {
    k_quotient<<<grid_for(c->m, 256, c->launch_sms, 4), 256, 0, c->stream>>>(c->mask, c->m, c->kwp, c->k, qbits);
    ++c->kernel_launches;
  }
  k_schedule<<<1, 32, 0, c->stream>>>(qbits, c->k, c->kwp, pairs, round_of, counts);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
