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
// thread block (thread j owns block j): per round the blocks are sorted by
// (remaining degree desc, id asc); each one still unmatched in its turn
// takes its unmatched remaining neighbour of the largest remaining degree
// (ties to the smaller id).
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

// Bitonic sort of blockDim.x (a power of two >= k) keys in shared memory, ascending.
__device__ __forceinline__ void block_sort(uint32_t *key) {
  const int n = blockDim.x, t = threadIdx.x;
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int o = t ^ stride;
      if (o > t) {
        const bool up = (t & size) == 0;
        const uint32_t a = key[t], b = key[o];
        if ((a > b) == up) {
          key[t] = b;
          key[o] = a;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kMaxK) k_schedule(const uint32_t *q, int32_t k, int kwp, int32_t *pairs,
                                                     int32_t *round_of, int32_t *out_counts) {
  __shared__ uint32_t s_rem[kMaxK * 8];
  __shared__ uint32_t s_key[kMaxK];
  __shared__ int s_deg[kMaxK];
  __shared__ int s_matched[kMaxK];
  __shared__ int s_best[kMaxK / 32];
  __shared__ int s_np, s_left;
  const int j = threadIdx.x, lane = j & 31, wid = j >> 5;
  for (int x = j; x < k * kwp; x += blockDim.x) s_rem[x] = q[x];
  __syncthreads();
  if (j < k) s_rem[j * kwp + (j >> 5)] &= ~(1u << (j & 31));  // no self pairs
  if (j == 0) s_np = 0;
  __syncthreads();
  int round = 0;
  for (;;) {
    int d = 0;
    if (j < k)
      for (int w = 0; w < kwp; ++w) d += __popc(s_rem[j * kwp + w]);
    s_deg[j] = d;
    s_matched[j] = 0;
    // (degree desc, id asc): ascending keys (255 - degree) << 8 | id; absent blocks sort last
    s_key[j] = j < k ? ((uint32_t)(255 - d) << 8) | (uint32_t)j : 0xffffffffu;
    if (j == 0) s_left = 0;
    __syncthreads();
    if (d) atomicAdd(&s_left, d);
    block_sort(s_key);  // ends with a barrier
    if (s_left == 0) break;
    for (int x = 0; x < k; ++x) {
      const int i = (int)(s_key[x] & 255);
      if (s_deg[i] == 0) break;  // the rest have no remaining edge
      if (s_matched[i]) continue;  // uniform: shared state
      // this thread's bid: its block j as i's partner
      const bool cand = j < k && !s_matched[j] && ((s_rem[i * kwp + (j >> 5)] >> (j & 31)) & 1u);
      int bid = cand ? (s_deg[j] << 8) | (255 - j) : -1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bid = max(bid, __shfl_xor_sync(kFull, bid, o));
      if (lane == 0) s_best[wid] = bid;
      __syncthreads();
      if (j == 0) {
        int b = -1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, s_best[w]);
        if (b >= 0) {
          const int p = 255 - (b & 255);
          s_matched[i] = s_matched[p] = 1;
          s_rem[i * kwp + (p >> 5)] &= ~(1u << (p & 31));
          s_rem[p * kwp + (i >> 5)] &= ~(1u << (i & 31));
          pairs[2 * s_np] = i;
          pairs[2 * s_np + 1] = p;
          round_of[s_np] = round;
          ++s_np;
        }
      }
      __syncthreads();
    }
    ++round;
    __syncthreads();
  }
  if (j == 0) {
    out_counts[0] = s_np;
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
  k_schedule<<<1, kMaxK, 0, c->stream>>>(qbits, c->k, c->kwp, pairs, round_of, counts);
  ++c->kernel_launches;
  return cudaGetLastError();
}

}  // namespace jet
