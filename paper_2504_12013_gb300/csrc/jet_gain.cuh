// Gain arithmetic shared by the candidate, rebalancing-target and batched
// kernels (Sections 4.1 and 4.3).
//
// gain(v, b) = conn(v, b) - A(v) for v in V_s, where conn(v, b) = sum of
// omega(e) over e in I(v) with phi_e[b] >= 1 and A(v) = sum of omega(e) over
// e in I(v) with phi_e[s] >= 2, both read from the two bitmasks of each edge.
// A light vertex keeps conn(v, .) for all k blocks as bit planes of k-bit
// words (kLightPlanes planes); an incident edge's Lambda(e) row is added with
// a ripple carry, and the argmax over a block set C is a top-down bit-serial
// filter whose lowest remaining block is the smallest-id maximiser.
#pragma once

#include "jet_internal.cuh"

namespace jet {

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

// Warp argmax of (conn desc, block asc); block -1 = none.  Result on all lanes.
__device__ __forceinline__ void warp_argmax(int32_t &c, int &b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int32_t c2 = __shfl_xor_sync(0xffffffffu, c, o);
    int b2 = __shfl_xor_sync(0xffffffffu, b, o);
    bool take = b2 >= 0 && (b < 0 || c2 > c || (c2 == c && b2 < b));
    if (take) { c = c2; b = b2; }
  }
}

// Exact rebalancing priority (Section 4.3) as an ascending key: gain * c for
// gain >= 0; for gain < 0 the ratio gain / c scaled by 2^30 and truncated.
// With c <= 2^15 two distinct ratios differ by >= 2^-30, so the scaled values
// differ by >= 1 and the truncation keeps their order; equal ratios stay
// equal.  All gain < 0 keys are <= -2^15 < 0 <= every gain >= 0 key, so the
// classes keep their order.  U = INT64_MAX - P (mod 2^64) turns "priority
// desc" into "U asc".  Compact form: with L = lcm(1..cmax), gain/c =
// gain*(L/c) / L, so gain*(L/c) orders the gain < 0 class exactly (equal
// ratios stay equal) and stays <= -1 < 0 <= gain*c of the gain >= 0 class;
// Pmax - P is then below 2^32 (checked by the context) and needs far fewer
// key bits.
__device__ __forceinline__ uint64_t rb_priority_key(int compact, long long L, long long Pmax, int32_t g, int32_t c) {
  if (compact) {
    const long long P = g >= 0 ? (long long)g * c : (long long)g * (L / c);
    return (uint64_t)(Pmax - P);
  }
  const long long P = g >= 0 ? (long long)g * c : ((long long)g * (1ll << kPrioShift)) / c;
  return (uint64_t)0x7fffffffffffffffull - (uint64_t)P;
}

}  // namespace jet
