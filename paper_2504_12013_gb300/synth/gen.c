/*
 * Seeded synthetic hypergraph generators.
 *
 * This file only produces inputs (CSR hypergraphs, weights, initial
 * partitions).  It holds none of the refinement method's arithmetic and is
 * shared by the CPU oracle tests, the CUDA parity tests and the benchmark.
 *
 * Random numbers: splitmix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; constants as published by
 * S. Vigna).  Bounded integers use Lemire's multiply-shift with rejection
 * (unbiased).  Discrete distributions are sampled by binary search over an
 * integer cumulative table, so the same seed gives the same instance on any
 * little- or big-endian, signed- or unsigned-char platform.  The log-normal
 * length table uses no libm function: its log, exp and normal CDF are
 * series in IEEE-754 double +, -, *, / (correctly rounded everywhere, built
 * without FMA contraction), so x86 and Arm hosts produce identical tables
 * and therefore identical instances.
 *
 * Every generated hyperedge holds distinct pins, sorted by vertex id.  The
 * vertex-major CSR (incidence lists I(v)) is the exact transpose, listing the
 * hyperedges of each vertex in increasing id order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG */
typedef struct { uint64_t s; } sm64;

static uint64_t sm_next(sm64 *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform integer in [0, n), n >= 1 (Lemire 2019, with rejection) */
static uint64_t sm_below(sm64 *r, uint64_t n) {
  uint64_t x = sm_next(r);
  __uint128_t mm = (__uint128_t)x * n;
  uint64_t l = (uint64_t)mm;
  if (l < n) {
    uint64_t t = (0 - n) % n;
    while (l < t) {
      x = sm_next(r);
      mm = (__uint128_t)x * n;
      l = (uint64_t)mm;
    }
  }
  return (uint64_t)(mm >> 64);
}

/* true with probability num/den */
static int sm_bern(sm64 *r, uint64_t num, uint64_t den) { return sm_below(r, den) < num; }

/* uniform double in [0,1) with 53 random bits */
static double sm_unit(sm64 *r) { return (double)(sm_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* sample index i with probability (cum[i]-cum[i-1])/cum[len-1] */
static int64_t sample_cum(sm64 *r, const uint64_t *cum, int64_t len) {
  uint64_t u = sm_below(r, cum[len - 1]);
  int64_t lo = 0, hi = len - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (cum[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* floor(sqrt(x)) for a 128-bit x whose root is below 2^63, by bisection */
static uint64_t isqrt_u128(__uint128_t x) {
  uint64_t lo = 0, hi = 1ULL << 63;
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if ((__uint128_t)mid * mid <= x) lo = mid; else hi = mid;
  }
  return lo;
}

/* ------------------------------------------- host-independent log/exp/CDF */
static const double kLn2 = 0.69314718055994530942;

/* natural log for x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)), then
   log m = 2 atanh((m-1)/(m+1)) by its series */
static double det_log(double x) {
  int e = 0;
  double m = frexp(x, &e); /* exact: x = m * 2^e, m in [0.5, 1) */
  if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
  const double u = (m - 1.0) / (m + 1.0), u2 = u * u;
  double term = u, sum = 0.0;
  for (int k = 1; k < 80; k += 2) {
    sum += term / k;
    term *= u2;
  }
  return 2.0 * sum + e * kLn2;
}

/* e^x: x = n ln2 + r with |r| <= ln2/2, Taylor series of e^r, exact scaling by 2^n */
static double det_exp(double x) {
  const double n = floor(x / kLn2 + 0.5);
  const double r = x - n * kLn2;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= r / k;
    sum += term;
  }
  return ldexp(sum, (int)n);
}

/* standard normal CDF: 1/2 + phi(z) (z + z^3/3 + z^5/(3*5) + ...), phi the density */
static double det_normal_cdf(double z) {
  const double phi = det_exp(-0.5 * z * z) * 0.39894228040143267794;
  double term = z, sum = z;
  for (int k = 1; k < 400; ++k) {
    term *= z * z / (2 * k + 1);
    sum += term;
    if (term < 1e-30 * sum && k > 2 * (int)(z * z)) break;
  }
  double F = 0.5 + phi * sum;
  return F < 0.0 ? 0.0 : (F > 1.0 ? 1.0 : F);
}

/* ---------------------------------------------------------------- output */
typedef struct {
  int32_t n, m;
  int64_t P;
  int64_t *eptr; /* m+1 */
  int32_t *pins; /* P   */
  int64_t *vptr; /* n+1 */
  int32_t *inc;  /* P   */
  int32_t *vwgt; /* n   */
  int32_t *ewgt; /* m   */
} synth_hg;

void synth_free(synth_hg *h) {
  if (!h) return;
  free(h->eptr); free(h->pins); free(h->vptr); free(h->inc); free(h->vwgt); free(h->ewgt);
  memset(h, 0, sizeof(*h));
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Build vptr/inc as the transpose of eptr/pins (counting sort, stable). */
static int build_transpose(synth_hg *h) {
  h->vptr = (int64_t *)calloc((size_t)h->n + 1, sizeof(int64_t));
  h->inc = (int32_t *)malloc((size_t)(h->P > 0 ? h->P : 1) * sizeof(int32_t));
  if (!h->vptr || !h->inc) return -1;
  for (int64_t p = 0; p < h->P; ++p) h->vptr[h->pins[p] + 1]++;
  for (int32_t v = 0; v < h->n; ++v) h->vptr[v + 1] += h->vptr[v];
  int64_t *cur = (int64_t *)malloc((size_t)h->n * sizeof(int64_t) + 8);
  if (!cur) return -1;
  memcpy(cur, h->vptr, (size_t)h->n * sizeof(int64_t));
  for (int32_t e = 0; e < h->m; ++e)
    for (int64_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) h->inc[cur[h->pins[p]]++] = e;
  free(cur);
  return 0;
}

/*
 * Fill pins of all edges given sizes[]: each pin drawn by `draw` until it is
 * new to the edge (stamp array), then the edge is sorted by vertex id.
 */
typedef int32_t (*draw_fn)(sm64 *r, void *ctx, int32_t e);

static int fill_pins(synth_hg *h, const int32_t *sizes, sm64 *r, draw_fn draw, void *dctx) {
  h->eptr = (int64_t *)malloc(((size_t)h->m + 1) * sizeof(int64_t));
  if (!h->eptr) return -1;
  h->eptr[0] = 0;
  for (int32_t e = 0; e < h->m; ++e) h->eptr[e + 1] = h->eptr[e] + sizes[e];
  h->P = h->eptr[h->m];
  h->pins = (int32_t *)malloc((size_t)(h->P > 0 ? h->P : 1) * sizeof(int32_t));
  int32_t *stamp = (int32_t *)malloc((size_t)h->n * sizeof(int32_t));
  if (!h->pins || !stamp) { free(stamp); return -1; }
  for (int32_t v = 0; v < h->n; ++v) stamp[v] = -1;
  for (int32_t e = 0; e < h->m; ++e) {
    int32_t *pe = h->pins + h->eptr[e];
    for (int32_t i = 0; i < sizes[e]; ++i) {
      int32_t v;
      do { v = draw(r, dctx, e); } while (stamp[v] == e);
      stamp[v] = e;
      pe[i] = v;
    }
    qsort(pe, (size_t)sizes[e], sizeof(int32_t), cmp_i32);
  }
  free(stamp);
  return 0;
}

static int alloc_weights(synth_hg *h) {
  h->vwgt = (int32_t *)malloc((size_t)(h->n > 0 ? h->n : 1) * sizeof(int32_t));
  h->ewgt = (int32_t *)malloc((size_t)(h->m > 0 ? h->m : 1) * sizeof(int32_t));
  return (h->vwgt && h->ewgt) ? 0 : -1;
}

static void draw_weights(synth_hg *h, sm64 *r, int32_t c_max, int32_t w_max) {
  for (int32_t v = 0; v < h->n; ++v) h->vwgt[v] = c_max <= 1 ? 1 : 1 + (int32_t)sm_below(r, (uint64_t)c_max);
  for (int32_t e = 0; e < h->m; ++e) h->ewgt[e] = w_max <= 1 ? 1 : 1 + (int32_t)sm_below(r, (uint64_t)w_max);
}

static int32_t draw_uniform(sm64 *r, void *ctx, int32_t e) {
  (void)e;
  return (int32_t)sm_below(r, (uint64_t)*(int32_t *)ctx);
}

/*
 * Uniform random hypergraph: |e| = base + G, G ~ Geometric(p = geo_num/geo_den)
 * counted as failures before the first success, |e| capped at size_cap and at
 * n; pins uniform without repeats; c ~ U{1..c_max}, omega ~ U{1..w_max}.
 * Weights are drawn after the pins from the same stream.
 */
int synth_uniform(uint64_t seed, int32_t n, int32_t m, int32_t base, uint32_t geo_num,
                  uint32_t geo_den, int32_t size_cap, int32_t c_max, int32_t w_max, synth_hg *out) {
  memset(out, 0, sizeof(*out));
  if (n < 1 || m < 0 || base < 0 || geo_den == 0 || geo_num == 0 || geo_num > geo_den) return -2;
  sm64 r = {seed};
  out->n = n; out->m = m;
  int32_t *sizes = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!sizes) return -1;
  int32_t cap = size_cap < n ? size_cap : n;
  for (int32_t e = 0; e < m; ++e) {
    int32_t s = base;
    while (s < cap && !sm_bern(&r, geo_num, geo_den)) ++s;
    sizes[e] = s < cap ? s : cap;
  }
  int rc = fill_pins(out, sizes, &r, draw_uniform, &n);
  free(sizes);
  if (rc || alloc_weights(out) || build_transpose(out)) { synth_free(out); return -1; }
  draw_weights(out, &r, c_max, w_max);
  return 0;
}

/*
 * VLSI-netlist-shaped hypergraph: sizes ~ discrete power law P(s) ~ s^(-alpha)
 * on [smin, smax] with alpha = alpha_x2 / 2, tabulated as floor(2^60 /
 * s^alpha) in exact integer arithmetic; every edge has a uniform centre x and each pin is, with
 * probability loc_num/loc_den, uniform in [x - window, x + window] mod n, else
 * uniform in [0, n).  c ~ U{1..c_max}, omega = 1.
 */
typedef struct { int32_t n, window; uint32_t loc_num, loc_den; int32_t *centre; } vlsi_ctx;

static int32_t draw_vlsi(sm64 *r, void *ctx, int32_t e) {
  vlsi_ctx *c = (vlsi_ctx *)ctx;
  if (sm_bern(r, c->loc_num, c->loc_den)) {
    int64_t off = (int64_t)sm_below(r, (uint64_t)(2 * (int64_t)c->window + 1)) - c->window;
    int64_t v = ((int64_t)c->centre[e] + off) % c->n;
    if (v < 0) v += c->n;
    return (int32_t)v;
  }
  return (int32_t)sm_below(r, (uint64_t)c->n);
}

int synth_vlsi(uint64_t seed, int32_t n, int32_t m, int32_t smin, int32_t smax, int32_t alpha_x2,
               int32_t window, uint32_t loc_num, uint32_t loc_den, int32_t c_max, synth_hg *out) {
  memset(out, 0, sizeof(*out));
  if (n < 1 || m < 0 || smin < 1 || smax < smin || smax > n || alpha_x2 < 1 || loc_den == 0) return -2;
  /* an edge larger than its window needs the non-local draws to fill it */
  if (loc_num >= loc_den && (int64_t)smax > 2 * (int64_t)window + 1) return -2;
  /* s^alpha_x2 must fit in 64 bits */
  if ((double)alpha_x2 * log2((double)smax) >= 63.0) return -2;
  sm64 r = {seed};
  out->n = n; out->m = m;
  int64_t len = (int64_t)smax - smin + 1;
  uint64_t *cum = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
  int32_t *sizes = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t *centre = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!cum || !sizes || !centre) { free(cum); free(sizes); free(centre); return -1; }
  uint64_t acc = 0;
  for (int64_t i = 0; i < len; ++i) {
    /* weight floor(2^60 / s^(alpha_x2/2)) = floor(sqrt(floor(2^120 / s^alpha_x2))) */
    uint64_t s = (uint64_t)(smin + i), p = 1;
    for (int32_t j = 0; j < alpha_x2; ++j) p *= s;
    acc += isqrt_u128((((__uint128_t)1) << 120) / p);
    cum[i] = acc;
  }
  for (int32_t e = 0; e < m; ++e) {
    sizes[e] = smin + (int32_t)sample_cum(&r, cum, len);
    centre[e] = (int32_t)sm_below(&r, (uint64_t)n);
  }
  vlsi_ctx c = {n, window, loc_num, loc_den, centre};
  int rc = fill_pins(out, sizes, &r, draw_vlsi, &c);
  free(cum); free(sizes); free(centre);
  if (rc || alloc_weights(out) || build_transpose(out)) { synth_free(out); return -1; }
  draw_weights(out, &r, c_max, 1);
  return 0;
}

/*
 * Sparse-matrix row-net-shaped hypergraph: n columns (vertices), m rows
 * (hyperedges); n_hubs rows at seeded distinct positions get a length
 * U{hub_min..hub_max}; every other row has length round(LogNormal(mu, sigma))
 * clamped to [1, n].  Columns uniform.  c = omega = 1.
 */
int synth_rownet(uint64_t seed, int32_t n, int32_t m, int32_t n_hubs, int32_t hub_min,
                 int32_t hub_max, double mu, double sigma, synth_hg *out) {
  memset(out, 0, sizeof(*out));
  if (n < 1 || m < 1 || n_hubs < 0 || n_hubs > m || hub_min < 1 || hub_max < hub_min || hub_max > n ||
      !(sigma > 0))
    return -2;
  sm64 r = {seed};
  out->n = n; out->m = m;
  /* length table: P(L = l) = P(l - 1/2 <= X < l + 1/2), l >= 2; l = 1 takes X < 3/2 */
  int64_t tlen = 1 << 16;
  if (tlen > n) tlen = n;
  uint64_t *cum = (uint64_t *)malloc((size_t)tlen * sizeof(uint64_t));
  int32_t *sizes = (int32_t *)malloc((size_t)m * sizeof(int32_t));
  uint8_t *is_hub = (uint8_t *)calloc((size_t)m, 1);
  if (!cum || !sizes || !is_hub) { free(cum); free(sizes); free(is_hub); return -1; }
  uint64_t acc = 0;
  double prev = 0.0;
  for (int64_t l = 1; l <= tlen; ++l) {
    double z = (det_log((double)l + 0.5) - mu) / sigma;
    double F = det_normal_cdf(z);
    if (l == tlen) F = 1.0;
    double p = F - prev;
    prev = F;
    acc += (uint64_t)llround(p * 4611686018427387904.0);
    cum[l - 1] = acc;
  }
  int32_t placed = 0;
  while (placed < n_hubs) {
    int32_t e = (int32_t)sm_below(&r, (uint64_t)m);
    if (!is_hub[e]) { is_hub[e] = 1; ++placed; }
  }
  for (int32_t e = 0; e < m; ++e) {
    if (is_hub[e]) sizes[e] = hub_min + (int32_t)sm_below(&r, (uint64_t)(hub_max - hub_min + 1));
    else sizes[e] = 1 + (int32_t)sample_cum(&r, cum, tlen);
  }
  int rc = fill_pins(out, sizes, &r, draw_uniform, &n);
  free(cum); free(sizes); free(is_hub);
  if (rc || alloc_weights(out) || build_transpose(out)) { synth_free(out); return -1; }
  draw_weights(out, &r, 1, 1);
  return 0;
}

/* Initial partition: block of vertex i is (i * 2654435761 + seed) mod k in uint64. */
void synth_part_hash(uint64_t seed, int32_t n, int32_t k, int32_t *part) {
  for (int32_t i = 0; i < n; ++i) part[i] = (int32_t)(((uint64_t)i * 2654435761ULL + seed) % (uint64_t)k);
}

/* Initial partition: seeded Fisher-Yates permutation pi; block of pi(i) is i mod k. */
int synth_part_perm(uint64_t seed, int32_t n, int32_t k, int32_t *part) {
  int32_t *pi = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!pi) return -1;
  sm64 r = {seed};
  for (int32_t i = 0; i < n; ++i) pi[i] = i;
  for (int32_t i = n - 1; i > 0; --i) {
    int32_t j = (int32_t)sm_below(&r, (uint64_t)i + 1);
    int32_t t = pi[i]; pi[i] = pi[j]; pi[j] = t;
  }
  for (int32_t i = 0; i < n; ++i) part[pi[i]] = i % k;
  free(pi);
  return 0;
}

/* Uniform random partition (not balanced): block ~ U{0..k-1}. */
void synth_part_random(uint64_t seed, int32_t n, int32_t k, int32_t *part) {
  sm64 r = {seed};
  for (int32_t i = 0; i < n; ++i) part[i] = (int32_t)sm_below(&r, (uint64_t)k);
}

/* Raw stream access, for seeded choices made by the Python side (job mixes, sizes). */
uint64_t synth_stream(uint64_t seed, int64_t index) {
  sm64 r = {seed};
  uint64_t x = 0;
  for (int64_t i = 0; i <= index; ++i) x = sm_next(&r);
  return x;
}

void synth_fill_u64(uint64_t seed, int64_t count, uint64_t *out) {
  sm64 r = {seed};
  for (int64_t i = 0; i < count; ++i) out[i] = sm_next(&r);
}

void synth_fill_unit(uint64_t seed, int64_t count, double *out) {
  sm64 r = {seed};
  for (int64_t i = 0; i < count; ++i) out[i] = sm_unit(&r);
}
