/*
 * CPU ORACLE for deterministic Jet refinement (connectivity metric).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  The product path (the
 * CUDA library) never calls it and shares no code, header, table or constant
 * with it.
 *
 * Plain, slow, single-threaded, integer-only.  Every function follows the
 * paper (arXiv 2504.12013) step by step, in its order and notation:
 *   Section 2 ("Preliminaries")         hypergraph, partition, balance, (lambda-1)
 *   Section 4.1, Algorithm 1            Jet loop: candidates, afterburner, apply, rebalance
 *   Section 4.2, Algorithm 2            hypergraph afterburner (sort + replay)
 *   Section 4.3                         deterministic rebalancing, deadzone, heavy vertices
 *   Section 7.2                         three temperatures 0.75 -> 0, 8 iterations
 *   Section 5 (matching schedule)       quotient graph, rounds of maximal matchings
 *   Section 6, Algorithm 4              synchronous clustering, contraction
 * Readings where the paper is silent or ambiguous (each marked READING below):
 *   R1  blocks are 0-based, [k] = {0..k-1}.
 *   R2  L_max = floor((1+eps) * ceil(c(V)/k)), eps = eps_num/eps_den exactly.
 *   R3  gain(v,b) is the connectivity gain: sum over e in I(v) of
 *       omega(e) * ([phi_e(s) = 1] - [phi_e(b) = 0]), s = Pi(v)  (the +-omega
 *       rule of Algorithm 2).
 *   R4  move candidates consider blocks b != s adjacent to v (phi_e(b) >= 1 for
 *       some e in I(v)); t(v) = argmax gain, ties to the smallest block id; a
 *       vertex with no adjacent block is not a candidate.
 *   R5  the temperature test is  gain >= -tau * A(v)  with tau = tau_num/tau_den
 *       and A(v) = sum of omega(e) over e in I(v) with |e cap V_s| > 1,
 *       evaluated exactly in integers.
 *   R6  the afterburner order is gain descending, ties to the smaller vertex id.
 *   R7  locking: the vertices moved by the afterburner-approved moves of an
 *       iteration are excluded from the candidates of the next iteration; the
 *       rebalancer ignores locks; locks are cleared at the start of each
 *       temperature phase.
 *   R8  rebalancing targets: all blocks b != s with c(V_b) + c(v) <= L_max that
 *       are not in the deadzone (c(V_b) >= L_max - d*eps*ceil(c(V)/k), with the
 *       real-valued L_max = (1+eps)*ceil(c(V)/k), compared exactly); ties of the
 *       best gain go to the smallest block id; non-adjacent blocks count.
 *   R9  rebalancing priority: gain*c(v) if gain >= 0, gain/c(v) otherwise,
 *       compared exactly; every gain >= 0 vertex precedes every gain < 0 one;
 *       ties to the smaller vertex id; per overloaded block the minimal prefix
 *       of this order whose weight reaches c(V_s) - L_max is moved (all
 *       candidates if the prefix never reaches it).
 *   R10 rebalancing rounds stop when no block is overloaded, when a round moves
 *       nothing, or after max_rebalance_rounds rounds.
 *   R11 "quality improved" means balanced and strictly smaller (lambda-1) than
 *       the best balanced partition seen so far; at the end of each temperature
 *       phase the best balanced partition is restored (rollback).
 *   R12 an empty hyperedge contributes 0 to (lambda-1).
 *   R17 the matching schedule of the quotient graph (Section 5): see
 *       ojet_schedule.
 *   R19..R25 coarsening (Section 6, Algorithm 4) and contraction: see
 *       ojet_subrounds, ojet_cluster and ojet_contract.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n, m;
  int64_t P;
  const int64_t *eptr; /* pins of e: pins[eptr[e] .. eptr[e+1]) */
  const int32_t *pins;
  const int64_t *vptr; /* I(v): inc[vptr[v] .. vptr[v+1]) */
  const int32_t *inc;
  const int32_t *vwgt; /* c(v)     */
  const int32_t *ewgt; /* omega(e) */
} ojet_hg;

typedef struct {
  int32_t k;
  int32_t eps_num, eps_den;
  int32_t d_num, d_den;
  int32_t max_rebalance_rounds;
} ojet_params;

typedef struct {
  int64_t candidates;       /* |M| after the temperature filter      */
  int64_t approved;         /* moves kept by the afterburner          */
  int64_t rebalance_rounds; /* rounds that found an overloaded block  */
  int64_t rebalance_moves;  /* vertices moved by the rebalancer       */
  int64_t objective;        /* (lambda-1) after the iteration         */
  int64_t max_block_weight;
  int64_t imbalanced;       /* 1 if some block is above L_max          */
} ojet_stats;

/* ------------------------------------------------------------ Section 2 */

/* c(V) */
int64_t ojet_total_weight(const ojet_hg *h) {
  int64_t W = 0;
  for (int32_t v = 0; v < h->n; ++v) W += h->vwgt[v];
  return W;
}

/* ceil(c(V)/k), the average block weight rounded up (Section 2, R2) */
int64_t ojet_avg_block(const ojet_hg *h, int32_t k) {
  int64_t W = ojet_total_weight(h);
  return (W + k - 1) / k;
}

/* L_max = floor((1 + eps) * ceil(c(V)/k))  (Section 2, R2) */
int64_t ojet_lmax(const ojet_hg *h, const ojet_params *p) {
  __int128 A = ojet_avg_block(h, p->k);
  return (int64_t)(((__int128)(p->eps_den + p->eps_num) * A) / p->eps_den);
}

/* phi_e[i] = |e cap V_i| for every edge and block; c(V_i) for every block (Section 2) */
void ojet_pincounts(const ojet_hg *h, int32_t k, const int32_t *part, int32_t *phi, int64_t *bw) {
  memset(phi, 0, sizeof(int32_t) * (size_t)h->m * (size_t)k);
  for (int32_t e = 0; e < h->m; ++e)
    for (int64_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) phi[(int64_t)e * k + part[h->pins[p]]] += 1;
  for (int32_t b = 0; b < k; ++b) bw[b] = 0;
  for (int32_t v = 0; v < h->n; ++v) bw[part[v]] += h->vwgt[v];
}

/* (lambda-1)(Pi) = sum_e (lambda(e) - 1) omega(e), lambda(e) = |{i : phi_e[i] > 0}| (Section 2, R12) */
int64_t ojet_connectivity(const ojet_hg *h, int32_t k, const int32_t *phi) {
  int64_t total = 0;
  for (int32_t e = 0; e < h->m; ++e) {
    int64_t lambda = 0;
    for (int32_t b = 0; b < k; ++b)
      if (phi[(int64_t)e * k + b] > 0) lambda += 1;
    if (lambda > 0) total += (lambda - 1) * (int64_t)h->ewgt[e];
  }
  return total;
}

/* gain of moving v from its block to b (Section 4.1 "gain", R3) */
int64_t ojet_gain(const ojet_hg *h, int32_t k, const int32_t *part, const int32_t *phi, int32_t v, int32_t b) {
  int32_t s = part[v];
  int64_t g = 0;
  for (int64_t j = h->vptr[v]; j < h->vptr[v + 1]; ++j) {
    int32_t e = h->inc[j];
    if (phi[(int64_t)e * k + s] == 1) g += h->ewgt[e];
    if (phi[(int64_t)e * k + b] == 0) g -= h->ewgt[e];
  }
  return g;
}

/* A(v) = sum of omega(e), e in I(v), with |e cap V_s| > 1  (threshold of Section 4.1, R5) */
int64_t ojet_affinity(const ojet_hg *h, int32_t k, const int32_t *part, const int32_t *phi, int32_t v) {
  int32_t s = part[v];
  int64_t a = 0;
  for (int64_t j = h->vptr[v]; j < h->vptr[v + 1]; ++j) {
    int32_t e = h->inc[j];
    if (phi[(int64_t)e * k + s] > 1) a += h->ewgt[e];
  }
  return a;
}

/* ------------------------------------------------------------ Section 4.1 */

/*
 * ComputeMoveCandidates (Section 4.1): for every unlocked v, the target t(v)
 * with the highest gain ignoring balance (R4), against the current partition
 * as if no other vertex moved; v joins M iff gain >= -tau * A(v) (R5).
 * Returns |M|.  target[v]/gain[v] hold t(v) and its gain for every unlocked
 * vertex with an adjacent block (in M or not); target[v] = -1 otherwise.
 */
int64_t ojet_candidates(const ojet_hg *h, int32_t k, const int32_t *part, const int32_t *phi, const uint8_t *locked,
                        int32_t tau_num, int32_t tau_den, int32_t *target, int64_t *gain, uint8_t *in_m) {
  uint8_t *adjacent = (uint8_t *)malloc((size_t)k);
  int64_t count = 0;
  for (int32_t v = 0; v < h->n; ++v) {
    target[v] = -1;
    gain[v] = 0;
    in_m[v] = 0;
    if (locked[v]) continue;
    int32_t s = part[v];
    memset(adjacent, 0, (size_t)k);
    for (int64_t j = h->vptr[v]; j < h->vptr[v + 1]; ++j) {
      int32_t e = h->inc[j];
      for (int32_t b = 0; b < k; ++b)
        if (phi[(int64_t)e * k + b] > 0) adjacent[b] = 1;
    }
    int32_t best = -1;
    int64_t best_gain = 0;
    for (int32_t b = 0; b < k; ++b) {
      if (b == s || !adjacent[b]) continue;
      int64_t g = ojet_gain(h, k, part, phi, v, b);
      if (best < 0 || g > best_gain) { best = b; best_gain = g; }
    }
    if (best < 0) continue;
    int64_t A = ojet_affinity(h, k, part, phi, v);
    target[v] = best;
    gain[v] = best_gain;
    if ((__int128)tau_den * best_gain >= -(__int128)tau_num * A) {
      in_m[v] = 1;
      count += 1;
    }
  }
  free(adjacent);
  return count;
}

/* ------------------------------------------------------------ Section 4.2 */

typedef struct { int64_t gain; int32_t v; } ab_item;

/* the move order of M: gain descending, ties to the smaller vertex id (R6) */
static int ab_order(const void *a, const void *b) {
  const ab_item *x = (const ab_item *)a, *y = (const ab_item *)b;
  if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

/*
 * Hypergraph afterburner (Algorithm 2).  For every edge: start from the pin
 * counts of the current partition, sort e cap M by the move order, replay the
 * moves; a pin whose departure empties its block in e earns +omega(e), a pin
 * whose arrival makes its target non-empty in e pays -omega(e).  Every earlier
 * pin of M counts as moved, whether or not it is approved itself.
 * rg[] receives the recomputed gains; approved[v] = v in M and rg[v] > 0.
 * Returns the number of approved moves.
 */
int64_t ojet_afterburner(const ojet_hg *h, int32_t k, const int32_t *part, const int32_t *phi, const int32_t *target,
                         const int64_t *gain, const uint8_t *in_m, int64_t *rg, uint8_t *approved) {
  int32_t *phi_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int64_t max_size = 0;
  for (int32_t e = 0; e < h->m; ++e)
    if (h->eptr[e + 1] - h->eptr[e] > max_size) max_size = h->eptr[e + 1] - h->eptr[e];
  ab_item *L = (ab_item *)malloc(sizeof(ab_item) * (size_t)(max_size > 0 ? max_size : 1));
  for (int32_t v = 0; v < h->n; ++v) rg[v] = 0;
  for (int32_t e = 0; e < h->m; ++e) {
    for (int32_t b = 0; b < k; ++b) phi_e[b] = phi[(int64_t)e * k + b];
    int64_t len = 0;
    for (int64_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) {
      int32_t v = h->pins[p];
      if (in_m[v]) { L[len].gain = gain[v]; L[len].v = v; ++len; }
    }
    qsort(L, (size_t)len, sizeof(ab_item), ab_order);
    for (int64_t i = 0; i < len; ++i) {
      int32_t v = L[i].v;
      phi_e[part[v]] -= 1;
      if (phi_e[part[v]] == 0) rg[v] += h->ewgt[e];
      phi_e[target[v]] += 1;
      if (phi_e[target[v]] == 1) rg[v] -= h->ewgt[e];
    }
  }
  int64_t count = 0;
  for (int32_t v = 0; v < h->n; ++v) {
    approved[v] = (uint8_t)(in_m[v] && rg[v] > 0);
    count += approved[v];
  }
  free(phi_e);
  free(L);
  return count;
}

/* ApplyMoves (Algorithm 1): move every flagged v to target[v] at once; update phi and c(V_i). */
void ojet_apply(const ojet_hg *h, int32_t k, int32_t *part, int32_t *phi, int64_t *bw, const uint8_t *move,
                const int32_t *target) {
  for (int32_t v = 0; v < h->n; ++v) {
    if (!move[v]) continue;
    int32_t s = part[v], t = target[v];
    for (int64_t j = h->vptr[v]; j < h->vptr[v + 1]; ++j) {
      int32_t e = h->inc[j];
      phi[(int64_t)e * k + s] -= 1;
      phi[(int64_t)e * k + t] += 1;
    }
    bw[s] -= h->vwgt[v];
    bw[t] += h->vwgt[v];
    part[v] = t;
  }
}

/* ------------------------------------------------------------ Section 4.3 */

/* deadzone test: c(V_b) >= L_max - d*eps*ceil(c(V)/k) with the real L_max = (1+eps)ceil(c(V)/k) (R8) */
static int in_deadzone(const ojet_params *p, int64_t A, int64_t bwb) {
  __int128 lhs = (__int128)p->eps_den * p->d_den * bwb;
  __int128 rhs = (__int128)p->d_den * (p->eps_den + p->eps_num) * A - (__int128)p->d_num * p->eps_num * A;
  return lhs >= rhs;
}

typedef struct { int64_t gain; int32_t c; int32_t v; int32_t t; } rb_item;

/* priority order (R9): higher priority first, ties to the smaller vertex id */
static int rb_order(const void *a, const void *b) {
  const rb_item *x = (const rb_item *)a, *y = (const rb_item *)b;
  int cx = x->gain >= 0, cy = y->gain >= 0;
  if (cx != cy) return cx ? -1 : 1;
  __int128 lx, ly;
  if (cx) { /* gain * c(v) */
    lx = (__int128)x->gain * x->c;
    ly = (__int128)y->gain * y->c;
  } else { /* gain / c(v):  gx/cx > gy/cy  <=>  gx*cy > gy*cx  (c > 0) */
    lx = (__int128)x->gain * y->c;
    ly = (__int128)y->gain * x->c;
  }
  if (lx != ly) return lx > ly ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

/*
 * One rebalancing round (Section 4.3), computed from the state at the start
 * of the round.  Per vertex v of an overloaded block s that is not too heavy
 * (2 c(v) <= 3 (c(V_s) - ceil(c(V)/k))): its best valid target (R8) and
 * priority (R9).  Per overloaded block: sort by priority, prefix sums of c(v),
 * the minimal prefix restoring balance.  All selected vertices move at once.
 * Returns the number of moved vertices, or -1 if no block is overloaded.
 * moved_flag/moved_target (n entries, may be NULL) receive the selection.
 */
int64_t ojet_rebalance_round(const ojet_hg *h, const ojet_params *p, int32_t *part, int32_t *phi, int64_t *bw,
                             uint8_t *moved_flag, int32_t *moved_target) {
  const int32_t k = p->k;
  const int64_t A = ojet_avg_block(h, k);
  const int64_t Lmax = ojet_lmax(h, p);
  int any = 0;
  for (int32_t b = 0; b < k; ++b) any |= bw[b] > Lmax;
  if (moved_flag) memset(moved_flag, 0, (size_t)h->n);
  if (!any) return -1;

  int64_t *cnt = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  for (int32_t v = 0; v < h->n; ++v) cnt[part[v]] += 1;
  rb_item **list = (rb_item **)calloc((size_t)k, sizeof(rb_item *));
  int64_t *len = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  for (int32_t b = 0; b < k; ++b)
    if (bw[b] > Lmax) list[b] = (rb_item *)malloc(sizeof(rb_item) * (size_t)(cnt[b] > 0 ? cnt[b] : 1));

  for (int32_t v = 0; v < h->n; ++v) {
    int32_t s = part[v];
    if (bw[s] <= Lmax) continue;
    int64_t c = h->vwgt[v];
    if (2 * c > 3 * (bw[s] - A)) continue; /* heavy vertex: never moved */
    int32_t best = -1;
    int64_t best_gain = 0;
    for (int32_t b = 0; b < k; ++b) {
      if (b == s) continue;
      if (bw[b] + c > Lmax) continue;
      if (in_deadzone(p, A, bw[b])) continue;
      int64_t g = ojet_gain(h, k, part, phi, v, b);
      if (best < 0 || g > best_gain) { best = b; best_gain = g; }
    }
    if (best < 0) continue;
    rb_item it = {best_gain, (int32_t)c, v, best};
    list[s][len[s]++] = it;
  }

  size_t nn = (size_t)(h->n > 0 ? h->n : 1);
  uint8_t *mv = (uint8_t *)calloc(nn, 1);
  int32_t *tg = (int32_t *)malloc(sizeof(int32_t) * nn);
  int64_t moved = 0;
  for (int32_t s = 0; s < k; ++s) {
    if (!list[s]) continue;
    qsort(list[s], (size_t)len[s], sizeof(rb_item), rb_order);
    int64_t excess = bw[s] - Lmax, prefix = 0;
    for (int64_t i = 0; i < len[s] && prefix < excess; ++i) {
      prefix += list[s][i].c;
      mv[list[s][i].v] = 1;
      tg[list[s][i].v] = list[s][i].t;
      moved += 1;
    }
  }
  ojet_apply(h, k, part, phi, bw, mv, tg);
  if (moved_flag) memcpy(moved_flag, mv, (size_t)h->n);
  if (moved_target)
    for (int32_t v = 0; v < h->n; ++v) moved_target[v] = mv[v] ? tg[v] : -1;
  for (int32_t b = 0; b < k; ++b) free(list[b]);
  free(list); free(len); free(cnt); free(mv); free(tg);
  return moved;
}

/* Rebalancing rounds until balanced, a round moves nothing, or the round cap (R10). */
int64_t ojet_rebalance(const ojet_hg *h, const ojet_params *p, int32_t *part, int32_t *phi, int64_t *bw,
                       int64_t *moves_out) {
  int64_t rounds = 0, moves = 0;
  while (rounds < p->max_rebalance_rounds) {
    int64_t moved = ojet_rebalance_round(h, p, part, phi, bw, NULL, NULL);
    if (moved < 0) break;
    rounds += 1;
    moves += moved;
    if (moved == 0) break;
  }
  if (moves_out) *moves_out = moves;
  return rounds;
}

/* ------------------------------------------------------------ Algorithm 1 */

static void fill_stats(const ojet_hg *h, const ojet_params *p, const int32_t *phi, const int64_t *bw,
                       ojet_stats *st) {
  int64_t Lmax = ojet_lmax(h, p), mx = 0;
  for (int32_t b = 0; b < p->k; ++b) mx = bw[b] > mx ? bw[b] : mx;
  st->objective = ojet_connectivity(h, p->k, phi);
  st->max_block_weight = mx;
  st->imbalanced = mx > Lmax;
}

/*
 * One Jet iteration (the body of Algorithm 1): candidates, afterburner, apply
 * (locking the approved vertices, R7), and rebalancing if a block is above
 * L_max.  part/phi/bw/locked are updated in place.
 */
void ojet_refine_round(const ojet_hg *h, const ojet_params *p, int32_t tau_num, int32_t tau_den, int32_t *part,
                       int32_t *phi, int64_t *bw, uint8_t *locked, ojet_stats *st) {
  const int32_t n = h->n, k = p->k;
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *target = (int32_t *)malloc(sizeof(int32_t) * nn);
  int64_t *gain = (int64_t *)malloc(sizeof(int64_t) * nn);
  int64_t *rg = (int64_t *)malloc(sizeof(int64_t) * nn);
  uint8_t *in_m = (uint8_t *)malloc(nn);
  uint8_t *approved = (uint8_t *)malloc(nn);
  memset(st, 0, sizeof(*st));
  st->candidates = ojet_candidates(h, k, part, phi, locked, tau_num, tau_den, target, gain, in_m);
  st->approved = ojet_afterburner(h, k, part, phi, target, gain, in_m, rg, approved);
  ojet_apply(h, k, part, phi, bw, approved, target);
  for (int32_t v = 0; v < n; ++v) locked[v] = approved[v];
  int64_t Lmax = ojet_lmax(h, p);
  int over = 0;
  for (int32_t b = 0; b < k; ++b) over |= bw[b] > Lmax;
  if (over) st->rebalance_rounds = ojet_rebalance(h, p, part, phi, bw, &st->rebalance_moves);
  fill_stats(h, p, phi, bw, st);
  free(target); free(gain); free(rg); free(in_m); free(approved);
}

/*
 * Algorithm 1 with the temperature schedule of Section 7.2: for each tau in
 * the schedule, iterate until `limit` iterations pass without a strictly
 * better balanced partition (R11), then roll back to the best balanced
 * partition seen.  tau is given as pairs (num, den).  part is updated in
 * place.  Returns the number of iterations executed; *best_objective gets the
 * (lambda-1) of the returned partition.
 */
int64_t ojet_refine(const ojet_hg *h, const ojet_params *p, const int32_t *tau_pairs, int32_t n_tau, int32_t limit,
                    int32_t *part, int64_t *objective_out, int64_t *phase_iters) {
  const int32_t n = h->n, k = p->k;
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)h->m * (size_t)k + 4);
  int64_t *bw = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
  uint8_t *locked = (uint8_t *)malloc(nn);
  int32_t *best = (int32_t *)malloc(sizeof(int32_t) * nn);
  ojet_pincounts(h, k, part, phi, bw);
  int64_t Lmax = ojet_lmax(h, p);
  int have_best = 1;
  for (int32_t b = 0; b < k; ++b) have_best &= bw[b] <= Lmax;
  int64_t best_obj = have_best ? ojet_connectivity(h, k, phi) : 0;
  if (have_best) memcpy(best, part, sizeof(int32_t) * (size_t)n);
  int64_t iterations = 0;
  for (int32_t ti = 0; ti < n_tau; ++ti) {
    memset(locked, 0, nn);
    int32_t it = 0;
    int64_t in_phase = 0;
    while (it < limit) {
      ojet_stats st;
      ojet_refine_round(h, p, tau_pairs[2 * ti], tau_pairs[2 * ti + 1], part, phi, bw, locked, &st);
      iterations += 1;
      in_phase += 1;
      it += 1;
      if (!st.imbalanced && (!have_best || st.objective < best_obj)) {
        have_best = 1;
        best_obj = st.objective;
        memcpy(best, part, sizeof(int32_t) * (size_t)n);
        it = 0;
      }
    }
    if (phase_iters) phase_iters[ti] = in_phase;
    if (have_best) { /* rollback to the best balanced partition */
      memcpy(part, best, sizeof(int32_t) * (size_t)n);
      ojet_pincounts(h, k, part, phi, bw);
    }
  }
  if (objective_out) *objective_out = ojet_connectivity(h, k, phi);
  free(phi); free(bw); free(locked); free(best);
  return iterations;
}

/*
 * Section 5 ("K-Way Refinement: Matching Schedule").  The quotient graph Q
 * has the k blocks as vertices and an edge {i, j} (i != j) when some
 * hyperedge has pins in both V_i and V_j, i.e. phi_e(i) >= 1 and
 * phi_e(j) >= 1.  qadj[i*k + j] = qadj[j*k + i] = 1 for those pairs, by
 * definition from phi.
 */
void ojet_quotient(const ojet_hg *h, int32_t k, const int32_t *phi, uint8_t *qadj) {
  memset(qadj, 0, (size_t)k * (size_t)k);
  for (int32_t e = 0; e < h->m; ++e) {
    const int32_t *row = phi + (size_t)e * (size_t)k;
    for (int32_t i = 0; i < k; ++i) {
      if (row[i] < 1) continue;
      for (int32_t j = 0; j < k; ++j)
        if (j != i && row[j] >= 1) qadj[(size_t)i * k + j] = 1;
    }
  }
}

/*
 * Section 5 ("K-Way Refinement: Matching Schedule"): block pairs are
 * scheduled in rounds; each round is a maximal matching in the quotient
 * edges not scheduled yet, and rounds repeat until every quotient edge is
 * scheduled.  Edges of high-degree blocks go first.
 * READING R17: each round takes the blocks in order of their degree in the
 * remaining quotient graph at the start of the round (descending, ties to
 * the smaller id); a block that is still unmatched is paired with its
 * unmatched remaining neighbour of the largest such degree (ties to the
 * smaller id).  Output in selection order: pairs[2p] = the visited block,
 * pairs[2p+1] = its partner, round_of[p] = the round.  Returns the number of
 * pairs; *n_rounds gets the number of rounds.
 */
int64_t ojet_schedule(int32_t k, const uint8_t *qadj, int32_t *pairs, int32_t *round_of, int32_t *n_rounds) {
  uint8_t *rem = (uint8_t *)malloc((size_t)k * (size_t)k + 1);
  int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)k + 4);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)k + 4);
  uint8_t *matched = (uint8_t *)malloc((size_t)k + 1);
  memcpy(rem, qadj, (size_t)k * (size_t)k);
  for (int32_t i = 0; i < k; ++i) rem[(size_t)i * k + i] = 0;
  int64_t np = 0;
  int32_t round = 0;
  for (;;) {
    int64_t left = 0;
    for (int32_t i = 0; i < k; ++i) {
      deg[i] = 0;
      for (int32_t j = 0; j < k; ++j) deg[i] += rem[(size_t)i * k + j];
      left += deg[i];
      order[i] = i;
    }
    if (left == 0) break;
    /* insertion sort by (degree desc, id asc) */
    for (int32_t x = 1; x < k; ++x) {
      const int32_t b = order[x];
      int32_t y = x - 1;
      while (y >= 0 && (deg[order[y]] < deg[b] || (deg[order[y]] == deg[b] && order[y] > b))) {
        order[y + 1] = order[y];
        --y;
      }
      order[y + 1] = b;
    }
    memset(matched, 0, (size_t)k);
    for (int32_t x = 0; x < k; ++x) {
      const int32_t i = order[x];
      if (deg[i] == 0 || matched[i]) continue;
      int32_t best = -1;
      for (int32_t j = 0; j < k; ++j)
        if (rem[(size_t)i * k + j] && !matched[j] && (best < 0 || deg[j] > deg[best])) best = j;
      if (best < 0) continue;
      matched[i] = matched[best] = 1;
      rem[(size_t)i * k + best] = rem[(size_t)best * k + i] = 0;
      pairs[2 * np] = i;
      pairs[2 * np + 1] = best;
      round_of[np] = round;
      ++np;
    }
    ++round;
  }
  if (n_rounds) *n_rounds = round;
  free(rem); free(deg); free(order); free(matched);
  return np;
}

/*
 * Section 6 ("Improving Deterministic Coarsening"), Algorithm 4: the sizes
 * of the synchronous sub-rounds (prefix doubling).  READING R21: n_single
 * sub-rounds of one vertex, then sizes 2, 4, 8, ... up to
 * cap = max(1, floor(n / cap_div)) (cap_div = 100: one percent of the
 * vertices), the last sub-round ragged.  bounds (may be NULL) receives the
 * start of every sub-round and n at the end.  Returns the number of
 * sub-rounds.
 */
int64_t ojet_subrounds(int32_t n, int32_t n_single, int32_t cap_div, int32_t *bounds) {
  int64_t cap = n / (cap_div > 0 ? cap_div : 1);
  if (cap < 1) cap = 1;
  int64_t pos = 0, r = 0, size = 1;
  while (pos < n) {
    if (r < n_single) size = 1;
    else if (r == n_single) size = 2;
    else size *= 2;
    if (size > cap) size = cap;
    if (bounds) bounds[r] = (int32_t)pos;
    pos += size > n - pos ? n - pos : size;
    ++r;
  }
  if (bounds) bounds[r] = n;
  return r;
}

/* The heavy-edge rating term of one hyperedge (READING R19): omega(e)/(|e|-1)
 * in fixed point with 32 fraction bits, rounded down. */
static uint64_t rating_term(int32_t w, int64_t size) { return ((uint64_t)(uint32_t)w << 32) / (uint64_t)(size - 1); }

static const int32_t *g_cw_vwgt;
static const int32_t *g_cw_target;
static int approve_order(const void *a, const void *b) {
  const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  if (g_cw_target[x] != g_cw_target[y]) return g_cw_target[x] < g_cw_target[y] ? -1 : 1;
  if (g_cw_vwgt[x] != g_cw_vwgt[y]) return g_cw_vwgt[x] < g_cw_vwgt[y] ? -1 : 1;
  return (x > y) - (x < y);
}

/*
 * Section 6, Algorithm 4: one level of synchronous clustering with the
 * heavy-edge rating (corrected: an edge counts once per cluster), prefix-
 * doubling sub-rounds and swap prevention.  Clusters are label classes;
 * label[v] starts as v.  Per sub-round, from the state at its start:
 *   1. every vertex u of the sub-round that is still a singleton cluster
 *      (READING R22: no vertex joined it; it has not moved) rates the
 *      clusters C of its neighbours: r(C) = sum over e in I(u) with
 *      2 <= |e| <= rmax that have a pin other than u in C of the term of e
 *      (READING R19), over clusters with c(C) + c(u) <= cmax (READING R20);
 *      T[u] = argmax, ties to the smaller label, none if no cluster qualifies;
 *   2. swap prevention (READING R23): for u, v of the sub-round with
 *      T[u] = v and T[v] = u, the vertex whose cluster would be heavier (its
 *      weight plus that of the other proposers to it) stays and the other
 *      joins it; equal weights: the smaller id stays;
 *   3. approval (READING R24): the proposers of each target label j, in
 *      order of (c(u) asc, u asc), move while their weight sum stays within
 *      cmax - c(C_j);
 *   4. all approved vertices move at once.
 * order (n entries, a permutation) is the random split of the vertices.
 * Returns 0, or -1 when a vertex's rating sum could reach 2^63 (overflow).
 */
int64_t ojet_cluster(const ojet_hg *h, int64_t cmax, int32_t rmax, int32_t n_single, int32_t cap_div,
                     const int32_t *order, int32_t *label) {
  const int32_t n = h->n;
  const size_t nn = (size_t)n + 1;
  for (int32_t u = 0; u < n; ++u) {
    uint64_t s = 0;
    for (int64_t i = h->vptr[u]; i < h->vptr[u + 1]; ++i) {
      const int32_t e = h->inc[i];
      const int64_t size = h->eptr[e + 1] - h->eptr[e];
      if (size < 2 || size > rmax) continue;
      s += rating_term(h->ewgt[e], size);
      if (s >= ((uint64_t)1 << 63)) return -1;
    }
  }
  int64_t *cw = (int64_t *)malloc(sizeof(int64_t) * nn);
  int32_t *csize = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *T = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *T2 = (int32_t *)malloc(sizeof(int32_t) * nn);
  int64_t *pw = (int64_t *)calloc(nn, sizeof(int64_t));
  uint64_t *acc = (uint64_t *)calloc(nn, sizeof(uint64_t));
  int32_t *last = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *members = (int32_t *)malloc(sizeof(int32_t) * nn);
  const int64_t rounds = ojet_subrounds(n, n_single, cap_div, NULL);
  int32_t *bounds = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rounds + 1));
  ojet_subrounds(n, n_single, cap_div, bounds);
  for (int32_t v = 0; v < n; ++v) {
    label[v] = v;
    cw[v] = h->vwgt[v];
    csize[v] = 1;
    T[v] = T2[v] = -1;
    last[v] = -1;
  }
  for (int64_t r = 0; r < rounds; ++r) {
    const int32_t a = bounds[r], b = bounds[r + 1];
    /* 1. target clusters */
    for (int32_t x = a; x < b; ++x) {
      const int32_t u = order[x];
      if (csize[u] != 1 || label[u] != u) continue;
      int32_t nt = 0;
      for (int64_t i = h->vptr[u]; i < h->vptr[u + 1]; ++i) {
        const int32_t e = h->inc[i];
        const int64_t size = h->eptr[e + 1] - h->eptr[e];
        if (size < 2 || size > rmax) continue;
        const uint64_t t = rating_term(h->ewgt[e], size);
        for (int64_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) {
          const int32_t v = h->pins[p];
          if (v == u) continue;
          const int32_t C = label[v];
          if (C == u || last[C] == e) continue; /* once per edge and cluster */
          if (last[C] < 0) touched[nt++] = C;
          last[C] = e;
          acc[C] += t;
        }
      }
      int32_t best = -1;
      for (int32_t q = 0; q < nt; ++q) {
        const int32_t C = touched[q];
        if (cw[C] + h->vwgt[u] <= cmax && (best < 0 || acc[C] > acc[best] || (acc[C] == acc[best] && C < best)))
          best = C;
      }
      for (int32_t q = 0; q < nt; ++q) {
        acc[touched[q]] = 0;
        last[touched[q]] = -1;
      }
      T[u] = best;
    }
    /* 2. swap prevention, decided on the proposals as made */
    for (int32_t x = a; x < b; ++x) {
      const int32_t u = order[x];
      if (T[u] >= 0) pw[T[u]] += h->vwgt[u];
    }
    for (int32_t x = a; x < b; ++x) {
      const int32_t u = order[x];
      const int32_t v = T[u];
      T2[u] = v;
      if (v < 0 || T[v] != u) continue;
      const int64_t wu = h->vwgt[u] + pw[u] - h->vwgt[v];
      const int64_t wv = h->vwgt[v] + pw[v] - h->vwgt[u];
      if (wu > wv || (wu == wv && u < v)) T2[u] = -1; /* u stays, v joins u */
    }
    /* 3. approval per target label */
    int32_t nm = 0;
    for (int32_t x = a; x < b; ++x)
      if (T2[order[x]] >= 0) members[nm++] = order[x];
    g_cw_vwgt = h->vwgt;
    g_cw_target = T2;
    qsort(members, (size_t)nm, sizeof(int32_t), approve_order);
    int32_t nmove = 0;
    for (int32_t q = 0; q < nm;) {
      const int32_t j = T2[members[q]];
      const int64_t room = cmax - cw[j];
      int64_t sum = 0;
      int32_t z = q;
      for (; z < nm && T2[members[z]] == j; ++z) {
        sum += h->vwgt[members[z]];
        if (sum <= room) members[nmove++] = members[z]; /* a prefix: weights ascend */
        else sum = room + 1;
      }
      q = z;
    }
    /* 4. move */
    for (int32_t q = 0; q < nmove; ++q) {
      const int32_t u = members[q], j = T2[u];
      label[u] = j;
      cw[j] += h->vwgt[u];
      cw[u] -= h->vwgt[u];
      csize[j] += 1;
      csize[u] -= 1;
    }
    for (int32_t x = a; x < b; ++x) {
      const int32_t u = order[x];
      if (T[u] >= 0) pw[T[u]] = 0;
      T[u] = T2[u] = -1;
    }
  }
  free(cw); free(csize); free(T); free(T2); free(pw); free(acc); free(last); free(touched); free(members);
  free(bounds);
  return 0;
}

static const int64_t *g_ct_eptr;
static const int32_t *g_ct_pins;
static int contract_order(const void *a, const void *b) {
  const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  const int64_t sx = g_ct_eptr[x + 1] - g_ct_eptr[x], sy = g_ct_eptr[y + 1] - g_ct_eptr[y];
  if (sx != sy) return sx < sy ? -1 : 1;
  for (int64_t i = 0; i < sx; ++i) {
    const int32_t px = g_ct_pins[g_ct_eptr[x] + i], py = g_ct_pins[g_ct_eptr[y] + i];
    if (px != py) return px < py ? -1 : 1;
  }
  return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
  const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/*
 * Contraction of the clusters (Section 6 reuses the contraction of the
 * earlier deterministic partitioner; READING R25): the non-empty label
 * classes become the coarse vertices, numbered in increasing label order,
 * with c(C) the sum of their members' weights; map[v] is v's coarse vertex.
 * Every hyperedge keeps its distinct coarse pins in increasing order and is
 * dropped when fewer than two remain; hyperedges with identical pin sets are
 * merged into the one of smallest id, their weights summed; coarse edges
 * follow the order of those ids; the incidences of a coarse vertex are in
 * increasing coarse edge id.  Output arrays are sized as the input's (n+1,
 * P, n+1, P, n, m).  Returns 0, or -1 when a coarse weight leaves int32.
 */
int64_t ojet_contract(const ojet_hg *h, const int32_t *label, int32_t *map, int64_t *ceptr, int32_t *cpins,
                      int64_t *cvptr, int32_t *cinc, int32_t *cvwgt, int32_t *cewgt, int32_t *nc_out,
                      int32_t *mc_out, int64_t *pc_out) {
  const int32_t n = h->n, m = h->m;
  int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int64_t *w = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) cid[v] = -1;
  for (int32_t v = 0; v < n; ++v) cid[label[v]] = 0;
  int32_t nc = 0;
  for (int32_t l = 0; l < n; ++l)
    if (cid[l] == 0) cid[l] = nc++;
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) {
    map[v] = cid[label[v]];
    w[map[v]] += h->vwgt[v];
  }
  for (int32_t c = 0; c < nc; ++c) {
    if (w[c] > INT32_MAX) rc = -1;
    cvwgt[c] = (int32_t)w[c];
  }
  /* distinct coarse pins of every edge, ascending */
  int64_t *teptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
  int32_t *tpins = (int32_t *)malloc(sizeof(int32_t) * ((size_t)h->P + 1));
  teptr[0] = 0;
  for (int32_t e = 0; e < m; ++e) {
    const int64_t o = teptr[e];
    int64_t len = 0;
    for (int64_t p = h->eptr[e]; p < h->eptr[e + 1]; ++p) tpins[o + len++] = map[h->pins[p]];
    qsort(tpins + o, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t d = 0;
    for (int64_t i = 0; i < len; ++i)
      if (d == 0 || tpins[o + i] != tpins[o + d - 1]) tpins[o + d++] = tpins[o + i];
    teptr[e + 1] = o + d;
  }
  /* identical pin sets: sort the kept edges by (size, pins, id); runs share a pin set */
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
  int32_t *rep = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m + 1));
  int64_t *ew = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
  int32_t nk = 0;
  for (int32_t e = 0; e < m; ++e) {
    rep[e] = -1;
    if (teptr[e + 1] - teptr[e] >= 2) ord[nk++] = e;
  }
  g_ct_eptr = teptr;
  g_ct_pins = tpins;
  qsort(ord, (size_t)nk, sizeof(int32_t), contract_order);
  for (int32_t i = 0; i < nk; ++i) {
    const int32_t e = ord[i];
    const int32_t f = i > 0 ? ord[i - 1] : -1;
    const int64_t size = teptr[e + 1] - teptr[e];
    const int same = f >= 0 && teptr[f + 1] - teptr[f] == size &&
                     memcmp(tpins + teptr[f], tpins + teptr[e], sizeof(int32_t) * (size_t)size) == 0;
    rep[e] = same ? rep[f] : e; /* a run's first edge has the smallest id */
    ew[rep[e]] += h->ewgt[e];
  }
  /* coarse edges in order of their representative's id */
  int32_t mc = 0;
  int64_t pc = 0;
  ceptr[0] = 0;
  for (int32_t e = 0; e < m; ++e) {
    if (rep[e] != e) continue;
    if (ew[e] > INT32_MAX) rc = -1;
    cewgt[mc] = (int32_t)ew[e];
    for (int64_t i = teptr[e]; i < teptr[e + 1]; ++i) cpins[pc++] = tpins[i];
    ceptr[++mc] = pc;
  }
  /* incidences by coarse vertex, in increasing coarse edge id */
  for (int32_t c = 0; c <= nc; ++c) cvptr[c] = 0;
  for (int64_t i = 0; i < pc; ++i) cvptr[cpins[i] + 1] += 1;
  for (int32_t c = 0; c < nc; ++c) cvptr[c + 1] += cvptr[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nc + 1));
  for (int32_t c = 0; c < nc; ++c) fill[c] = cvptr[c];
  for (int32_t f = 0; f < mc; ++f)
    for (int64_t i = ceptr[f]; i < ceptr[f + 1]; ++i) cinc[fill[cpins[i]]++] = f;
  *nc_out = nc;
  *mc_out = mc;
  *pc_out = pc;
  free(cid); free(w); free(teptr); free(tpins); free(ord); free(rep); free(ew); free(fill);
  return rc;
}
