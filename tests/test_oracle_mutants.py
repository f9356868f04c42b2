"""Planted mistakes in copies of the oracle must each fail a pin.

Each mutant below is a plausible slip in the oracle (a dropped term, a wrong
sign or threshold, a flipped tie-break, a transposed operand).  The test
writes the mutated source to a temporary directory, compiles it, and runs the
whole pin suite against it in a child process (a mutant may crash).  A mutant
that passes every pin would mean the pins cannot tell that slip from the
paper's method.
"""
import os
import subprocess
import sys

from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "jet_oracle.c")

MUTANTS = {
    # Section 2
    "lmax_uses_floor_average": ("return (W + k - 1) / k;", "return W / k;"),
    "lmax_drops_eps": ("return (int64_t)(((__int128)(p->eps_den + p->eps_num) * A) / p->eps_den);",
                       "return (int64_t)(((__int128)(p->eps_den) * A) / p->eps_den);"),
    "pincount_wrong_row": ("phi[(int64_t)e * k + part[h->pins[p]]] += 1;", "phi[(int64_t)e + part[h->pins[p]]] += 1;"),
    "connectivity_counts_lambda": ("total += (lambda - 1) * (int64_t)h->ewgt[e];", "total += lambda * (int64_t)h->ewgt[e];"),
    "connectivity_drops_weight": ("total += (lambda - 1) * (int64_t)h->ewgt[e];", "total += (lambda - 1);"),
    # Section 4.1
    "gain_source_threshold": ("if (phi[(int64_t)e * k + s] == 1) g += h->ewgt[e];", "if (phi[(int64_t)e * k + s] == 2) g += h->ewgt[e];"),
    "gain_target_sign": ("if (phi[(int64_t)e * k + b] == 0) g -= h->ewgt[e];", "if (phi[(int64_t)e * k + b] == 0) g += h->ewgt[e];"),
    "affinity_threshold": ("if (phi[(int64_t)e * k + s] > 1) a += h->ewgt[e];", "if (phi[(int64_t)e * k + s] >= 1) a += h->ewgt[e];"),
    "candidate_tie_largest_block": ("if (best < 0 || g > best_gain) { best = b; best_gain = g; }\n    }\n    if (best < 0) continue;\n    int64_t A",
                                    "if (best < 0 || g >= best_gain) { best = b; best_gain = g; }\n    }\n    if (best < 0) continue;\n    int64_t A"),
    "candidate_strict_tau": ("if ((__int128)tau_den * best_gain >= -(__int128)tau_num * A) {", "if ((__int128)tau_den * best_gain > -(__int128)tau_num * A) {"),
    "candidate_ignores_lock": ("    if (locked[v]) continue;\n    int32_t s = part[v];\n    memset", "    int32_t s = part[v];\n    memset"),
    "candidate_tau_transposed": ("if ((__int128)tau_den * best_gain >= -(__int128)tau_num * A) {", "if ((__int128)tau_num * best_gain >= -(__int128)tau_den * A) {"),
    # Section 4.2
    "ab_order_ascending": ("if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;", "if (x->gain != y->gain) return x->gain < y->gain ? -1 : 1;"),
    "ab_tie_larger_id": ("return (x->v > y->v) - (x->v < y->v);\n}\n\n/*\n * Hypergraph", "return (x->v < y->v) - (x->v > y->v);\n}\n\n/*\n * Hypergraph"),
    "ab_departure_dropped": ("if (phi_e[part[v]] == 0) rg[v] += h->ewgt[e];", ""),
    "ab_arrival_threshold": ("if (phi_e[target[v]] == 1) rg[v] -= h->ewgt[e];", "if (phi_e[target[v]] == 2) rg[v] -= h->ewgt[e];"),
    "ab_no_sort": ("qsort(L, (size_t)len, sizeof(ab_item), ab_order);", ""),
    "ab_approve_nonnegative": ("approved[v] = (uint8_t)(in_m[v] && rg[v] > 0);", "approved[v] = (uint8_t)(in_m[v] && rg[v] >= 0);"),
    # apply
    "apply_bw_sign": ("    bw[s] -= h->vwgt[v];\n    bw[t] += h->vwgt[v];", "    bw[s] += h->vwgt[v];\n    bw[t] -= h->vwgt[v];"),
    # Section 4.3
    "rb_heavy_rule_dropped": ("if (2 * c > 3 * (bw[s] - A)) continue;", ""),
    "rb_deadzone_dropped": ("if (in_deadzone(p, A, bw[b])) continue;", ""),
    "rb_deadzone_sign": ("- (__int128)p->d_num * p->eps_num * A;", "+ (__int128)p->d_num * p->eps_num * A;"),
    "rb_deadzone_strict": ("  return lhs >= rhs;", "  return lhs > rhs;"),
    "rb_target_may_overload": ("if (bw[b] + c > Lmax) continue;", "if (bw[b] > Lmax) continue;"),
    "rb_positive_uses_ratio": ("lx = (__int128)x->gain * x->c;\n    ly = (__int128)y->gain * y->c;", "lx = (__int128)x->gain * y->c;\n    ly = (__int128)y->gain * x->c;"),
    "rb_negative_uses_product": ("lx = (__int128)x->gain * y->c;\n    ly = (__int128)y->gain * x->c;\n  }", "lx = (__int128)x->gain * x->c;\n    ly = (__int128)y->gain * y->c;\n  }"),
    "rb_class_order_flipped": ("if (cx != cy) return cx ? -1 : 1;", "if (cx != cy) return cx ? 1 : -1;"),
    "rb_tie_larger_id": ("  if (lx != ly) return lx > ly ? -1 : 1;\n  return (x->v > y->v) - (x->v < y->v);", "  if (lx != ly) return lx > ly ? -1 : 1;\n  return (x->v < y->v) - (x->v > y->v);"),
    "rb_prefix_one_too_many": ("for (int64_t i = 0; i < len[s] && prefix < excess; ++i) {", "for (int64_t i = 0; i < len[s] && prefix <= excess; ++i) {"),
    "rb_stops_after_one_round": ("    if (moved == 0) break;\n  }", "    break;\n  }"),
    # Algorithm 1
    "loop_non_strict_improvement": ("if (!st.imbalanced && (!have_best || st.objective < best_obj)) {", "if (!st.imbalanced && (!have_best || st.objective <= best_obj)) {"),
    "loop_no_rollback": ("      memcpy(part, best, sizeof(int32_t) * (size_t)n);\n      ojet_pincounts(h, k, part, phi, bw);\n    }", "    }"),
    "loop_no_locking": ("for (int32_t v = 0; v < n; ++v) locked[v] = approved[v];", ""),
    "loop_locks_kept_across_phases": ("    memset(locked, 0, nn);\n    int32_t it = 0;", "    int32_t it = 0;"),
    "loop_counter_not_reset": ("        memcpy(best, part, sizeof(int32_t) * (size_t)n);\n        it = 0;", "        memcpy(best, part, sizeof(int32_t) * (size_t)n);"),
    # Section 5 (matching schedule)
    "quotient_needs_two_pins": ("if (j != i && row[j] >= 1) qadj[(size_t)i * k + j] = 1;", "if (j != i && row[j] >= 2) qadj[(size_t)i * k + j] = 1;"),
    "schedule_degree_ascending": ("while (y >= 0 && (deg[order[y]] < deg[b] ||", "while (y >= 0 && (deg[order[y]] > deg[b] ||"),
    "schedule_tie_larger_id": ("(deg[order[y]] == deg[b] && order[y] > b))) {", "(deg[order[y]] == deg[b] && order[y] < b))) {"),
    "schedule_partner_lowest_degree": ("(best < 0 || deg[j] > deg[best])) best = j;", "(best < 0 || deg[j] < deg[best])) best = j;"),
    "schedule_one_pair_per_round": ("      round_of[np] = round;\n      ++np;\n    }", "      round_of[np] = round;\n      ++np;\n      break;\n    }"),
    # Section 6, Algorithm 4 (coarsening) and contraction
    "subrounds_no_doubling": ("    else size *= 2;\n", "\n"),
    "subrounds_cap_ignored": ("    if (size > cap) size = cap;\n", "\n"),
    "rating_counts_per_pin": ("if (C == u || last[C] == e) continue; /* once per edge and cluster */", "if (C == u) continue;"),
    "rating_divides_by_size": ("/ (uint64_t)(size - 1); }", "/ (uint64_t)size; }"),
    "rating_ignores_edge_limit": ("      if (size < 2 || size > rmax) continue;\n        const uint64_t t", "      if (size < 2) continue;\n        const uint64_t t"),
    "cluster_tie_larger_label": ("(acc[C] == acc[best] && C < best)", "(acc[C] == acc[best] && C > best)"),
    "cluster_ignores_weight_bound": ("if (cw[C] + h->vwgt[u] <= cmax && (best < 0", "if ((best < 0"),
    "cluster_moves_non_singletons": ("if (csize[u] != 1 || label[u] != u) continue;", "if (label[u] != u) continue;"),
    "swap_not_prevented": ("if (wu > wv || (wu == wv && u < v)) T2[u] = -1; /* u stays, v joins u */", ""),
    "swap_lighter_stays": ("if (wu > wv || (wu == wv && u < v)) T2[u] = -1;", "if (wu < wv || (wu == wv && u < v)) T2[u] = -1;"),
    "approve_heavier_first": ("if (g_cw_vwgt[x] != g_cw_vwgt[y]) return g_cw_vwgt[x] < g_cw_vwgt[y] ? -1 : 1;",
                              "if (g_cw_vwgt[x] != g_cw_vwgt[y]) return g_cw_vwgt[x] > g_cw_vwgt[y] ? -1 : 1;"),
    "approve_room_ignores_cluster": ("const int64_t room = cmax - cw[j];", "const int64_t room = cmax;"),
    "contract_keeps_single_pin_edges": ("if (teptr[e + 1] - teptr[e] >= 2) ord[nk++] = e;", "if (teptr[e + 1] - teptr[e] >= 1) ord[nk++] = e;"),
    "contract_no_merge": ("rep[e] = same ? rep[f] : e;", "rep[e] = e;"),
    "contract_merge_drops_weight": ("ew[rep[e]] += h->ewgt[e];", "ew[rep[e]] = h->ewgt[e];"),
    "contract_no_dedupe": ("if (d == 0 || tpins[o + i] != tpins[o + d - 1]) tpins", "if (1) tpins"),
    "round_always_rebalances_once": ("  if (over) st->rebalance_rounds = ojet_rebalance(h, p, part, phi, bw, &st->rebalance_moves);",
                                     "  if (over) { st->rebalance_rounds = 1; ojet_rebalance_round(h, p, part, phi, bw, NULL, NULL); }"),
}

RUNNER = """
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, pins
try:
    pins.run_all(oracle.Oracle, oracle.Params, source={src!r})
except AssertionError:
    sys.exit(3)
sys.exit(0)
"""


def test_every_mutant_applies_exactly_once():
    src = open(SRC).read()
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, name


def _run_variant(src_text, tmpdir, timeout):
    os.makedirs(tmpdir, exist_ok=True)
    path = os.path.join(tmpdir, "jet_oracle_variant.c")
    with open(path, "w") as f:
        f.write(src_text)
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), src=path)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return "timeout"  # e.g. an improvement test that always resets the counter never ends
    return r.returncode


def test_every_mutant_is_caught(tmp_path):
    src = open(SRC).read()
    jobs = {}
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as pool:
        for name, (old, new) in sorted(MUTANTS.items()):
            assert src.count(old) == 1, name
            jobs[name] = pool.submit(_run_variant, src.replace(old, new), str(tmp_path / name), 45)
        survivors = [name for name, fut in jobs.items() if fut.result() == 0]
    assert not survivors, f"mutants that pass every pin: {survivors}"


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: an unchanged copy passes, so failures above are the mutations'."""
    assert _run_variant(open(SRC).read(), str(tmp_path / "copy"), 300) == 0
