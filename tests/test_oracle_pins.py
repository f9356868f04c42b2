"""The CPU oracle against what the paper and mathematics fix (no GPU needed).

Each test runs one family of independent pins from ``pins.py`` on seeded tiny
hypergraphs: brute-force objective differences (gain, A(v), t(v)), the global
sequential replay that Algorithm 2 is defined to approximate exactly per edge,
closed forms of the connectivity metric, exact-rational rebalancing selection,
and a hand-worked example.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pins
from paper_2504_12013_gb300 import synth

INSTANCES = pins.small_instances(count=10)


def make(hg):
    return oracle.Oracle(hg)


def test_hand_example():
    pins.check_hand_example(make(pins.hand_example()[0]), oracle.Params)


def test_connectivity_closed_forms():
    pins.check_connectivity_closed_forms(make)


def test_balance_hand_values():
    pins.check_balance_hand_values(make)


@pytest.mark.parametrize("idx", range(6))
def test_rebalance_medium_blocks(idx):
    hg, k, part, eps, d = pins.medium_instances()[idx]
    o = make(hg)
    params = oracle.Params(k, eps=eps, d=d)
    pins.check_rebalance_round(o, params, hg, part)
    pins.check_rebalance_loop(o, params, hg, part)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_pincounts(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_pincounts(make(hg), hg, k, part)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_gain_and_affinity_brute_force(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_gain_and_affinity(make(hg), hg, k, part)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
@pytest.mark.parametrize("tau", [(0, 1), (3, 8), (3, 4), (1, 1)])
def test_candidates(idx, tau):
    hg, k, part = INSTANCES[idx]
    locked = (synth.stream_u64(idx + 5, hg.n) % np.uint64(4) == 0).astype(np.uint8)
    pins.check_candidates(make(hg), hg, k, part, locked, tau)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
@pytest.mark.parametrize("tau", [(0, 1), (3, 8), (3, 4), (1, 1)])
def test_afterburner_is_sequential_replay(idx, tau):
    hg, k, part = INSTANCES[idx]
    pins.check_afterburner(make(hg), hg, k, part, tau)


def test_afterburner_single_candidate_edges_give_plain_gain():
    # every edge holds at most one candidate -> recomputed gain = plain gain
    hg = synth.from_edges(8, [[0, 1], [2, 3], [4, 5], [6, 7], [1, 2]], ewgt=[1, 2, 3, 1, 5])
    part = np.array([0, 1, 0, 1, 1, 0, 0, 1], np.int32)
    o = make(hg)
    k = 2
    phi, _ = o.pincounts(k, part)
    in_m = np.array([1, 0, 0, 1, 1, 0, 1, 0], np.uint8)  # no edge holds two of {0,3,4,6}
    target = (1 - part).astype(np.int32)
    gain = np.array([o.gain(k, part, phi, v, 1 - part[v]) for v in range(8)], np.int64)
    _, rg, _ = o.afterburner(k, part, phi, target, gain, in_m)
    assert all(rg[v] == gain[v] for v in range(8) if in_m[v])


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_apply_matches_rebuild(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_apply(make(hg), hg, k, part, seed=idx + 3)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_rebalance_round_exact_selection(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_rebalance_round(make(hg), oracle.Params(k), hg, part)


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_rebalance_loop(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_rebalance_loop(make(hg), oracle.Params(k), hg, part)


def test_rebalance_exhaustive_tiny():
    """Every partition of a 7-vertex hypergraph into 3 blocks (3^7 = 2187)."""
    hg = synth.uniform(77, 7, 9, base=2, geo=(1, 2), size_cap=4, c_max=3, w_max=2)
    o = make(hg)
    params = oracle.Params(3)
    for code in range(3 ** 7):
        part = np.array([(code // 3 ** i) % 3 for i in range(7)], np.int32)
        pins.check_rebalance_round(o, params, hg, part)


def test_rebalance_deadzone_and_heavy_vertices():
    # one heavy vertex (c=10) in an overloaded block must never move; blocks
    # inside the deadzone must never receive a vertex
    edges = [[0, 1, 2], [2, 3], [3, 4, 5], [5, 6, 7], [7, 8, 0], [1, 9]]
    vw = [10, 1, 1, 1, 1, 1, 1, 1, 1, 1]
    hg = synth.from_edges(10, edges, vwgt=vw)
    o = make(hg)
    params = oracle.Params(3)
    for code in range(3 ** 10):
        part = np.array([(code // 3 ** i) % 3 for i in range(10)], np.int32)
        if code % 7:
            continue
        p2 = part.copy()
        phi, bw = o.pincounts(3, p2)
        bw0 = bw.copy()
        W, A, Lmax, dz = pins.balance_constants(hg, 3)
        moved, flag, tgt = o.rebalance_round(params, p2, np.ascontiguousarray(phi), bw)
        for v in np.nonzero(flag)[0]:
            s, t = part[v], tgt[v]
            assert bw0[s] > Lmax
            assert 2 * vw[v] <= 3 * (bw0[s] - A)
            assert bw0[t] + vw[v] <= Lmax and bw0[t] < dz


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_refine_round_stats(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_refine_round_stats(make(hg), oracle.Params(k), hg, part, (3, 4))


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_refine_loop(idx):
    hg, k, part = INSTANCES[idx]
    pins.check_refine_loop(make(hg), oracle.Params(k), hg, part, oracle.TAU_SCHEDULE, 3)


def test_refine_loop_random_10k():
    hg, k, part = synth.config_random_10k(1)
    pins.check_refine_loop(make(hg), oracle.Params(k), hg, part, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT)


def test_refine_random_10k_invariants():
    """The 10,000-vertex workload: balanced start, so no loss and balance kept."""
    hg, k, part = synth.config_random_10k(1)
    o = make(hg)
    params = oracle.Params(k)
    p = part.copy()
    iters, obj, phase = o.refine(params, p)
    assert obj == pins.objective_sets(hg, p)
    assert obj < o.objective(k, part)
    assert np.bincount(p, weights=hg.vwgt, minlength=k).max() <= o.lmax(params)
    assert all(int(x) >= oracle.ITERATION_LIMIT for x in phase)
    p2 = part.copy()
    assert o.refine(params, p2)[:2] == (iters, obj) and np.array_equal(p, p2)


# ---------------------------------------------------------------- Section 5: matching schedule
def test_schedule_hand_example():
    pins.check_schedule_hand(make(pins.hand_example()[0]))


@pytest.mark.parametrize("idx", range(len(INSTANCES)))
def test_quotient_and_schedule_of_partitions(idx):
    hg, k, part = INSTANCES[idx]
    o = make(hg)
    pins.check_schedule_invariants(o, pins.check_quotient(o, hg, k, part))


@pytest.mark.parametrize("q_idx", range(8))
def test_schedule_invariants_random_quotients(q_idx):
    q = pins.random_quotients()[q_idx]
    pins.check_schedule_invariants(make(pins.hand_example()[0]), q)


def test_schedule_of_a_complete_quotient():
    """K_k: all k(k-1)/2 pairs are scheduled, in at least k - 1 rounds (every block has k - 1 quotient
    edges and meets at most one per round)."""
    for k in (2, 4, 8, 16):
        q = np.ones((k, k), np.uint8) - np.eye(k, dtype=np.uint8)
        pairs, rnd, nr = oracle.schedule(q)
        assert len(pairs) == k * (k - 1) // 2
        assert nr >= k - 1


# Section 6, Algorithm 4 (coarsening) and contraction

def test_coarsen_hand_examples():
    pins.check_coarsen_hand(make)


def test_subround_schedule():
    pins.check_subrounds(make(pins.hand_example()[0]))


def test_clustering_against_restatements():
    pins.check_clustering(make)


def test_clustering_edge_cases():
    """No edges: every vertex stays alone.  One vertex heavier than the bound: it never joins and no
    cluster it would grow is rated.  All sub-rounds of one vertex equal the sequential restatement."""
    hg = synth.from_edges(5, [])
    assert list(make(hg).cluster(10, np.arange(5, dtype=np.int32))) == [0, 1, 2, 3, 4]
    hg = synth.from_edges(3, [[0, 1, 2]], vwgt=[9, 1, 1])
    lab = make(hg).cluster(5, np.arange(3, dtype=np.int32))
    assert lab[0] == 0 and lab[1] == lab[2]
    c, mp = make(hg).contract(lab)
    assert c.n == 2 and c.m == 1 and list(c.vwgt) == [9, 2]


def test_rating_overflow_is_reported():
    # a vertex in three edges of weight 2^31 - 1 and size 2: three terms of about 2^63
    hg = synth.from_edges(2, [[0, 1]] * 3, ewgt=[2 ** 31 - 1] * 3)
    with pytest.raises(OverflowError):
        make(hg).cluster(10, np.arange(2, dtype=np.int32))


def test_projection_keeps_objective_over_levels():
    hg = synth.uniform(8, 2000, 2300, base=2, geo=(1, 2), size_cap=30, c_max=3, w_max=2)
    order = synth.stream_u64(8, hg.n).argsort(kind="stable").astype(np.int32)
    for _ in range(3):
        o = make(hg)
        c = pins.check_contraction(o, hg, o.cluster(int(hg.vwgt.sum()) // 50, order))
        assert c.n < hg.n
        hg = c
        order = synth.stream_u64(9, hg.n).argsort(kind="stable").astype(np.int32)


def test_graph_afterburner_is_a_neighbour_sum():
    """On graphs (two-pin edges), Algorithm 2's recomputed gain of a candidate v equals the sum over
    its neighbours u of omega(e) * ([b'(u) != s] - [b'(u) != t]), where b'(u) is u's target if u is a
    candidate ordered before v (gain desc, id asc), else Pi(u): the graph path's afterburner (R27)."""
    for seed in range(6):
        g = synth.graph(seed, 300, 1200, local=0.6, window=12, w_max=4)
        k = (2, 4, 8)[seed % 3]
        part = synth.part_random(seed + 40, g.n, k)
        o = make(g)
        phi, _ = o.pincounts(k, part)
        for tau in ((3, 4), (0, 1)):
            _, target, gain, in_m = o.candidates(k, part, phi, np.zeros(g.n, np.uint8), tau)
            _, rg, _ = o.afterburner(k, part, phi, target, gain, in_m)
            for v in np.flatnonzero(in_m):
                s, t, acc = part[v], target[v], 0
                for e in g.inc[g.vptr[v]:g.vptr[v + 1]]:
                    a, b = g.pins[g.eptr[e]:g.eptr[e + 1]]
                    u = b if a == v else a
                    before = in_m[u] and (gain[u] > gain[v] or (gain[u] == gain[v] and u < v))
                    bu = target[u] if before else part[u]
                    acc += int(g.ewgt[e]) * (int(bu != s) - int(bu != t))
                assert acc == rg[v], (seed, tau, int(v))


def test_graph_candidates_from_neighbour_blocks():
    """On graphs, conn(v, b) = sum of omega over neighbours in b and A(v) = conn(v, Pi(v)), so the best
    target (ties to the smaller block), its gain and the temperature filter follow from the neighbours'
    blocks alone (R27); they must equal the oracle's phi-based candidates."""
    for seed in range(6):
        g = synth.graph(seed + 20, 250, 1000, local=0.5, window=9, w_max=5)
        k = (3, 8, 16)[seed % 3]
        part = synth.part_random(seed + 60, g.n, k)
        o = make(g)
        phi, _ = o.pincounts(k, part)
        for tau in ((3, 4), (3, 8), (0, 1)):
            _, target, gain, in_m = o.candidates(k, part, phi, np.zeros(g.n, np.uint8), tau)
            for v in range(g.n):
                s = part[v]
                conn = {}
                for e in g.inc[g.vptr[v]:g.vptr[v + 1]]:
                    a, b = g.pins[g.eptr[e]:g.eptr[e + 1]]
                    u = b if a == v else a
                    conn[part[u]] = conn.get(part[u], 0) + int(g.ewgt[e])
                A = conn.get(s, 0)
                adj = [b for b in conn if b != s]
                if not adj:
                    assert not in_m[v]
                    continue
                t = min(adj, key=lambda b: (-conn[b], b))
                gv = conn[t] - A
                keep = Fraction(gv) >= -Fraction(tau[0], tau[1]) * A
                assert bool(in_m[v]) == keep, (seed, tau, v)
                if keep:
                    assert (target[v], gain[v]) == (t, gv), (seed, tau, v)
