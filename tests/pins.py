"""Independent pins for the CPU oracle.

Every check here recomputes what the oracle computes by a *different route*
than the oracle's own arithmetic: full objective recomputation from vertex
sets instead of pin counts, objective differences instead of the gain rule,
a global sequential replay instead of the per-edge afterburner, exact
``fractions.Fraction`` priorities instead of cross-multiplied integers, closed
forms (edge cut of a graph, all-in-one-block, singleton blocks) and a
hand-worked example.  The checks are plain functions raising AssertionError so
that ``test_oracle_mutants.py`` can run them against deliberately broken
copies of the oracle and confirm that each planted mistake is caught.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from paper_2504_12013_gb300 import synth


# ------------------------------------------------------------------ helpers

def lam_sets(hg, part, e):
    """lambda(e) = number of distinct blocks among the pins of e (Section 2)."""
    return len({int(part[v]) for v in hg.edge(e)})


def objective_sets(hg, part):
    """(lambda-1) recomputed from vertex sets; empty edges contribute 0."""
    tot = 0
    for e in range(hg.m):
        lam = lam_sets(hg, part, e)
        if lam:
            tot += (lam - 1) * int(hg.ewgt[e])
    return tot


def moved(part, v, b):
    q = np.array(part, dtype=np.int32, copy=True)
    q[v] = b
    return q


def brute_gain(hg, part, v, b):
    """gain(v,b) = objective before - objective after moving v to b.

    Only the edges of I(v) change when v moves, so the difference is taken
    over them, each lambda recounted from the vertex sets before and after.
    """
    after = moved(part, v, b)
    d = 0
    for e in hg.incident(v):
        e = int(e)
        d += (lam_sets(hg, part, e) - lam_sets(hg, after, e)) * int(hg.ewgt[e])
    return d


def brute_gain_full(hg, part, v, b):
    """The same difference by recomputing the whole objective twice."""
    return objective_sets(hg, part) - objective_sets(hg, moved(part, v, b))


def brute_affinity(hg, part, k, v):
    """A(v) = -(gain of moving v into a block that no edge of v touches).

    A fresh block id k (outside [0,k)) is never adjacent, so the objective
    difference of that move is exactly -sum of omega(e) over e in I(v) with
    |e cap V_s| > 1.
    """
    return -brute_gain(hg, part, v, k)


def adjacent_blocks(hg, part, v):
    s = int(part[v])
    out = set()
    for e in hg.incident(v):
        for u in hg.edge(int(e)):
            out.add(int(part[u]))
    out.discard(s)
    return out


def balance_constants(hg, k, eps=(3, 100), d=(1, 10)):
    W = int(np.sum(hg.vwgt, dtype=np.int64))
    A = -(-W // k)
    lmax_real = (1 + Fraction(*eps)) * A
    Lmax = int(lmax_real)  # floor, positive
    dz = lmax_real - Fraction(*d) * Fraction(*eps) * A
    return W, A, Lmax, dz


def small_instances(count=6, base_seed=11):
    """Tiny seeded hypergraphs with ties (unit weights) and without (random weights)."""
    out = []
    for i in range(count):
        seed = base_seed + i
        n = 10 + 4 * i
        m = 12 + 3 * i
        k = 2 + i % 4
        cw = 1 if i % 2 == 0 else 3
        hg = synth.uniform(seed, n, m, base=1 if i % 3 == 0 else 2, geo=(1, 2), size_cap=6, c_max=cw, w_max=cw)
        part = synth.part_random(seed * 7 + 1, n, k)
        out.append((hg, k, part))
    return out


# ------------------------------------------------------------------ Section 2

def check_pincounts(orc, hg, k, part):
    phi, bw = orc.pincounts(k, part)
    sizes = np.diff(hg.eptr)
    assert np.array_equal(phi.sum(axis=1), sizes), "row sums of phi must equal |e|"
    deg = np.diff(hg.vptr)
    col = np.bincount(part, weights=deg, minlength=k).astype(np.int64)
    assert np.array_equal(phi.sum(axis=0), col), "column sums of phi must equal the incidences of each block"
    assert np.array_equal(bw, np.bincount(part, weights=hg.vwgt, minlength=k).astype(np.int64)), "c(V_i)"
    # lambda(e) from phi must equal the distinct-block count of the edge
    for e in range(hg.m):
        assert int(np.count_nonzero(phi[e])) == lam_sets(hg, part, e)


def check_connectivity_closed_forms(make):
    """make(hg) returns an oracle bound to hg."""
    # graph (all |e| = 2): (lambda-1) is the weighted edge cut
    g = synth.uniform(5, 40, 90, base=2, geo=(1, 1), size_cap=2, w_max=5)
    assert np.all(np.diff(g.eptr) == 2)
    orc = make(g)
    for k in (2, 3, 7):
        part = synth.part_random(17 + k, g.n, k)
        u, v = g.pins[0::2], g.pins[1::2]
        cut = int(np.sum(g.ewgt[part[u] != part[v]], dtype=np.int64))
        assert orc.objective(k, part) == cut, "edge cut of a graph"
    h = synth.uniform(6, 30, 40, base=1, geo=(1, 3), size_cap=8, w_max=4)
    sizes = np.diff(h.eptr)
    orc = make(h)
    # everything in one block: 0
    assert orc.objective(3, np.full(h.n, 2, np.int32)) == 0
    # every vertex its own block: sum (|e|-1) omega(e) over non-empty edges
    want = int(np.sum((sizes - 1).clip(min=0) * h.ewgt, dtype=np.int64))
    assert orc.objective(h.n, np.arange(h.n, dtype=np.int32)) == want
    # relabelling blocks leaves (lambda-1) unchanged
    part = synth.part_random(3, h.n, 5)
    perm = np.array([3, 0, 4, 1, 2], dtype=np.int32)
    assert orc.objective(5, part) == orc.objective(5, perm[part])
    # empty edges contribute 0
    e = synth.from_edges(4, [[0, 1], [], [2, 3]], ewgt=[2, 9, 3])
    assert make(e).objective(2, np.array([0, 1, 0, 0], np.int32)) == 2


# ------------------------------------------------------------------ Section 4.1

def check_gain_and_affinity(orc, hg, k, part):
    phi, _ = orc.pincounts(k, part)
    for v in range(hg.n):
        for b in range(k):
            if b == part[v]:
                continue
            g = orc.gain(k, part, phi, v, b)
            assert g == brute_gain(hg, part, v, b), (v, b)
            if v < 8:
                assert g == brute_gain_full(hg, part, v, b), (v, b)
        assert orc.affinity(k, part, phi, v) == brute_affinity(hg, part, k, v), v


def check_candidates(orc, hg, k, part, locked, tau):
    phi, _ = orc.pincounts(k, part)
    cnt, target, gain, in_m = orc.candidates(k, part, phi, locked, tau)
    t = Fraction(*tau)
    want_count = 0
    for v in range(hg.n):
        if locked[v]:
            assert not in_m[v]
            continue
        adj = adjacent_blocks(hg, part, v)
        if not adj:
            assert target[v] == -1 and not in_m[v]
            continue
        gains = {b: brute_gain(hg, part, v, b) for b in adj}
        best = max(gains.values())
        tb = min(b for b in adj if gains[b] == best)
        assert target[v] == tb, (v, target[v], tb)
        assert gain[v] == best
        A = brute_affinity(hg, part, k, v)
        want = best >= -t * A
        assert bool(in_m[v]) == want, (v, best, A, tau)
        want_count += want
    assert cnt == want_count


# ------------------------------------------------------------------ Section 4.2

def sequential_replay(hg, part, target, gain, in_m):
    """Move M one vertex at a time in the order (gain desc, id asc); the
    recomputed gain of v is the objective drop of its own move, by full
    recomputation, with every earlier vertex of M already moved."""
    order = sorted((v for v in range(hg.n) if in_m[v]), key=lambda v: (-int(gain[v]), v))
    cur = np.array(part, dtype=np.int32, copy=True)
    rg = np.zeros(hg.n, dtype=np.int64)
    obj = objective_sets(hg, cur)
    for v in order:
        cur[v] = target[v]
        nxt = objective_sets(hg, cur)
        rg[v] = obj - nxt
        obj = nxt
    return rg


def check_afterburner(orc, hg, k, part, tau, locked=None):
    phi, _ = orc.pincounts(k, part)
    locked = np.zeros(hg.n, np.uint8) if locked is None else locked
    _, target, gain, in_m = orc.candidates(k, part, phi, locked, tau)
    cnt, rg, approved = orc.afterburner(k, part, phi, target, gain, in_m)
    want = sequential_replay(hg, part, target, gain, in_m)
    for v in range(hg.n):
        if in_m[v]:
            assert rg[v] == want[v], (v, rg[v], want[v])
        else:
            assert rg[v] == 0
    assert np.array_equal(approved.astype(bool), (in_m.astype(bool) & (want > 0)))
    assert cnt == int(np.count_nonzero(approved))
    # invariance: pin order inside edges and edge order do not change the result
    hp, _ = synth.permuted(hg, 99)
    orp = type(orc)(hp, orc.source)
    phip, _ = orp.pincounts(k, part)
    _, rgp, app2 = orp.afterburner(k, part, phip, target, gain, in_m)
    assert np.array_equal(rgp, rg) and np.array_equal(app2, approved)


def check_apply(orc, hg, k, part, seed):
    phi, bw = orc.pincounts(k, part)
    rng = synth.stream_u64(seed, 2 * hg.n)
    move = (rng[:hg.n] % 3 == 0).astype(np.uint8)
    target = (rng[hg.n:] % np.uint64(k)).astype(np.int32)
    target = np.where(target == part, (target + 1) % k, target).astype(np.int32)
    p2 = np.array(part, np.int32, copy=True)
    phi2 = np.ascontiguousarray(phi.copy())
    bw2 = bw.copy()
    orc.apply(k, p2, phi2, bw2, move, target)
    want = np.where(move.astype(bool), target, part).astype(np.int32)
    assert np.array_equal(p2, want)
    ref_phi, ref_bw = orc.pincounts(k, want)
    assert np.array_equal(phi2, ref_phi)
    assert np.array_equal(bw2, np.bincount(want, weights=hg.vwgt, minlength=k).astype(np.int64))
    assert orc.connectivity(k, phi2) == objective_sets(hg, want)


# ------------------------------------------------------------------ Section 4.3

def expected_rebalance_round(hg, k, part, eps=(3, 100), d=(1, 10)):
    """Section 4.3 with Fractions and brute-force gains; returns {v: target}."""
    W, A, Lmax, dz = balance_constants(hg, k, eps, d)
    bw = np.bincount(part, weights=hg.vwgt, minlength=k).astype(np.int64)
    over = [b for b in range(k) if bw[b] > Lmax]
    if not over:
        return None
    per_block = {b: [] for b in over}
    for v in range(hg.n):
        s = int(part[v])
        if s not in per_block:
            continue
        c = int(hg.vwgt[v])
        if c > Fraction(3, 2) * (int(bw[s]) - A):
            continue
        elig = [b for b in range(k) if b != s and bw[b] + c <= Lmax and not (bw[b] >= dz)]
        if not elig:
            continue
        gains = {b: brute_gain(hg, part, v, b) for b in elig}
        g = max(gains.values())
        t = min(b for b in elig if gains[b] == g)
        prio = (1, Fraction(g * c)) if g >= 0 else (0, Fraction(g, c))
        per_block[s].append((prio, v, c, t))
    sel = {}
    for s, items in per_block.items():
        items.sort(key=lambda it: (-it[0][0], -it[0][1], it[1]))
        excess = int(bw[s]) - Lmax
        acc = 0
        for prio, v, c, t in items:
            if acc >= excess:
                break
            sel[v] = t
            acc += c
    return sel


def check_rebalance_round(orc, params, hg, part):
    k = params.k
    p2 = np.array(part, np.int32, copy=True)
    phi, bw = orc.pincounts(k, p2)
    phi = np.ascontiguousarray(phi)
    want = expected_rebalance_round(hg, k, part, params.eps, params.d)
    moved_cnt, flag, tgt = orc.rebalance_round(params, p2, phi, bw)
    if want is None:
        assert moved_cnt == -1 and not flag.any()
        return
    got = {int(v): int(tgt[v]) for v in np.nonzero(flag)[0]}
    assert got == want, (got, want)
    assert moved_cnt == len(want)
    exp_part = np.array(part, np.int32, copy=True)
    for v, t in want.items():
        exp_part[v] = t
    assert np.array_equal(p2, exp_part)
    ref_phi, ref_bw = orc.pincounts(k, exp_part)
    assert np.array_equal(phi, ref_phi) and np.array_equal(bw, ref_bw)


def check_rebalance_loop(orc, params, hg, part):
    k = params.k
    p2 = np.array(part, np.int32, copy=True)
    phi, bw = orc.pincounts(k, p2)
    phi = np.ascontiguousarray(phi)
    rounds, moves = orc.rebalance(params, p2, phi, bw)
    # replay round by round with the independent selection
    cur = np.array(part, np.int32, copy=True)
    r = mv = 0
    while r < params.max_rebalance_rounds:
        sel = expected_rebalance_round(hg, k, cur, params.eps, params.d)
        if sel is None:
            break
        r += 1
        mv += len(sel)
        for v, t in sel.items():
            cur[v] = t
        if not sel:
            break
    assert (rounds, moves) == (r, mv)
    assert np.array_equal(p2, cur)


# ------------------------------------------------------------------ Algorithm 1

def check_refine_round_stats(orc, params, hg, part, tau):
    k = params.k
    p2 = np.array(part, np.int32, copy=True)
    phi, bw = orc.pincounts(k, p2)
    phi = np.ascontiguousarray(phi)
    locked = np.zeros(hg.n, np.uint8)
    st = orc.refine_round(params, tau, p2, phi, bw, locked)
    assert st["objective"] == objective_sets(hg, p2)
    _, _, Lmax, _ = balance_constants(hg, k, params.eps, params.d)
    bwr = np.bincount(p2, weights=hg.vwgt, minlength=k).astype(np.int64)
    assert np.array_equal(bw, bwr)
    assert st["max_block_weight"] == int(bwr.max())
    assert st["imbalanced"] == int(bwr.max() > Lmax)
    ref_phi, _ = orc.pincounts(k, p2)
    assert np.array_equal(phi, ref_phi)
    # locks are exactly the afterburner-approved vertices of this iteration
    phi0, _ = orc.pincounts(k, part)
    _, target, gain, in_m = orc.candidates(k, part, phi0, np.zeros(hg.n, np.uint8), tau)
    _, rg, approved = orc.afterburner(k, part, phi0, target, gain, in_m)
    assert np.array_equal(locked, approved)
    assert st["candidates"] == int(in_m.sum()) and st["approved"] == int(approved.sum())


def check_refine_loop(orc, params, hg, part, schedule, limit):
    """Algorithm 1 restated in Python over oracle iterations must match ojet_refine."""
    k = params.k
    p1 = np.array(part, np.int32, copy=True)
    iters, obj, phase = orc.refine(params, p1, schedule, limit)
    # Python restatement of the loop control (R7, R11)
    cur = np.array(part, np.int32, copy=True)
    phi, bw = orc.pincounts(k, cur)
    phi = np.ascontiguousarray(phi)
    _, _, Lmax, _ = balance_constants(hg, k, params.eps, params.d)
    best = cur.copy() if bw.max() <= Lmax else None
    best_obj = objective_sets(hg, cur) if best is not None else None
    total = 0
    for tau in schedule:
        locked = np.zeros(hg.n, np.uint8)
        it = 0
        while it < limit:
            st = orc.refine_round(params, tau, cur, phi, bw, locked)
            total += 1
            it += 1
            if not st["imbalanced"] and (best is None or st["objective"] < best_obj):
                best, best_obj, it = cur.copy(), st["objective"], 0
        if best is not None:
            cur = best.copy()
            phi, bw = orc.pincounts(k, cur)
            phi = np.ascontiguousarray(phi)
    assert total == iters
    assert np.array_equal(cur, p1)
    assert obj == objective_sets(hg, p1)
    assert int(phase.sum()) == iters and all(int(x) >= limit for x in phase)
    bw0 = np.bincount(part, weights=hg.vwgt, minlength=k)
    if bw0.max() <= Lmax:  # rollback guarantees no loss and balance
        assert obj <= objective_sets(hg, part)
        assert np.bincount(p1, weights=hg.vwgt, minlength=k).max() <= Lmax
    # determinism
    p3 = np.array(part, np.int32, copy=True)
    assert orc.refine(params, p3, schedule, limit)[:2] == (iters, obj) and np.array_equal(p1, p3)


# ------------------------------------------------------------------ hand-worked example

def hand_example():
    """6 vertices, 4 edges, k=2, omega(e2)=2, Pi = [0,0,1,1,1,0].

    Worked by hand from the definitions of Section 2 and Algorithm 2:
      phi: e0={0,1,2}:[2,1]  e1={2,3}:[0,2]  e2={3,4,5}:[1,2] (w=2)  e3={1,4}:[1,1]
      (lambda-1) = 1 + 0 + 2 + 1 = 4
      gains to the other block: v0 0, v1 +1, v2 0, v3 -1, v4 +1, v5 +2
      A(v): v0 1, v1 1, v2 1, v3 3, v4 2, v5 0
    tau = 1/2: every vertex is a candidate (v3: -1 >= -3/2); order 5,1,4,0,2,3;
      per-edge replay: e0 -> v1 0, v0 +1, v2 -1; e1 -> v2 -1, v3 +1;
      e2 -> v5 +2, v4 -2, v3 0; e3 -> v1 +1, v4 -1
      recomputed gains v0..v5 = 1, 1, -2, 1, -3, 2  -> approved {0,1,3,5}
      after the moves Pi = [1,1,1,0,1,1], c(V) = [1,5], (lambda-1) = 3;
      A = ceil(6/2) = 3, L_max = floor(1.03*3) = 3 -> block 1 overloaded by 2;
      block 0 eligible (1000*1 < 1027*3); gains to 0: v0 -1, v1 -2, v2 0, v4 -1, v5 0
      priority order v2, v5, v0, v4, v1 -> move {v2, v5} -> Pi = [1,1,0,0,1,0],
      c(V) = [3,3], (lambda-1) = 3; one rebalancing round, two moves.
    tau = 0: v3 (-1 < 0) drops out; recomputed gains v0 1, v1 1, v2 -2, v4 -3, v5 2
      -> approved {0,1,5} -> all in block 1, (lambda-1) = 0, c(V) = [0,6];
      rebalancing (excess 3) gains to 0: v0 -1, v1 -2, v2 -2, v3 -3, v4 -3, v5 -2
      order v0, v1, v2, v5, v3, v4 -> move {v0,v1,v2} -> Pi = [0,0,0,1,1,1],
      (lambda-1) = 2.
    """
    hg = synth.from_edges(6, [[0, 1, 2], [2, 3], [3, 4, 5], [1, 4]], ewgt=[1, 1, 2, 1])
    part = np.array([0, 0, 1, 1, 1, 0], np.int32)
    return hg, part


def check_hand_example(orc, params_cls):
    hg, part = hand_example()
    k = 2
    params = params_cls(k)
    phi, bw = orc.pincounts(k, part)
    assert phi.tolist() == [[2, 1], [0, 2], [1, 2], [1, 1]]
    assert bw.tolist() == [3, 3]
    assert orc.connectivity(k, phi) == 4
    assert [orc.gain(k, part, phi, v, 1 - part[v]) for v in range(6)] == [0, 1, 0, -1, 1, 2]
    assert [orc.affinity(k, part, phi, v) for v in range(6)] == [1, 1, 1, 3, 2, 0]
    assert orc.lmax(params) == 3 and orc.avg_block(k) == 3
    z = np.zeros(6, np.uint8)
    cnt, target, gain, in_m = orc.candidates(k, part, phi, z, (1, 2))
    assert cnt == 6 and target.tolist() == [1, 1, 0, 0, 0, 1]
    cnt, rg, approved = orc.afterburner(k, part, phi, target, gain, in_m)
    assert rg.tolist() == [1, 1, -2, 1, -3, 2] and approved.tolist() == [1, 1, 0, 1, 0, 1] and cnt == 4
    p2, phi2, bw2 = part.copy(), np.ascontiguousarray(phi.copy()), bw.copy()
    st = orc.refine_round(params, (1, 2), p2, phi2, bw2, z.copy())
    assert p2.tolist() == [1, 1, 0, 0, 1, 0]
    assert st == {"candidates": 6, "approved": 4, "rebalance_rounds": 1, "rebalance_moves": 2,
                  "objective": 3, "max_block_weight": 3, "imbalanced": 0}
    p3, phi3, bw3 = part.copy(), np.ascontiguousarray(phi.copy()), bw.copy()
    st = orc.refine_round(params, (0, 1), p3, phi3, bw3, z.copy())
    assert p3.tolist() == [0, 0, 0, 1, 1, 1]
    assert st == {"candidates": 5, "approved": 3, "rebalance_rounds": 1, "rebalance_moves": 3,
                  "objective": 2, "max_block_weight": 3, "imbalanced": 0}


def check_balance_hand_values(make):
    """Hand values of Section 2's balance bound: ceil(c(V)/k) and floor((1+eps)ceil(c(V)/k))."""
    h = synth.uniform(1, 10_000, 10, base=2, geo=(1, 2), size_cap=4)  # c(V) = 10,000
    o = make(h)
    assert o.total_weight() == 10_000
    assert o.avg_block(8) == 1250 and o.lmax(_P(8)) == 1287          # 1.03 * 1250 = 1287.5
    assert o.avg_block(3) == 3334 and o.lmax(_P(3)) == 3434          # 1.03 * 3334 = 3434.02
    assert o.lmax(_P(8, eps=(1, 10))) == 1375                         # 1.1 * 1250
    assert o.lmax(_P(7, eps=(0, 1))) == 1429                          # eps = 0: ceil(10000/7)


class _P:
    def __init__(self, k, eps=(3, 100), d=(1, 10), max_rebalance_rounds=32):
        self.k, self.eps, self.d, self.max_rebalance_rounds = k, eps, d, max_rebalance_rounds

    def c(self):
        import oracle
        return oracle.OParams(self.k, self.eps[0], self.eps[1], self.d[0], self.d[1], self.max_rebalance_rounds)


def medium_instances():
    """Larger blocks (ceil(c(V)/k) ~ 100) so that eps bites; the last two use
    eps = 1/5, d = 1/2 so that the deadzone (width d*eps*ceil(c(V)/k)) spans
    several weight units and excludes blocks that still have room."""
    out = []
    for i, (n, k, cmax, eps, d) in enumerate(((160, 3, 2, (3, 100), (1, 10)), (200, 4, 3, (3, 100), (1, 10)),
                                              (150, 2, 1, (3, 100), (1, 10)))):
        hg = synth.uniform(40 + i, n, n + n // 4, base=2, geo=(1, 2), size_cap=5, c_max=cmax, w_max=2)
        part = synth.part_random(90 + i, n, k)
        # skew: push a slice of vertices into block 0 so it is overloaded
        part[: n // 5] = 0
        out.append((hg, k, part, eps, d))
    # unit weights, c(V) = 180, k = 3: ceil = 60, L_max = floor(1.2 * 60) = 72, deadzone from
    # 72 - 0.5 * 0.2 * 60 = 66.  Block 1 holds 68 (in the deadzone, room for 4), or exactly 66
    # (on the deadzone boundary, which the deadzone includes); block 0 is overloaded.
    for i, sizes in enumerate(((90, 68, 22), (80, 70, 30), (94, 66, 20))):
        n, k = 180, 3
        hg = synth.uniform(60 + i, n, 240, base=2, geo=(1, 2), size_cap=5, w_max=2)
        order = np.argsort(synth.stream_u64(70 + i, n), kind="stable")
        part = np.empty(n, np.int32)
        part[order] = np.repeat(np.arange(k, dtype=np.int32), sizes)
        out.append((hg, k, part, (1, 5), (1, 2)))
    return out


# ------------------------------------------------------------------ suite

# ---------------------------------------------------------------- Section 5: matching schedule
def schedule_hand_example():
    """Quotient graph on 4 blocks with edges {0,1}, {1,2}, {2,3}, {1,3}; expected schedule by hand.

    Round 0: degrees 0:1, 1:3, 2:2, 3:2, so block 1 goes first; its unmatched neighbours of the
    largest degree are 2 and 3 (both 2), the smaller id wins: (1, 2).  Blocks 3 and 0 then find no
    unmatched neighbour.  Round 1: remaining {0,1}, {2,3}, {1,3}; degrees 0:1, 1:2, 2:1, 3:2; block 1
    first, its neighbours 0 (degree 1) and 3 (degree 2): (1, 3); 0 and 2 find nothing.  Round 2:
    {0,1} and {2,3}, all degrees 1: (0, 1) then (2, 3).
    """
    q = np.zeros((4, 4), np.uint8)
    for i, j in ((0, 1), (1, 2), (2, 3), (1, 3)):
        q[i, j] = q[j, i] = 1
    return q, [(1, 2), (1, 3), (0, 1), (2, 3)], [0, 1, 2, 2], 3


def check_schedule_hand(orc):
    q, want_pairs, want_rounds, want_n = schedule_hand_example()
    pairs, rnd, nr = orc.schedule(q)
    assert [tuple(int(x) for x in p) for p in pairs] == want_pairs, pairs
    assert list(rnd) == want_rounds and nr == want_n, (rnd, nr)


def check_quotient(orc, hg, k, part):
    """Q from phi equals the block pairs that share a hyperedge, counted from the partition."""
    phi, _ = orc.pincounts(k, part)
    q = orc.quotient(k, phi)
    want = np.zeros((k, k), np.uint8)
    for e in range(hg.m):
        bl = sorted({int(part[v]) for v in hg.edge(e)})
        for i in bl:
            for j in bl:
                if i != j:
                    want[i, j] = 1
    assert np.array_equal(q, want)
    return q


def check_schedule_invariants(orc, q):
    """Every quotient edge exactly once; each round a matching that is maximal in the edges left at its
    start; each round opens with a block of the largest remaining degree (smallest such id)."""
    k = q.shape[0]
    pairs, rnd, nr = orc.schedule(q)
    edges = {(i, j) for i in range(k) for j in range(i + 1, k) if q[i, j]}
    got = [tuple(sorted((int(a), int(b)))) for a, b in pairs]
    assert len(got) == len(set(got)) and set(got) == edges
    assert list(rnd) == sorted(rnd) and (nr == (int(rnd[-1]) + 1 if len(rnd) else 0))
    remaining = set(edges)
    for r in range(nr):
        this = [got[x] for x in range(len(got)) if rnd[x] == r]
        used = [b for p in this for b in p]
        assert len(used) == len(set(used)), "a block in two pairs of one round"
        deg = np.zeros(k, np.int64)
        for i, j in remaining:
            deg[i] += 1
            deg[j] += 1
        first = int(pairs[list(rnd).index(r)][0])
        assert deg[first] == deg.max() and first == int(np.argmax(deg)), (r, first)
        free = set(range(k)) - set(used)
        assert not any(i in free and j in free for i, j in remaining - set(this)), "round not maximal"
        remaining -= set(this)
    assert not remaining


def random_quotients(count=8, seed=71):
    u = synth.stream_u64(seed, 4096)
    out = []
    for t in range(count):
        k = 2 + int(u[t] % np.uint64(39))
        dens = 1 + int(u[100 + t] % np.uint64(9))  # percent-in-ten of edges present
        bits = synth.stream_u64(seed + 17 * t + 1, k * k)
        q = np.zeros((k, k), np.uint8)
        for i in range(k):
            for j in range(i + 1, k):
                if int(bits[i * k + j] % np.uint64(10)) < dens:
                    q[i, j] = q[j, i] = 1
        out.append(q)
    return out


def run_all(orc_cls, params_cls, source=None):
    """Every pin; raises AssertionError on the first failure."""
    def O(hg):
        return orc_cls(hg, source)

    check_hand_example(O(hand_example()[0]), params_cls)
    check_balance_hand_values(O)
    check_connectivity_closed_forms(O)
    for hg, k, part, eps, d in medium_instances():
        o = O(hg)
        params = params_cls(k, eps=eps, d=d)
        check_rebalance_round(o, params, hg, part)
        check_rebalance_loop(o, params, hg, part)
    hg, k, part = synth.config_random_10k(1)
    check_refine_loop(O(hg), params_cls(k), hg, part, ((3, 4), (3, 8), (0, 1)), 8)
    for i, (hg, k, part) in enumerate(small_instances()):
        o = O(hg)
        check_pincounts(o, hg, k, part)
        check_gain_and_affinity(o, hg, k, part)
        for tau in ((0, 1), (3, 8), (3, 4), (1, 1)):
            locked = (synth.stream_u64(i + 5, hg.n) % np.uint64(4) == 0).astype(np.uint8)
            check_candidates(o, hg, k, part, locked, tau)
            check_afterburner(o, hg, k, part, tau)
        check_apply(o, hg, k, part, seed=i + 3)
        params = params_cls(k)
        check_rebalance_round(o, params, hg, part)
        check_rebalance_loop(o, params, hg, part)
        check_refine_round_stats(o, params, hg, part, (3, 4))
        check_refine_loop(o, params, hg, part, ((3, 4), (3, 8), (0, 1)), 3)
        check_schedule_invariants(o, check_quotient(o, hg, k, part))
    o = O(hand_example()[0])
    check_schedule_hand(o)
    for q in random_quotients():
        check_schedule_invariants(o, q)
    check_coarsen_hand(O)
    check_subrounds(o)
    check_clustering(O)


# ------------------------------------------------------------------ Section 6 (coarsening)

def rating_term(w, size):
    """omega(e)/(|e|-1) with 32 fraction bits, rounded down (reading R19)."""
    return (int(w) << 32) // (int(size) - 1)


def coarsen_hand_examples():
    """(name, hypergraph, c_max, order, n_single, cap_div, expected labels), worked by hand.

    A (unit weights, c_max 2, one vertex per sub-round, order 0..5):
      edges {0,1} w4, {1,2,3} w2, {2,3} w3, {3,4,5} w2, {4,5} w1
      u0: cluster 1 rated 4 -> joins 1 (weight 2);  u1: cluster {0,1} is not a singleton, stays
      u2: cluster 1 rated 1 (over the bound: 2+1 > 2), cluster 3 rated 1+3 = 4 -> joins 3
      u3: not a singleton;  u4: cluster 3 rated 1 (over the bound), cluster 5 rated 1+1 -> joins 5
      labels [1,1,3,3,5,5]; contraction: edges {0,1} w2 and {1,2} w2, weights [2,2,2]
    B (the corrected rating; c_max 10; order 1,0,2,3):
      edges {0,1,2} w3, {0,3} w2, {1,2} w10
      u1: cluster 2 rated 1.5 + 10, cluster 0 rated 1.5 -> joins 2
      u0: edge {0,1,2} has two pins of cluster 2 but counts once: cluster 2 rated 1.5 < cluster 3
          rated 2 -> joins 3 (counting per pin would give 3 > 2 and pick cluster 2)
      labels [3,2,2,3]
    C (ties to the smaller label): edges {0,1} w1, {0,2} w1; u0 rates clusters 1 and 2 equally -> 1;
      u1 is no longer a singleton; u2 rates cluster 1 (through pin 0) -> joins it.  labels [1,1,1]
      (ties to the larger label would give [2,2,2])
    D (swap prevention and approval; weights [1,2,1,1], c_max 4, sub-rounds {0,1}, {2,3}):
      edges {0,1} w5, {1,2} w1, {0,3} w1
      sub-round {0,1}: T[0] = 1, T[1] = 0 (a swap); cluster 0 would weigh 1, cluster 1 weighs 2
      -> 1 stays, 0 joins 1 (cluster 1 weighs 3)
      sub-round {2,3}: both propose cluster 1 (3+1 <= 4); room 4-3 = 1; order (c, id): 2, 3
      -> 2 joins, 3 stays.  labels [1,1,1,3]
    E (approval by weight; weights [1,2,1,2], c_max 3, order 2,1,3,0, sub-rounds {2,1}, {3,0}):
      edges {0,1} w1, {0,2} w1, {0,3} w1
      sub-round {2,1}: both propose cluster 0; room 3-1 = 2; order (c, id): 2 (c 1), 1 (c 2):
      sums 1, 3 -> only 2 joins.  sub-round {3,0}: cluster 0 weighs 2, 2+2 > 3: 3 stays;
      0 is no longer a singleton.  labels [0,1,0,3]
    """
    ex = []
    hg = synth.from_edges(6, [[0, 1], [1, 2, 3], [2, 3], [3, 4, 5], [4, 5]], ewgt=[4, 2, 3, 2, 1])
    ex.append(("A", hg, 2, [0, 1, 2, 3, 4, 5], 100, 100, [1, 1, 3, 3, 5, 5]))
    hg = synth.from_edges(4, [[0, 1, 2], [0, 3], [1, 2]], ewgt=[3, 2, 10])
    ex.append(("B", hg, 10, [1, 0, 2, 3], 100, 100, [3, 2, 2, 3]))
    hg = synth.from_edges(3, [[0, 1], [0, 2]])
    ex.append(("C", hg, 10, [0, 1, 2], 100, 100, [1, 1, 1]))
    hg = synth.from_edges(4, [[0, 1], [1, 2], [0, 3]], vwgt=[1, 2, 1, 1], ewgt=[5, 1, 1])
    ex.append(("D", hg, 4, [0, 1, 2, 3], 0, 2, [1, 1, 1, 3]))
    hg = synth.from_edges(4, [[0, 1], [0, 2], [0, 3]], vwgt=[1, 2, 1, 2])
    ex.append(("E", hg, 3, [2, 1, 3, 0], 0, 2, [0, 1, 0, 3]))
    return ex


def check_coarsen_hand(make):
    for name, hg, cmax, order, n_single, cap_div, want in coarsen_hand_examples():
        o = make(hg)
        got = o.cluster(cmax, np.array(order, np.int32), n_single=n_single, cap_div=cap_div)
        assert list(got) == want, f"example {name}: {list(got)} != {want}"
    name, hg, cmax, order, n_single, cap_div, want = coarsen_hand_examples()[0]
    c, mp = make(hg).contract(np.array(want, np.int32))
    assert list(mp) == [0, 0, 1, 1, 2, 2]
    assert (c.n, c.m, list(c.eptr), list(c.pins), list(c.ewgt), list(c.vwgt)) == \
        (3, 2, [0, 2, 4], [0, 1, 1, 2], [2, 2], [2, 2, 2])
    assert list(c.vptr) == [0, 1, 3, 4] and list(c.inc) == [0, 0, 1, 1]


def check_subrounds(orc):
    """The prefix-doubling schedule against its statement: n_single sizes of 1, then 2, 4, 8, ... capped
    at floor(n / cap_div) (at least 1), the last one ragged."""
    assert list(np.diff(orc.subrounds(1000)))[:106] == [1] * 100 + [2, 4, 8, 10, 10, 10]
    for n, ns, cd in ((1000, 100, 100), (7, 100, 100), (5000, 3, 10), (64, 0, 1), (1, 0, 1), (300, 10, 1000)):
        cap = max(1, n // cd)
        sizes, j = [], 0
        while sum(sizes) < n:
            s = 1 if len(sizes) < ns else min(2 ** (len(sizes) - ns + 1), cap)
            sizes.append(min(s, n - sum(sizes)))
        b = orc.subrounds(n, ns, cd)
        assert list(np.diff(b)) == sizes and b[0] == 0 and b[-1] == n, (n, ns, cd)


def sequential_clustering(hg, cmax, rmax, order):
    """Clustering with every sub-round of one vertex, restated from Section 6 with sets: each singleton
    vertex in turn joins its best-rated cluster within the weight bound (ties to the smaller label)."""
    label = list(range(hg.n))
    members = {v: {v} for v in range(hg.n)}
    weight = {v: int(hg.vwgt[v]) for v in range(hg.n)}
    for u in order:
        if members[u] != {u}:
            continue
        rating = {}
        for e in hg.inc[hg.vptr[u]:hg.vptr[u + 1]]:
            pins = hg.pins[hg.eptr[e]:hg.eptr[e + 1]]
            if len(pins) < 2 or len(pins) > rmax:
                continue
            for C in {label[v] for v in pins if v != u}:
                rating[C] = rating.get(C, 0) + rating_term(hg.ewgt[e], len(pins))
        ok = [C for C in rating if weight[C] + int(hg.vwgt[u]) <= cmax]
        if not ok:
            continue
        best = min(ok, key=lambda C: (-rating[C], C))
        members[u].discard(u)
        members[best].add(u)
        weight[best] += int(hg.vwgt[u])
        weight[u] -= int(hg.vwgt[u])
        label[u] = best
    return label


def synchronous_clustering(hg, cmax, rmax, order, bounds):
    """Algorithm 4 restated with dictionaries, one sub-round at a time from the state at its start:
    selection as above, swap pairs resolved by the would-be cluster weights, then per target the
    longest prefix in (weight, id) order that fits the bound."""
    label = list(range(hg.n))
    size = [1] * hg.n
    weight = [int(x) for x in hg.vwgt]
    c = [int(x) for x in hg.vwgt]
    for a, b in zip(bounds[:-1], bounds[1:]):
        B = [int(u) for u in order[a:b]]
        T = {}
        for u in B:
            if size[u] != 1:
                continue
            rating = {}
            for e in hg.inc[hg.vptr[u]:hg.vptr[u + 1]]:
                pins = hg.pins[hg.eptr[e]:hg.eptr[e + 1]]
                if 2 <= len(pins) <= rmax:
                    for C in {label[v] for v in pins if v != u}:
                        rating[C] = rating.get(C, 0) + rating_term(hg.ewgt[e], len(pins))
            ok = [C for C in rating if weight[C] + c[u] <= cmax]
            if ok:
                T[u] = min(ok, key=lambda C: (-rating[C], C))
        incoming = {}
        for u, j in T.items():
            incoming[j] = incoming.get(j, 0) + c[u]
        T2 = dict(T)
        for u, v in T.items():
            if T.get(v) == u:
                wu = c[u] + incoming.get(u, 0) - c[v]
                wv = c[v] + incoming.get(v, 0) - c[u]
                if (wu, -u) > (wv, -v):
                    del T2[u]
        groups = {}
        for u, j in T2.items():
            groups.setdefault(j, []).append(u)
        moves = []
        for j, us in groups.items():
            total = 0
            for u in sorted(us, key=lambda x: (c[x], x)):
                total += c[u]
                if total > cmax - weight[j]:
                    break
                moves.append((u, j))
        for u, j in moves:
            label[u] = j
            weight[j] += c[u]
            weight[u] -= c[u]
            size[j] += 1
            size[u] -= 1
    return label


def expected_contraction(hg, label):
    """The contracted hypergraph from its definition (reading R25), by dictionaries over pin sets."""
    used = sorted(set(int(x) for x in label))
    cid = {l: i for i, l in enumerate(used)}
    mp = [cid[int(label[v])] for v in range(hg.n)]
    vw = [0] * len(used)
    for v in range(hg.n):
        vw[mp[v]] += int(hg.vwgt[v])
    sets = {}
    for e in range(hg.m):
        s = tuple(sorted({mp[v] for v in hg.pins[hg.eptr[e]:hg.eptr[e + 1]]}))
        if len(s) >= 2:
            if s not in sets:
                sets[s] = [e, 0]
            sets[s][1] += int(hg.ewgt[e])
    edges = sorted(sets.items(), key=lambda kv: kv[1][0])
    return mp, vw, [list(s) for s, _ in edges], [w for _, (_, w) in edges]


def check_contraction(orc, hg, label, k=5, seed=3):
    c, mp = orc.contract(label)
    emp, evw, eedges, eew = expected_contraction(hg, label)
    assert list(mp) == emp
    assert list(c.vwgt) == evw and c.n == len(evw)
    assert c.m == len(eedges) and list(c.ewgt) == eew
    assert [list(c.pins[c.eptr[f]:c.eptr[f + 1]]) for f in range(c.m)] == eedges
    inc = [[f for f in range(c.m) if v in eedges[f]] for v in range(c.n)]
    assert [list(c.inc[c.vptr[v]:c.vptr[v + 1]]) for v in range(c.n)] == inc
    # projection keeps (lambda-1) and the block weights of any partition of the coarse vertices
    for s in range(3):
        pc = (synth.stream_u64(seed + s, c.n) % np.uint64(k)).astype(np.int32)
        pf = pc[mp]
        assert objective_sets(c, pc) == objective_sets(hg, pf)
        assert np.array_equal(np.bincount(pc, weights=c.vwgt, minlength=k), np.bincount(pf, weights=hg.vwgt, minlength=k))
    return c


def coarsen_instances(seed=41):
    out = []
    for i, (n, m, cap, cm, wm) in enumerate(((150, 170, 6, 1, 1), (200, 260, 12, 4, 3), (320, 300, 40, 3, 2),
                                             (90, 400, 3, 2, 5))):
        hg = synth.uniform(seed + i, n, m, base=2, geo=(1, 2), size_cap=cap, c_max=cm, w_max=wm)
        order = synth.stream_u64(seed + 10 + i, n).argsort(kind="stable").astype(np.int32)
        out.append((hg, order))
    return out


def check_clustering(make):
    for i, (hg, order) in enumerate(coarsen_instances()):
        o = make(hg)
        W = int(hg.vwgt.sum())
        for cmax in (2, 4, max(3, W // 20), W):
            for rmax in (1000, 4):
                got = o.cluster(cmax, order, rmax=rmax, n_single=hg.n, cap_div=100)
                assert list(got) == sequential_clustering(hg, cmax, rmax, order), (i, cmax, rmax, "sequential")
                for ns, cd in ((100, 100), (0, 1), (3, 8)):
                    got = o.cluster(cmax, order, rmax=rmax, n_single=ns, cap_div=cd)
                    want = synchronous_clustering(hg, cmax, rmax, order, list(o.subrounds(hg.n, ns, cd)))
                    assert list(got) == want, (i, cmax, rmax, ns, cd)
                    # invariants: clusters of several vertices within the bound; no label swaps
                    lab = np.asarray(got)
                    w = np.bincount(lab, weights=hg.vwgt, minlength=hg.n)
                    cnt = np.bincount(lab, minlength=hg.n)
                    assert np.all(w[cnt > 1] <= cmax)
                    assert not np.any((lab != np.arange(hg.n)) & (lab[lab] == np.arange(hg.n)))
            check_contraction(o, hg, o.cluster(cmax, order), seed=i)
