"""The fixed test hierarchy (vertex pairs contracted level by level) against
what projection must preserve (the multilevel scheme of §2/§7.2): the
(lambda-1) objective and the block weights of a partition equal those of its
projection to the finer level, on the oracle's own connectivity and block
weights.  This pins the input builder that the uncoarsening tests use."""
import numpy as np

import oracle
from paper_2504_12013_gb300 import synth


def _brute_objective(h, part):
    tot = 0
    for e in range(h.m):
        blocks = {int(part[v]) for v in h.pins[h.eptr[e]:h.eptr[e + 1]]}
        tot += int(h.ewgt[e]) * (len(blocks) - 1)
    return tot


def test_contraction_structure():
    h = synth.uniform(3, 801, 900, base=2, geo=(1, 2), size_cap=12, c_max=3, w_max=4)
    c, mp = synth.contract_pairs(h)
    assert c.n == 401 and mp.dtype == np.int32 and mp.shape == (h.n,)
    assert np.array_equal(mp, np.arange(h.n) // 2)
    assert int(c.vwgt.sum()) == int(h.vwgt.sum())
    for e in range(c.m):
        pins = c.pins[c.eptr[e]:c.eptr[e + 1]]
        assert len(pins) >= 2 and np.all(np.diff(pins) > 0)
    # the vertex view lists exactly the edge view's incidences
    inc = sorted((int(v), e) for e in range(c.m) for v in c.pins[c.eptr[e]:c.eptr[e + 1]])
    inc2 = sorted((v, int(e)) for v in range(c.n) for e in c.inc[c.vptr[v]:c.vptr[v + 1]])
    assert inc == inc2


def test_projection_preserves_objective_and_block_weights():
    h = synth.uniform(4, 3000, 3300, base=2, geo=(1, 2), size_cap=40, c_max=3, w_max=3)
    hs, maps = synth.hierarchy(h, 4)
    assert [x.n for x in hs] == [375, 750, 1500, 3000]
    k = 7
    p = synth.part_perm(9, hs[0].n, k)
    for l in range(len(hs)):
        if l:
            q = p[maps[l - 1]]
            o_c, o_f = oracle.Oracle(hs[l - 1]), oracle.Oracle(hs[l])
            assert o_f.objective(k, q) == o_c.objective(k, p) == _brute_objective(hs[l], q)
            assert np.array_equal(o_f.pincounts(k, q)[1], o_c.pincounts(k, p)[1])
            p = q
