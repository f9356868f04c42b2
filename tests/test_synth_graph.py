"""The graph generator (two-pin edges) used by the graph-path tests and the graph workload."""
import numpy as np

from paper_2504_12013_gb300 import synth


def test_from_pairs_equals_general_builder():
    h = synth.graph(3, 80, 300, local=0.6, window=7, c_max=3, w_max=5)
    edges = [list(h.pins[h.eptr[e]:h.eptr[e + 1]]) for e in range(h.m)]
    g = synth.from_edges(h.n, edges, vwgt=h.vwgt, ewgt=h.ewgt)
    for f in ("eptr", "pins", "vptr", "inc", "vwgt", "ewgt"):
        assert np.array_equal(getattr(h, f), getattr(g, f)), f


def test_graph_edges_are_pairs_of_distinct_vertices():
    h = synth.graph(5, 1000, 5000, local=0.8, window=20, c_max=4, w_max=9)
    sizes = np.diff(h.eptr)
    assert np.all(sizes == 2) and h.P == 2 * h.m
    a, b = h.pins[0::2], h.pins[1::2]
    assert np.all(a < b) and a.min() >= 0 and b.max() < h.n
    assert 1 <= h.vwgt.min() and h.vwgt.max() <= 4 and 1 <= h.ewgt.min() and h.ewgt.max() <= 9
    # about 80 % of the edges join vertices at most 20 ids apart (mod n)
    d = np.minimum(b - a, h.n - (b - a))
    assert 0.75 < np.mean(d <= 20) < 0.9


def test_graph_is_deterministic():
    a, b = synth.graph(9, 500, 2000), synth.graph(9, 500, 2000)
    assert np.array_equal(a.pins, b.pins) and np.array_equal(a.inc, b.inc)
    assert not np.array_equal(a.pins, synth.graph(10, 500, 2000).pins)
