"""Properties of the seeded input generators (no method arithmetic)."""
import numpy as np

from paper_2504_12013_gb300 import synth


def _check_csr(h):
    sizes = np.diff(h.eptr)
    assert h.eptr[0] == 0 and np.all(sizes >= 0) and h.eptr[-1] == h.pins.size
    assert h.vptr[0] == 0 and h.vptr[-1] == h.inc.size == h.pins.size
    assert h.pins.min(initial=0) >= 0 and (h.pins.size == 0 or h.pins.max() < h.n)
    for e in range(min(h.m, 2000)):
        pe = h.edge(e)
        assert np.all(np.diff(pe) > 0)  # distinct, sorted by id
    # transpose: (v, e) pairs of both views are identical
    edge_of = np.repeat(np.arange(h.m), np.diff(h.eptr))
    a = np.lexsort((edge_of, h.pins))
    assert np.array_equal(h.inc, edge_of[a])
    assert np.array_equal(np.diff(h.vptr), np.bincount(h.pins, minlength=h.n))


def test_uniform_shape_and_determinism():
    h1 = synth.uniform(3, 500, 700, base=2, geo=(1, 2), size_cap=64, c_max=4, w_max=3)
    h2 = synth.uniform(3, 500, 700, base=2, geo=(1, 2), size_cap=64, c_max=4, w_max=3)
    _check_csr(h1)
    for a, b in zip((h1.eptr, h1.pins, h1.vwgt, h1.ewgt), (h2.eptr, h2.pins, h2.vwgt, h2.ewgt)):
        assert np.array_equal(a, b)
    sizes = np.diff(h1.eptr)
    assert sizes.min() >= 2 and sizes.max() <= 64
    assert 2.7 < sizes.mean() < 3.3  # 2 + Geometric(1/2) failures: mean 3
    assert h1.vwgt.min() >= 1 and h1.vwgt.max() <= 4 and h1.ewgt.max() <= 3
    h3 = synth.uniform(4, 500, 700)
    assert not np.array_equal(h1.pins[:100], h3.pins[:100])


def test_random_10k_config():
    h, k, part = synth.config_random_10k(1)
    _check_csr(h)
    assert (h.n, h.m, k) == (10_000, 12_000, 8)
    assert np.all(np.bincount(part, minlength=k) == 1250)  # the hash is a bijection mod 8
    assert np.all(h.vwgt == 1) and np.all(h.ewgt == 1)


def test_vlsi_small_shape():
    h = synth.vlsi(2, 20_000, 22_000, smax=500, window=200)
    _check_csr(h)
    sizes = np.diff(h.eptr)
    assert sizes.min() >= 2 and sizes.max() <= 500
    assert 3.0 < sizes.mean() < 6.0
    assert set(np.unique(h.vwgt)) <= {1, 2, 3, 4}


def test_rownet_small_shape():
    h = synth.rownet(5, 20_000, 20_000, n_hubs=3, hub_min=2_000, hub_max=5_000)
    _check_csr(h)
    sizes = np.diff(h.eptr)
    assert int(np.sum(sizes >= 2_000)) >= 3
    body = sizes[sizes < 2_000]
    assert body.min() >= 1 and 8 < body.mean() < 17  # E[round(LogNormal(2,1))] ~ e^2.5 ~ 12.2


def test_partitions():
    assert np.all(np.bincount(synth.part_perm(9, 1000, 7), minlength=7) >= 142)
    p = synth.part_hash(5, 1000, 8)
    assert np.array_equal(p, ((np.arange(1000, dtype=np.uint64) * np.uint64(2654435761) + np.uint64(5))
                              % np.uint64(8)).astype(np.int32))


def test_from_edges_and_permuted():
    h = synth.from_edges(5, [[0, 3], [4, 1, 2], [], [2]])
    assert h.inc.tolist() == [0, 1, 1, 3, 0, 1]
    assert h.vptr.tolist() == [0, 1, 2, 4, 5, 6]
    hp, eperm = synth.permuted(h, 7)
    for i, old in enumerate(eperm):
        assert sorted(hp.edge(i).tolist()) == sorted(h.edge(int(old)).tolist())
