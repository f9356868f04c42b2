"""Coarsening (Section 6, Algorithm 4) and contraction on the GPU vs the oracle.

Cluster labels must equal the oracle's bit for bit for every parameter
setting (weight bound, rating edge limit, sub-round schedule), and the
contracted hypergraph (map, CSR in both directions, weights) must equal the
oracle's contraction of the same labels exactly, over several levels.
"""
import numpy as np
import pytest

import oracle
from paper_2504_12013_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12013_gb300 import jet  # noqa: E402


def _instances():
    return [
        ("uniform", synth.uniform(61, 20_000, 23_000, base=2, geo=(1, 2), size_cap=64, c_max=3, w_max=3)),
        ("wide", synth.uniform(62, 6_000, 5_000, base=2, geo=(1, 8), size_cap=300, c_max=2, w_max=5)),
        ("vlsi", synth.vlsi(63, 40_000, 44_000)),
        ("rownet", synth.rownet(64, 30_000, 30_000, n_hubs=4, hub_min=1_500, hub_max=4_000)),
    ]


INST = _instances()


def _same_hg(a, b, what):
    assert (a.n, a.m, a.P) == (b.n, b.m, b.P), what
    for f in ("eptr", "pins", "vptr", "inc", "vwgt", "ewgt"):
        assert np.array_equal(np.asarray(getattr(a, f)), np.asarray(getattr(b, f))), f"{what}: {f}"


def _bound(h, frac):
    return max(2, int(h.vwgt.sum()) // frac)


@pytest.mark.parametrize("idx", range(len(INST)))
@pytest.mark.parametrize("frac,rmax,ns,cd", [(200, 1000, 100, 100), (50, 1000, 0, 1), (2000, 8, 100, 100),
                                             (400, 1000, 5, 20)])
def test_cluster_matches_oracle(idx, frac, rmax, ns, cd):
    name, h = INST[idx]
    cmax = _bound(h, frac)
    order = synth.vertex_order(7 + idx, h.n)
    want = oracle.Oracle(h).cluster(cmax, order, rmax=rmax, n_single=ns, cap_div=cd)
    dh = jet.DeviceHypergraph(h)
    got = jet.jet_cluster(dh, cmax, torch.as_tensor(order).cuda(), rmax=rmax, n_single=ns, cap_div=cd)
    assert np.array_equal(got.cpu().numpy(), want), f"{name}: labels differ at {np.flatnonzero(got.cpu().numpy() != want)[:10]}"


@pytest.mark.parametrize("idx", range(len(INST)))
def test_contract_matches_oracle(idx):
    name, h = INST[idx]
    o = oracle.Oracle(h)
    label = o.cluster(_bound(h, 200), synth.vertex_order(3, h.n))
    want, want_map = o.contract(label)
    coarse, mp = jet.jet_contract(jet.DeviceHypergraph(h), torch.as_tensor(label).cuda())
    assert np.array_equal(mp.cpu().numpy(), want_map)
    _same_hg(coarse.to_host(), want, name)


def test_three_levels_match_oracle():
    _, h = INST[2]
    dh = jet.DeviceHypergraph(h)
    for level in range(3):
        cmax = _bound(h, 300)
        order = synth.vertex_order(20 + level, h.n)
        want, want_map, want_label = oracle.Oracle(h).coarsen(cmax, order)
        dh, mp, label = jet.jet_coarsen(dh, cmax, torch.as_tensor(order).cuda())
        assert np.array_equal(label.cpu().numpy(), want_label), f"level {level}: labels"
        assert np.array_equal(mp.cpu().numpy(), want_map), f"level {level}: map"
        _same_hg(dh.to_host(), want, f"level {level}")
        assert want.n < h.n
        h = want


def test_degenerate_inputs():
    # no edges: every vertex stays alone; single-pin edges only: nothing is rated, all edges dropped
    for edges in ([], [[0], [3], [5]]):
        h = synth.from_edges(6, edges)
        dh = jet.DeviceHypergraph(h)
        order = torch.as_tensor(synth.vertex_order(1, 6)).cuda()
        coarse, mp, label = jet.jet_coarsen(dh, 4, order)
        assert list(label.cpu().numpy()) == list(range(6))
        assert (coarse.n, coarse.m, coarse.P) == (6, 0, 0)
        assert list(coarse.vptr.cpu().numpy()) == [0] * 7 and list(coarse.eptr.cpu().numpy()) == [0]
    # everything in one cluster: all edges collapse and are dropped
    h = synth.from_edges(4, [[0, 1], [1, 2, 3]])
    coarse, mp = jet.jet_contract(jet.DeviceHypergraph(h), torch.zeros(4, dtype=torch.int32, device="cuda"))
    assert (coarse.n, coarse.m) == (1, 0) and list(mp.cpu().numpy()) == [0, 0, 0, 0]
    assert list(coarse.vwgt.cpu().numpy()) == [4]


def test_errors_are_reported():
    _, h = INST[0]
    dh = jet.DeviceHypergraph(h)
    order = synth.vertex_order(1, h.n)
    bad = order.copy()
    bad[5] = bad[6]  # not a permutation
    with pytest.raises(jet.JetError) as ei:
        jet.jet_cluster(dh, 10, torch.as_tensor(bad).cuda())
    assert ei.value.code == -5
    with pytest.raises(jet.JetError) as ei:
        jet.jet_cluster(dh, 0, torch.as_tensor(order).cuda())
    assert ei.value.code == -1
    with pytest.raises(jet.JetError) as ei:
        jet.jet_cluster(dh, 10, torch.as_tensor(order).cuda(), rmax=1)
    assert ei.value.code == -1
    lab = torch.zeros(h.n, dtype=torch.int32, device="cuda")
    lab[7] = h.n
    with pytest.raises(jet.JetError) as ei:
        jet.jet_contract(dh, lab)
    assert ei.value.code == -5
    big = synth.from_edges(2, [[0, 1]] * 3, ewgt=[2 ** 31 - 1] * 3)
    with pytest.raises(jet.JetError) as ei:
        jet.jet_cluster(jet.DeviceHypergraph(big), 10, torch.arange(2, dtype=torch.int32, device="cuda"))
    assert ei.value.code == -4


def test_full_size_vlsi_level_matches_oracle():
    """One level of the 2M-vertex VLSI workload, in the configuration the benchmark coarsens."""
    h, k, _ = synth.config_vlsi_2m(1)
    cmax = -(-int(h.vwgt.sum()) // (160 * k))
    order = synth.vertex_order(1, h.n)
    want, want_map, want_label = oracle.Oracle(h).coarsen(cmax, order)
    coarse, mp, label = jet.jet_coarsen(jet.DeviceHypergraph(h), cmax, torch.as_tensor(order).cuda())
    assert np.array_equal(label.cpu().numpy(), want_label)
    assert np.array_equal(mp.cpu().numpy(), want_map)
    _same_hg(coarse.to_host(), want, "vlsi_2m level 1")
