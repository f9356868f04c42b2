"""CUDA path vs the CPU oracle, element by element, on seeded instances.

Each instance is small enough for the oracle to finish in seconds but spans
many thread blocks and ragged tails, and together they exercise every size
class of the kernels: light and heavy vertices (weighted degree below / at
least 64), tiny (<= 8), warp (9..2048, including edges with more than 32
candidates that are handed to the block path) and block (> 2048) edges,
k with 1, 2, 4 and 8 mask words (k = 2, 11, 27, 64, 128, 256), vertex and
edge weights, empty and single-pin edges and isolated vertices.  The bar is
bit-exact equality: all arithmetic is integer.
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


def _with_empty_edges():
    hg = synth.uniform(31, 3000, 2500, base=1, geo=(1, 3), size_cap=12, c_max=2, w_max=3)
    edges = [list(hg.edge(e)) for e in range(hg.m)]
    for i in range(0, len(edges), 97):
        edges[i] = []
    return synth.from_edges(hg.n + 50, edges, np.concatenate([hg.vwgt, np.ones(50, np.int32)]), hg.ewgt)


def make_instances():
    inst = {}
    h, k, p = synth.config_random_10k(1)
    inst["random10k_k8"] = (h, k, p)
    h = synth.uniform(2, 20_000, 24_000, base=2, geo=(1, 2), size_cap=64, c_max=4, w_max=3)
    inst["weighted_k11"] = (h, 11, synth.part_perm(2, h.n, 11))
    inst["weighted_k27"] = (h, 27, synth.part_perm(3, h.n, 27))
    h = synth.uniform(4, 8_000, 9_000, base=2, geo=(2, 5), size_cap=256)
    inst["geo04_k64"] = (h, 64, synth.part_perm(4, h.n, 64))
    inst["geo04_k2"] = (h, 2, synth.part_hash(4, h.n, 2))
    h = synth.uniform(5, 6_000, 7_000, base=2, geo=(1, 2), size_cap=64, w_max=40)  # heavy vertices
    inst["heavy_k128"] = (h, 128, synth.part_perm(5, h.n, 128))
    inst["heavy_k256"] = (h, 256, synth.part_perm(6, h.n, 256))
    h = synth.rownet(7, 20_000, 20_000, n_hubs=5, hub_min=3_000, hub_max=8_000)  # block + deferred edges
    inst["rownet_k32"] = (h, 32, synth.part_perm(7, h.n, 32))
    h = synth.vlsi(8, 30_000, 33_000, smax=3_000, window=300)
    inst["vlsi_k64"] = (h, 64, synth.part_perm(8, h.n, 64))
    h = _with_empty_edges()
    inst["empty_edges_k4"] = (h, 4, synth.part_random(9, h.n, 4))
    # vertex weights up to 1000: lcm(1..1000) is huge, so rebalancing uses the 96-bit priority keys
    h = synth.uniform(10, 12_000, 14_000, base=2, geo=(1, 2), size_cap=32, c_max=1000, w_max=2)
    inst["bigc_k16"] = (h, 16, synth.part_perm(10, h.n, 16))
    return inst


INSTANCES = make_instances() if torch.cuda.is_available() else {}
NAMES = ["random10k_k8", "weighted_k11", "weighted_k27", "geo04_k64", "geo04_k2", "heavy_k128", "heavy_k256",
         "rownet_k32", "vlsi_k64", "empty_edges_k4", "bigc_k16"]


def setup(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hg, k, part = INSTANCES[name]
    dh = jet.DeviceHypergraph(hg)
    ctx = jet.jet_ctx_create(dh, jet.params(k))
    return hg, k, part, ctx


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("name", NAMES)
def test_pincounts_and_connectivity(name):
    hg, k, part, ctx = setup(name)
    st = jet.JetState(ctx, part)
    orc = oracle.Oracle(hg)
    phi_ref, bw_ref = orc.pincounts(k, part)
    assert np.array_equal(host(st.phi)[: hg.m * k].reshape(hg.m, k), phi_ref)
    assert np.array_equal(host(st.block_w), bw_ref)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    jet.jet_connectivity(ctx, st.phi, out)
    assert int(out.item()) == orc.connectivity(k, phi_ref)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("tau", [(0, 1), (3, 8), (3, 4)])
def test_candidates_and_afterburner(name, tau):
    hg, k, part, ctx = setup(name)
    st = jet.JetState(ctx, part)
    locked_np = (synth.stream_u64(11, hg.n) % np.uint64(5) == 0).astype(np.uint8)
    locked = dev(locked_np, torch.uint8)
    n = hg.n
    target = torch.empty(n, dtype=torch.int32, device="cuda")
    gain = torch.empty(n, dtype=torch.int32, device="cuda")
    in_m = torch.empty(n, dtype=torch.uint8, device="cuda")
    jet.jet_candidates(ctx, tau, st.part, st.phi, locked, target, gain, in_m)
    orc = oracle.Oracle(hg)
    phi_ref, _ = orc.pincounts(k, part)
    cnt, t_ref, g_ref, m_ref = orc.candidates(k, part, phi_ref, locked_np, tau)
    m = host(in_m).astype(bool)
    assert np.array_equal(m, m_ref.astype(bool)), int((m != m_ref.astype(bool)).sum())
    assert int(m.sum()) == cnt
    assert np.array_equal(host(target)[m], t_ref[m])
    assert np.array_equal(host(gain)[m].astype(np.int64), g_ref[m])
    rg = torch.empty(n, dtype=torch.int32, device="cuda")
    approved = torch.empty(n, dtype=torch.uint8, device="cuda")
    jet.jet_afterburner(ctx, st.part, st.phi, rg, approved)
    acnt, rg_ref, ap_ref = orc.afterburner(k, part, phi_ref, t_ref, g_ref, m_ref)
    assert np.array_equal(host(rg).astype(np.int64)[m], rg_ref[m])
    assert np.array_equal(host(approved), ap_ref)
    # rg is zeroed for the next call: a second run gives the same answer
    jet.jet_afterburner(ctx, st.part, st.phi, rg, approved)
    assert np.array_equal(host(rg).astype(np.int64)[m], rg_ref[m])


def _compare_state(hg, k, st, ost, where):
    assert np.array_equal(host(st.part)[: hg.n], ost.part), f"{where}: partition"
    assert np.array_equal(host(st.phi)[: hg.m * k].reshape(hg.m, k), ost.phi), f"{where}: phi"
    assert np.array_equal(host(st.block_w), ost.bw), f"{where}: block weights"
    assert np.array_equal(host(st.locked)[: hg.n], ost.locked), f"{where}: locks"


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("mode", ["graph", "eager"])
def test_refine_rounds_state(name, mode):
    hg, k, part, ctx = setup(name)
    jet.jet_set_graph_mode(ctx, mode == "graph")
    st = jet.JetState(ctx, part)
    orc = oracle.Oracle(hg)
    ost = oracle.State(orc, k, part)
    params = oracle.Params(k)
    for r, tau in enumerate([(3, 4), (3, 4), (3, 4), (3, 8), (0, 1), (0, 1)]):
        st.round(tau)
        want = orc.refine_round(params, tau, ost.part, ost.phi, ost.bw, ost.locked)
        got = st.stats_dict()
        assert got == want, f"round {r}: {got} != {want}"
        _compare_state(hg, k, st, ost, f"round {r}")


@pytest.mark.parametrize("name", NAMES)
def test_rebalance_from_random_partition(name):
    hg, k, _, ctx = setup(name)
    part = synth.part_random(101, hg.n, k)
    part[: hg.n // 6] = 0  # overload block 0
    st = jet.JetState(ctx, part)
    jet.jet_rebalance(ctx, st.part, st.phi, st.block_w, st.stats)
    orc = oracle.Oracle(hg)
    ost = oracle.State(orc, k, part)
    rounds, moves = orc.rebalance(oracle.Params(k), ost.part, ost.phi, ost.bw)
    got = st.stats_dict()
    assert (got["rebalance_rounds"], got["rebalance_moves"]) == (rounds, moves)
    assert got["objective"] == orc.connectivity(k, ost.phi)
    assert np.array_equal(host(st.part)[: hg.n], ost.part)
    assert np.array_equal(host(st.phi)[: hg.m * k].reshape(hg.m, k), ost.phi)
    assert np.array_equal(host(st.block_w), ost.bw)


@pytest.mark.parametrize("graph", [True, False], ids=["device_loop", "host_loop"])
@pytest.mark.parametrize("name", ["random10k_k8", "weighted_k11", "geo04_k2", "heavy_k128", "rownet_k32",
                                  "empty_edges_k4", "bigc_k16"])
def test_refine_to_convergence(name, graph):
    hg, k, part, ctx = setup(name)
    jet.jet_set_graph_mode(ctx, graph)
    st = jet.JetState(ctx, part)
    res = jet.jet_refine(ctx, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, st.part, st.phi, st.block_w)
    orc = oracle.Oracle(hg)
    p_ref = part.copy()
    iters, obj, phase = orc.refine(oracle.Params(k), p_ref)
    assert res["iterations"] == iters and res["objective"] == obj
    assert res["phase_iterations"][:3] == [int(x) for x in phase]
    assert np.array_equal(host(st.part)[: hg.n], p_ref)
    phi_ref, bw_ref = orc.pincounts(k, p_ref)
    assert np.array_equal(host(st.phi)[: hg.m * k].reshape(hg.m, k), phi_ref)
    assert np.array_equal(host(st.block_w), bw_ref)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random10k_seeds_match_oracle_fixture(seed):
    """The 10,000-vertex workload to convergence against the committed oracle trajectory."""
    import json
    import os
    fix = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "random_10k_oracle.json")))
    want = [r for r in fix["runs"] if r["seed"] == seed][0]
    hg, k, part = synth.config_random_10k(seed)
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(k))
    st = jet.JetState(ctx, part)
    res = jet.jet_refine(ctx, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, st.part, st.phi, st.block_w)
    import hashlib
    p = host(st.part)[: hg.n].astype("<i4")
    assert res["iterations"] == want["iterations"]
    assert res["objective"] == want["final_objective"]
    assert hashlib.sha256(p.tobytes()).hexdigest() == want["final_partition_sha256"]


def test_runs_are_bit_identical():
    hg, k, part, ctx = setup("rownet_k32")
    outs = []
    for _ in range(2):
        st = jet.JetState(ctx, part)
        for tau in [(3, 4)] * 3 + [(0, 1)] * 2:
            st.round(tau)
        outs.append((host(st.part).copy(), host(st.phi).copy(), host(st.block_w).copy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_host_buffer_entry_point():
    hg, k, part = synth.config_random_10k(2)
    p = part.copy()
    res = jet.jet_refine_host(hg, jet.params(k), oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, p)
    orc = oracle.Oracle(hg)
    p_ref = part.copy()
    iters, obj, _ = orc.refine(oracle.Params(k), p_ref)
    assert res["iterations"] == iters and res["objective"] == obj and np.array_equal(p, p_ref)


@pytest.mark.parametrize("name", ["vlsi_k64", "heavy_k128"])
def test_rounds_host_entry_point(name):
    """jet_rounds_host (host buffers, a fixed number of iterations) equals the same iterations of the oracle."""
    hg, k, part = INSTANCES[name]
    p = part.copy()
    st = jet.jet_rounds_host(hg, jet.params(k), (3, 4), 3, p)
    orc = oracle.Oracle(hg)
    ost = oracle.State(orc, k, part)
    for _ in range(3):
        want = orc.refine_round(oracle.Params(k), (3, 4), ost.part, ost.phi, ost.bw, ost.locked)
    assert np.array_equal(p, ost.part)
    assert all(st[f] == want[f] for f in ("candidates", "approved", "rebalance_rounds", "rebalance_moves",
                                          "objective", "max_block_weight", "imbalanced")), (st, want)
    with pytest.raises(jet.JetError) as ei:
        jet.jet_rounds_host(hg, jet.params(k), (3, 4), -1, p)
    assert ei.value.code == -1


def test_release_memory_between_host_calls():
    """The library's pools may be emptied between calls: a host-buffer call after jet_release_memory gives the
    same partition and statistics as before it."""
    hg, k, part = INSTANCES["random10k_k8"]
    p1, p2 = part.copy(), part.copy()
    st1 = jet.jet_rounds_host(hg, jet.params(k), (3, 4), 2, p1)
    jet.jet_release_memory()
    st2 = jet.jet_rounds_host(hg, jet.params(k), (3, 4), 2, p2)
    jet.jet_release_memory()
    assert np.array_equal(p1, p2) and st1 == st2


def test_errors_are_reported():
    hg, k, part, ctx = setup("random10k_k8")
    st = jet.JetState(ctx, part)
    with pytest.raises(jet.JetError) as ei:
        jet.jet_refine_round(ctx, (1, 1), st.part, st.phi, st.block_w, st.locked)  # tau = 1 is outside [0,1)
    assert ei.value.code == -1
    bad = part.copy()
    bad[17] = k  # out of range
    pb = dev(bad, torch.int32)
    jet.jet_build_pincounts(ctx, pb, st.phi, st.block_w)
    with pytest.raises(jet.JetError) as ei:
        jet.jet_rebalance(ctx, pb, st.phi, st.block_w)
    assert ei.value.code == -5
    # the context stays usable
    st2 = jet.JetState(ctx, part)
    st2.round((3, 4))
    # bad CSR: a pin out of range is caught at context creation
    h2 = synth.from_edges(5, [[0, 1], [2, 3, 4]])
    d2 = jet.DeviceHypergraph(h2)
    d2.pins[1] = 7
    with pytest.raises(jet.JetError) as ei:
        jet.jet_ctx_create(d2, jet.params(2))
    assert ei.value.code == -5
    # weighted degree beyond the int32 gain range
    h3 = synth.from_edges(3, [[0, 1], [1, 2]], ewgt=[2 ** 30, 2 ** 30])
    with pytest.raises(jet.JetError) as ei:
        jet.jet_ctx_create(jet.DeviceHypergraph(h3), jet.params(2))
    assert ei.value.code == -4


def test_degenerate_inputs():
    # all vertices in one block: no candidates move, rebalancing restores balance
    hg = synth.uniform(12, 500, 600, base=2, geo=(1, 2), size_cap=8)
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(4))
    part = np.zeros(hg.n, np.int32)
    st = jet.JetState(ctx, part)
    st.round((3, 4))
    orc = oracle.Oracle(hg)
    ost = oracle.State(orc, 4, part)
    want = orc.refine_round(oracle.Params(4), (3, 4), ost.part, ost.phi, ost.bw, ost.locked)
    assert st.stats_dict() == want
    _compare_state(hg, 4, st, ost, "one block")
    # a hypergraph without edges
    h0 = synth.from_edges(10, [])
    ctx0 = jet.jet_ctx_create(jet.DeviceHypergraph(h0), jet.params(2))
    st0 = jet.JetState(ctx0, synth.part_hash(1, 10, 2))
    st0.round((0, 1))
    assert st0.stats_dict()["objective"] == 0
