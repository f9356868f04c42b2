"""The graph path (every edge two pins: neighbour blocks instead of phi) vs the oracle.

The oracle runs the same hypergraph method on the graph.  Every round's
partition, block weights and statistics, and every whole refinement's
summary, partition and final phi must equal the oracle's, in both
execution forms, with and without a phi table.
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

GRAPHS = [
    (synth.graph(71, 6_000, 24_000), 8),
    (synth.graph(72, 5_000, 30_000, local=0.5, window=50, c_max=4, w_max=20), 64),  # heavy vertices
    (synth.graph(73, 3_000, 12_000, local=0.9, window=10, w_max=3), 256),
    (synth.graph(74, 4_000, 8_000, local=0.0), 2),
]


def _ctx(h, k, graph_mode=True):
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(h), jet.params(k))
    jet.jet_set_graph_mode(ctx, graph_mode)
    jet.jet_set_graph_path(ctx, True)
    return ctx


@pytest.mark.parametrize("idx", range(len(GRAPHS)))
@pytest.mark.parametrize("graph_mode", [True, False])
def test_rounds_match_oracle(idx, graph_mode):
    h, k = GRAPHS[idx]
    part0 = synth.part_perm(idx, h.n, k)
    orc = oracle.Oracle(h)
    ost = oracle.State(orc, k, part0)
    prm = oracle.Params(k)
    st = jet.JetState(_ctx(h, k, graph_mode), part0, with_phi=False)
    for r, tau in enumerate(((3, 4), (3, 4), (3, 8), (0, 1), (0, 1))):
        want = orc.refine_round(prm, tau, ost.part, ost.phi, ost.bw, ost.locked)
        st.round(tau)
        assert st.stats_dict() == want, f"round {r}"
        assert np.array_equal(st.part.cpu().numpy()[: h.n], ost.part), f"round {r}: partition"
        assert np.array_equal(st.block_w.cpu().numpy(), ost.bw), f"round {r}: block weights"
        assert np.array_equal(st.locked.cpu().numpy()[: h.n], ost.locked), f"round {r}: locks"


@pytest.mark.parametrize("idx", range(len(GRAPHS)))
@pytest.mark.parametrize("graph_mode", [True, False])
def test_refine_matches_oracle(idx, graph_mode):
    h, k = GRAPHS[idx]
    part0 = synth.part_random(idx + 10, h.n, k)
    p = part0.copy()
    orc = oracle.Oracle(h)
    iters, obj, phase = orc.refine(oracle.Params(k), p)
    phi, bw = orc.pincounts(k, p)
    st = jet.JetState(_ctx(h, k, graph_mode), part0)
    res = jet.jet_refine(st.ctx, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, st.part, st.phi, st.block_w)
    assert res["iterations"] == iters and res["objective"] == obj
    assert res["phase_iterations"][:3] == [int(x) for x in phase]
    assert np.array_equal(st.part.cpu().numpy()[: h.n], p)
    assert np.array_equal(st.block_w.cpu().numpy(), bw)
    assert np.array_equal(st.phi.cpu().numpy()[: h.m * k].reshape(h.m, k), phi), "final phi is rebuilt"
    # without a phi table
    st2 = jet.JetState(st.ctx, part0, with_phi=False)
    res2 = jet.jet_refine(st.ctx, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, st2.part, None, st2.block_w)
    assert res2 == res and np.array_equal(st2.part.cpu().numpy()[: h.n], p)


def test_batch_of_graph_path_contexts():
    insts = [(h, k, synth.part_perm(i, h.n, k)) for i, (h, k) in enumerate(GRAPHS)]
    ctxs = [_ctx(h, k) for h, k, _ in insts]
    states = [jet.JetState(c, p, with_phi=False) for c, (_, _, p) in zip(ctxs, insts)]
    b = jet.jet_batch_create(ctxs)
    res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for (h, k, part0), r, st in zip(insts, res, states):
        p = part0.copy()
        iters, obj, _ = oracle.Oracle(h).refine(oracle.Params(k), p)
        assert r["iterations"] == iters and r["objective"] == obj
        assert np.array_equal(st.part.cpu().numpy()[: h.n], p)
    b.close()


def test_graph_path_errors():
    h = synth.uniform(5, 500, 600, base=2, geo=(1, 2), size_cap=8)  # edges of more than two pins
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(h), jet.params(4))
    with pytest.raises(jet.JetError) as ei:
        jet.jet_set_graph_path(ctx, True)
    assert ei.value.code == -1
    g, k = GRAPHS[0]
    ctx = _ctx(g, k)
    st = jet.JetState(ctx, synth.part_perm(1, g.n, k), with_phi=False)
    with pytest.raises(jet.JetError) as ei:  # the schedule reads phi, which the graph path does not keep
        jet.jet_quotient_schedule(ctx, torch.zeros(g.m * k, dtype=torch.int32, device="cuda"))
    assert ei.value.code == -1
    # back to the hypergraph path: phi must be rebuilt first, then rounds match the oracle again
    jet.jet_set_graph_path(ctx, False)
    st = jet.JetState(ctx, synth.part_perm(1, g.n, k))
    orc = oracle.Oracle(g)
    ost = oracle.State(orc, k, synth.part_perm(1, g.n, k))
    want = orc.refine_round(oracle.Params(k), (3, 4), ost.part, ost.phi, ost.bw, ost.locked)
    st.round((3, 4))
    assert st.stats_dict() == want


def test_uncoarsening_of_a_graph_hierarchy_on_the_graph_path():
    """The oracle coarsens a graph twice (every coarse level is a graph again); jet_uncoarsen refines
    the hierarchy with graph-path contexts and no phi tables, and every level must equal the oracle's
    projection and refinement."""
    g = synth.graph(75, 6_000, 20_000, local=0.7, window=40)
    k = 16
    hs, maps = [g], []
    for level in range(2):
        coarse, mp, _ = oracle.Oracle(hs[0]).coarsen(40, synth.vertex_order(level, hs[0].n))
        assert np.all(np.diff(coarse.eptr) == 2)
        hs.insert(0, coarse)
        maps.insert(0, mp)
    part0 = synth.part_perm(3, hs[0].n, k)
    want, p = [], part0.copy()
    for l, h in enumerate(hs):
        if l:
            p = p[maps[l - 1]].astype(np.int32)
        iters, obj, _ = oracle.Oracle(h).refine(oracle.Params(k), p)
        want.append((iters, obj, p.copy()))
    ctxs = [_ctx(h, k) for h in hs]
    states = [jet.JetState(ctxs[0], part0, with_phi=False)] + [
        jet.JetState(c, np.zeros(h.n, np.int32), with_phi=False) for c, h in zip(ctxs[1:], hs[1:])]
    res = jet.jet_uncoarsen(ctxs, [torch.as_tensor(m).cuda() for m in maps], oracle.TAU_SCHEDULE,
                            oracle.ITERATION_LIMIT, states)
    for l, (h, r, st, (iters, obj, p)) in enumerate(zip(hs, res, states, want)):
        assert (r["iterations"], r["objective"]) == (iters, obj), f"level {l}"
        assert np.array_equal(st.part.cpu().numpy()[: h.n], p), f"level {l}: partition"
