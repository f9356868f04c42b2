"""The uncoarsening driver (project, then Algorithm 1, level by level, as one graph) vs the oracle.

The hierarchy is a fixed test input (synth.hierarchy: vertices paired level by
level), not the paper's coarsening.  Every level's refined partition, pin
counts, block weights and summary must equal the oracle's projection and
refinement of the same levels.
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


def _run(h, k, levels, seed):
    hs, maps = synth.hierarchy(h, levels)
    part0 = synth.part_perm(seed, hs[0].n, k)
    # oracle: refine the coarsest level, then project and refine each finer one
    want, p = [], part0.copy()
    for l, hl in enumerate(hs):
        if l:
            p = p[maps[l - 1]].astype(np.int32)
        o = oracle.Oracle(hl)
        iters, obj, phase = o.refine(oracle.Params(k), p)
        phi, bw = o.pincounts(k, p)
        want.append((iters, obj, [int(x) for x in phase], p.copy(), phi, bw))
    ctxs = [jet.jet_ctx_create(jet.DeviceHypergraph(hl), jet.params(k)) for hl in hs]
    states = [jet.JetState(ctxs[0], part0)] + [jet.JetState(c, np.zeros(hl.n, np.int32))
                                                for c, hl in zip(ctxs[1:], hs[1:])]
    dmaps = [torch.as_tensor(m).cuda() for m in maps]
    res = jet.jet_uncoarsen(ctxs, dmaps, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for l, (hl, r, st, w) in enumerate(zip(hs, res, states, want)):
        iters, obj, phase, p, phi, bw = w
        assert r["iterations"] == iters and r["objective"] == obj, f"level {l}"
        assert r["phase_iterations"][:3] == phase, f"level {l}"
        if l:  # projection keeps (lambda-1): the contraction keeps edge weights, drops one-vertex edges
            assert r["initial_objective"] == res[l - 1]["objective"], f"level {l}: projected objective"
        assert np.array_equal(st.part.cpu().numpy()[: hl.n], p), f"level {l}: partition"
        assert np.array_equal(st.phi.cpu().numpy()[: hl.m * k].reshape(hl.m, k), phi), f"level {l}: phi"
        assert np.array_equal(st.block_w.cpu().numpy(), bw), f"level {l}: block weights"
    return ctxs, states, dmaps


@pytest.mark.parametrize("k,levels", [(8, 3), (27, 2), (64, 4)])
def test_uncoarsen_matches_oracle(k, levels):
    h = synth.uniform(50 + k, 6000, 6600, base=2, geo=(1, 2), size_cap=48, c_max=3, w_max=2)
    _run(h, k, levels, seed=k)


def test_bad_map_is_reported():
    h = synth.uniform(9, 2000, 2200, base=2, geo=(1, 2), size_cap=16)
    hs, maps = synth.hierarchy(h, 2)
    k = 4
    ctxs = [jet.jet_ctx_create(jet.DeviceHypergraph(hl), jet.params(k)) for hl in hs]
    states = [jet.JetState(ctxs[0], synth.part_perm(1, hs[0].n, k)), jet.JetState(ctxs[1], np.zeros(hs[1].n, np.int32))]
    bad = maps[0].copy()
    bad[17] = hs[0].n  # outside the coarser level
    with pytest.raises(jet.JetError) as ei:
        jet.jet_uncoarsen(ctxs, [torch.as_tensor(bad).cuda()], oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    assert ei.value.code == -5
    with pytest.raises(jet.JetError) as ei:  # levels with different k
        c8 = jet.jet_ctx_create(jet.DeviceHypergraph(hs[1]), jet.params(8))
        jet.jet_uncoarsen([ctxs[0], c8], [torch.as_tensor(maps[0]).cuda()], oracle.TAU_SCHEDULE, 8,
                          [states[0], jet.JetState(c8, np.zeros(hs[1].n, np.int32))])
    assert ei.value.code == -1
