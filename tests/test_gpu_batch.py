"""Batched refinement (one graph launch for many instances) vs the oracle.

Every instance of a batch must come out exactly as the oracle's Algorithm 1
on that instance alone: same partition, objective, iteration counts, pin
counts and block weights, whatever the work split.  The device-side
refinement graph (jet_refine in graph mode) is checked the same way.
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
    inst = synth.config_batched(seed=5, count=9, n_lo=300, n_hi=6_000)
    h = synth.uniform(41, 3_000, 3_300, base=2, geo=(1, 2), size_cap=64, c_max=4, w_max=3)
    inst.append((h, 11, synth.part_perm(41, h.n, 11)))
    h = synth.uniform(42, 2_000, 2_200, base=2, geo=(1, 2), size_cap=64, w_max=40)  # heavy vertices
    inst.append((h, 128, synth.part_perm(42, h.n, 128)))
    h = synth.rownet(43, 6_000, 6_000, n_hubs=3, hub_min=2_100, hub_max=3_000)  # block-path edges
    inst.append((h, 32, synth.part_random(43, h.n, 32)))
    return inst


INST = _instances()


def _oracle(hg, k, part):
    orc = oracle.Oracle(hg)
    p = part.copy()
    iters, obj, phase = orc.refine(oracle.Params(k), p)
    phi, bw = orc.pincounts(k, p)
    return iters, obj, [int(x) for x in phase], p, phi, bw


EXPECTED = [_oracle(*x) for x in INST]


def _check(i, res, st):
    hg, k, _ = INST[i]
    iters, obj, phase, p, phi, bw = EXPECTED[i]
    assert res["iterations"] == iters and res["objective"] == obj, f"instance {i}"
    assert res["phase_iterations"][:3] == phase, f"instance {i}"
    assert np.array_equal(st.part.cpu().numpy()[: hg.n], p), f"instance {i}: partition"
    assert np.array_equal(st.phi.cpu().numpy()[: hg.m * k].reshape(hg.m, k), phi), f"instance {i}: phi"
    assert np.array_equal(st.block_w.cpu().numpy(), bw), f"instance {i}: block weights"


def _contexts():
    return [jet.jet_ctx_create(jet.DeviceHypergraph(h), jet.params(k)) for h, k, _ in INST]


@pytest.mark.parametrize("split", [0, 1, 4])
def test_batch_matches_oracle(split):
    ctxs = _contexts()
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, INST)]
    b = jet.jet_batch_create(ctxs)
    jet.jet_batch_set_split(b, split)
    res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for i, (r, st) in enumerate(zip(res, states)):
        _check(i, r, st)
    # a second launch of the cached graph from fresh partitions gives the same
    for st, (_, _, p) in zip(states, INST):
        st.part.copy_(torch.as_tensor(p))
    res2 = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for i, (r, st) in enumerate(zip(res2, states)):
        _check(i, r, st)
    b.close()


def test_batch_tune_restores_partitions_and_picks_a_split():
    ctxs = _contexts()
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, INST)]
    b = jet.jet_batch_create(ctxs)
    chosen, ms = jet.jet_batch_tune(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states, [0, 1, 2])
    assert chosen in (0, 1, 2) and set(ms) == {0, 1, 2} and all(t > 0 for t in ms.values())
    for st, (hg, _, p) in zip(states, INST):
        assert np.array_equal(st.part.cpu().numpy()[: hg.n], p)
    res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for i, (r, st) in enumerate(zip(res, states)):
        _check(i, r, st)


@pytest.mark.parametrize("graph", [True, False])
def test_refine_graph_and_host_loop_match_oracle(graph):
    for i in (0, 9, 10, 11):
        hg, k, part = INST[i]
        ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(k))
        jet.jet_set_graph_mode(ctx, graph)
        st = jet.JetState(ctx, part)
        res = jet.jet_refine(ctx, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, st.part, st.phi, st.block_w)
        _check(i, res, st)


def test_batch_argument_errors():
    c = jet.jet_ctx_create(jet.DeviceHypergraph(INST[0][0]), jet.params(INST[0][1]))
    with pytest.raises(jet.JetError) as ei:
        jet.jet_batch_create([c, c])
    assert ei.value.code == -1
    b = jet.jet_batch_create([c])
    with pytest.raises(jet.JetError) as ei:
        jet.jet_batch_set_split(b, -1)
    assert ei.value.code == -1
    st = jet.JetState(c, INST[0][2])
    with pytest.raises(jet.JetError) as ei:
        jet.jet_batch_refine(b, [(1, 1)], 8, [st])
    assert ei.value.code == -1


@pytest.mark.parametrize("shape", [(1, 256, 0), (1, 1024, 0), (2, 512, 0), (4, 1024, 0), (8, 256, 0),
                                   (8, 256, 8_000), (4, 512, 60_000)])
def test_persistent_batch_matches_oracle(shape):
    """The persistent form (one kernel, teams of `shape` blocks x threads, a device work queue; with a split,
    instances below that many pins run on single blocks of a cluster): every instance equals the oracle's
    Algorithm 1 on it alone, also on a second launch of the cached graph."""
    ctxs = _contexts()
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, INST)]
    b = jet.jet_batch_create(ctxs)
    jet.jet_batch_set_team(b, *shape)
    assert jet.jet_batch_get_team(b) == shape
    for _ in range(2):
        for st, (_, _, p) in zip(states, INST):
            st.part.copy_(torch.as_tensor(p))
        res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
        for i, (r, st) in enumerate(zip(res, states)):
            _check(i, r, st)
    b.close()


def test_persistent_autotune_restores_partitions_and_picks_a_shape():
    ctxs = _contexts()
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, INST)]
    b = jet.jet_batch_create(ctxs)
    shapes = ((1, 256, 0), (1, 1024, 0), (2, 512, 0), (2, 512, 10_000))
    chosen, trials = jet.jet_batch_autotune(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states, shapes,
                                            sample=5, trial_iterations=3)
    assert chosen in shapes and set(trials) == set(shapes)
    assert all(ms > 0 and rate > 0 for ms, rate in trials.values())
    for st, (hg, _, p) in zip(states, INST):
        assert np.array_equal(st.part.cpu().numpy()[: hg.n], p)
    res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for i, (r, st) in enumerate(zip(res, states)):
        _check(i, r, st)
    b.close()


def test_persistent_batch_errors():
    ctxs = _contexts()[:3]
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, INST[:3])]
    b = jet.jet_batch_create(ctxs)
    for ctas, threads, split in ((3, 256, 0), (1, 100, 0), (1, 2048, 0), (2, 256, -1)):
        with pytest.raises(jet.JetError) as ei:
            jet.jet_batch_set_team(b, ctas, threads, split)
        assert ei.value.code == -1
    jet.jet_batch_set_team(b, 1, 256)
    bad = INST[1][2].copy()
    bad[7] = INST[1][1]  # block id k: outside [0, k)
    states[1].part.copy_(torch.as_tensor(bad))
    with pytest.raises(jet.JetError) as ei:
        jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    assert ei.value.code == -5 and "instance 1" in str(ei.value)
    # the batch stays usable (the other instances were refined by the failed launch: start them over)
    for st, (_, _, p) in zip(states, INST[:3]):
        st.part.copy_(torch.as_tensor(p))
    res = jet.jet_batch_refine(b, oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, states)
    for i, (r, st) in enumerate(zip(res, states)):
        _check(i, r, st)
    b.close()
