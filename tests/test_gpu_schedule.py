"""Matching schedule of k-way refinement (Section 5) on the GPU vs the oracle.

The quotient graph and every round of the schedule must equal the oracle's,
pair by pair and in the same order, for k from 2 to 256, for the seeded start
partitions and for partitions after a few Jet iterations (sparser quotient
graphs), and for the degenerate partition with a single block.
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
from test_gpu_parity import INSTANCES, NAMES  # noqa: E402


def _oracle_schedule(hg, k, part):
    o = oracle.Oracle(hg)
    phi, _ = o.pincounts(k, part)
    return o.schedule(o.quotient(k, phi))


def _check(hg, k, part, ctx, st):
    got = jet.jet_quotient_schedule(ctx, st.phi)
    want = _oracle_schedule(hg, k, part)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]) and got[2] == want[2]
    return got


@pytest.mark.parametrize("name", NAMES)
def test_schedule_matches_oracle(name):
    hg, k, part = INSTANCES[name]
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(k))
    st = jet.JetState(ctx, part)
    _check(hg, k, part, ctx, st)
    for tau in ((3, 4), (3, 4), (0, 1)):  # refined partitions: fewer cut pairs
        st.round(tau)
    _check(hg, k, st.part.cpu().numpy()[: hg.n], ctx, st)
    ctx.close()


def test_single_block_has_empty_schedule():
    hg = synth.uniform(3, 400, 500, base=2, geo=(1, 2), size_cap=8)
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(8))
    st = jet.JetState(ctx, np.zeros(hg.n, np.int32))
    pairs, rnd, nr = jet.jet_quotient_schedule(ctx, st.phi)
    assert len(pairs) == 0 and nr == 0
    ctx.close()
