"""The serving loop: jobs admitted by memory footprint and run concurrently.

Each job's refined partition must be the same when it runs in a mix of
concurrent jobs as when it runs alone, and the same as the oracle's
Algorithm 1 on that job.
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

JOBS = []
for j in range(10):
    h = synth.served_instance(500 + j, P_lo=2_000, P_hi=40_000)
    k = 2 << (j % 8)
    JOBS.append((h, k, synth.part_perm(900 + j, h.n, k)))


def _oracle(h, k, part):
    p = part.copy()
    iters, obj, _ = oracle.Oracle(h).refine(oracle.Params(k), p)
    return iters, obj, p


EXPECTED = [_oracle(*j) for j in JOBS]


def _run(slots, budget):
    server = jet.jet_server_create(budget, slots)
    parts = [p.copy() for _, _, p in JOBS]
    ids = {jet.jet_server_submit(server, h, jet.params(k), oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, parts[i]): i
           for i, (h, k, _) in enumerate(JOBS)}
    done = []
    while len(done) < len(JOBS):
        done += jet.jet_server_wait(server, timeout_ms=10_000)
    server.close()
    return parts, {ids[d["id"]]: d for d in done}


def test_jobs_match_alone_and_oracle():
    fp = max(jet.jet_job_footprint(h.n, h.m, h.P, k) for h, k, _ in JOBS)
    mixed, dm = _run(4, int(2.5 * fp))   # at most two jobs fit the budget at a time
    alone, da = _run(1, int(1.1 * fp))
    for i, ((h, k, _), (iters, obj, p)) in enumerate(zip(JOBS, EXPECTED)):
        assert dm[i]["status"] == 0 and da[i]["status"] == 0
        assert np.array_equal(mixed[i], p), f"job {i}: mixed run differs from the oracle"
        assert np.array_equal(alone[i], p), f"job {i}: alone run differs from the oracle"
        assert dm[i]["result"]["iterations"] == iters and dm[i]["result"]["objective"] == obj
        assert dm[i]["latency_ms"] >= dm[i]["queue_ms"] >= 0
        assert dm[i]["message"] == ""
        assert 0 <= dm[i]["device_start_ms"] <= dm[i]["device_end_ms"]
    # continuous batching: jobs admitted together had work in flight on the GPU at the same time
    spans = sorted((d["device_start_ms"], d["device_end_ms"]) for d in dm.values())
    overlaps = sum(1 for (a0, a1), (b0, b1) in zip(spans, spans[1:]) if b0 < a1)
    assert overlaps >= 1, f"no two jobs overlapped on the device: {spans}"
    # one slot: the jobs ran one after another
    spans = sorted((d["device_start_ms"], d["device_end_ms"]) for d in da.values())
    assert all(b0 >= a1 for (a0, a1), (b0, b1) in zip(spans, spans[1:])), spans


def test_submit_errors():
    with pytest.raises(jet.JetError) as ei:
        jet.jet_server_create(1 << 30, 0)
    assert ei.value.code == -1
    h, k, p = JOBS[0]
    server = jet.jet_server_create(1024, 1)  # smaller than any job's footprint
    with pytest.raises(jet.JetError) as ei:
        jet.jet_server_submit(server, h, jet.params(k), oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, p.copy())
    assert ei.value.code == -2
    assert jet.jet_server_load(server) == {"pending": 0, "running": 0, "reserved_bytes": 0}
    server.close()


def test_failed_job_reports_its_reason():
    """A job whose partition holds a block id outside [0, k) fails with JET_ERR_DATA, and its report carries the
    reason; the jobs around it are unaffected."""
    server = jet.jet_server_create(1 << 34, 2)
    parts = [p.copy() for _, _, p in JOBS[:3]]
    parts[1][5] = JOBS[1][1]  # block id k: out of range
    ids = {jet.jet_server_submit(server, h, jet.params(k), oracle.TAU_SCHEDULE, oracle.ITERATION_LIMIT, parts[i]): i
           for i, (h, k, _) in enumerate(JOBS[:3])}
    done = []
    while len(done) < 3:
        done += jet.jet_server_wait(server, timeout_ms=10_000)
    server.close()
    by = {ids[d["id"]]: d for d in done}
    assert by[1]["status"] == -5 and "partition" in by[1]["message"], by[1]
    for i in (0, 2):
        assert by[i]["status"] == 0 and by[i]["message"] == ""
        assert np.array_equal(parts[i], EXPECTED[i][2])
