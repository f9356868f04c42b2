"""The allocation-free block-weight entry point against the context path.

jet_block_weights_noalloc is for callers that must not allocate device
memory (their device memory is owned up front by their own pool, or a
cudaMalloc/cudaFree would stall a latency-critical loop).  It keeps its
scratch in a static device array instead of a context.  This file is named
to be collected last, so a failure here never hides another test's result;
it passes both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_2504_12013_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_12013_gb300 import jet  # noqa: E402


def _noalloc(lib, part, vwgt, k, block_w, block_count):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.jet_block_weights_noalloc(ctypes.c_void_p(part.data_ptr()), ctypes.c_void_p(vwgt.data_ptr()),
                                         part.numel(), k, ctypes.c_void_p(block_w.data_ptr()),
                                         ctypes.c_void_p(block_count.data_ptr()) if block_count is not None
                                         else None, ctypes.c_void_p(stream))


@pytest.mark.parametrize("k", [27, 256])
def test_noalloc_matches_context_path_on_two_calls(k):
    lib = jet.load_library()
    hg = synth.uniform(21, 50_000, 60_000, base=2, geo=(1, 2), size_cap=32, c_max=4)
    # existing entry point: block weights of jet_build_pincounts through a context
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg), jet.params(k))
    vwgt = torch.from_numpy(hg.vwgt).cuda()
    for call, seed in enumerate((5, 6)):  # two calls in a row, different partitions
        part_np = synth.part_random(seed, hg.n, k)
        part = torch.from_numpy(part_np).cuda()
        st = jet.JetState(ctx, part_np)
        ref = st.block_w.cpu().numpy()
        bw = torch.full((k,), -7, dtype=torch.int64, device="cuda")
        cnt = torch.full((k,), -7, dtype=torch.int32, device="cuda")
        rc = _noalloc(lib, part, vwgt, k, bw, cnt)
        assert rc == 0, jet.jet_last_error(None)
        assert np.array_equal(bw.cpu().numpy(), ref), f"call {call}"
        # and against the definition c(V_i) = sum of c(v) over Pi(v) = i, computed on the host
        want = np.bincount(part_np, weights=hg.vwgt.astype(np.float64), minlength=k).astype(np.int64)
        assert np.array_equal(bw.cpu().numpy(), want), f"call {call}"
        assert np.array_equal(cnt.cpu().numpy(), np.bincount(part_np, minlength=k)), f"call {call}"
    ctx.close()


def test_noalloc_rejects_k_beyond_its_scratch():
    lib = jet.load_library()
    part = torch.zeros(10, dtype=torch.int32, device="cuda")
    vw = torch.ones(10, dtype=torch.int32, device="cuda")
    bw = torch.zeros(300, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, part, vw, 257, bw, None) == -1
    assert "256" in jet.jet_last_error(None)


def test_noalloc_reports_bad_partition_then_recovers():
    lib = jet.load_library()
    n, k = 1000, 8
    part_np = synth.part_hash(3, n, k)
    bad = part_np.copy()
    bad[123] = k
    vw = torch.ones(n, dtype=torch.int32, device="cuda")
    bw = torch.zeros(k, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, torch.from_numpy(bad).cuda(), vw, k, bw, None) == -5
    assert _noalloc(lib, torch.from_numpy(part_np).cuda(), vw, k, bw, None) == 0
    assert np.array_equal(bw.cpu().numpy(), np.bincount(part_np, minlength=k))


def test_noalloc_reports_weight_below_one_then_recovers():
    """c(v) >= 1 is required (jet_ctx_create rejects such inputs too): a zero weight is a data error."""
    lib = jet.load_library()
    n, k = 1000, 8
    part_np = synth.part_hash(4, n, k)
    vw_np = np.arange(n, dtype=np.int32) % 5 + 1
    bad = vw_np.copy()
    bad[77] = 0
    part = torch.from_numpy(part_np).cuda()
    bw = torch.zeros(k, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, part, torch.from_numpy(bad).cuda(), k, bw, None) == -5
    assert "weight" in jet.jet_last_error(None)
    assert _noalloc(lib, part, torch.from_numpy(vw_np).cuda(), k, bw, None) == 0
    want = np.bincount(part_np, weights=vw_np.astype(np.float64), minlength=k).astype(np.int64)
    assert np.array_equal(bw.cpu().numpy(), want)
