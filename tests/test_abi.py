"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares (no GPU)."""
import ctypes
import os
import re

from paper_2504_12013_gb300 import build as cuda_build
from paper_2504_12013_gb300 import jet

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jet.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jet_[a-z_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(jet.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = cuda_build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_errors_without_gpu():
    lib = jet.load_library()
    # argument errors are detected on the host before any CUDA call
    out = ctypes.c_void_p()
    rc = lib.jet_ctx_create(ctypes.byref(out), None, None, None)
    assert rc == -1 and out.value is None
    assert "NULL" in jet.jet_last_error(None)
    hg = jet.JetHypergraph(4, 2, 4, 1, 1, 1, 1, 1, 1)
    for bad in (jet.params(1), jet.params(257), jet.params(8, eps=(1, 0)), jet.params(8, d=(-1, 10))):
        rc = lib.jet_ctx_create(ctypes.byref(out), ctypes.byref(hg), ctypes.byref(bad), None)
        assert rc == -1, (bad.k, bad.eps_den, bad.d_num)
    assert lib.jet_build_pincounts(None, None, None, None) == -1
    assert lib.jet_refine_round(None, 0, 1, None, None, None, None, None) == -1


def test_sources_target_sm_103a_only():
    assert cuda_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_coarsening_graph_path_and_uncoarsening_argument_errors_without_gpu():
    """The newer entry points reject bad arguments on the host, before any CUDA call."""
    lib = jet.load_library()
    hg = jet.JetHypergraph(4, 2, 4, 1, 1, 1, 1, 1, 1)  # sizes only; no pointer is dereferenced here
    assert lib.jet_cluster(None, None, None, None, None) == -1
    assert lib.jet_cluster(ctypes.byref(hg), None, None, None, None) == -1
    for bad in (jet.JetCoarsenParams(0, 1000, 100, 100), jet.JetCoarsenParams(10, 1, 100, 100),
                jet.JetCoarsenParams(10, 1000, -1, 100), jet.JetCoarsenParams(10, 1000, 100, 0)):
        assert lib.jet_cluster(ctypes.byref(hg), ctypes.byref(bad), 1, 1, None) == -1
    neg = jet.JetHypergraph(-1, 2, 4, 1, 1, 1, 1, 1, 1)
    ok = jet.JetCoarsenParams(10, 1000, 100, 100)
    assert lib.jet_cluster(ctypes.byref(neg), ctypes.byref(ok), 1, 1, None) == -1
    n, m, P = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    assert lib.jet_contract(None, None, None, None, ctypes.byref(n), ctypes.byref(m), ctypes.byref(P), None) == -1
    assert lib.jet_contract(ctypes.byref(hg), 1, 1, None, ctypes.byref(n), ctypes.byref(m), ctypes.byref(P),
                            None) == -1  # no output buffers
    assert lib.jet_set_graph_path(None, 1) == -1
    assert lib.jet_uncoarsen(None, 0, None, None, 0, 8, None, None, None, None, None) == -1
    assert lib.jet_quotient_schedule(None, None, None, None, None, None) == -1
