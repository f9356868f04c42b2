"""Python binding of libjet (``include/jet.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch tensors (device memory) where the C function takes device pointers.
All computation happens in the CUDA library; there is no CPU fallback.  If
``lib/libjet.so`` is missing, every call raises ``RuntimeError``: build it
with ``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libjet.so")

JET_OK = 0
ERRORS = {-1: "JET_ERR_INVALID_ARG", -2: "JET_ERR_OOM", -3: "JET_ERR_CUDA", -4: "JET_ERR_OVERFLOW", -5: "JET_ERR_DATA"}

# every symbol include/jet.h declares
EXPORTS = ("jet_ctx_create", "jet_ctx_destroy", "jet_last_error", "jet_build_pincounts", "jet_connectivity",
           "jet_refine_round", "jet_rebalance", "jet_refine", "jet_candidates", "jet_afterburner",
           "jet_refine_host", "jet_profile_enable", "jet_profile_read", "jet_block_weights_noalloc",
           "jet_set_graph_mode", "jet_batch_create", "jet_batch_destroy", "jet_batch_last_error",
           "jet_batch_refine", "jet_batch_set_split", "jet_batch_get_split", "jet_batch_tune",
           "jet_job_footprint", "jet_server_create", "jet_server_submit", "jet_server_wait", "jet_server_load",
           "jet_server_last_error", "jet_server_destroy", "jet_profile_work", "jet_quotient_schedule",
           "jet_uncoarsen", "jet_cluster", "jet_contract", "jet_set_graph_path", "jet_rounds_host",
           "jet_batch_set_team", "jet_batch_get_team", "jet_batch_autotune", "jet_release_memory")

PROF_FAMILIES = ("pincounts", "candidates", "afterburner", "approve", "apply", "rebalance_targets",
                 "rebalance_select", "rebalance_control", "objective", "other")

_P = ctypes.c_void_p


class JetHypergraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("P", ctypes.c_int64),
                ("eptr", _P), ("pins", _P), ("vptr", _P), ("inc", _P), ("vwgt", _P), ("ewgt", _P)]


class JetCoarsenParams(ctypes.Structure):
    _fields_ = [("max_cluster_weight", ctypes.c_int64), ("rating_max_edge", ctypes.c_int32),
                ("single_subrounds", ctypes.c_int32), ("subround_cap_div", ctypes.c_int32)]


class JetHypergraphOut(ctypes.Structure):
    _fields_ = [("eptr", _P), ("pins", _P), ("vptr", _P), ("inc", _P), ("vwgt", _P), ("ewgt", _P)]


class JetParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("eps_num", ctypes.c_int32), ("eps_den", ctypes.c_int32),
                ("d_num", ctypes.c_int32), ("d_den", ctypes.c_int32), ("max_rebalance_rounds", ctypes.c_int32)]


STATS_FIELDS = ("candidates", "approved", "rebalance_rounds", "rebalance_moves", "objective", "max_block_weight",
                "imbalanced", "reserved")


class JetRoundStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in STATS_FIELDS]


class JetRefineResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("objective", ctypes.c_int64),
                ("initial_objective", ctypes.c_int64), ("balanced", ctypes.c_int64),
                ("phase_iterations", ctypes.c_int64 * 8)]

    def as_dict(self):
        return {"iterations": self.iterations, "objective": self.objective,
                "initial_objective": self.initial_objective, "balanced": self.balanced,
                "phase_iterations": list(self.phase_iterations)}


class JetJobDone(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("device_start_ms", ctypes.c_double), ("device_end_ms", ctypes.c_double),
                ("result", JetRefineResult), ("message", ctypes.c_char * 128)]


class JetError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load_library():
    """Load libjet.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library has not been built "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(LIB_PATH)
            i32, i64, pp = ctypes.c_int32, ctypes.c_int64, ctypes.POINTER
            lib.jet_ctx_create.argtypes = [pp(_P), pp(JetHypergraph), pp(JetParams), _P]
            lib.jet_ctx_destroy.argtypes = [_P]
            lib.jet_ctx_destroy.restype = None
            lib.jet_last_error.argtypes = [_P]
            lib.jet_last_error.restype = ctypes.c_char_p
            lib.jet_build_pincounts.argtypes = [_P, _P, _P, _P]
            lib.jet_connectivity.argtypes = [_P, _P, _P]
            lib.jet_refine_round.argtypes = [_P, i32, i32, _P, _P, _P, _P, _P]
            lib.jet_rebalance.argtypes = [_P, _P, _P, _P, _P]
            lib.jet_refine.argtypes = [_P, pp(i32), i32, i32, _P, _P, _P, pp(JetRefineResult)]
            lib.jet_candidates.argtypes = [_P, i32, i32, _P, _P, _P, _P, _P, _P]
            lib.jet_afterburner.argtypes = [_P, _P, _P, _P, _P]
            lib.jet_refine_host.argtypes = [pp(JetHypergraph), pp(JetParams), pp(i32), i32, i32, _P,
                                            pp(JetRefineResult)]
            lib.jet_rounds_host.argtypes = [pp(JetHypergraph), pp(JetParams), i32, i32, i32, _P, pp(JetRoundStats)]
            lib.jet_profile_enable.argtypes = [_P, ctypes.c_int]
            lib.jet_profile_read.argtypes = [_P, pp(ctypes.c_double), pp(i64), pp(i64), ctypes.c_int]
            lib.jet_block_weights_noalloc.argtypes = [_P, _P, i32, i32, _P, _P, _P]
            lib.jet_set_graph_mode.argtypes = [_P, ctypes.c_int]
            lib.jet_set_graph_path.argtypes = [_P, ctypes.c_int]
            lib.jet_profile_work.argtypes = [_P, pp(i64), i32]
            lib.jet_quotient_schedule.argtypes = [_P, _P, _P, _P, pp(i32), pp(i32)]
            lib.jet_uncoarsen.argtypes = [pp(_P), i32, pp(_P), pp(i32), i32, i32, pp(_P), pp(_P), pp(_P),
                                          pp(JetRefineResult), _P]
            lib.jet_cluster.argtypes = [pp(JetHypergraph), pp(JetCoarsenParams), _P, _P, _P]
            lib.jet_contract.argtypes = [pp(JetHypergraph), _P, _P, pp(JetHypergraphOut), pp(i32), pp(i32), pp(i64),
                                         _P]
            lib.jet_batch_create.argtypes = [pp(_P), pp(_P), i32, _P]
            lib.jet_batch_destroy.argtypes = [_P]
            lib.jet_batch_destroy.restype = None
            lib.jet_batch_last_error.argtypes = [_P]
            lib.jet_batch_last_error.restype = ctypes.c_char_p
            lib.jet_batch_refine.argtypes = [_P, pp(i32), i32, i32, pp(_P), pp(_P), pp(_P), pp(JetRefineResult)]
            lib.jet_batch_set_split.argtypes = [_P, i32]
            lib.jet_batch_get_split.argtypes = [_P]
            lib.jet_batch_tune.argtypes = [_P, pp(i32), i32, i32, pp(_P), pp(_P), pp(_P), pp(i32), i32,
                                           pp(ctypes.c_float)]
            lib.jet_batch_set_team.argtypes = [_P, i32, i32, i32]
            lib.jet_batch_get_team.argtypes = [_P, pp(i32), pp(i32), pp(i32)]
            lib.jet_batch_autotune.argtypes = [_P, pp(i32), i32, i32, pp(_P), pp(_P), pp(_P), pp(i32), i32, i32, i32,
                                               pp(ctypes.c_float), pp(ctypes.c_double)]
            sz = ctypes.c_size_t
            lib.jet_job_footprint.argtypes = [i32, i32, i64, i32]
            lib.jet_job_footprint.restype = sz
            lib.jet_server_create.argtypes = [pp(_P), sz, i32]
            lib.jet_server_submit.argtypes = [_P, pp(JetHypergraph), pp(JetParams), pp(i32), i32, i32, _P, pp(i64)]
            lib.jet_server_wait.argtypes = [_P, pp(JetJobDone), i32, pp(i32), i32]
            lib.jet_server_load.argtypes = [_P, pp(i32), pp(i32), pp(sz)]
            lib.jet_server_last_error.argtypes = [_P]
            lib.jet_server_last_error.restype = ctypes.c_char_p
            lib.jet_server_destroy.argtypes = [_P]
            lib.jet_server_destroy.restype = None
            for f in EXPORTS:
                if f not in ("jet_ctx_destroy", "jet_last_error", "jet_batch_destroy", "jet_batch_last_error",
                             "jet_job_footprint", "jet_server_last_error", "jet_server_destroy"):
                    getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _check(rc, ctx=None):
    if rc != JET_OK:
        raise JetError(rc, jet_last_error(ctx))


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class DeviceHypergraph:
    """A host ``synth.Hypergraph`` uploaded to torch device tensors."""

    def __init__(self, hg, device="cuda"):
        import torch
        self.n, self.m, self.P = hg.n, hg.m, hg.P
        self.host = hg
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.eptr, self.pins, self.vptr, self.inc = t(hg.eptr), t(hg.pins), t(hg.vptr), t(hg.inc)
        self.vwgt, self.ewgt = t(hg.vwgt), t(hg.ewgt)

    @classmethod
    def from_tensors(cls, n, m, P, eptr, pins, vptr, inc, vwgt, ewgt):
        """A hypergraph already on the device (e.g. a contraction's output), trimmed to its sizes."""
        self = cls.__new__(cls)
        self.n, self.m, self.P = int(n), int(m), int(P)
        self.host = None
        self.eptr, self.pins, self.vptr, self.inc = eptr[: m + 1], pins[:P], vptr[: n + 1], inc[:P]
        self.vwgt, self.ewgt = vwgt[:n], ewgt[:m]
        return self

    def to_host(self):
        from . import synth
        c = lambda t: t.cpu().numpy().copy()
        return synth.Hypergraph(n=self.n, m=self.m, eptr=c(self.eptr), pins=c(self.pins), vptr=c(self.vptr),
                                inc=c(self.inc), vwgt=c(self.vwgt), ewgt=c(self.ewgt))

    def c(self) -> JetHypergraph:
        import torch
        return JetHypergraph(self.n, self.m, self.P, _ptr(self.eptr, torch.int64), _ptr(self.pins, torch.int32),
                             _ptr(self.vptr, torch.int64), _ptr(self.inc, torch.int32),
                             _ptr(self.vwgt, torch.int32), _ptr(self.ewgt, torch.int32))


RATING_MAX_EDGE = 1000   # edges with more pins add nothing to a coarsening rating
SINGLE_SUBROUNDS = 100   # one-vertex sub-rounds at the start of a clustering level (Section 6)
SUBROUND_CAP_DIV = 100   # sub-rounds grow to 1% of the vertices (Section 6)


def jet_cluster(dh, cmax, order, rmax=RATING_MAX_EDGE, n_single=SINGLE_SUBROUNDS, cap_div=SUBROUND_CAP_DIV,
                stream=None):
    """One level of synchronous clustering (Section 6, Algorithm 4): the label tensor (int32, n)."""
    import torch
    label = torch.empty(max(dh.n, 1), dtype=torch.int32, device=dh.eptr.device)
    prm = JetCoarsenParams(int(cmax), int(rmax), int(n_single), int(cap_div))
    _check(load_library().jet_cluster(ctypes.byref(dh.c()), ctypes.byref(prm), _ptr(order, torch.int32, "order"),
                                      _ptr(label, torch.int32), _stream_ptr(stream)))
    return label[: dh.n]


def jet_contract(dh, label, stream=None):
    """Contraction of the label classes: (coarse DeviceHypergraph, map tensor)."""
    import torch
    dev = dh.eptr.device
    e = lambda n, dt: torch.empty(max(n, 1), dtype=dt, device=dev)
    eptr, pins, vptr, inc = e(dh.m + 1, torch.int64), e(dh.P, torch.int32), e(dh.n + 1, torch.int64), e(dh.P, torch.int32)
    vwgt, ewgt, mp = e(dh.n, torch.int32), e(dh.m, torch.int32), e(dh.n, torch.int32)
    out = JetHypergraphOut(_ptr(eptr), _ptr(pins), _ptr(vptr), _ptr(inc), _ptr(vwgt), _ptr(ewgt))
    nc, mc, pc = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    _check(load_library().jet_contract(ctypes.byref(dh.c()), _ptr(label, torch.int32, "label"), _ptr(mp),
                                       ctypes.byref(out), ctypes.byref(nc), ctypes.byref(mc), ctypes.byref(pc),
                                       _stream_ptr(stream)))
    coarse = DeviceHypergraph.from_tensors(nc.value, mc.value, pc.value, eptr, pins, vptr, inc, vwgt, ewgt)
    return coarse, mp[: dh.n]


def jet_coarsen(dh, cmax, order, stream=None, **kw):
    """One coarsening level: (coarse DeviceHypergraph, map, labels)."""
    label = jet_cluster(dh, cmax, order, stream=stream, **kw)
    coarse, mp = jet_contract(dh, label, stream)
    return coarse, mp, label


def params(k, eps=(3, 100), d=(1, 10), max_rebalance_rounds=32) -> JetParams:
    return JetParams(k, eps[0], eps[1], d[0], d[1], max_rebalance_rounds)


class Ctx:
    """Owning handle of a jet_ctx; keeps the hypergraph tensors alive."""

    def __init__(self, handle, hg, params_):
        self.handle = handle
        self.hg = hg
        self.params = params_

    @property
    def k(self):
        return self.params.k

    def close(self):
        if self.handle:
            load_library().jet_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- C ABI names

def jet_last_error(ctx=None) -> str:
    h = ctx.handle if isinstance(ctx, Ctx) else ctx
    return load_library().jet_last_error(h).decode()


def jet_ctx_create(hg: DeviceHypergraph, p: JetParams, stream=None) -> Ctx:
    lib = load_library()
    out = _P()
    chg = hg.c()
    rc = lib.jet_ctx_create(ctypes.byref(out), ctypes.byref(chg), ctypes.byref(p), _stream_ptr(stream))
    _check(rc)
    return Ctx(out, hg, p)


def jet_ctx_destroy(ctx: Ctx):
    ctx.close()


def jet_build_pincounts(ctx: Ctx, part, phi, block_w):
    import torch
    _check(load_library().jet_build_pincounts(ctx.handle, _ptr(part, torch.int32, "part"),
                                              _ptr(phi, torch.int32, "phi"), _ptr(block_w, torch.int64, "block_w")),
           ctx)


def jet_connectivity(ctx: Ctx, phi, objective_out):
    import torch
    _check(load_library().jet_connectivity(ctx.handle, _ptr(phi, torch.int32, "phi"),
                                           _ptr(objective_out, torch.int64, "objective_out")), ctx)


def jet_refine_round(ctx: Ctx, tau, part, phi, block_w, locked, stats=None):
    import torch
    _check(load_library().jet_refine_round(ctx.handle, int(tau[0]), int(tau[1]), _ptr(part, torch.int32, "part"),
                                           _ptr(phi, torch.int32, "phi"), _ptr(block_w, torch.int64, "block_w"),
                                           _ptr(locked, torch.uint8, "locked"), _ptr(stats, torch.int64, "stats")),
           ctx)


def jet_rebalance(ctx: Ctx, part, phi, block_w, stats=None):
    import torch
    _check(load_library().jet_rebalance(ctx.handle, _ptr(part, torch.int32, "part"), _ptr(phi, torch.int32, "phi"),
                                        _ptr(block_w, torch.int64, "block_w"), _ptr(stats, torch.int64, "stats")),
           ctx)


def jet_refine(ctx: Ctx, schedule, limit, part, phi, block_w) -> dict:
    import torch
    pairs = (ctypes.c_int32 * (2 * len(schedule)))(*[int(x) for t in schedule for x in t])
    res = JetRefineResult()
    _check(load_library().jet_refine(ctx.handle, pairs, len(schedule), int(limit), _ptr(part, torch.int32, "part"),
                                     _ptr(phi, torch.int32, "phi"), _ptr(block_w, torch.int64, "block_w"),
                                     ctypes.byref(res)), ctx)
    return res.as_dict()


def jet_candidates(ctx: Ctx, tau, part, phi, locked, target, gain, in_m):
    import torch
    _check(load_library().jet_candidates(ctx.handle, int(tau[0]), int(tau[1]), _ptr(part, torch.int32, "part"),
                                         _ptr(phi, torch.int32, "phi"), _ptr(locked, torch.uint8, "locked"),
                                         _ptr(target, torch.int32, "target"), _ptr(gain, torch.int32, "gain"),
                                         _ptr(in_m, torch.uint8, "in_m")), ctx)


def jet_afterburner(ctx: Ctx, part, phi, rg, approved):
    import torch
    _check(load_library().jet_afterburner(ctx.handle, _ptr(part, torch.int32, "part"), _ptr(phi, torch.int32, "phi"),
                                          _ptr(rg, torch.int32, "rg"), _ptr(approved, torch.uint8, "approved")), ctx)


def jet_refine_host(hg, p: JetParams, schedule, limit, part: np.ndarray) -> dict:
    """Host buffers in and out: ``hg`` is a ``synth.Hypergraph`` (numpy), ``part`` int32[n] is refined in place."""
    assert part.dtype == np.int32 and part.flags.c_contiguous
    arrs = [np.ascontiguousarray(a) for a in (hg.eptr, hg.pins, hg.vptr, hg.inc, hg.vwgt, hg.ewgt)]
    ch = JetHypergraph(hg.n, hg.m, hg.P, *[a.ctypes.data for a in arrs])
    pairs = (ctypes.c_int32 * (2 * len(schedule)))(*[int(x) for t in schedule for x in t])
    res = JetRefineResult()
    rc = load_library().jet_refine_host(ctypes.byref(ch), ctypes.byref(p), pairs, len(schedule), int(limit),
                                        part.ctypes.data, ctypes.byref(res))
    _check(rc)
    return res.as_dict()


def jet_rounds_host(hg, p: JetParams, tau, n_rounds, part: np.ndarray) -> dict:
    """Host buffers in and out: n_rounds Jet iterations at temperature tau from ``part`` (int32[n], updated in
    place); returns the last iteration's statistics."""
    assert part.dtype == np.int32 and part.flags.c_contiguous
    arrs = [np.ascontiguousarray(a) for a in (hg.eptr, hg.pins, hg.vptr, hg.inc, hg.vwgt, hg.ewgt)]
    ch = JetHypergraph(hg.n, hg.m, hg.P, *[a.ctypes.data for a in arrs])
    st = JetRoundStats()
    _check(load_library().jet_rounds_host(ctypes.byref(ch), ctypes.byref(p), int(tau[0]), int(tau[1]),
                                          int(n_rounds), part.ctypes.data, ctypes.byref(st)))
    return {f: int(getattr(st, f)) for f in STATS_FIELDS[:7]}


def jet_set_graph_mode(ctx: Ctx, enable: bool = True):
    _check(load_library().jet_set_graph_mode(ctx.handle, 1 if enable else 0), ctx)


def jet_set_graph_path(ctx: Ctx, enable: bool = True):
    """Graph path (every edge two distinct pins): neighbour blocks instead of phi; phi is not maintained."""
    _check(load_library().jet_set_graph_path(ctx.handle, 1 if enable else 0), ctx)


def jet_release_memory():
    """Return the device memory the library keeps in its pools (one per device) to the driver."""
    _check(load_library().jet_release_memory())


def jet_profile_enable(ctx: Ctx, enable: bool = True):
    _check(load_library().jet_profile_enable(ctx.handle, 1 if enable else 0), ctx)


def jet_profile_read(ctx: Ctx, reset: bool = True) -> dict:
    """Per kernel family: device ms (while enabled), timed calls, kernel launches."""
    n = len(PROF_FAMILIES)
    ms = (ctypes.c_double * n)()
    calls = (ctypes.c_int64 * n)()
    launches = (ctypes.c_int64 * n)()
    _check(load_library().jet_profile_read(ctx.handle, ms, calls, launches, 1 if reset else 0), ctx)
    return {f: {"ms": ms[i], "calls": calls[i], "launches": launches[i]} for i, f in enumerate(PROF_FAMILIES)}


def jet_uncoarsen(ctxs, maps, schedule, limit, states, stream=None) -> list:
    """Project and refine level by level, coarsest first (states[0].part holds the coarsest partition);
    maps[l] (int32 tensor) maps the vertices of level l+1 to level l.  One graph launch."""
    import torch
    n = len(ctxs)
    hs = (_P * n)(*[c.handle for c in ctxs])
    mp = (_P * max(n - 1, 1))(*([_ptr(m, torch.int32, "map") for m in maps] or [None]))
    part, phi, bw = _state_arrays(states)
    res = (JetRefineResult * n)()
    rc = load_library().jet_uncoarsen(hs, n, mp, _pairs(schedule), len(schedule), int(limit), part, phi, bw, res,
                                      _stream_ptr(stream))
    if rc != JET_OK:
        raise JetError(rc, jet_last_error(None))
    return [r.as_dict() for r in res]


def jet_quotient_schedule(ctx: Ctx, phi):
    """Matching schedule of the quotient graph: (pairs int32[p, 2], round int32[p], rounds) on the host."""
    import torch
    k = ctx.k
    cap = max(k * (k - 1) // 2, 1)
    dev = phi.device
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device=dev)
    rnd = torch.zeros(cap, dtype=torch.int32, device=dev)
    npairs, nr = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().jet_quotient_schedule(ctx.handle, _ptr(phi, torch.int32, "phi"), _ptr(pairs), _ptr(rnd),
                                                ctypes.byref(npairs), ctypes.byref(nr)), ctx)
    p = npairs.value
    return pairs[: 2 * p].cpu().numpy().reshape(-1, 2), rnd[:p].cpu().numpy(), nr.value


WORK_FIELDS = ("rebalance_over", "rebalance_evaluated", "rebalance_evaluated_pins", "moved_pins", "select_levels")


def jet_profile_work(ctx: Ctx) -> dict:
    out = (ctypes.c_int64 * 5)()
    _check(load_library().jet_profile_work(ctx.handle, out, 5), ctx)
    return dict(zip(WORK_FIELDS, [int(x) for x in out]))


def jet_block_weights_noalloc(part, vwgt, k, block_w, block_count=None, stream=None):
    """c(V_i) (and |V_i|) with no device allocation; scratch is a static device array (k <= 256)."""
    import torch
    n = part.numel()
    _check(load_library().jet_block_weights_noalloc(_ptr(part, torch.int32, "part"), _ptr(vwgt, torch.int32, "vwgt"),
                                                    n, int(k), _ptr(block_w, torch.int64, "block_w"),
                                                    _ptr(block_count, torch.int32, "block_count"),
                                                    _stream_ptr(stream)))


class Batch:
    """Owning handle of a jet_batch; keeps its contexts alive."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)

    def close(self):
        if self.handle:
            load_library().jet_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_check(rc, batch):
    if rc != JET_OK:
        raise JetError(rc, load_library().jet_batch_last_error(batch.handle if batch else None).decode())


def jet_batch_create(ctxs, stream=None) -> Batch:
    lib = load_library()
    out = _P()
    arr = (_P * len(ctxs))(*[c.handle for c in ctxs])
    _batch_check(lib.jet_batch_create(ctypes.byref(out), arr, len(ctxs), _stream_ptr(stream)), None)
    return Batch(out, ctxs)


def jet_batch_destroy(batch: Batch):
    batch.close()


def _state_arrays(states):
    import torch
    part = (_P * len(states))(*[_ptr(s.part, torch.int32, "part") for s in states])
    phi = (_P * len(states))(*[_ptr(s.phi, torch.int32, "phi") for s in states])
    bw = (_P * len(states))(*[_ptr(s.block_w, torch.int64, "block_w") for s in states])
    return part, phi, bw


def _pairs(schedule):
    return (ctypes.c_int32 * max(2 * len(schedule), 1))(*[int(x) for t in schedule for x in t])


def jet_batch_refine(batch: Batch, schedule, limit, states) -> list:
    """Refine every instance (states[i]: a JetState of batch.ctxs[i]) with one graph launch."""
    part, phi, bw = _state_arrays(states)
    res = (JetRefineResult * len(states))()
    _batch_check(load_library().jet_batch_refine(batch.handle, _pairs(schedule), len(schedule), int(limit), part, phi,
                                                  bw, res), batch)
    return [r.as_dict() for r in res]


def jet_batch_set_split(batch: Batch, split: int):
    _batch_check(load_library().jet_batch_set_split(batch.handle, int(split)), batch)


def jet_batch_get_split(batch: Batch) -> int:
    return int(load_library().jet_batch_get_split(batch.handle))


def jet_batch_tune(batch: Batch, schedule, limit, states, splits) -> tuple:
    """Time the batch under each split; keep the fastest.  Returns (chosen split, {split: ms})."""
    part, phi, bw = _state_arrays(states)
    sp = (ctypes.c_int32 * len(splits))(*[int(x) for x in splits])
    ms = (ctypes.c_float * len(splits))()
    _batch_check(load_library().jet_batch_tune(batch.handle, _pairs(schedule), len(schedule), int(limit), part, phi,
                                               bw, sp, len(splits), ms), batch)
    return jet_batch_get_split(batch), {int(s): float(t) for s, t in zip(splits, ms)}


# team shapes (blocks per team, threads per block) the persistent form's autotuner tries; multi-block shapes are
# tried with no split and with splits at quantiles of the batch's instance sizes
TEAM_SHAPES = ((1, 256), (1, 512), (1, 1024), (2, 1024), (4, 1024), (8, 1024))
TEAM_SPLIT_QUANTILES = (0.25, 0.5, 0.75)


def jet_batch_set_team(batch: Batch, ctas: int, threads: int = 1024, split_pins: int = 0):
    """Persistent form with teams of `ctas` blocks of `threads` threads; with ctas > 1, instances of fewer than
    split_pins pins run on single blocks (ctas = 0: the branch-graph form)."""
    _batch_check(load_library().jet_batch_set_team(batch.handle, int(ctas), int(threads), int(split_pins)), batch)


def jet_batch_get_team(batch: Batch) -> tuple:
    c, t, sp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _batch_check(load_library().jet_batch_get_team(batch.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(sp)),
                 batch)
    return c.value, t.value, sp.value


def team_candidates(batch: Batch, shapes=TEAM_SHAPES, quantiles=TEAM_SPLIT_QUANTILES) -> list:
    """(blocks, threads, split_pins) triples: every shape without a split, and the multi-block shapes of the
    largest block size with splits at the given quantiles of the instances' pin counts."""
    pins = sorted(int(c.hg.P) for c in batch.ctxs)
    out = [(c, t, 0) for c, t in shapes]
    big = max((s for s in shapes if s[0] > 1), default=None)
    if big and pins:
        for q in quantiles:
            sp = pins[min(len(pins) - 1, int(q * len(pins)))]
            if sp > 0 and (big[0], big[1], sp) not in out:
                out.append((big[0], big[1], sp))
    return out


def jet_batch_autotune(batch: Batch, schedule, limit, states, shapes=None, sample=24, trial_iterations=8):
    """Choose the persistent form's team shape from short trials on a sample; returns
    ((blocks, threads, split_pins), {shape: (ms, rate)})."""
    shapes = [tuple(s) if len(s) == 3 else (s[0], s[1], 0) for s in (shapes or team_candidates(batch))]
    part, phi, bw = _state_arrays(states)
    sh = (ctypes.c_int32 * (3 * len(shapes)))(*[int(x) for p in shapes for x in p])
    ms = (ctypes.c_float * len(shapes))()
    rate = (ctypes.c_double * len(shapes))()
    _batch_check(load_library().jet_batch_autotune(batch.handle, _pairs(schedule), len(schedule), int(limit), part, phi,
                                                   bw, sh, len(shapes), int(sample), int(trial_iterations), ms, rate),
                 batch)
    return jet_batch_get_team(batch), {p: (float(m), float(r)) for p, m, r in zip(shapes, ms, rate)}


def jet_job_footprint(n, m, P, k) -> int:
    return int(load_library().jet_job_footprint(int(n), int(m), int(P), int(k)))


class Server:
    """Owning handle of a jet_server.  Keeps every submitted job's host arrays alive until it is reported."""

    def __init__(self, handle):
        self.handle = handle
        self.keep = {}

    def close(self):
        if self.handle:
            load_library().jet_server_destroy(self.handle)
            self.handle = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _server_check(rc, server):
    if rc != JET_OK:
        raise JetError(rc, load_library().jet_server_last_error(server.handle if server else None).decode())


def jet_server_create(hbm_budget: int, max_active: int) -> Server:
    out = _P()
    _server_check(load_library().jet_server_create(ctypes.byref(out), int(hbm_budget), int(max_active)), None)
    return Server(out)


def jet_server_destroy(server: Server):
    server.close()


def jet_server_submit(server: Server, hg, p: JetParams, schedule, limit, part: np.ndarray) -> int:
    """Submit a job on host arrays (hg: synth.Hypergraph; part: int32[n], refined in place)."""
    if part.dtype != np.int32 or not part.flags["C_CONTIGUOUS"] or part.shape[0] != hg.n:
        raise ValueError("part must be a contiguous int32 array of n entries")
    arrs = [np.ascontiguousarray(a) for a in (hg.eptr, hg.pins, hg.vptr, hg.inc, hg.vwgt, hg.ewgt)]
    hh = JetHypergraph(hg.n, hg.m, hg.P, *[a.ctypes.data for a in arrs])
    pairs = (ctypes.c_int32 * max(2 * len(schedule), 1))(*[int(x) for t in schedule for x in t])
    jid = ctypes.c_int64()
    _server_check(load_library().jet_server_submit(server.handle, ctypes.byref(hh), ctypes.byref(p), pairs,
                                                   len(schedule), int(limit), part.ctypes.data, ctypes.byref(jid)),
                  server)
    server.keep[jid.value] = (arrs, part, hh, pairs)
    return jid.value


def jet_server_wait(server: Server, max_done: int = 64, timeout_ms: int = -1) -> list:
    """Finished jobs as dicts (id, status, latency_ms, queue_ms, service_ms, device_start_ms, device_end_ms,
    message, result)."""
    buf = (JetJobDone * max_done)()
    nd = ctypes.c_int32()
    _server_check(load_library().jet_server_wait(server.handle, buf, max_done, ctypes.byref(nd), int(timeout_ms)),
                  server)
    out = []
    for d in buf[: nd.value]:
        server.keep.pop(d.id, None)
        out.append({"id": d.id, "status": d.status, "latency_ms": d.latency_ms, "queue_ms": d.queue_ms,
                    "service_ms": d.latency_ms - d.queue_ms, "device_start_ms": d.device_start_ms,
                    "device_end_ms": d.device_end_ms, "message": d.message.decode(errors="replace"),
                    "result": d.result.as_dict()})
    return out


def jet_server_load(server: Server) -> dict:
    pend, run, res = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _server_check(load_library().jet_server_load(server.handle, ctypes.byref(pend), ctypes.byref(run),
                                                 ctypes.byref(res)), server)
    return {"pending": pend.value, "running": run.value, "reserved_bytes": res.value}


# ---------------------------------------------------------------- state helper

class JetState:
    """Device state of one refinement: Pi, phi, c(V_i), locks and a stats slot."""

    def __init__(self, ctx: Ctx, part, with_phi: bool = True):
        import torch
        dev = ctx.hg.eptr.device
        self.ctx = ctx
        self.part = torch.as_tensor(part, dtype=torch.int32).to(dev).contiguous()
        # without phi (graph path only): no m*k table at all
        self.phi = torch.empty(max(ctx.hg.m * ctx.k, 1), dtype=torch.int32, device=dev) if with_phi else None
        self.block_w = torch.empty(ctx.k, dtype=torch.int64, device=dev)
        self.locked = torch.zeros(max(ctx.hg.n, 1), dtype=torch.uint8, device=dev)
        self.stats = torch.zeros(8, dtype=torch.int64, device=dev)
        jet_build_pincounts(ctx, self.part, self.phi, self.block_w)

    def round(self, tau):
        jet_refine_round(self.ctx, tau, self.part, self.phi, self.block_w, self.locked, self.stats)

    def stats_dict(self):
        return dict(zip(STATS_FIELDS[:7], [int(x) for x in self.stats.cpu().tolist()[:7]]))
