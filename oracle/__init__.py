"""CPU oracle for deterministic Jet refinement -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it, and the two share no code.

``jet_oracle.c`` is plain single-threaded integer C that follows the paper
(arXiv 2504.12013) step by step: Section 2 (definitions), Algorithm 1 (Jet
loop), Algorithm 2 (hypergraph afterburner), Section 4.3 (deterministic
rebalancing) and the schedule of Section 7.2.  Its readings of points the
paper leaves open are listed in the C file's header (R1..R25).  Section 5's
matching schedule and Section 6's coarsening (Algorithm 4, contraction) are
here too.

Parity pins: every oracle function is checked by ``tests/test_oracle_pins.py``
against brute force, closed forms, invariants and hand-worked fixtures.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jet_oracle.c")
_lock = threading.Lock()
_libs: dict = {}

I32P = ctypes.POINTER(ctypes.c_int32)
I64P = ctypes.POINTER(ctypes.c_int64)
U8P = ctypes.POINTER(ctypes.c_uint8)


def build(source=None, force: bool = False) -> str:
    """Compile the oracle (or a variant source file, used by the mutation tests)."""
    src = source or _SRC
    if source is None:
        out = os.path.join(_HERE, "_build", "libjet_oracle.so")
    else:
        out = os.path.join(os.path.dirname(os.path.abspath(source)), "libjet_oracle_variant.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


class OHG(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("P", ctypes.c_int64),
        ("eptr", I64P), ("pins", I32P), ("vptr", I64P), ("inc", I32P), ("vwgt", I32P), ("ewgt", I32P),
    ]


class OParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("eps_num", ctypes.c_int32), ("eps_den", ctypes.c_int32),
                ("d_num", ctypes.c_int32), ("d_den", ctypes.c_int32), ("max_rebalance_rounds", ctypes.c_int32)]


class OStats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("approved", ctypes.c_int64),
                ("rebalance_rounds", ctypes.c_int64), ("rebalance_moves", ctypes.c_int64),
                ("objective", ctypes.c_int64), ("max_block_weight", ctypes.c_int64),
                ("imbalanced", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def load(source=None):
    key = source
    with _lock:
        if key not in _libs:
            lib = ctypes.CDLL(build(source))
            H, Pp, S = ctypes.POINTER(OHG), ctypes.POINTER(OParams), ctypes.POINTER(OStats)
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.ojet_total_weight.argtypes = [H]; lib.ojet_total_weight.restype = i64
            lib.ojet_avg_block.argtypes = [H, i32]; lib.ojet_avg_block.restype = i64
            lib.ojet_lmax.argtypes = [H, Pp]; lib.ojet_lmax.restype = i64
            lib.ojet_pincounts.argtypes = [H, i32, I32P, I32P, I64P]; lib.ojet_pincounts.restype = None
            lib.ojet_connectivity.argtypes = [H, i32, I32P]; lib.ojet_connectivity.restype = i64
            lib.ojet_gain.argtypes = [H, i32, I32P, I32P, i32, i32]; lib.ojet_gain.restype = i64
            lib.ojet_affinity.argtypes = [H, i32, I32P, I32P, i32]; lib.ojet_affinity.restype = i64
            lib.ojet_candidates.argtypes = [H, i32, I32P, I32P, U8P, i32, i32, I32P, I64P, U8P]
            lib.ojet_candidates.restype = i64
            lib.ojet_afterburner.argtypes = [H, i32, I32P, I32P, I32P, I64P, U8P, I64P, U8P]
            lib.ojet_afterburner.restype = i64
            lib.ojet_apply.argtypes = [H, i32, I32P, I32P, I64P, U8P, I32P]; lib.ojet_apply.restype = None
            lib.ojet_rebalance_round.argtypes = [H, Pp, I32P, I32P, I64P, U8P, I32P]
            lib.ojet_rebalance_round.restype = i64
            lib.ojet_rebalance.argtypes = [H, Pp, I32P, I32P, I64P, I64P]; lib.ojet_rebalance.restype = i64
            lib.ojet_refine_round.argtypes = [H, Pp, i32, i32, I32P, I32P, I64P, U8P, S]
            lib.ojet_refine_round.restype = None
            lib.ojet_refine.argtypes = [H, Pp, I32P, i32, i32, I32P, I64P, I64P]; lib.ojet_refine.restype = i64
            lib.ojet_quotient.argtypes = [H, i32, I32P, U8P]; lib.ojet_quotient.restype = None
            lib.ojet_schedule.argtypes = [i32, U8P, I32P, I32P, I32P]; lib.ojet_schedule.restype = i64
            lib.ojet_subrounds.argtypes = [i32, i32, i32, I32P]; lib.ojet_subrounds.restype = i64
            lib.ojet_cluster.argtypes = [H, i64, i32, i32, i32, I32P, I32P]; lib.ojet_cluster.restype = i64
            lib.ojet_contract.argtypes = [H, I32P, I32P, I64P, I32P, I64P, I32P, I32P, I32P, I32P, I32P, I64P]
            lib.ojet_contract.restype = i64
            _libs[key] = lib
    return _libs[key]


def _p(a, t):
    return a.ctypes.data_as(t)


@dataclass
class Params:
    k: int
    eps: tuple = (3, 100)
    d: tuple = (1, 10)
    max_rebalance_rounds: int = 32

    def c(self) -> OParams:
        return OParams(self.k, self.eps[0], self.eps[1], self.d[0], self.d[1], self.max_rebalance_rounds)


TAU_SCHEDULE = ((3, 4), (3, 8), (0, 1))  # three temperatures 0.75 -> 0, equidistant (Section 7.2)
ITERATION_LIMIT = 8                      # iterations without improvement (Section 7.2)
SINGLE_SUBROUNDS = 100                   # one-vertex sub-rounds at the start of clustering (Section 6)
SUBROUND_CAP_DIV = 100                   # sub-rounds grow to 1% of the vertices (Section 6)
RATING_MAX_EDGE = 1000                   # larger edges add nothing to the rating (reading R19)


class Oracle:
    """Bound oracle for one hypergraph.  Arrays are numpy; state is updated in place."""

    def __init__(self, hg, source=None):
        self.lib = load(source)
        self.source = source
        self.hg = hg
        # keep contiguous copies alive
        self._arrs = [np.ascontiguousarray(a) for a in (hg.eptr, hg.pins, hg.vptr, hg.inc, hg.vwgt, hg.ewgt)]
        e, p, vp, inc, vw, ew = self._arrs
        self.h = OHG(hg.n, hg.m, int(e[-1]) if e.size else 0, _p(e, I64P), _p(p, I32P), _p(vp, I64P),
                     _p(inc, I32P), _p(vw, I32P), _p(ew, I32P))

    # Section 2
    def total_weight(self):
        return self.lib.ojet_total_weight(ctypes.byref(self.h))

    def avg_block(self, k):
        return self.lib.ojet_avg_block(ctypes.byref(self.h), k)

    def lmax(self, params: Params):
        return self.lib.ojet_lmax(ctypes.byref(self.h), ctypes.byref(params.c()))

    def pincounts(self, k, part):
        part = np.ascontiguousarray(part, dtype=np.int32)
        phi = np.zeros(self.hg.m * k, dtype=np.int32)
        bw = np.zeros(k, dtype=np.int64)
        self.lib.ojet_pincounts(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), _p(bw, I64P))
        return phi.reshape(self.hg.m, k), bw

    def connectivity(self, k, phi):
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        return self.lib.ojet_connectivity(ctypes.byref(self.h), k, _p(phi, I32P))

    def objective(self, k, part):
        return self.connectivity(k, self.pincounts(k, part)[0])

    def gain(self, k, part, phi, v, b):
        part = np.ascontiguousarray(part, dtype=np.int32)
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        return self.lib.ojet_gain(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), v, b)

    def affinity(self, k, part, phi, v):
        part = np.ascontiguousarray(part, dtype=np.int32)
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        return self.lib.ojet_affinity(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), v)

    # Section 4.1
    def candidates(self, k, part, phi, locked, tau):
        n = self.hg.n
        part = np.ascontiguousarray(part, dtype=np.int32)
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        locked = np.ascontiguousarray(locked, dtype=np.uint8)
        target = np.empty(n, np.int32); gain = np.empty(n, np.int64); in_m = np.empty(n, np.uint8)
        cnt = self.lib.ojet_candidates(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), _p(locked, U8P),
                                       tau[0], tau[1], _p(target, I32P), _p(gain, I64P), _p(in_m, U8P))
        return cnt, target, gain, in_m

    # Section 4.2
    def afterburner(self, k, part, phi, target, gain, in_m):
        n = self.hg.n
        part = np.ascontiguousarray(part, dtype=np.int32)
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        target = np.ascontiguousarray(target, dtype=np.int32)
        gain = np.ascontiguousarray(gain, dtype=np.int64)
        in_m = np.ascontiguousarray(in_m, dtype=np.uint8)
        rg = np.empty(n, np.int64); approved = np.empty(n, np.uint8)
        cnt = self.lib.ojet_afterburner(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), _p(target, I32P),
                                        _p(gain, I64P), _p(in_m, U8P), _p(rg, I64P), _p(approved, U8P))
        return cnt, rg, approved

    def apply(self, k, part, phi, bw, move, target):
        """In place on part (int32[n]), phi (int32[m,k]), bw (int64[k])."""
        move = np.ascontiguousarray(move, dtype=np.uint8)
        target = np.ascontiguousarray(target, dtype=np.int32)
        self.lib.ojet_apply(ctypes.byref(self.h), k, _p(part, I32P), _p(phi, I32P), _p(bw, I64P), _p(move, U8P),
                            _p(target, I32P))

    # Section 4.3
    def rebalance_round(self, params: Params, part, phi, bw):
        n = self.hg.n
        flag = np.empty(n, np.uint8); tgt = np.empty(n, np.int32)
        moved = self.lib.ojet_rebalance_round(ctypes.byref(self.h), ctypes.byref(params.c()), _p(part, I32P),
                                              _p(phi, I32P), _p(bw, I64P), _p(flag, U8P), _p(tgt, I32P))
        return moved, flag, tgt

    def rebalance(self, params: Params, part, phi, bw):
        moves = ctypes.c_int64(0)
        rounds = self.lib.ojet_rebalance(ctypes.byref(self.h), ctypes.byref(params.c()), _p(part, I32P),
                                         _p(phi, I32P), _p(bw, I64P), ctypes.byref(moves))
        return rounds, moves.value

    # Section 5 (matching schedule)
    def quotient(self, k, phi):
        """Quotient graph adjacency (k x k uint8) of the partition whose pin counts are phi."""
        phi = np.ascontiguousarray(phi, dtype=np.int32)
        q = np.zeros((k, k), np.uint8)
        self.lib.ojet_quotient(ctypes.byref(self.h), k, _p(phi, I32P), _p(q, U8P))
        return q

    def schedule(self, qadj):
        """Rounds of maximal matchings covering the quotient edges: (pairs int32[p, 2], round int32[p], rounds)."""
        return schedule(qadj, self.lib)

    # Section 6, Algorithm 4 (coarsening)
    def cluster(self, cmax, order, rmax=RATING_MAX_EDGE, n_single=SINGLE_SUBROUNDS, cap_div=SUBROUND_CAP_DIV):
        """Cluster labels (int32[n]) of one level of synchronous clustering; order is the vertex split."""
        order = np.ascontiguousarray(order, dtype=np.int32)
        label = np.zeros(self.hg.n, np.int32)
        rc = self.lib.ojet_cluster(ctypes.byref(self.h), int(cmax), int(rmax), int(n_single), int(cap_div),
                                   _p(order, I32P), _p(label, I32P))
        if rc != 0:
            raise OverflowError("rating sum overflow")
        return label

    def contract(self, label):
        """(coarse Hypergraph, map int32[n]) of the label classes."""
        hg = self.hg
        label = np.ascontiguousarray(label, dtype=np.int32)
        P = int(hg.eptr[-1]) if hg.m else 0
        mp = np.zeros(hg.n, np.int32)
        ce, cp = np.zeros(hg.m + 1, np.int64), np.zeros(max(P, 1), np.int32)
        cv, ci = np.zeros(hg.n + 1, np.int64), np.zeros(max(P, 1), np.int32)
        cvw, cew = np.zeros(max(hg.n, 1), np.int32), np.zeros(max(hg.m, 1), np.int32)
        nc, mc, pc = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
        rc = self.lib.ojet_contract(ctypes.byref(self.h), _p(label, I32P), _p(mp, I32P), _p(ce, I64P),
                                    _p(cp, I32P), _p(cv, I64P), _p(ci, I32P), _p(cvw, I32P), _p(cew, I32P),
                                    ctypes.byref(nc), ctypes.byref(mc), ctypes.byref(pc))
        if rc != 0:
            raise OverflowError("coarse weight overflow")
        nc, mc, pc = nc.value, mc.value, pc.value
        from paper_2504_12013_gb300.synth import Hypergraph
        coarse = Hypergraph(n=nc, m=mc, eptr=ce[: mc + 1].copy(), pins=cp[:pc].copy(), vptr=cv[: nc + 1].copy(),
                            inc=ci[:pc].copy(), vwgt=cvw[:nc].copy(), ewgt=cew[:mc].copy())
        return coarse, mp

    def subrounds(self, n, n_single=SINGLE_SUBROUNDS, cap_div=SUBROUND_CAP_DIV):
        return subrounds(n, n_single, cap_div, self.lib)

    def coarsen(self, cmax, order, **kw):
        """One coarsening level: (coarse Hypergraph, map, labels)."""
        label = self.cluster(cmax, order, **kw)
        coarse, mp = self.contract(label)
        return coarse, mp, label

    # Algorithm 1
    def refine_round(self, params: Params, tau, part, phi, bw, locked):
        st = OStats()
        self.lib.ojet_refine_round(ctypes.byref(self.h), ctypes.byref(params.c()), tau[0], tau[1], _p(part, I32P),
                                   _p(phi, I32P), _p(bw, I64P), _p(locked, U8P), ctypes.byref(st))
        return st.as_dict()

    def refine(self, params: Params, part, schedule=TAU_SCHEDULE, limit=ITERATION_LIMIT):
        pairs = np.array([x for t in schedule for x in t], dtype=np.int32)
        obj = ctypes.c_int64(0)
        phase = np.zeros(len(schedule), np.int64)
        iters = self.lib.ojet_refine(ctypes.byref(self.h), ctypes.byref(params.c()), _p(pairs, I32P),
                                     len(schedule), limit, _p(part, I32P), ctypes.byref(obj), _p(phase, I64P))
        return iters, obj.value, phase


class State:
    """Mutable Jet state (Pi, phi, c(V_i), locks) for stepping the oracle round by round."""

    def __init__(self, orc: Oracle, k: int, part):
        self.part = np.array(part, dtype=np.int32, copy=True)
        phi, bw = orc.pincounts(k, self.part)
        self.phi = np.ascontiguousarray(phi)
        self.bw = bw
        self.locked = np.zeros(orc.hg.n, dtype=np.uint8)


def subrounds(n, n_single=SINGLE_SUBROUNDS, cap_div=SUBROUND_CAP_DIV, lib=None):
    """Sub-round bounds of the prefix-doubling schedule (Section 6): int32[r + 1], starts and n at the end."""
    lib = lib or load()
    r = lib.ojet_subrounds(int(n), int(n_single), int(cap_div), None)
    b = np.zeros(r + 1, np.int32)
    lib.ojet_subrounds(int(n), int(n_single), int(cap_div), _p(b, I32P))
    return b


def schedule(qadj, lib=None):
    """The matching schedule (Section 5) of a quotient graph given as a k x k 0/1 matrix."""
    lib = lib or load()
    q = np.ascontiguousarray(qadj, dtype=np.uint8)
    k = q.shape[0]
    cap = max(k * (k - 1) // 2, 1)
    pairs = np.zeros(2 * cap, np.int32)
    rnd = np.zeros(cap, np.int32)
    nr = ctypes.c_int32(0)
    npairs = lib.ojet_schedule(k, _p(q, U8P), _p(pairs, I32P), _p(rnd, I32P), ctypes.byref(nr))
    return pairs[: 2 * npairs].reshape(-1, 2), rnd[:npairs], nr.value
