"""Seeded synthetic hypergraph instances (inputs only).

The generators live in ``gen.c`` (splitmix64, integer samplers) and are
compiled on first use with the host C compiler into ``_build/``.  This module
holds no arithmetic of the refinement method: it makes CSR hypergraphs,
weights and initial partitions, and is the only code shared by the CPU oracle
tests, the CUDA parity tests and the benchmark.

Shapes follow the workloads of the paper's experiments (Section 7.1): random
hypergraphs, VLSI-netlist-like power-law hypergraphs with locality, and
sparse-matrix row-net hypergraphs with hub rows.  The paper's benchmark sets
are not available here; these seeded generators stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT = os.path.join(_HERE, "_build", "libjet_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared object (host compiler, portable flags)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _SynthHG(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("P", ctypes.c_int64),
        ("eptr", ctypes.POINTER(ctypes.c_int64)), ("pins", ctypes.POINTER(ctypes.c_int32)),
        ("vptr", ctypes.POINTER(ctypes.c_int64)), ("inc", ctypes.POINTER(ctypes.c_int32)),
        ("vwgt", ctypes.POINTER(ctypes.c_int32)), ("ewgt", ctypes.POINTER(ctypes.c_int32)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, i64 = ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
            P = ctypes.POINTER
            lib.synth_uniform.argtypes = [u64, i32, i32, i32, ctypes.c_uint32, ctypes.c_uint32, i32, i32, i32,
                                          P(_SynthHG)]
            lib.synth_vlsi.argtypes = [u64, i32, i32, i32, i32, i32, i32, ctypes.c_uint32, ctypes.c_uint32, i32,
                                       P(_SynthHG)]
            lib.synth_rownet.argtypes = [u64, i32, i32, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                         P(_SynthHG)]
            lib.synth_free.argtypes = [P(_SynthHG)]
            lib.synth_part_hash.argtypes = [u64, i32, i32, P(i32)]
            lib.synth_part_perm.argtypes = [u64, i32, i32, P(i32)]
            lib.synth_part_random.argtypes = [u64, i32, i32, P(i32)]
            lib.synth_fill_u64.argtypes = [u64, i64, P(u64)]
            lib.synth_fill_unit.argtypes = [u64, i64, P(ctypes.c_double)]
            for f in ("synth_uniform", "synth_vlsi", "synth_rownet", "synth_part_perm"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Hypergraph:
    """Host CSR hypergraph H = (V, E, c, omega) (Section 2).

    ``eptr``/``pins``: pins of edge e are ``pins[eptr[e]:eptr[e+1]]``.
    ``vptr``/``inc``: incident edges I(v) are ``inc[vptr[v]:vptr[v+1]]``.
    """
    n: int
    m: int
    eptr: np.ndarray  # int64[m+1]
    pins: np.ndarray  # int32[P]
    vptr: np.ndarray  # int64[n+1]
    inc: np.ndarray   # int32[P]
    vwgt: np.ndarray  # int32[n]
    ewgt: np.ndarray  # int32[m]

    @property
    def P(self) -> int:
        return int(self.eptr[-1])

    def edge(self, e: int) -> np.ndarray:
        return self.pins[self.eptr[e]:self.eptr[e + 1]]

    def incident(self, v: int) -> np.ndarray:
        return self.inc[self.vptr[v]:self.vptr[v + 1]]

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.eptr, self.pins, self.vptr, self.inc, self.vwgt, self.ewgt))


def _take(h: _SynthHG) -> Hypergraph:
    lib = _load()
    n, m, P = h.n, h.m, h.P
    def arr(ptr, count, dtype):
        if count == 0:
            return np.zeros(0, dtype=dtype)
        return np.ctypeslib.as_array(ptr, shape=(count,)).copy()
    out = Hypergraph(n=n, m=m, eptr=arr(h.eptr, m + 1, np.int64), pins=arr(h.pins, P, np.int32),
                     vptr=arr(h.vptr, n + 1, np.int64), inc=arr(h.inc, P, np.int32),
                     vwgt=arr(h.vwgt, n, np.int32), ewgt=arr(h.ewgt, m, np.int32))
    lib.synth_free(ctypes.byref(h))
    return out


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what}: generator returned {rc} (invalid arguments or out of memory)")


def uniform(seed: int, n: int, m: int, *, base: int = 2, geo=(1, 2), size_cap: int = 64,
            c_max: int = 1, w_max: int = 1) -> Hypergraph:
    """|e| = base + Geometric(p) failures (capped); pins uniform without repeats."""
    h = _SynthHG()
    _check(_load().synth_uniform(seed, n, m, base, geo[0], geo[1], size_cap, c_max, w_max, ctypes.byref(h)),
           "uniform")
    return _take(h)


def vlsi(seed: int, n: int, m: int, *, smin: int = 2, smax: int = 5000, alpha_x2: int = 5,
         window: int = 20000, loc=(4, 5), c_max: int = 4) -> Hypergraph:
    """Power-law sizes (exponent alpha_x2/2), 80 % of pins within +-window of a centre."""
    h = _SynthHG()
    _check(_load().synth_vlsi(seed, n, m, smin, smax, alpha_x2, window, loc[0], loc[1], c_max, ctypes.byref(h)),
           "vlsi")
    return _take(h)


def rownet(seed: int, n: int, m: int, *, n_hubs: int = 200, hub_min: int = 50000, hub_max: int = 200000,
           mu: float = 2.0, sigma: float = 1.0) -> Hypergraph:
    """Row-net of a sparse matrix: log-normal row lengths plus hub rows."""
    h = _SynthHG()
    _check(_load().synth_rownet(seed, n, m, n_hubs, hub_min, hub_max, mu, sigma, ctypes.byref(h)), "rownet")
    return _take(h)


def part_hash(seed: int, n: int, k: int) -> np.ndarray:
    """Block of vertex i = (i * 2654435761 + seed) mod k (uint64 arithmetic)."""
    out = np.empty(n, dtype=np.int32)
    _load().synth_part_hash(seed, n, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def part_perm(seed: int, n: int, k: int) -> np.ndarray:
    """Seeded Fisher-Yates permutation pi; block of pi(i) = i mod k (balanced)."""
    out = np.empty(n, dtype=np.int32)
    _check(_load().synth_part_perm(seed, n, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "part_perm")
    return out


def part_random(seed: int, n: int, k: int) -> np.ndarray:
    """Uniform random blocks (generally imbalanced)."""
    out = np.empty(n, dtype=np.int32)
    _load().synth_part_random(seed, n, k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def stream_u64(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().synth_fill_u64(seed, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def stream_unit(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().synth_fill_unit(seed, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def from_edges(n: int, edges, vwgt=None, ewgt=None) -> Hypergraph:
    """Build both CSR views from a list of pin lists (hand-made test cases).

    Pins of each edge are kept in the given order; I(v) lists edges in
    increasing id order.
    """
    m = len(edges)
    sizes = np.array([len(e) for e in edges], dtype=np.int64)
    eptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=eptr[1:])
    pins = np.array([v for e in edges for v in e], dtype=np.int32) if m else np.zeros(0, np.int32)
    if pins.size and (pins.min() < 0 or pins.max() >= n):
        raise ValueError("pin out of range")
    for e in edges:
        if len(set(e)) != len(e):
            raise ValueError("repeated pin in an edge")
    edge_of = np.repeat(np.arange(m, dtype=np.int32), sizes)
    order = np.lexsort((edge_of, pins))  # by vertex, then edge id
    inc = edge_of[order].astype(np.int32)
    deg = np.bincount(pins, minlength=n) if pins.size else np.zeros(n, np.int64)
    vptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=vptr[1:])
    vw = np.ones(n, np.int32) if vwgt is None else np.asarray(vwgt, dtype=np.int32)
    ew = np.ones(m, np.int32) if ewgt is None else np.asarray(ewgt, dtype=np.int32)
    return Hypergraph(n=n, m=m, eptr=eptr, pins=pins, vptr=vptr, inc=inc, vwgt=vw, ewgt=ew)


def permuted(h: Hypergraph, seed: int, *, pins_within_edges=True, edge_order=True) -> tuple[Hypergraph, np.ndarray]:
    """Same hypergraph with pin order inside edges and/or edge ids permuted.

    Returns the new hypergraph and ``eperm`` with new edge id ``i`` = old edge
    ``eperm[i]``.  Vertex ids are unchanged.
    """
    u = stream_u64(seed, h.m + h.P + 1)
    eperm = np.argsort(u[:h.m], kind="stable") if edge_order else np.arange(h.m)
    edges = []
    pos = h.m
    for old in eperm:
        pe = list(h.edge(int(old)))
        if pins_within_edges and len(pe) > 1:
            key = u[pos:pos + len(pe)]
            pe = [pe[i] for i in np.argsort(key, kind="stable")]
        pos += len(pe)
        edges.append(pe)
    return from_edges(h.n, edges, h.vwgt, h.ewgt[eperm]), eperm


# Workload shapes of the benchmark configurations.
def config_random_10k(seed: int = 1):
    """n=10,000, m=12,000, |e| = 2 + Geometric(1/2) capped at 64, unit weights, k=8, hash partition."""
    h = uniform(seed, 10_000, 12_000, base=2, geo=(1, 2), size_cap=64)
    return h, 8, part_hash(seed, h.n, 8)


def config_vlsi_2m(seed: int = 1):
    """n=2,000,000, m=2,200,000, power-law 2.5 sizes on [2,5000], 80 % pins in +-20,000, c in 1..4, k=64."""
    h = vlsi(seed, 2_000_000, 2_200_000)
    return h, 64, part_perm(seed, h.n, 64)


def config_rownet_4m(seed: int = 1):
    """4,000,000 columns x 4,000,000 rows, log-normal(2,1) lengths + 200 hubs of 50k-200k pins, k=128."""
    h = rownet(seed, 4_000_000, 4_000_000)
    return h, 128, part_perm(seed, h.n, 128)


def config_batched(seed: int = 1, count: int = 256, n_lo: int = 1_000, n_hi: int = 200_000):
    """Independent instances of the batched workload: n log-uniform in [n_lo, n_hi], m = round(1.1 n),
    |e| = 2 + Geometric(2/5) failures capped at 256, unit weights, k uniform from {2, 8, 32},
    hash partition with the instance's seed.  Returns a list of (hypergraph, k, partition)."""
    import math
    u = stream_u64(seed * 1_000_003 + 17, 2 * count)
    out = []
    for i in range(count):
        frac = float(u[2 * i] >> np.uint64(11)) / float(1 << 53)
        n = int(round(math.exp(math.log(n_lo) + frac * (math.log(n_hi) - math.log(n_lo)))))
        k = (2, 8, 32)[int(u[2 * i + 1] % np.uint64(3))]
        s = seed * 100_003 + i
        h = uniform(s, n, int(round(1.1 * n)), base=2, geo=(2, 5), size_cap=256)
        out.append((h, k, part_hash(s, h.n, k)))
    return out


def served_instance(seed: int, P_lo: int = 10_000, P_hi: int = 5_000_000):
    """One request of the served workload: pins P log-uniform in [P_lo, P_hi], n = round(P / 3.85),
    m = round(1.1 n), |e| = 2 + Geometric(2/5) failures capped at 256, c in 1..8, unit edge weights."""
    import math
    u = stream_u64(seed * 7_919 + 3, 1)
    frac = float(u[0] >> np.uint64(11)) / float(1 << 53)
    P = math.exp(math.log(P_lo) + frac * (math.log(P_hi) - math.log(P_lo)))
    n = max(int(round(P / 3.85)), 2)
    return uniform(seed, n, int(round(1.1 * n)), base=2, geo=(2, 5), size_cap=256, c_max=8)


def served_jobs(seed: int, count: int, rate_per_s: float = 200.0, pool: int = 32):
    """The request stream of the served workload: Poisson arrivals (seeded exponential gaps) at rate_per_s;
    job j refines instance j % pool of a pool of `pool` served_instance hypergraphs, with k from
    {2, 4, ..., 256} and a balanced random partition (seeded permutation).  Returns (pool instances,
    [(arrival_s, pool index, k, partition)])."""
    import math
    insts = [served_instance(seed * 1_000 + i) for i in range(pool)]
    u = stream_u64(seed * 104_729 + 11, 2 * count)
    t, jobs = 0.0, []
    for j in range(count):
        frac = (float(u[2 * j] >> np.uint64(11)) + 0.5) / float(1 << 53)
        t += -math.log(frac) / rate_per_s
        k = 2 << int(u[2 * j + 1] % np.uint64(8))
        h = insts[j % pool]
        jobs.append((t, j % pool, k, part_perm(seed * 31 + j, h.n, k)))
    return insts, jobs


def contract_pairs(h: Hypergraph) -> tuple[Hypergraph, np.ndarray]:
    """One level of a fixed test hierarchy (an input builder, not the paper's coarsening): vertex v of h
    becomes vertex v // 2; every edge keeps its distinct mapped pins (in increasing order) and is dropped
    when fewer than two remain; coarse vertex weights are the sums, edge weights are kept.  Returns
    (coarse hypergraph, map int32[h.n] from h's vertices to the coarse ones)."""
    nc = (h.n + 1) // 2
    mp = (np.arange(h.n, dtype=np.int64) // 2).astype(np.int32)
    sizes = np.diff(h.eptr)
    eid = np.repeat(np.arange(h.m, dtype=np.int64), sizes)
    cp = mp[h.pins].astype(np.int64)
    order = np.lexsort((cp, eid))
    eid, cp = eid[order], cp[order]
    keep = np.ones(len(cp), bool)
    if len(cp):
        keep[1:] = (eid[1:] != eid[:-1]) | (cp[1:] != cp[:-1])
    eid, cp = eid[keep], cp[keep]
    cnt = np.bincount(eid, minlength=h.m)
    big = cnt >= 2
    sel = big[eid]
    eid, cp = eid[sel], cp[sel]
    newid = np.cumsum(big) - 1
    eid = newid[eid]
    mc = int(big.sum())
    eptr = np.zeros(mc + 1, np.int64)
    np.cumsum(np.bincount(eid, minlength=mc), out=eptr[1:])
    pins = cp.astype(np.int32)
    o2 = np.lexsort((eid, cp))  # incidences by vertex, then edge id
    inc = eid[o2].astype(np.int32)
    vptr = np.zeros(nc + 1, np.int64)
    np.cumsum(np.bincount(cp, minlength=nc), out=vptr[1:])
    vw = np.zeros(nc, np.int64)
    np.add.at(vw, mp, h.vwgt.astype(np.int64))
    return Hypergraph(n=nc, m=mc, eptr=eptr, pins=pins, vptr=vptr, inc=inc, vwgt=vw.astype(np.int32),
                      ewgt=h.ewgt[big].astype(np.int32)), mp


def hierarchy(h: Hypergraph, levels: int) -> tuple[list, list]:
    """levels hypergraphs from the coarsest to h, and the maps between consecutive ones (contract_pairs)."""
    hs, maps = [h], []
    for _ in range(levels - 1):
        c, mp = contract_pairs(hs[0])
        hs.insert(0, c)
        maps.insert(0, mp)
    return hs, maps


def vertex_order(seed: int, n: int) -> np.ndarray:
    """A seeded permutation of [0, n) (the random vertex split of a clustering level)."""
    return stream_u64(seed, n).argsort(kind="stable").astype(np.int32)


def from_pairs(n: int, u: np.ndarray, v: np.ndarray, vwgt=None, ewgt=None) -> Hypergraph:
    """A graph as a hypergraph of two-pin edges (pins of each edge ascending), both CSR views."""
    m = len(u)
    lo = np.minimum(u, v).astype(np.int32)
    hi = np.maximum(u, v).astype(np.int32)
    pins = np.empty(2 * m, np.int32)
    pins[0::2], pins[1::2] = lo, hi
    eptr = (2 * np.arange(m + 1, dtype=np.int64))
    eid = np.repeat(np.arange(m, dtype=np.int32), 2)
    order = np.lexsort((eid, pins))
    inc = eid[order]
    vptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(pins, minlength=n), out=vptr[1:])
    vw = np.ones(n, np.int32) if vwgt is None else np.asarray(vwgt, np.int32)
    ew = np.ones(m, np.int32) if ewgt is None else np.asarray(ewgt, np.int32)
    return Hypergraph(n=n, m=m, eptr=eptr, pins=pins, vptr=vptr, inc=inc, vwgt=vw, ewgt=ew)


def graph(seed: int, n: int, m: int, *, local: float = 0.8, window: int = 1000, c_max: int = 1,
          w_max: int = 1) -> Hypergraph:
    """Seeded graph with m edges {u, v}, u != v: u uniform; with probability `local` v is u plus an offset
    uniform in [1, window] (mod n), otherwise uniform over the other vertices.  Parallel edges may occur.
    c uniform in 1..c_max, omega uniform in 1..w_max."""
    r = stream_u64(seed, 4 * m + n)
    u = (r[:m] % np.uint64(n)).astype(np.int64)
    is_local = (r[m:2 * m] % np.uint64(1 << 20)).astype(np.float64) < local * (1 << 20)
    off_local = 1 + (r[2 * m:3 * m] % np.uint64(min(window, n - 1))).astype(np.int64)
    off_far = 1 + (r[2 * m:3 * m] % np.uint64(n - 1)).astype(np.int64)
    v = (u + np.where(is_local, off_local, off_far)) % n
    ew = 1 + (r[3 * m:4 * m] % np.uint64(w_max)).astype(np.int32)
    vw = 1 + (r[4 * m:4 * m + n] % np.uint64(c_max)).astype(np.int32)
    return from_pairs(n, u, v, vwgt=vw, ewgt=ew)


def config_graph_16m(seed: int = 1):
    """n=4,000,000, m=16,000,000 two-pin edges (80 % within +-1,000 ids), unit weights, k=64."""
    h = graph(seed, 4_000_000, 16_000_000)
    return h, 64, part_perm(seed, h.n, 64)
