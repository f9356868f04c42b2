#!/usr/bin/env python
"""Benchmark of deterministic Jet refinement rounds (connectivity metric) on GB300.

A step is one Jet iteration (the body of Algorithm 1: candidates,
afterburner, apply, rebalancing if needed, objective) on the whole
hypergraph; the metric is pins/s = P * steps / time.  The default workload is
the largest one-GPU configuration, the sparse-matrix row-net hypergraph
(n = m = 4,000,000, log-normal(2, 1) row lengths plus 200 hub rows of
50,000-200,000 pins, unit weights, k = 128, eps = 3/100), started from a
seeded balanced partition; the timed steps are the first K iterations at
temperature 3/4.  The VLSI-shaped hypergraph (n = 2,000,000, k = 64) is
measured the same way and reported beside it.

One JSON line on stdout (rank 0).  --impl reference times the CPU oracle
(single-threaded, test infrastructure) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_12013_gb300 import synth  # noqa: E402

WORKLOADS = {
    "vlsi_2m": ("VLSI-shaped hypergraph n=2,000,000 m=2,200,000 power-law(2.5)[2,5000] sizes, 80% pins "
                "within +-20,000, c in 1..4, k=64, eps=3/100", synth.config_vlsi_2m),
    "rownet_4m": ("sparse-matrix row-net n=m=4,000,000, log-normal(2,1) rows + 200 hubs of 50k-200k pins, "
                  "k=128, eps=3/100", synth.config_rownet_4m),
    "random_10k": ("random hypergraph n=10,000 m=12,000 |e|=2+Geometric(1/2)<=64, k=8, eps=3/100",
                   synth.config_random_10k),
    # the VLSI shape at a quarter of the size (phi 141 MB, still larger than L2), for multi-pass ncu captures
    "vlsi_500k": ("VLSI-shaped hypergraph n=500,000 m=550,000 power-law(2.5)[2,5000] sizes, 80% pins within +-5,000, "
                  "c in 1..4, k=64, eps=3/100",
                  lambda seed: (lambda h: (h, 64, synth.part_perm(seed, h.n, 64)))(
                      synth.vlsi(seed, 500_000, 550_000, window=5_000))),
    # the row-net shape at a quarter of the size (phi 512 MB), for multi-pass ncu captures
    "rownet_1m": ("sparse-matrix row-net n=m=1,000,000, log-normal(2,1) rows + 50 hubs of 50k-200k pins, k=128, "
                  "eps=3/100",
                  lambda seed: (lambda h: (h, 128, synth.part_perm(seed, h.n, 128)))(
                      synth.rownet(seed, 1_000_000, 1_000_000, n_hubs=50))),
}
TAU = (3, 4)
SCHEDULE = ((3, 4), (3, 8), (0, 1))
LIMIT = 8


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names[1:], f[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- byte model
def kernel_bytes(hg, k, deg, st_before, round_stats):
    """Compulsory (algorithmic) bytes of the candidate kernels for one round.

    Each array counts once per launch: the streamed CSR arrays by the bytes
    read, and every gathered table by min(gathers x element, table size).
    st_before: locked (bool[n]) before the round.
    """
    n, m, P = hg.n, hg.m, hg.P
    kw = (k + 31) // 32
    unlocked = ~st_before
    Pu = int(deg[unlocked].sum())
    b = 8 * (n + 1) + 4 * n + n + n                         # vptr, partition, heavy flags, locks
    b += 4 * Pu                                              # incidences of unlocked vertices
    b += min(4 * Pu, 4 * m)                                  # omega(e) gathers
    b += min(8 * kw * Pu, 8 * kw * m)                        # bitmask rows (phi >= 1, phi >= 2) gathers
    b += 8 * n                                               # candidate records written
    return b


def graph_cand_bytes(hg, deg, st_before):
    """Compulsory bytes of the graph path's candidate kernels for one round: the bitmask rows are replaced
    by the neighbour ids (4 B per incidence) and their blocks (a gather from the 4n-byte partition)."""
    n, m = hg.n, hg.m
    Pu = int(deg[~st_before].sum())
    b = 8 * (n + 1) + 4 * n + n + n + 8 * n                  # vptr, partition, heavy flags, locks, records
    b += 4 * Pu + min(4 * Pu, 4 * n)                         # neighbour ids, their blocks
    if not ctx_unit_weights(hg):
        b += 4 * Pu + min(4 * Pu, 4 * m)                     # incidences and omega(e) gathers
    return b


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    return float(peaks.get("hbm_gbs", 6800.0)), "measured" if "hbm_gbs" in peaks else "fallback"


def ctx_unit_weights(hg):
    return bool(hg.m == 0 or int(hg.ewgt.max()) <= 1)


def rebalance_target_bytes(hg, k, stats, work, unit):
    """Algorithmic bytes of the rebalancing target kernels over one iteration (all its rounds), gathers
    counted at their element size: per round a scan of the partition and heavy flags; per vertex of an
    overloaded block its weight; per evaluated vertex its offsets and its record (16 B key, vertex,
    weight/target) and first-level histogram update (8 B); per incidence of an evaluated vertex the edge id,
    the edge's bitmask row (2 ceil(k/32) words, rounded to 8/16/32/64 B) and omega(e) unless unit."""
    kw = (k + 31) // 32
    row = 4 * 2 * (1 if kw <= 1 else 2 if kw <= 2 else 4 if kw <= 4 else 8)
    rounds = stats["rebalance_rounds"]
    b = rounds * (4 * hg.n + hg.n)
    b += 4 * work["rebalance_over"]
    b += (8 + 16 + 8) * work["rebalance_evaluated"]
    b += (4 + row + (0 if unit else 4)) * work["rebalance_evaluated_pins"]
    return b


def afterburner_bytes(hg, unit):
    """Algorithmic bytes of the afterburner over one iteration: the edge offsets and pins streamed once; the
    candidate records (8 B per vertex) and the partition (4 B per vertex) gathered per pin, each table counted
    once (min(gathers, table)); omega(e) per edge unless unit; the recomputed gains written (4 B per vertex)."""
    n, m, P = hg.n, hg.m, hg.P
    return 8 * (m + 1) + 4 * P + min(8 * P, 8 * n) + min(4 * P, 4 * n) + (0 if unit else 4 * m) + 4 * n


def approve_bytes(hg, stats):
    """Approval and locks over one iteration: per vertex its record (8 B), recomputed gain (4 B read, 4 B
    cleared) and lock (1 B); per approved move its move-list entry (8 B)."""
    return 17 * hg.n + 8 * stats["approved"]


def selection_bytes(work):
    """Rebalancing selection over one iteration: every record (16 B: key, vertex, weight and blocks) is read
    once per radix level after the first (the first level's histogram is built by the target kernels).  The
    per-block histogram rows the pick kernels scan are not counted."""
    return 16 * max(work["select_levels"] - 1, 0) * work["rebalance_evaluated"]


def objective_bytes(hg, k, unit):
    """(lambda-1) from the compact bitmasks: one Lambda(e) row (ceil(k/32) words, rounded to 1/2/4/8) per edge,
    plus omega(e) unless unit."""
    kw = (k + 31) // 32
    kwp = 1 if kw <= 1 else 2 if kw <= 2 else 4 if kw <= 4 else 8
    return 4 * hg.m * kwp + (0 if unit else 4 * hg.m)


def apply_move_bytes(stats, work):
    """Algorithmic bytes of the apply kernels over one iteration: per Jet move its list entry (vertex,
    source/target), the partition write, c(v) and the offsets; per rebalancing record (the rebalancing
    apply reads every record and moves the selected ones) the record, and per rebalancing move the
    partition write and the offsets; per incidence of a moved vertex the edge id and two phi
    read-modify-writes (4 B each way).  The bitmask toggles at phi crossings are not counted."""
    return (stats["approved"] * (4 + 4 + 4 + 4 + 16) + work["rebalance_evaluated"] * 16
            + stats["rebalance_moves"] * (4 + 16) + work["moved_pins"] * (4 + 2 * 8))


def ncu_traffic(workload, kernel="k_cand_light"):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or None if the kernel source
    changed since that capture (or no capture exists for this workload)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", kernel + ".md")
    src = os.path.join(ROOT, "paper_2504_12013_gb300", "csrc", "k_moves.cu" if kernel == "k_apply" else "k_cand.cu")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_source_sha256 = ([0-9a-f]{64})", txt)
    if not m or m.group(1) != hashlib.sha256(open(src, "rb").read()).hexdigest():
        return None
    m = re.search(r"traffic_per_launch\[" + re.escape(workload) + r"\] = (\d+)", txt)
    return int(m.group(1)) if m else None


# ---------------------------------------------------------------- replicas
def max_over_ranks(ms, world, device=None):
    """The slowest rank's time (every rank runs its own replica; the job takes as long as the slowest)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import torch

    from paper_2504_12013_gb300 import jet

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    desc, make = WORKLOADS[args.workload]
    t0 = time.time()
    hg, k, part0 = make(args.seed)
    log(f"[rank {rank}] workload {args.workload}: n={hg.n} m={hg.m} P={hg.P} k={k} (generated in "
        f"{time.time() - t0:.1f}s)")
    dh = jet.DeviceHypergraph(hg, dev)
    stream = torch.cuda.current_stream(dev)
    ctx = jet.jet_ctx_create(dh, jet.params(k), stream)
    if args.eager:
        jet.jet_set_graph_mode(ctx, False)
    st = jet.JetState(ctx, part0)
    part_init = st.part.clone()
    phi_init = st.phi.clone()
    bw_init = st.block_w.clone()

    def reset():
        st.part.copy_(part_init)
        st.phi.copy_(phi_init)
        st.block_w.copy_(bw_init)
        st.locked.zero_()
        jet.jet_build_pincounts(ctx, st.part, st.phi, st.block_w)  # also refreshes the context's bitmasks

    for _ in range(args.warmup):
        st.round(TAU)
    reset()
    torch.cuda.synchronize(dev)
    jet.jet_profile_read(ctx, reset=True)
    jet.jet_profile_enable(ctx, True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            st.round(TAU)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    prof_timed = jet.jet_profile_read(ctx, reset=True)  # graph mode: the candidate kernels, timed in the graphs
    ms = max_over_ranks(ms, world, dev)
    final_stats = st.stats_dict()

    # untimed replay of the same K steps, kernel by kernel (results are bit-identical): per-family device
    # times and kernel launches from the profiler, and per-step locks and stats for the byte model
    reset()
    jet.jet_set_graph_mode(ctx, False)
    if args.eager:  # the timed region already ran kernel by kernel: its family times are the ones
        prof_eager_timed = prof_timed
    jet.jet_profile_read(ctx, reset=True)
    deg = np.diff(hg.vptr)
    unit = ctx_unit_weights(hg)
    model_bytes = 0
    rb_bytes = 0
    apply_bytes = 0
    fam_bytes = {"candidates": 0, "afterburner": 0, "approve": 0, "apply": 0, "rebalance_targets": 0,
                 "rebalance_select": 0, "objective": 0}
    trace = []
    for _ in range(args.steps):
        locked_before = st.locked.cpu().numpy()[: hg.n].astype(bool)
        st.round(TAU)
        s = st.stats_dict()
        trace.append(s)
        cb = kernel_bytes(hg, k, deg, locked_before, s)
        model_bytes += cb
        work = jet.jet_profile_work(ctx)
        rb = rebalance_target_bytes(hg, k, s, work, unit)
        ap = apply_move_bytes(s, work)
        rb_bytes += rb
        apply_bytes += ap
        for f, b in (("candidates", cb), ("afterburner", afterburner_bytes(hg, unit)), ("approve", approve_bytes(hg, s)),
                     ("apply", ap), ("rebalance_targets", rb), ("rebalance_select", selection_bytes(work)),
                     ("objective", objective_bytes(hg, k, unit))):
            fam_bytes[f] += b
    prof = jet.jet_profile_read(ctx, reset=True)
    if args.eager:
        prof = prof_eager_timed
    jet.jet_profile_enable(ctx, False)
    assert trace[-1] == final_stats, "replay diverged from the timed run"
    sched = schedule_timing(jet, ctx, st, stream, dev)

    result = {"ms": ms, "prof": prof, "prof_timed": prof_timed, "model_bytes": model_bytes, "rb_bytes": rb_bytes,
              "apply_bytes": apply_bytes, "fam_bytes": fam_bytes, "workload": args.workload,
              "trace": trace, "schedule": sched,
              "clocks": clk.summary(), "hg": hg, "k": k, "part0": part0, "desc": desc, "dev": dev}
    ctx.close()
    return result


def schedule_timing(jet, ctx, st, stream, dev):
    """Matching schedule of the quotient graph (Section 5) of the partition after the timed steps: the
    quotient kernel over every edge bitmask row plus the one-warp schedule kernel.  Device time from the
    context's event pairs around the two kernels; the call time adds the host's result copies."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    jet.jet_profile_read(ctx, reset=True)
    jet.jet_profile_enable(ctx, True)
    for _ in range(3):
        ev0.record(stream)
        pairs, rnd, nr = jet.jet_quotient_schedule(ctx, st.phi)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(ev0.elapsed_time(ev1))
    prof = jet.jet_profile_read(ctx, reset=True)["other"]
    jet.jet_profile_enable(ctx, False)
    return {"ms": prof["ms"] / max(prof["calls"], 1), "call_ms": min(times), "pairs": int(len(pairs)),
            "rounds": int(nr), "launches_per_call": prof["launches"] / max(prof["calls"], 1),
            "what": "quotient graph of the partition after the timed steps and its rounds of maximal matchings "
                    "(jet_quotient_schedule, Section 5): device time of the kernels; call_ms with the host copies"}


def pinned_hypergraph(hg):
    """The hypergraph's arrays copied into pinned host memory (the fastest host->device copies)."""
    import torch
    pinned = {}
    for name in ("eptr", "pins", "vptr", "inc", "vwgt", "ewgt"):
        a = getattr(hg, name)
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
        t.numpy()[:] = a
        pinned[name] = t.numpy()
    return synth.Hypergraph(hg.n, hg.m, **pinned)


def run_e2e(args, hg, k, part0, dev):
    """End to end through the C ABI on pinned host buffers, the same K iterations as the device-timed value:
    jet_rounds_host copies the hypergraph and the partition to the device, creates the context (validation,
    size classes), builds phi, runs K iterations at tau = 3/4 and copies the partition back, per call.  Also
    the whole temperature schedule through jet_refine_host (e2e_schedule)."""
    import torch

    from paper_2504_12013_gb300 import jet
    hp = pinned_hypergraph(hg)
    part_t = torch.empty(hg.n, dtype=torch.int32, pin_memory=True)
    part = part_t.numpy()
    part[:] = part0
    jet.jet_rounds_host(hp, jet.params(k), TAU, args.steps, part)  # warm-up (allocator pools, module load)
    times = []
    for _ in range(args.e2e_steps):
        part[:] = part0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st = jet.jet_rounds_host(hp, jet.params(k), TAU, args.steps, part)
        times.append(time.perf_counter() - t0)
    bi = hg.nbytes() + 4 * hg.n
    bo = 4 * hg.n
    out = {"value": hg.P * args.steps / (sum(times) / len(times)), "unit": "pins/s", "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": bo, "iterations_per_call": args.steps, "seconds_per_call": sum(times) / len(times),
           "objective": st["objective"],
           "what": "jet_rounds_host on pinned host buffers: upload, context set-up, pin counts, the same K iterations "
                   "at tau 3/4 as value, download of the partition; wall time per call, mean of the calls"}
    if not args.no_e2e_schedule:
        part[:] = part0
        jet.jet_refine_host(hp, jet.params(k), SCHEDULE, LIMIT, part)  # warm-up
        stimes, iters = [], []
        for _ in range(args.e2e_steps):
            part[:] = part0
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            res = jet.jet_refine_host(hp, jet.params(k), SCHEDULE, LIMIT, part)
            stimes.append(time.perf_counter() - t0)
            iters.append(res["iterations"])
        out["e2e_schedule"] = {"value": hg.P * sum(iters) / sum(stimes), "unit": "pins/s",
                               "iterations_per_call": iters[-1], "seconds_per_call": min(stimes),
                               "objective": res["objective"],
                               "what": "jet_refine_host: the whole temperature schedule (Algorithm 1 to convergence, "
                                       "later iterations are cheap), copies and set-up included"}
    return out


def run_batched(args, dev):
    """The batched form: 256 independent random hypergraphs (n log-uniform in [1k, 200k], m = 1.1 n,
    |e| = 2 + Geometric(0.4) <= 256, k in {2, 8, 32}, unit weights), each refined to convergence
    (Algorithm 1, schedule 3/4, 3/8, 0, limit 8) -- all of them by ONE batch-graph launch per step, against
    the plain path (jet_refine on each instance in turn).  Each step restores the initial partitions first.
    The end-to-end figure also re-uploads every hypergraph and partition from pinned host memory and reads
    the partitions back, per step."""
    import torch

    from paper_2504_12013_gb300 import jet
    t0 = time.time()
    insts = synth.config_batched(args.seed)
    stream = torch.cuda.current_stream(dev)
    dhs = [jet.DeviceHypergraph(h, dev) for h, _, _ in insts]
    ctxs = [jet.jet_ctx_create(d, jet.params(k), stream) for d, (_, k, _) in zip(dhs, insts)]
    states = [jet.JetState(c, p) for c, (_, _, p) in zip(ctxs, insts)]
    init = [st.part.clone() for st in states]
    pins = [h.P for h, _, _ in insts]
    log(f"batched: {len(insts)} instances, sum n={sum(h.n for h, _, _ in insts)}, sum P={sum(pins)} "
        f"(set up in {time.time() - t0:.1f}s)")

    def restore():
        for st, p in zip(states, init):
            st.part.copy_(p)

    b = jet.jet_batch_create(ctxs, stream)
    split, tune_ms = jet.jet_batch_tune(b, SCHEDULE, LIMIT, states, [0, 1, 2, 4, 8])
    for _ in range(max(args.warmup, 1)):
        restore()
        res = jet.jet_batch_refine(b, SCHEDULE, LIMIT, states)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.batch_steps):
        restore()
        res = jet.jet_batch_refine(b, SCHEDULE, LIMIT, states)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_batch = ev0.elapsed_time(ev1) / args.batch_steps
    pin_rounds = sum(p * r["iterations"] for p, r in zip(pins, res))
    parts_batch = [st.part[: h.n].cpu().numpy().copy() for st, (h, _, _) in zip(states, insts)]

    # persistent form: one kernel, teams chosen by the autotuner from short trials on a sample
    restore()
    t_tune = time.perf_counter()
    shape, trials = jet.jet_batch_autotune(b, SCHEDULE, LIMIT, states, sample=args.tune_sample,
                                           trial_iterations=args.tune_iterations)
    tune_s = time.perf_counter() - t_tune
    for _ in range(max(args.warmup, 1)):
        restore()
        jet.jet_batch_refine(b, SCHEDULE, LIMIT, states)
    torch.cuda.synchronize(dev)
    tms = []
    for _ in range(args.batch_steps):
        restore()
        ev0.record(stream)
        res_team = jet.jet_batch_refine(b, SCHEDULE, LIMIT, states)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        tms.append(ev0.elapsed_time(ev1))
    ms_team = sum(tms) / len(tms)
    same_team = all(a["iterations"] == r["iterations"] and a["objective"] == r["objective"]
                    for a, r in zip(res_team, res))
    same_team = same_team and all(np.array_equal(st.part[: h.n].cpu().numpy(), pb)
                                  for st, (h, _, _), pb in zip(states, insts, parts_batch))
    persistent = {"value": pin_rounds / (ms_team / 1e3), "unit": "pins/s", "ms_per_step": ms_team,
                  "team": {"blocks": shape[0], "threads": shape[1], "split_pins": shape[2]},
                  "autotuner": {"sample_instances": args.tune_sample, "trial_iterations": args.tune_iterations,
                                "seconds": tune_s,
                                "trials": [{"blocks": c, "threads": t, "split_pins": sp, "ms": ms,
                                            "pin_iterations_per_s": rate}
                                           for (c, t, sp), (ms, rate) in trials.items()]},
                  "results_identical_to_branch_graph": bool(same_team),
                  "how": "jet_batch_refine with jet_batch_set_team: ONE persistent kernel in a CUDA graph; teams "
                         "(thread-block clusters) take instances from a device queue, largest first, and run all "
                         "of Algorithm 1 with cluster barriers between phases; below split_pins pins every block "
                         "of a cluster takes instances on its own"}
    jet.jet_batch_set_team(b, 0)
    b.close()

    # plain path: one jet_refine (device-side loop, one graph launch and one synchronization) per instance
    for c, st in zip(ctxs[:8], states[:8]):  # warm the per-context graphs
        jet.jet_refine(c, SCHEDULE, LIMIT, st.part, st.phi, st.block_w)
    restore()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    res_plain = [jet.jet_refine(c, SCHEDULE, LIMIT, st.part, st.phi, st.block_w) for c, st in zip(ctxs, states)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_plain = ev0.elapsed_time(ev1)
    same = all(a["iterations"] == r["iterations"] and a["objective"] == r["objective"] for a, r in zip(res_plain, res))
    same = same and all(np.array_equal(st.part[: h.n].cpu().numpy(), pb)
                        for st, (h, _, _), pb in zip(states, insts, parts_batch))

    # end to end: inputs from pinned host memory every step
    host_bufs = []
    for d, (h, _, p) in zip(dhs, insts):
        bufs = {}
        for name in ("eptr", "pins", "vptr", "inc", "vwgt", "ewgt"):
            a = getattr(h, name)
            t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
            t.numpy()[:] = a
            bufs[name] = t
        pt = torch.empty(h.n, dtype=torch.int32, pin_memory=True)
        pt.numpy()[:] = p
        host_bufs.append((bufs, pt))
    out_parts = [torch.empty(h.n, dtype=torch.int32, pin_memory=True) for h, _, _ in insts]
    b = jet.jet_batch_create(ctxs, stream)
    jet.jet_batch_set_split(b, split)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for _ in range(args.batch_steps):
        for d, st, (bufs, pt) in zip(dhs, states, host_bufs):
            for name, t in bufs.items():
                getattr(d, name).copy_(t, non_blocking=True)
            st.part[: pt.numel()].copy_(pt, non_blocking=True)
        jet.jet_batch_refine(b, SCHEDULE, LIMIT, states)
        for st, o in zip(states, out_parts):
            o.copy_(st.part[: o.numel()], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t1) / args.batch_steps
    b.close()
    h2d = sum(h.nbytes() + 4 * h.n for h, _, _ in insts)
    d2h = sum(4 * h.n for h, _, _ in insts)
    for c in ctxs:
        c.close()
    return {"metric": "Jet-round pins/s, batched (256 instances to convergence, one graph launch per step: the "
                      "branch graph in value, the persistent kernel in persistent)",
            "value": pin_rounds / (ms_batch / 1e3), "unit": "pins/s", "ms_per_step": ms_batch,
            "steps": args.batch_steps, "instances": len(insts), "pins": sum(pins),
            "jet_iterations": sum(r["iterations"] for r in res),
            "plain": {"value": pin_rounds / (ms_plain / 1e3), "unit": "pins/s", "ms_per_step": ms_plain,
                      "how": "jet_refine on each instance in turn (one graph launch + synchronization each)"},
            "speedup_vs_plain": ms_plain / ms_batch, "results_identical_to_plain": bool(same),
            "persistent": persistent, "persistent_speedup_vs_plain": ms_plain / ms_team,
            "persistent_speedup_vs_branch_graph": ms_batch / ms_team,
            "work_split": {"chosen": split, "tuned_ms": tune_ms},
            "e2e": {"value": pin_rounds / e2e_s, "unit": "pins/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "config": "256 random hypergraphs, n log-uniform [1k, 200k], m = 1.1 n, |e| = 2 + Geometric(0.4) <= 256, "
                      "k from {2, 8, 32}, unit weights, eps = 3/100, hash partitions"}


def run_convergence_10k(args, dev):
    """The plain configuration to convergence: random_10k (n 10,000, m 12,000, k 8), Algorithm 1 with the
    schedule 3/4, 3/8, 0 and limit 8 as one graph launch (jet_refine), against the oracle's Algorithm 1 on the
    same input (one host core); the partitions must be identical."""
    import torch

    import oracle
    from paper_2504_12013_gb300 import jet
    hg, k, part0 = synth.config_random_10k(args.seed)
    stream = torch.cuda.current_stream(dev)
    ctx = jet.jet_ctx_create(jet.DeviceHypergraph(hg, dev), jet.params(k), stream)
    st = jet.JetState(ctx, part0)
    jet.jet_refine(ctx, SCHEDULE, LIMIT, st.part, st.phi, st.block_w)  # warm-up: graph capture
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(5):
        st.part.copy_(torch.as_tensor(part0))
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        res = jet.jet_refine(ctx, SCHEDULE, LIMIT, st.part, st.phi, st.block_w)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(ev0.elapsed_time(ev1))
    gpu_part = st.part.cpu().numpy()[: hg.n].copy()
    ctx.close()
    p = part0.copy()
    t0 = time.perf_counter()
    iters, obj, _ = oracle.Oracle(hg).refine(oracle.Params(k), p)
    osec = time.perf_counter() - t0
    return {"ms": sorted(times)[len(times) // 2], "iterations": res["iterations"], "objective": res["objective"],
            "initial_objective": res["initial_objective"], "pins": hg.P,
            "pin_iterations_per_s": hg.P * res["iterations"] / (sorted(times)[len(times) // 2] / 1e3),
            "oracle_seconds": osec, "oracle_iterations": iters, "oracle_objective": obj,
            "identical_to_oracle": bool(iters == res["iterations"] and obj == res["objective"]
                                        and np.array_equal(gpu_part, p)),
            "what": "random_10k to convergence (jet_refine, one graph launch, median of 5) and the oracle's "
                    "Algorithm 1 on one host core"}


def run_multilevel(args, hg, k, dev, coarsen_only=False, graph_path=False):
    """The multilevel pass of the paper (Sections 6 and 7.2) on the workload: deterministic coarsening on the
    GPU (jet_cluster + jet_contract per level; c_max = ceil(c(V) / (160 k)), until at most 160 k vertices
    remain or a level shrinks by less than 1%), a balanced hash partition of the coarsest level standing in
    for initial partitioning, then the uncoarsening (projection + Algorithm 1 at every level) as one graph
    launch (jet_uncoarsen).  Each level's vertex order is a seeded permutation generated beforehand."""
    import torch

    from paper_2504_12013_gb300 import jet
    stream = torch.cuda.current_stream(dev)
    limit = 160 * k
    # contexts take c(v) <= 32767, and a cluster never exceeds c_max: keep the coarse levels refinable
    cmax = min(-(-int(hg.vwgt.astype(np.int64).sum()) // limit), 32767)
    orders = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def coarsen_all():
        levels, maps, rows = [jet.DeviceHypergraph(hg, dev)], [], []
        while levels[-1].n > limit:
            cur = levels[-1]
            if len(levels) not in orders:
                orders[len(levels)] = torch.as_tensor(synth.vertex_order(args.seed + len(levels), cur.n)).to(dev)
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            label = jet.jet_cluster(cur, cmax, orders[len(levels)], stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            t_cl = ev0.elapsed_time(ev1)
            ev0.record(stream)
            coarse, mp = jet.jet_contract(cur, label, stream)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            sz = (cur.eptr[1:] - cur.eptr[:-1]).double()
            rated = sz[(sz >= 2) & (sz <= jet.RATING_MAX_EDGE)]
            visits = int((rated * rated).sum().item())
            rows.append({"n": cur.n, "m": cur.m, "pins": cur.P, "cluster_ms": t_cl, "contract_ms": ev0.elapsed_time(ev1),
                         "rating_pin_visits_bound": visits,
                         "rating_gbs": 8 * visits / (t_cl / 1e3) / 1e9 if t_cl > 0 else None})
            if coarse.n > 0.99 * cur.n:
                break
            levels.append(coarse)
            maps.append(mp)
        return levels, maps, rows

    coarsen_all()  # warm-up (module load, allocator pools); same orders, same result
    t0 = time.perf_counter()
    levels, maps, rows = coarsen_all()
    coarsen_s = time.perf_counter() - t0
    coarsening = {"levels": rows, "seconds": coarsen_s, "max_cluster_weight": cmax,
                  "pins_per_s": sum(r["pins"] for r in rows) / coarsen_s,
                  "what": "jet_cluster + jet_contract per level, wall time of all levels (host syncs included), "
                          "per-level device times in levels; rating_pin_visits_bound = sum of |e|^2 over the "
                          "rated edges (each vertex of a rated edge visits its pins)"}
    if coarsen_only:
        return {"coarsening": coarsening}
    hs, mps = levels[::-1], maps[::-1]
    ctxs = [jet.jet_ctx_create(h, jet.params(k), stream) for h in hs]
    if graph_path:  # every level of a graph's hierarchy is a graph (contraction drops one-pin edges)
        for c in ctxs:
            jet.jet_set_graph_path(c, True)
    p0 = synth.part_perm(args.seed, hs[0].n, k)
    states = [jet.JetState(ctxs[0], p0, with_phi=not graph_path)] + [
        jet.JetState(c, np.zeros(h.n, np.int32), with_phi=not graph_path) for c, h in zip(ctxs[1:], hs[1:])]
    init = states[0].part.clone()
    times = []
    for it in range(1 + max(args.batch_steps, 1)):
        states[0].part.copy_(init)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        res = jet.jet_uncoarsen(ctxs, mps, SCHEDULE, LIMIT, states, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if it:
            times.append(ev0.elapsed_time(ev1))
    ms = sum(times) / len(times)
    for c in ctxs:
        c.close()
    work = sum(h.P * r["iterations"] for h, r in zip(hs, res))
    fine = res[-1]
    return {"coarsening": coarsening,
            "uncoarsening": {"ms": ms, "pin_iterations_per_s": work / (ms / 1e3),
                             "levels": [{"n": h.n, "pins": h.P, "iterations": r["iterations"],
                                         "initial_objective": r["initial_objective"], "objective": r["objective"],
                                         "balanced": r["balanced"]} for h, r in zip(hs, res)],
                             "what": "projection + Algorithm 1 per level, one graph launch; mean over timed launches"},
            "objective": fine["objective"], "balanced": fine["balanced"],
            "seconds_total": coarsen_s + ms / 1e3}


def run_graph(args, dev):
    """The graph path (jet_set_graph_path) against the hypergraph path on a graph: 4M vertices, 16M two-pin
    edges (80 % local), k = 64.  The same K Jet iterations at tau = 3/4 from the same partition, each path
    one graph launch per iteration, CUDA events; the final partitions must be identical."""
    import torch

    from paper_2504_12013_gb300 import jet
    t0 = time.time()
    hg, k, part0 = synth.config_graph_16m(args.seed)
    gen_s = time.time() - t0
    stream = torch.cuda.current_stream(dev)
    dh = jet.DeviceHypergraph(hg, dev)
    deg = np.diff(hg.vptr)
    out = {}
    parts = {}
    for name, graph_path in (("hypergraph_path", False), ("graph_path", True)):
        ctx = jet.jet_ctx_create(dh, jet.params(k), stream)
        if args.eager:
            jet.jet_set_graph_mode(ctx, False)
        if graph_path:
            jet.jet_set_graph_path(ctx, True)
        st = jet.JetState(ctx, part0, with_phi=not graph_path)
        for _ in range(max(args.warmup, 1)):
            st.round(TAU)
        st = jet.JetState(ctx, part0, with_phi=not graph_path)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            st.round(TAU)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1) / args.steps
        stats = st.stats_dict()
        parts[name] = st.part.cpu().numpy()[: hg.n]
        # untimed kernel-by-kernel replay of the same steps: device time per kernel family
        st = jet.JetState(ctx, part0, with_phi=not graph_path)
        jet.jet_set_graph_mode(ctx, False)
        jet.jet_profile_read(ctx, reset=True)
        jet.jet_profile_enable(ctx, True)
        cand_bytes = 0
        for _ in range(args.steps):
            locked_before = st.locked.cpu().numpy()[: hg.n].astype(bool)
            if graph_path:
                cand_bytes += graph_cand_bytes(hg, deg, locked_before)
            else:
                cand_bytes += kernel_bytes(hg, k, deg, locked_before, None)
            st.round(TAU)
        prof = jet.jet_profile_read(ctx, reset=True)
        jet.jet_profile_enable(ctx, False)
        assert st.stats_dict() == stats, "replay diverged from the timed run"
        peak, peak_src = hbm_peak()
        cms = prof["candidates"]["ms"]
        cand_gbs = cand_bytes / (cms / 1e3) / 1e9 if cms > 0 else None
        out[name] = {"ms_per_step": ms, "pins_per_s": hg.P / (ms / 1e3), "objective": stats["objective"],
                     "phi_bytes": 0 if graph_path else hg.m * k * 4,
                     "candidates_roofline": {"bound": "hbm", "achieved": cand_gbs, "peak": peak, "unit": "GB/s",
                                             "frac": cand_gbs / peak if cand_gbs else None,
                                             "bytes_per_step": cand_bytes / args.steps, "peak_source": peak_src,
                                             "timing": "kernel-by-kernel replay, CUDA events around the launches"},
                     "family_ms_per_step_replay": {f: round(v["ms"] / args.steps, 4) for f, v in prof.items()
                                                   if v["ms"] > 0}}
        ctx.close()
        del st
    out["speedup"] = out["hypergraph_path"]["ms_per_step"] / out["graph_path"]["ms_per_step"]
    out["results_identical"] = bool(np.array_equal(parts["hypergraph_path"], parts["graph_path"]))
    if not args.no_multilevel:  # the multilevel pass on the graph, graph path at every level
        ml = run_multilevel(args, hg, k, dev, graph_path=True)
        flat_ctx = jet.jet_ctx_create(dh, jet.params(k), stream)
        jet.jet_set_graph_path(flat_ctx, True)
        st = jet.JetState(flat_ctx, part0, with_phi=False)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        flat = jet.jet_refine(flat_ctx, SCHEDULE, LIMIT, st.part, None, st.block_w)
        flat_s = time.perf_counter() - t1
        flat_ctx.close()
        ml["flat_refinement"] = {"objective": flat["objective"], "iterations": flat["iterations"],
                                 "seconds": flat_s, "what": "Algorithm 1 on the finest level from the hash "
                                                            "partition (graph path, one graph launch)"}
        out["multilevel"] = ml
    out["config"] = {"n": hg.n, "m": hg.m, "pins": hg.P, "k": k, "steps": args.steps, "tau": "3/4",
                     "generated_s": round(gen_s, 1),
                     "workload": "graph: u uniform, v = u + U[1, 1000] (80 %) or uniform (20 %), unit weights"}
    return out


def run_served(args, dev):
    """The served form: refinement requests (P log-uniform in [10k, 5M], n = P / 3.85, m = 1.1 n,
    |e| = 2 + Geometric(0.4) <= 256, c in 1..8, k from {2, 4, ..., 256}, balanced random partitions, each
    refined to convergence) arrive as a Poisson stream at 200/s.  The server admits them by device-memory
    footprint into up to `serve_slots` concurrent slots (continuous batching); the serial arm is the same
    queue with one slot (the plain path, one job after another).  Latency = arrival to refined partition back
    in host memory."""
    import threading

    import torch

    from paper_2504_12013_gb300 import jet
    insts, jobs = synth.served_jobs(args.seed, args.serve_jobs)
    pinned = []
    for h in insts:
        arrs = {}
        for name in ("eptr", "pins", "vptr", "inc", "vwgt", "ewgt"):
            a = getattr(h, name)
            t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
            t.numpy()[:] = a
            arrs[name] = t.numpy()
        pinned.append(synth.Hypergraph(h.n, h.m, **arrs))
    budget = int(args.serve_budget_gb * (1 << 30))
    out = {}
    finals = {}
    for arm, slots in (("served", args.serve_slots), ("serial", 1)):
        server = jet.jet_server_create(budget, slots)
        warm = [np.ascontiguousarray(jobs[i][3].copy()) for i in range(min(4, len(jobs)))]
        for i, w in enumerate(warm):
            jet.jet_server_submit(server, pinned[jobs[i][1]], jet.params(jobs[i][2]), SCHEDULE, LIMIT, w)
        got = 0
        while got < len(warm):
            got += len(jet.jet_server_wait(server))
        parts = [np.ascontiguousarray(j[3].copy()) for j in jobs]
        ids = {}
        t0 = time.perf_counter()

        def submit():
            for idx, (arr_s, pi, k, _) in enumerate(jobs):
                delay = t0 + arr_s - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                ids[jet.jet_server_submit(server, pinned[pi], jet.params(k), SCHEDULE, LIMIT, parts[idx])] = idx

        th = threading.Thread(target=submit)
        th.start()
        done = []
        while len(done) < len(jobs):
            done += jet.jet_server_wait(server, timeout_ms=1000)
        wall = time.perf_counter() - t0
        th.join()
        server.close()
        bad = [d for d in done if d["status"] != 0]
        if bad:
            raise RuntimeError(f"served job failed: {bad[0]}")
        def pct(xs, q):
            xs = sorted(xs)
            return xs[min(len(xs) - 1, (q * len(xs)) // 100)]

        lat = [d["latency_ms"] for d in done]
        serv = [d["service_ms"] for d in done]
        pr = sum(insts[jobs[ids[d["id"]]][1]].P * d["result"]["iterations"] for d in done)
        spans = sorted((d["device_start_ms"], d["device_end_ms"]) for d in done if d["device_start_ms"] >= 0)
        conc = 0
        if spans:  # most jobs in flight on the device at once (from the jobs' GPU-timeline intervals)
            ev = sorted([(a, 1) for a, _ in spans] + [(b, -1) for _, b in spans], key=lambda x: (x[0], x[1]))
            cur = 0
            for _, d_ in ev:
                cur += d_
                conc = max(conc, cur)
        out[arm] = {"slots": slots, "jobs": len(done), "seconds": wall, "jobs_per_s": len(done) / wall,
                    "pin_rounds_per_s": pr / wall,
                    "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
                    "service_ms_p50": pct(serv, 50), "service_ms_p99": pct(serv, 99),
                    "queue_ms_mean": sum(d["queue_ms"] for d in done) / len(done),
                    "max_jobs_in_flight_on_device": conc}
        finals[arm] = parts
        torch.cuda.synchronize(dev)
    same = all(np.array_equal(a, b) for a, b in zip(finals["served"], finals["serial"]))
    return {"metric": "served refinement: throughput and p50/p99 latency, continuous batching vs serial queue",
            "latency": "arrival to refined partition in host memory (queueing included); service: admission to "
                       "completion",
            "served": out["served"], "serial": out["serial"],
            "p99_speedup": out["serial"]["latency_ms_p99"] / out["served"]["latency_ms_p99"],
            "throughput_speedup": out["served"]["jobs_per_s"] / out["serial"]["jobs_per_s"],
            "results_identical_alone_and_in_mix": bool(same),
            "config": f"{len(jobs)} jobs, Poisson arrivals at 200/s, P log-uniform [10k, 5M] over a pool of "
                      f"{len(insts)} seeded instances, k from {{2..256}} (powers of two), c in 1..8, balanced "
                      f"random partitions, memory budget {args.serve_budget_gb} GB"}


def host_cpu():
    """The host the oracle ran on: its logical CPU count and model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_baseline(hg, k, part0, budget_s):
    """The oracle as it stands (single thread), iterations at tau = 3/4 from the same start until budget_s (at
    least one)."""
    import oracle
    orc = oracle.Oracle(hg)
    st = oracle.State(orc, k, part0)
    prm = oracle.Params(k)
    rounds, t0 = 0, time.perf_counter()
    while True:
        orc.refine_round(prm, TAU, st.part, st.phi, st.bw, st.locked)
        rounds += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return dict({"value": hg.P * rounds / el, "unit": "pins/s", "cores": 1, "kind": "oracle",
                 "sample": f"first {rounds} Jet iteration(s) at tau=3/4 of the same workload, {el:.1f} s"},
                **host_cpu())


def roofline_block(args, r, hbm, peak_src):
    """The roofline object of one measured workload: the dominant kernel family's (the larger device time per
    step of the rebalancing-target kernels and the apply kernels, from the kernel-by-kernel replay), the others
    beside it, and `round`: the algorithmic bytes of every family of the iteration over the timed ms per step."""
    prof = r["prof"]
    fam_ms = {f: v["ms"] for f, v in prof.items()}
    total_fam = sum(fam_ms.values())
    dom = max(fam_ms, key=fam_ms.get)
    cand_ms = r["prof_timed"]["candidates"]["ms"]  # measured inside the timed region
    achieved = r["model_bytes"] / (cand_ms / 1e3) / 1e9 if cand_ms > 0 else None
    replay_note = ("CUDA events around each launch in the kernel-by-kernel replay of the timed steps (these kernels "
                   "also run inside conditional graph bodies, which cannot hold event nodes)")
    workload = r["workload"]

    def family_roofline(fam, kernel, nbytes, traffic_kernel):
        fms, fl = prof[fam]["ms"], prof[fam]["launches"]
        ach = nbytes / (fms / 1e3) / 1e9 if fms > 0 else None
        tr = ncu_traffic(workload, traffic_kernel) if traffic_kernel else None
        # the DRAM bytes the family moves at sector granularity (ncu mean per launch x launches) over its time
        tr_ach = tr * fl / (fms / 1e3) / 1e9 if tr and fms > 0 else None
        return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": (ach / hbm) if ach else None,
                "traffic": tr,
                "traffic_achieved": tr_ach, "traffic_frac": (tr_ach / hbm) if tr_ach else None,
                "traffic_frac_note": "measured DRAM bytes per launch (ncu, cold L2) x launches per step over the "
                                     "family's replay time: the share of HBM bandwidth the kernels use at sector "
                                     "granularity, beside frac, which counts algorithmic bytes only",
                "traffic_note": (f"mean DRAM bytes per launch, cold L2 (profiles/{traffic_kernel}.md); null when the "
                                 "kernel source changed since that capture" if traffic_kernel
                                 else "no capture for this kernel"),
                "bytes_per_step": nbytes / args.steps, "ms_per_step": fms / args.steps,
                "launches_per_step": fl / args.steps, "timing": replay_note, "peak_source": peak_src}

    fam_roof = {"rebalance_targets": family_roofline("rebalance_targets",
                                                     "rebalancing targets (k_rbcand_light/k_rbcand_heavy)",
                                                     r["rb_bytes"], "k_rbcand_light"),
                "apply": family_roofline("apply", "apply moves (k_apply, k_rb_apply)",
                                         r["apply_bytes"], "k_apply")}
    dom_kernel = max(fam_roof, key=lambda f: prof[f]["ms"])  # the kernel with the most device time per step
    launches = sum(v["launches"] for v in prof.values())
    ms_step = r["ms"] / args.steps
    fb = r["fam_bytes"]
    b_round = sum(fb.values()) / args.steps
    fams = {}
    for f, b in fb.items():
        fms = prof[f]["ms"] / args.steps
        ach = (b / args.steps) / (fms / 1e3) / 1e9 if fms > 0 else None
        fams[f] = {"bytes_per_step": b / args.steps, "ms_per_step_replay": fms,
                   "achieved": ach, "frac": ach / hbm if ach else None}
    round_ach = b_round / (ms_step / 1e3) / 1e9
    roof = dict(fam_roof[dom_kernel], **{
        "others": {f: v for f, v in fam_roof.items() if f != dom_kernel},
        "candidates": {"kernel": "k_cand_light/k_cand_heavy", "achieved": achieved,
                       "frac": (achieved / hbm) if achieved else None,
                       "traffic": ncu_traffic(workload),
                       "traffic_note": "DRAM bytes of the first timed launch (profiles/k_cand_light.md)",
                       "timing": "event-record nodes around the kernels inside the timed graphs",
                       "ms_per_step": cand_ms / args.steps,
                       "bytes_per_step": r["model_bytes"] / args.steps},
        "round": {"bound": "hbm", "achieved": round_ach, "peak": hbm, "unit": "GB/s", "frac": round_ach / hbm,
                  "bytes_per_step": b_round, "ms_per_step": ms_step, "peak_source": peak_src,
                  "what": "sum of every family's algorithmic bytes per iteration (candidates, afterburner, approval, "
                          "apply, rebalancing targets and selection, objective) over the timed ms per step (graph "
                          "form, CUDA events); per family: its bytes over its replay time",
                  "families": fams},
        "dominant_family": dom, "family_share": {f: round(v / total_fam, 4) for f, v in fam_ms.items()}
        if total_fam > 0 else {},
        "family_ms_per_step_replay": {f: round(v / args.steps, 4) for f, v in fam_ms.items()},
        "family_times": "kernel-by-kernel replay of the timed steps (identical work)"})
    return roof, launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rownet_4m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-second", action="store_true", help="skip the vlsi_2m object beside the headline")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e-schedule", action="store_true", help="skip the whole-schedule end-to-end figure")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds of oracle iterations in the reference arm (at least one iteration)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--tune-sample", type=int, default=24, help="instances in each autotuner trial")
    ap.add_argument("--tune-iterations", type=int, default=6, help="Jet iterations per instance in a trial")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=48.0)
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-multilevel", action="store_true")
    ap.add_argument("--no-convergence", action="store_true", help="skip the random_10k convergence object")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--graph-only", action="store_true",
                    help="time only the graph workload on both paths (with --eager: kernel by kernel) and print its line")
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the batched workload (branch graph, persistent kernel, plain launches)")
    ap.add_argument("--coarsen-only", action="store_true",
                    help="time only the GPU coarsening of the workload (Section 6) and print its JSON line")
    ap.add_argument("--eager", action="store_true",
                    help="time the kernel-by-kernel form instead of the CUDA graphs (same work and results; "
                         "ncu cannot profile kernels inside graphs with conditional nodes)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.coarsen_only:
        return run_coarsen_only(args, rank)
    if args.graph_only:
        return run_graph_only(args, rank)
    if args.batched_only:
        return run_batched_only(args, rank)

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    r = run_gpu(args, rank, world)
    hg, k = r["hg"], r["k"]
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return
    e2e = None if args.no_e2e else run_e2e(args, hg, k, r["part0"], r["dev"])
    batched = None if args.no_batched else run_batched(args, r["dev"])
    served = None if args.no_served else run_served(args, r["dev"])
    multilevel = None if args.no_multilevel else run_multilevel(args, hg, k, r["dev"])
    conv10k = None if args.no_convergence else run_convergence_10k(args, r["dev"])
    graph = None if args.no_graph else run_graph(args, r["dev"])
    cpu = None if args.no_cpu_baseline else cpu_baseline(hg, k, r["part0"], args.cpu_budget)

    hbm, peak_src = hbm_peak()
    ms = r["ms"]
    value = job_throughput(hg.P * args.steps, world, ms)
    roof, launches = roofline_block(args, r, hbm, peak_src)
    second = None
    if not args.no_second and args.workload != "vlsi_2m":
        import copy
        a2 = copy.copy(args)
        a2.workload = "vlsi_2m"
        r2 = run_gpu(a2, rank, 1)
        roof2, launches2 = roofline_block(a2, r2, hbm, peak_src)
        second = {"value": r2["hg"].P * args.steps / (r2["ms"] / 1e3), "unit": "pins/s",
                  "ms_per_step": r2["ms"] / args.steps, "steps": args.steps,
                  "config": {"workload": r2["desc"], "n": r2["hg"].n, "m": r2["hg"].m, "pins": r2["hg"].P,
                             "k": r2["k"], "tau": "3/4"},
                  "roofline": roof2, "gpu_launches": launches2, "clocks": r2["clocks"], "trace_first_steps": r2["trace"][:3],
                  "what": "the VLSI-shaped workload measured exactly like the headline (first K iterations at tau "
                          "3/4, one CUDA graph per iteration, CUDA events)"}
    line = {
        "metric": "Jet-round pins/s (bit-exact vs oracle)",
        "value": value,
        "unit": "pins/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded generator shaped like the paper's sparse-matrix and VLSI benchmark instances)",
        "config": {"workload": r["desc"], "n": hg.n, "m": hg.m, "pins": hg.P, "k": k, "tau": "3/4",
                   "step": "one Jet iteration (candidates, afterburner, apply, rebalancing, objective)",
                   "execution": "kernel by kernel" if args.eager else "one CUDA graph per iteration (device-side "
                                                                          "rebalancing loop)",
                   "l2": "inputs larger than L2 (phi %d MB)" % (hg.m * k * 4 // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "clocks": r["clocks"],
        "gpu_launches": launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "batched": batched,
        "served": served,
        "multilevel": multilevel,
        "graph": graph,
        "vlsi_2m": second,
        "random_10k_convergence": conv10k,
        "matching_schedule": r["schedule"],
        "trace_first_steps": r["trace"][:3],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_coarsen_only(args, rank):
    """Coarsening alone (one warm-up pass, one timed pass over all levels), for profiling."""
    import torch
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    desc, make = WORKLOADS[args.workload]
    hg, k, _ = make(args.seed)
    c = run_multilevel(args, hg, k, dev, coarsen_only=True)["coarsening"]
    print(json.dumps({"metric": "coarsening pins/s (all levels)", "value": c["pins_per_s"], "unit": "pins/s",
                      "config": {"workload": desc, "n": hg.n, "m": hg.m, "pins": hg.P, "k": k},
                      "coarsening": c}), flush=True)


def run_batched_only(args, rank):
    """The batched workload alone (for profiling and tuning)."""
    import torch
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    b = run_batched(args, dev)
    print(json.dumps({"metric": b["metric"], "value": b["value"], "unit": "pins/s", "batched": b}), flush=True)


def run_graph_only(args, rank):
    """The graph workload alone on both paths (for profiling)."""
    import torch
    if rank != 0:
        return
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g = run_graph(args, dev)
    print(json.dumps({"metric": "Jet-round pins/s on a graph (graph path)", "value": g["graph_path"]["pins_per_s"],
                      "unit": "pins/s", "graph": g}), flush=True)


def run_reference(args, rank, world):
    """The oracle (single thread) as the reference arm: each step one oracle Jet iteration at tau = 3/4 on the
    same workload, from the same start.  A CPU program has no device state to warm, so the warm-up steps are
    not run; and since one oracle iteration of the row-net workload takes most of a minute, the timed steps
    stop once --ref-budget seconds have passed (at least one step), and the line reports how many ran."""
    if rank != 0:
        return
    import oracle
    desc, make = WORKLOADS[args.workload]
    hg, k, part0 = make(args.seed)
    orc = oracle.Oracle(hg)
    st = oracle.State(orc, k, part0)
    prm = oracle.Params(k)
    done = 0
    t0 = time.perf_counter()
    while done < args.steps:
        orc.refine_round(prm, TAU, st.part, st.phi, st.bw, st.locked)
        done += 1
        if time.perf_counter() - t0 >= args.ref_budget:
            break
    el = time.perf_counter() - t0
    value = hg.P * done / el
    line = {"impl": "reference", "metric": "Jet-round pins/s (bit-exact vs oracle)", "value": value,
            "unit": "pins/s", "n_gpus": world, "steps": done, "steps_requested": args.steps, "warmup": 0,
            "warmup_requested": args.warmup,
            "ms_per_step": el * 1e3 / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": desc, "n": hg.n, "m": hg.m, "pins": hg.P, "k": k, "tau": "3/4"},
            "cpu_baseline": dict({"value": value, "unit": "pins/s", "cores": 1, "kind": "oracle",
                                  "sample": f"the first {done} of the {args.steps} requested Jet iterations at "
                                            f"tau=3/4 from the seeded start ({el:.1f} s; time budget "
                                            f"{args.ref_budget:.0f} s, no warm-up)"}, **host_cpu()),
            "e2e": {"value": value, "unit": "pins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
