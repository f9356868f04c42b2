"""Write oracle-only regression fixtures for the 10,000-vertex random workload.

Calls only ``oracle/`` and the seeded generator.  The paper prints no worked
example with numbers for this method (its results are aggregate timings and
quality ratios on datasets), so nothing here is a value from the paper: these
fixtures pin the oracle's own trajectory so that a later edit to the oracle's
arithmetic, or a different host (x86 here, Arm on the GPU machine), shows up
as a diff.

Usage:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2504_12013_gb300 import synth  # noqa: E402


def trajectory(seed):
    hg, k, part = synth.config_random_10k(seed)
    orc = oracle.Oracle(hg)
    params = oracle.Params(k)
    st = oracle.State(orc, k, part)
    first = [orc.refine_round(params, (3, 4), st.part, st.phi, st.bw, st.locked) for _ in range(3)]
    p = part.copy()
    iters, obj, phase = orc.refine(params, p)
    return {
        "seed": seed, "n": hg.n, "m": hg.m, "P": hg.P, "k": k,
        "initial_objective": int(orc.objective(k, part)),
        "first_rounds_tau_3_4": first,
        "iterations": int(iters), "phase_iterations": [int(x) for x in phase],
        "final_objective": int(obj),
        "final_block_weights": np.bincount(p, weights=hg.vwgt, minlength=k).astype(int).tolist(),
        "final_partition_sha256": hashlib.sha256(p.astype("<i4").tobytes()).hexdigest(),
    }


def coarsening(seed):
    """Three levels of the oracle's coarsening (Section 6, Algorithm 4) of the 10,000-vertex workload."""
    hg, k, _ = synth.config_random_10k(seed)
    levels = []
    for level in range(3):
        o = oracle.Oracle(hg)
        cmax = max(2, int(hg.vwgt.sum()) // 400)
        coarse, mp, label = o.coarsen(cmax, synth.vertex_order(seed * 10 + level, hg.n))
        levels.append({"n": hg.n, "m": hg.m, "P": hg.P, "max_cluster_weight": cmax,
                       "coarse": [coarse.n, coarse.m, coarse.P],
                       "labels_sha256": hashlib.sha256(label.astype("<i4").tobytes()).hexdigest(),
                       "coarse_pins_sha256": hashlib.sha256(coarse.pins.astype("<i4").tobytes()).hexdigest(),
                       "coarse_edge_weights_sum": int(coarse.ewgt.astype(np.int64).sum()),
                       "coarse_vertex_weight_max": int(coarse.vwgt.max())})
        hg = coarse
    return {"seed": seed, "levels": levels}


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out = {"workload": "random hypergraph n=10000 m=12000 |e|=2+Geometric(1/2)<=64, k=8, eps=3/100",
           "written_by": "tests/golden/make_golden.py (oracle only)",
           "runs": [trajectory(s) for s in (1, 2, 3)]}
    path = os.path.join(here, "random_10k_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)
    out = {"workload": "coarsening of the same workload, c_max = c(V) // 400, rating edge limit 1000, "
                       "100 one-vertex sub-rounds, sub-rounds up to 1 % (order: synth.vertex_order)",
           "written_by": "tests/golden/make_golden.py (oracle only)",
           "runs": [coarsening(s) for s in (1, 2)]}
    path = os.path.join(here, "coarsen_10k_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
