"""Write seg2d_1024_sweep_iterations.txt: the oracle's FGMRES(30) iteration
counts (rtol 1e-8, M_L with FP64 L1-Jacobi V-cycles, default AMG options) for
the nine contrasts of the 1024 x 1024 random-segment workload, and the range
of the counts over the input and two replicates with every k_m value moved by
one unit in the last place (multiplied by 1 + e 2^-52, e = +-1 per cell):
how far arithmetic that differs only in rounding can move the count.  Calls
only the oracle and the seeded generator (one process per solve; about half
an hour of CPU time in all)."""
import dataclasses
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2206_03203_gb300 import inputs  # noqa: E402

REPLICATES = 2


def count(task):
    c, r = task
    oracle.build()
    inst = inputs.random_segments_2d(contrast=c)
    if r > 0:
        e = np.where(np.random.default_rng(1000 + r).random(inst.km.shape[0]) < 0.5, -1.0, 1.0)
        inst = dataclasses.replace(inst, km=inst.km * (1.0 + e * 2.0 ** -52))
    res, *_ = oracle.solve(inst, maxit=5000)
    return c, r, res.iterations


if __name__ == "__main__":
    oracle.build()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seg2d_1024_sweep_iterations.txt")
    tasks = [(c, r) for c in inputs.CONTRASTS for r in range(REPLICATES + 1)]
    tasks.sort(key=lambda t: -abs(np.log10(t[0])))  # longest solves first
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        res = pool.map(count, tasks, chunksize=1)
    by = {}
    for c, r, it in res:
        by.setdefault(c, {})[r] = it
    lines = ["# contrast iterations min max (oracle, FGMRES(30) + M_L, FP64, rtol 1e-8; min / max over the input and "
             f"{REPLICATES} replicates with k_m moved by one ulp); make_sweep_iterations.py"]
    for c in inputs.CONTRASTS:
        v = by[c]
        lines.append(f"{c:g} {v[0]} {min(v.values())} {max(v.values())}")
    open(out, "w").write("\n".join(lines) + "\n")
    print("\n".join(lines))
