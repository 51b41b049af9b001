"""Write seg2d_1024_sweep_iterations.txt: the oracle's FGMRES(30) iteration
counts (rtol 1e-8, M_L with FP64 L1-Jacobi V-cycles, default AMG options) for
the nine contrasts of the 1024 x 1024 random-segment workload.  Calls only the
oracle (one process per contrast); about an hour of CPU time in all."""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2206_03203_gb300 import inputs  # noqa: E402


def count(c):
    res, *_ = oracle.solve(inputs.random_segments_2d(contrast=c), maxit=5000)
    return res.iterations


if __name__ == "__main__":
    oracle.build()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seg2d_1024_sweep_iterations.txt")
    with mp.get_context("spawn").Pool(min(9, os.cpu_count() or 1)) as pool:
        its = pool.map(count, inputs.CONTRASTS)
    lines = ["# contrast iterations (oracle, FGMRES(30) + M_L, FP64, rtol 1e-8); make_sweep_iterations.py"]
    lines += [f"{c:g} {i}" for c, i in zip(inputs.CONTRASTS, its)]
    open(out, "w").write("\n".join(lines) + "\n")
    print("\n".join(lines))
