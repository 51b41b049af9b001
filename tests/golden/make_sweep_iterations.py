"""Write seg2d_1024_sweep_iterations.txt: the oracle's FGMRES(30) iteration
counts (rtol 1e-8, M_L with FP64 L1-Jacobi V-cycles, default AMG options) for
the nine contrasts of the 1024 x 1024 random-segment workload.  Calls only the
oracle; takes about an hour of single-thread CPU time."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2206_03203_gb300 import inputs  # noqa: E402

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seg2d_1024_sweep_iterations.txt")
    lines = ["# contrast iterations (oracle, FGMRES(30) + M_L, FP64, rtol 1e-8); make_sweep_iterations.py"]
    for c in inputs.CONTRASTS:
        res, *_ = oracle.solve(inputs.random_segments_2d(contrast=c), maxit=5000)
        lines.append(f"{c:g} {res.iterations}")
        print(lines[-1], flush=True)
    open(out, "w").write("\n".join(lines) + "\n")
