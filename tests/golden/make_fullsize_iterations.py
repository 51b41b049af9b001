"""Write fullsize_iterations.json: the oracle's FGMRES(30) iteration counts
(rtol 1e-8, M_L, x0 = 0) at full workload sizes, each with the spread of
counts under rounding-level perturbations of the input, which bounds how far
an implementation whose arithmetic differs from the oracle's only in rounding
(summation order, fused multiply-adds, classical instead of modified
Gram-Schmidt) can land from the oracle's count.

A replicate multiplies every k_m value by (1 + e 2^-52), e = +-1 drawn per
cell, i.e. moves it by about one unit in the last place.  Calls only the
oracle and the seeded generator; about an hour of CPU time in all (one process
per solve).

Cases:
  planes3d_128: the 128^3 nine-plane instance, k_f in {1e-4, 1, 1e4}, FP64 and
      with FP32 V-cycles (the oracle's precision emulation);
  batch8_bf16: instances 0..7 of the 256-instance batch packed into one
      system (each coarsened as if alone), four right-hand sides each, FP32
      finest and BF16 row-scaled coarse levels;
  large3d_128_fp16: the 30-rectangle generator at 128^3, two right-hand
      sides, FP32 finest and FP16 row-scaled coarse levels.
"""
import dataclasses
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2206_03203_gb300 import inputs  # noqa: E402

REPLICATES = 2
PREC = {"fp64": 64, "fp32": 32, "bf16": 16, "fp16": 17}


def perturbed(inst, r):
    if r == 0:
        return inst
    e = np.where(np.random.default_rng(1000 + r).random(inst.km.shape[0]) < 0.5, -1.0, 1.0)
    return dataclasses.replace(inst, km=inst.km * (1.0 + e * 2.0 ** -52))


def packed(insts):
    import scipy.sparse as sp
    parts = [oracle.assemble(i) for i in insts]
    blocks = [oracle.split(A, i.n_m) for (A, _), i in zip(parts, insts)]
    A = sp.bmat([[sp.block_diag([b[0] for b in blocks]), sp.block_diag([b[1] for b in blocks])],
                 [sp.block_diag([b[2] for b in blocks]), sp.block_diag([b[3] for b in blocks])]], format="csr")
    A.sort_indices()
    nm = sum(i.n_m for i in insts)
    b = np.stack([np.concatenate([p[1][r][:i.n_m] for p, i in zip(parts, insts)] +
                                 [p[1][r][i.n_m:] for p, i in zip(parts, insts)]) for r in range(insts[0].nrhs)])
    mo = np.cumsum([0] + [i.n_m for i in insts])
    fo = np.cumsum([0] + [i.n_f for i in insts])
    return A, b, nm, mo, fo


def job(task):
    """One oracle solve (or, for the packed batch, every problem of one
    right-hand side); returns (key, replicate, counts)."""
    oracle.build()
    kind, key, r, arg = task
    if kind == "single":
        inst, prec, rhs = arg
        inst = perturbed(inst, r)
        A, b = oracle.assemble(inst)
        M = oracle.ML(A, inst.n_m, prec=PREC[prec])
        return key, r, [oracle.fgmres(A, b[c], M, rtol=1e-8, maxit=5000).iterations for c in range(rhs)]
    insts, prec, col = arg
    insts = [perturbed(i, r) for i in insts]
    A, b, nm, mo, fo = packed(insts)
    M = oracle.ML(A, nm, segments=(mo, fo), prec=PREC[prec])
    out = []
    for k in range(len(insts)):
        rows = np.r_[mo[k]:mo[k + 1], nm + fo[k]:nm + fo[k + 1]]
        be = np.zeros(A.shape[0])
        be[rows] = b[col][rows]
        out.append(oracle.fgmres(A, be, M, rtol=1e-8, maxit=5000).iterations)
    return key, r, out


def tasks():
    t = []
    for kf in (1e-4, 1.0, 1e4):
        inst = inputs.planes_3d(128, kf=kf)
        for prec in ("fp64", "fp32"):
            for r in range(REPLICATES + 1):
                t.append(("single", f"planes3d_128/kf={kf:g}/{prec}", r, (inst, prec, 1)))
    sub = [inputs.batch_instance(i, 256) for i in range(8)]
    for col in range(4):
        for r in range(REPLICATES + 1):
            t.append(("packed", f"batch8_bf16/col{col}", r, (sub, "bf16", col)))
    big = inputs.large_3d(128, nrhs=2)
    for r in range(REPLICATES + 1):
        t.append(("single", "large3d_128_fp16", r, (big, "fp16", 2)))
    return t


if __name__ == "__main__":
    oracle.build()
    T = tasks()
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        res = pool.map(job, T, chunksize=1)
    out = {}
    for key, r, counts in res:
        e = out.setdefault(key, {"oracle": None, "perturbed": []})
        if r == 0:
            e["oracle"] = counts
        else:
            e["perturbed"].append(counts)
    for e in out.values():
        allc = [e["oracle"]] + e["perturbed"]
        e["min"] = [min(c[i] for c in allc) for i in range(len(e["oracle"]))]
        e["max"] = [max(c[i] for c in allc) for i in range(len(e["oracle"]))]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_iterations.json")
    json.dump({"about": "oracle FGMRES(30) counts to rtol 1e-8 with M_L; min / max over the input and "
                        f"{REPLICATES} replicates with k_m moved by one unit in the last place; "
                        "make_fullsize_iterations.py", "cases": out}, open(path, "w"), indent=1)
    print(json.dumps(out))
