"""Placement of independent solves on ranks (one process per GPU).

The block solver couples nothing across instances: a batch of separate
mixed-dimensional problems (a parameter sweep over fracture permeability, or
many fracture networks, as in the paper's Sec. 4 studies) is a set of
independent linear systems.  Ranks therefore take disjoint subsets of the
instances and exchange no data on the solve path.  After the timed region the
ranks combine two numbers once: the slowest rank's time (max) and the number
of solves (sum).

A single instance is not split: a domain-decomposed solve would need halo
exchanges in every SpMV and smoother sweep and global reductions in every
Arnoldi step, which this solver does not do; several GPUs run replicas.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard_by_work(work: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time-first placement of instances on `world` ranks.

    Instances are taken in descending work (ties by ascending index) and each
    goes to the rank with the least work so far (ties to the lower rank).
    Returns, per rank, the ascending list of instance indices.  The result is
    a partition of range(len(work)); with world >= 1 the most loaded rank
    carries at most the mean load plus the largest single item.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(work[i])
    return [sorted(s) for s in out]


def instance_work(n_m: int, n_f: int) -> float:
    """Work estimate of one instance: its unknown count.  Iteration counts
    are not known before the solve; every kernel on the path is linear in the
    unknowns (and in the nonzeros, which track them on these stencils)."""
    return float(n_m + n_f)


def reduce_over_ranks(seconds: float, solves: float) -> Tuple[float, float]:
    """(max over ranks of seconds, sum over ranks of solves).

    Uses the default torch.distributed process group when one is initialised
    (NCCL on GPUs, gloo on CPU); returns the inputs unchanged otherwise.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(solves)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(solves)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())
