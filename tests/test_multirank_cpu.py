"""Multi-rank host logic on CPU (gloo, world size 2).

One process per GPU: independent instances are placed on ranks by
`sharding.shard_by_work` and the timed results are combined once by
`sharding.reduce_over_ranks` (max of times, sum of solves).  These tests run
two gloo ranks on the CPU; no GPU and no collective on the solve path.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2206_03203_gb300 import inputs, sharding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_by_work_partitions_and_balances():
    rng = np.random.default_rng(5)
    work = list(rng.integers(1, 1000, size=97).astype(float))
    for world in (1, 2, 3, 8, 128):
        sh = sharding.shard_by_work(work, world)
        assert len(sh) == world
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(work)))  # a partition
        loads = [sum(work[i] for i in s) for s in sh]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(work) / world + max(work) + 1e-9
        assert all(s == sorted(s) for s in sh)
    # deterministic, and equal work goes round-robin by index
    assert sharding.shard_by_work([1.0] * 4, 2) == [[0, 2], [1, 3]]
    assert sharding.shard_by_work([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        sharding.shard_by_work([1.0], 0)


def test_shard_batch_instances():
    """The 256-instance batch splits into two shards whose unknown counts
    differ by less than the largest instance."""
    sizes = inputs.batch_sizes(22060304, 256)
    work = [float(n ** 3) for n in sizes]
    a, b = sharding.shard_by_work(work, 2)
    la, lb = sum(work[i] for i in a), sum(work[i] for i in b)
    assert abs(la - lb) <= max(work)
    assert len(a) + len(b) == 256


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = [float(3 + (i * 7) % 11) for i in range(20)]
        shard = sharding.shard_by_work(work, world)[rank]
        # each rank "solves" its shard: time proportional to its work
        seconds = 0.5 + sum(work[i] for i in shard) / 100.0
        t, solves = sharding.reduce_over_ranks(seconds, len(shard))
        gathered = [None] * world
        dist.all_gather_object(gathered, shard)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"t": t, "solves": solves, "seconds": seconds, "shard": shard, "all": gathered}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # every rank sees the same combined numbers
    assert rs[0]["t"] == rs[1]["t"] == max(r["seconds"] for r in rs)
    assert rs[0]["solves"] == rs[1]["solves"] == 20
    # the shards gathered on each rank agree and partition the instances
    assert rs[0]["all"] == rs[1]["all"]
    assert sorted(i for s in rs[0]["all"] for i in s) == list(range(20))
    assert rs[0]["shard"] == rs[0]["all"][0] and rs[1]["shard"] == rs[1]["all"][1]


def _solve_rank_main(rank, world, port, out_dir):
    """One gloo rank: solve this rank's shard of a small uneven 3D batch with
    the oracle (assembly, M_L set-up, FGMRES(30) to 1e-8 for every
    right-hand side), then gather every rank's per-instance results."""
    import pickle

    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = inputs.batch_3d(count=6, lo=8, hi=12, nrhs=2)
        work = [sharding.instance_work(b.n_m, b.n_f) for b in batch]
        shard = sharding.shard_by_work(work, world)[rank]
        local = {}
        for i in shard:
            A, b = oracle.assemble(batch[i])
            M = oracle.ML(A, batch[i].n_m)
            res = [oracle.fgmres(A, b[k], M, rtol=1e-8, maxit=500) for k in range(b.shape[0])]
            local[i] = ([r.x for r in res], [r.iterations for r in res])
        t, solves = sharding.reduce_over_ranks(1.0 + rank, sum(len(v[1]) for v in local.values()))
        gathered = [None] * world
        dist.all_gather_object(gathered, local)
        with open(os.path.join(out_dir, f"solve{rank}.pkl"), "wb") as f:
            pickle.dump({"shard": shard, "all": gathered, "t": t, "solves": solves}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_solve_their_shards(tmp_path, oracle_mod):
    """Instance sharding with real solves: two gloo ranks each solve their
    shard of a six-instance batch with the oracle; the gathered solutions and
    iteration counts equal, bit for bit, those of one process solving every
    instance (the instances are independent and the oracle is sequential)."""
    import pickle
    world = 2
    mp.start_processes(_solve_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rs = [pickle.load(open(tmp_path / f"solve{r}.pkl", "rb")) for r in range(world)]
    assert all(len(r["shard"]) > 0 for r in rs)  # both ranks had work
    assert rs[0]["t"] == rs[1]["t"] == 2.0 and rs[0]["solves"] == rs[1]["solves"] == 12
    merged = {}
    for part in rs[0]["all"]:
        assert not set(part) & set(merged)  # no instance solved twice
        merged.update(part)
    assert sorted(merged) == list(range(6))
    batch = inputs.batch_3d(count=6, lo=8, hi=12, nrhs=2)
    for i, inst in enumerate(batch):
        A, b = oracle_mod.assemble(inst)
        M = oracle_mod.ML(A, inst.n_m)
        xs, its = merged[i]
        for k in range(b.shape[0]):
            ref = oracle_mod.fgmres(A, b[k], M, rtol=1e-8, maxit=500)
            assert ref.converged and its[k] == ref.iterations
            assert np.array_equal(xs[k], ref.x), (i, k)


def test_reduce_without_process_group_is_identity():
    assert sharding.reduce_over_ranks(1.25, 7) == (1.25, 7.0)


def test_reference_arm_other_ranks_exit_without_work(tmp_path):
    """Under torchrun the reference arm runs on rank 0 only; rank 1 prints
    nothing and exits 0 without building or running the oracle."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, cwd=str(tmp_path), capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
