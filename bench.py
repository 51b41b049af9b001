"""Benchmark: solves/s of the block-preconditioned FGMRES solver to 1e-8.

Headline workload (one step): 256 uneven 3D instances (cube side n ~ U{32..64},
1-12 random axis-aligned rectangular fractures each, log10 k_f ~ U(-4, 4),
log-normal k_m with sigma = 1), each with 4 random-Dirichlet right-hand sides:
1,024 solves.  A step packs the instances into one block-diagonal system:
GPU two-point-flux assembly from device-resident instance arrays, the Schur
complement S~ and both AMG hierarchies (FP32 finest level, BF16 row-scaled
coarse levels), and lockstep FP64 FGMRES(30) with M_L on the four interleaved
columns of every instance to a relative residual of 1e-8.  value = solves per
second over the timed steps.  Beside it, the same batch with every level in
FP64 (the plain GPU solve) is timed by the same protocol, and the ratio is
reported.

Secondary line: the 2D 1024 x 1024 instance with log-normal k_m and 64
random segments swept over nine contrasts (FP64 path), with its CPU oracle
timed on the whole sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--variants] [--no-sweep]

Under torchrun the instances of the batch are sharded across ranks by unknown
count (no collective on the solve path); value sums the ranks' solves over the
slowest rank's time.  ``--impl reference`` times the CPU oracle on a bounded
sample of the same batch instead (rank 0 only).

Accuracy: the true relative residual of every solve, and for sampled instances
the relative error of the GPU solutions against a sparse direct solve
(SuperLU) of the same assembled FP64 systems on the host, finished before the
timed region starts.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/s to 1e-8 rel-res (assemble + set-up + lockstep FGMRES; 256 instances x 4 RHS)"
UNIT = "solves/s"
FP64_PEAK_TFLOPS = 1.25
NRHS = 4
BATCH = 256
WORKLOAD = ("3D batch: 256 uneven instances (n ~ U{32..64}, 1-12 random rectangles, log10 k_f ~ U(-4,4), "
            "log-normal k_m sigma=1), 4 random-Dirichlet RHS each = 1,024 solves; packed TPFA assembly, S~, "
            "AMG (FP32 finest, BF16 row-scaled coarse), lockstep FP64 FGMRES(30) + M_L to rtol 1e-8")
SWEEP_WORKLOAD = ("2D 1024x1024 TPFA, log-normal k_m sigma=1, 64 random segments (k_f = c / 1/c, a = 1e-4), "
                  "contrast sweep c = 1e-4..1e4 (9 solves per step), FP64 FGMRES(30) + M_L, rtol 1e-8")
# approximate FGMRES iterations per contrast member of the sweep (for ordering)
SWEEP_WORK = [1700, 1420, 1610, 645, 226, 505, 1006, 1180, 1770]
CLASSES = ["spmv", "vc_resid", "vc_post", "vc_restrict", "gs_dot", "gs_axpy"]


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel_class: str, workload: str, avg_alg_bytes: float):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic.txt lines: '<class> <workload> <dram bytes> <algorithmic
    bytes of that launch>'), scaled to this run's average launch by the ratio
    of algorithmic bytes."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel_class and f[1] == workload:
            try:
                return float(f[2]) / float(f[3]) * avg_alg_bytes
            except (ValueError, ZeroDivisionError):
                return None
    return None


def _direct_instance(indptr, indices, data, B):
    """Sparse LU (SuperLU, COLAMD ordering) of one assembled FP64 system on the
    host, applied to every right-hand side row of B: the direct solutions the
    GPU results are compared with."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = sp.csc_matrix(sp.csr_matrix((data, indices, indptr), shape=(len(indptr) - 1,) * 2))
    lu = spla.splu(A, permc_spec="COLAMD")
    return np.stack([lu.solve(b) for b in B])


def class_rates(ctx, fn, peak, classes=CLASSES):
    """Per-class launch averages of one run of fn() with every launch of each
    class bracketed by events: achieved HBM GB/s and FP64 TFLOP/s, and each
    class's share of the bracketed time."""
    for c in classes:
        ctx.timing_enable(c, True)
    ctx.timing_sample_every(1)
    ctx.timing_reset()
    fn()
    out, tot = {}, 0.0
    for c in classes:
        n_t, ms_t, by_t, fl_t = ctx.timing_sampled(c)
        ctx.timing_enable(c, False)
        if n_t and ms_t > 0:
            gbs = by_t / (ms_t / 1e3) / 1e9
            tf = fl_t / (ms_t / 1e3) / 1e12
            out[c] = {"launches": n_t, "ms_total": round(ms_t, 3), "avg_launch_us": round(ms_t / n_t * 1e3, 2),
                      "algorithmic_bytes_per_launch": by_t / n_t, "hbm_gbs": round(gbs, 1),
                      "hbm_frac_of_measured": round(gbs / peak, 4), "fp64_tflops": round(tf, 4),
                      "fp64_frac_of_nominal": round(tf / FP64_PEAK_TFLOPS, 4)}
            tot += ms_t
    for c in out:
        out[c]["time_share"] = round(out[c]["ms_total"] / tot, 4) if tot else None
    return out


def roofline_of(ctx, cls, peak, peak_src, workload):
    """The roofline entry of one class from its launches bracketed since the
    last timing reset."""
    kl, kms, kbytes, kflops = ctx.timing_sampled(cls)
    avg_ms = kms / max(kl, 1)
    avg_bytes = kbytes / max(kl, 1)
    avg_flops = kflops / max(kl, 1)
    gbs = avg_bytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else None
    tflops = avg_flops / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else None
    hbm_frac = gbs / peak if gbs else None
    alu_frac = tflops / FP64_PEAK_TFLOPS if tflops else None
    if alu_frac and hbm_frac and alu_frac > hbm_frac:
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                "frac": alu_frac, "peak_source": "derived: 152 SMs x 2070 MHz x 4 FP64 flops per clock per SM "
                "(GB300 nominal 1.25 TFLOP/s; a dependent-FMA probe measured 1.20)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": hbm_frac,
                "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s"}
    roof.update({"traffic": profile_traffic(cls, workload, avg_bytes), "kernel_class": cls,
                 "algorithmic_bytes_per_launch": avg_bytes, "algorithmic_flops_per_launch": avg_flops,
                 "launches_timed": kl, "avg_launch_ms": avg_ms, "hbm_gbs": gbs, "hbm_frac_of_measured": hbm_frac,
                 "fp64_tflops": tflops, "fp64_frac_of_nominal": alu_frac})
    return roof


def _step_times(step, flush, steps):
    """Device-timed seconds of each of `steps` calls of step() (CUDA events on
    the current stream, L2 flushed by a 256 MB write before each)."""
    import torch
    out = []
    for s_ in range(steps):
        flush.fill_(float(s_))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(s_ == steps - 1)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / 1e3)
    return out


def run_gpu(args):
    import dataclasses

    import torch
    import torch.distributed as dist

    from paper_2206_03203_gb300 import build, inputs, mdsolve, sharding

    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    build.build()
    ctx = mdsolve.Context(local)
    peak, peak_src = measured_peaks()
    all_idx = list(range(BATCH))
    sizes = inputs.batch_sizes(22060304, BATCH)
    if world > 1:
        # instances are independent: each rank solves its own share, no exchange
        all_idx = sharding.shard_by_work([float(n ** 3) for n in sizes], world)[rank]
    batch = [inputs.batch_instance(i, BATCH) for i in all_idx]
    dev = [mdsolve.device_arrays(b) for b in batch]  # inputs resident in HBM before timing
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sopt = dict(rtol=1e-8, max_iters=5000, restart=30, nrhs=NRHS)
    s0 = ctx.assemble_batch(batch, device_arrays=dev)
    N, n_m, n_f = s0.N, s0.n_m, s0.n_f
    s0.close()
    x = torch.zeros(N * NRHS, dtype=torch.float64, device="cuda")
    last = {}
    phase_ev = []

    def make_step(prec):
        def step(collect=False):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if collect else None
            if ev:
                ev[0].record()
            s = ctx.assemble_batch(batch, device_arrays=dev)
            if ev:
                ev[1].record()
            p = ctx.setup(s, precision=prec, format="auto")
            if ev:
                ev[2].record()
            x.zero_()
            code, st = ctx.solve(s, p, None, x, **sopt)
            if ev:
                ev[3].record()
                phase_ev[:] = [ev]
            if code != 0:
                raise RuntimeError(f"batch solve ({prec}) returned {code}")
            if collect:
                last[prec] = (st, [p.info(0)["n"], p.info(1)["n"]])
            p.close()
            s.close()
        return step

    # direct references for sampled instances (host SuperLU in spawned
    # processes), finished before any timed step
    direct = {}
    if rank == 0 and not args.no_direct:
        import multiprocessing as mp
        pick = [k for k, b in enumerate(batch) if b.n <= 40][:4]
        jobs = []
        pool = mp.get_context("spawn").Pool(max(1, len(pick)))
        for k in pick:
            s = ctx.assemble(batch[k])
            (_, _, _, _, Ah), bh = s.to_host()
            s.close()
            jobs.append((k, pool.apply_async(_direct_instance, (Ah.indptr, Ah.indices, Ah.data, bh)), Ah, bh))
        for k, job, Ah, bh in jobs:
            try:
                direct[k] = (job.get(timeout=900), Ah, bh)
            except Exception as e:  # reported, never fatal
                direct[k] = (e, Ah, bh)
        pool.terminate()

    # ---- mixed-precision batch (the headline) ----
    step = make_step("bf16")
    step()  # first warm-up: storage autotuning, allocations
    classes_bf16 = class_rates(ctx, step, peak)  # second warm-up, every class bracketed
    share = {c: v["ms_total"] for c, v in classes_bf16.items()}
    dominant = max(share, key=share.get)
    for _ in range(max(0, args.warmup - 2)):
        step()
    torch.cuda.synchronize()
    for c in CLASSES:
        ctx.timing_enable(c, c == dominant)
    ctx.timing_sample_every(1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.timing_reset()
    launches0 = ctx.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    step_s = _step_times(step, flush, args.steps)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    roof = roofline_of(ctx, dominant, peak, peak_src, "batch3d-256")
    for c in CLASSES:
        ctx.timing_enable(c, False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_total, solves = sharding.reduce_over_ranks(sum(step_s), len(batch) * NRHS * args.steps)
    value = solves / t_total
    st_bf16, levels_bf16 = last["bf16"]
    its = [q.iterations for q in st_bf16]
    dof = [(b.n_m + b.n_f) for b in batch for _ in range(NRHS)]
    ph = phase_ev[0]
    phases = {"assemble_ms": ph[0].elapsed_time(ph[1]), "setup_ms": ph[1].elapsed_time(ph[2]),
              "solve_ms": ph[2].elapsed_time(ph[3])}
    phases["solve_only_solves_per_s"] = len(batch) * NRHS / (phases["solve_ms"] / 1e3)
    phases["dof_iter_per_s_solve_only"] = sum(d * i for d, i in zip(dof, its)) / (phases["solve_ms"] / 1e3)
    x_last = x.cpu().numpy().reshape(NRHS, N)

    # accuracy: every solve's true residual; sampled instances against direct
    accuracy = {"relres_true_max": max(q.relres_true for q in st_bf16),
                "relres_true_min": min(q.relres_true for q in st_bf16),
                "all_converged": all(q.status == 0 for q in st_bf16)}
    if direct:
        mo, fo = 0, 0
        offs = []
        for b in batch:
            offs.append((mo, fo))
            mo += b.n_m
            fo += b.n_f
        rows_of = {k: np.r_[offs[k][0]:offs[k][0] + batch[k].n_m, n_m + offs[k][1]:n_m + offs[k][1] + batch[k].n_f]
                   for k in direct}
        errs = {}
        for k, (xd, Ah, bh) in direct.items():
            if isinstance(xd, Exception):
                errs[int(all_idx[k])] = {"error": str(xd)}
                continue
            e = []
            for c in range(NRHS):
                xg = x_last[c][rows_of[k]]
                e.append({"rel_error": float(np.linalg.norm(xg - xd[c]) / np.linalg.norm(xd[c])),
                          "relres_direct": float(np.linalg.norm(bh[c] - Ah @ xd[c]) / np.linalg.norm(bh[c])),
                          "relres_gpu": float(np.linalg.norm(bh[c] - Ah @ xg) / np.linalg.norm(bh[c]))})
            errs[int(all_idx[k])] = e
        accuracy["vs_direct"] = {"instances": errs, "direct": "scipy splu (SuperLU, COLAMD) of each sampled "
                                 "instance's assembled FP64 system on the host; finished before the timed steps"}

    # ---- the same batch, FP64 throughout (the plain GPU solve), same protocol ----
    step64 = make_step("fp64")
    step64()
    classes_fp64 = class_rates(ctx, step64, peak)
    step64()
    k64 = max(10, min(args.steps, 10))
    if world > 1:
        dist.barrier()
    s64 = _step_times(step64, flush, k64)
    t64, solves64 = sharding.reduce_over_ranks(sum(s64), len(batch) * NRHS * k64)
    value64 = solves64 / t64
    st64, _ = last["fp64"]

    # ---- end to end through the C ABI with host buffers ----
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    batch_h = [dataclasses.replace(b, km=pinned(b.km), fc_axis=pinned(b.fc_axis), fc_pos=pinned(b.fc_pos),
                                   fc_kf=pinned(b.fc_kf), fc_a=pinned(b.fc_a), pD_left=pinned(b.pD_left),
                                   pD_right=pinned(b.pD_right)) for b in batch]
    xh = pinned(np.zeros(N * NRHS))

    def e2e_step():
        s = ctx.assemble_batch(batch_h)
        p = ctx.setup(s, precision="bf16", format="auto")
        code, _ = ctx.solve(s, p, None, xh, x0_zero=True, **sopt)  # x is output only
        p.close()
        s.close()
        if code != 0:
            raise RuntimeError(f"end-to-end batch solve returned {code}")

    # untimed warm-up steps: the first host-array step grows the context's
    # memory pool for the staged inputs and the host solution
    e2e_warmup, e2e_steps = 2, 3
    for _ in range(e2e_warmup):
        e2e_step()
    e2e_t = 0.0
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_t += time.perf_counter() - t0
    # one more step with a synchronisation after each phase: where the
    # end-to-end time goes (not part of the value)
    e2e_phases = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s_ = ctx.assemble_batch(batch_h)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    p_ = ctx.setup(s_, precision="bf16", format="auto")
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ctx.solve(s_, p_, None, xh, x0_zero=True, **sopt)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    p_.close()
    s_.close()
    t4 = time.perf_counter()
    e2e_phases = {"assemble_from_host_ms": (t1 - t0) * 1e3, "setup_ms": (t2 - t1) * 1e3,
                  "solve_to_host_ms": (t3 - t2) * 1e3, "release_ms": (t4 - t3) * 1e3}
    h2d = sum(b.km.nbytes + b.fc_axis.nbytes + b.fc_pos.nbytes + b.fc_kf.nbytes + b.fc_a.nbytes +
              b.pD_left.nbytes + b.pD_right.nbytes for b in batch)
    d2h = 8 * N * NRHS
    e2e_t, e2e_solves = sharding.reduce_over_ranks(e2e_t, len(batch) * NRHS * e2e_steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64+f32+bf16",
        "data": "synthetic (seeded generator; stands in for the paper's parameter studies of Sec. 4)",
        "config": {"workload": WORKLOAD, "precision": "FP64 assembly / set-up / FGMRES; FP32 finest V-cycle "
                   "level, BF16 row-scaled coarse levels", "nrhs_per_instance": NRHS,
                   "instances": len(batch) * world if world > 1 else len(batch), "N_packed": N,
                   "l2": "flushed between steps (256 MB write); inputs and working set far above the 129 MB L2",
                   "parallelism": f"instances sharded over {world} rank(s) by unknown count" if world > 1
                   else "one GPU, one packed batch"},
        "step_s": {"median": float(np.median(step_s)), "min": float(np.min(step_s)), "all": step_s},
        "dof_iter_per_s": sum(d * i for d, i in zip(dof, its)) * args.steps * world / t_total,
        "iterations": {"min": min(its), "mean": float(np.mean(its)), "max": max(its)},
        "phases_last_step": phases,
        "levels_last_step": levels_bf16,
        "fp64_batch": {"value": value64, "unit": UNIT, "steps": k64,
                       "step_s": {"median": float(np.median(s64)), "min": float(np.min(s64))},
                       "speedup_mixed_over_fp64": value / value64,
                       "iterations": {"min": min(q.iterations for q in st64),
                                      "mean": float(np.mean([q.iterations for q in st64])),
                                      "max": max(q.iterations for q in st64)},
                       "relres_true_max": max(q.relres_true for q in st64)},
        "classes": {"bf16": classes_bf16, "fp64": classes_fp64,
                    "note": "every launch of each class bracketed by events in one warm-up step; vc_* are the "
                            "finest-level V-cycle kernels of the S~ and A_ff hierarchies"},
        "accuracy": accuracy,
        "roofline": roof,
        "e2e": {"value": e2e_solves / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "host_buffers": "pinned; instance arrays in, 1,024 solution columns out (zero initial guess: x is "
                                "output only), every step; host clock", "steps": e2e_steps, "warmup": e2e_warmup,
                "phases_one_more_step": e2e_phases},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_sweep and rank == 0:
        line["sweep_1024"] = sweep_line(ctx, args, flush, peak, peak_src)
    if args.variants:
        insts = [inputs.random_segments_2d(contrast=c) for c in inputs.CONTRASTS]
        dev2 = [mdsolve.device_arrays(i) for i in insts]
        line["variants"] = variants(ctx, insts, dev2, [i.n_m + i.n_f for i in insts], flush)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def sweep_line(ctx, args, flush, peak, peak_src):
    """Secondary line: the nine-contrast 1024^2 sweep on the FP64 path (GPU
    assembly from device-resident arrays, set-up, FGMRES), 3 warm-up and
    min(K, 5) timed steps, with the CPU oracle timed on the whole sweep."""
    import torch

    from paper_2206_03203_gb300 import inputs, mdsolve
    insts = [inputs.random_segments_2d(contrast=c) for c in inputs.CONTRASTS]
    dev = [mdsolve.device_arrays(i) for i in insts]
    xs = [torch.zeros(i.n_m + i.n_f, dtype=torch.float64, device="cuda") for i in insts]
    its = []

    def step(collect=False):
        its.clear()
        for k, inst in enumerate(insts):
            s = ctx.assemble(inst, device_arrays=dev[k])
            p = ctx.setup(s, precision="fp64", format="stencil")
            xs[k].zero_()
            code, st = ctx.solve(s, p, None, xs[k], rtol=1e-8, max_iters=5000)
            if code != 0:
                raise RuntimeError(f"sweep solve failed at contrast {inputs.CONTRASTS[k]}")
            its.append(st[0].iterations)
            p.close()
            s.close()
    for _ in range(3):
        step()
    for c in CLASSES:
        ctx.timing_enable(c, c == "gs_axpy")
    ctx.timing_sample_every(4)
    ctx.timing_reset()
    k = max(1, min(args.steps, 5))
    ts = _step_times(step, flush, k)
    roof = roofline_of(ctx, "gs_axpy", peak, peak_src, "seg2d-1024")
    for c in CLASSES:
        ctx.timing_enable(c, False)
    out = {"workload": SWEEP_WORKLOAD, "value": len(insts) * k / sum(ts), "unit": UNIT, "steps": k, "warmup": 3,
           "step_s": {"median": float(np.median(ts)), "min": float(np.min(ts))},
           "iterations_per_contrast": list(its),
           "storage": "finest S~ level by stencil planes, CSR elsewhere (fixed formats: bitwise reproducible counts, "
                      "equal to CSR storage bit for bit)",
           "roofline_gs_axpy": roof}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sweep()
    return out


def _oracle_batch_instance(i):
    """The oracle on instance i of the batch: assembly, M_L set-up (FP64) and
    FGMRES(30) to 1e-8 for each of its right-hand sides; (seconds, counts)."""
    import oracle
    from paper_2206_03203_gb300 import inputs
    oracle.build()
    inst = inputs.batch_instance(i, BATCH)
    t0 = time.perf_counter()
    A, b = oracle.assemble(inst)
    M = oracle.ML(A, inst.n_m)
    its = []
    for r in range(b.shape[0]):
        res = oracle.fgmres(A, b[r], M, rtol=1e-8, maxit=5000)
        its.append(res.iterations)
    return time.perf_counter() - t0, its


def cpu_baseline_batch():
    """The oracle (plain sequential FP64 C, as it stands) on a bounded sample of
    the batch: 16 of its instances (every 16th), each assembled, set up and
    solved for its 4 right-hand sides, one process per host core at once."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    sample = list(range(0, BATCH, 16))
    cores = min(os.cpu_count() or 1, len(sample))
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        rs = pool.map(_oracle_batch_instance, sample)
        dt = time.perf_counter() - t0
    its = [i for _, r in rs for i in r]
    return {"value": len(sample) * NRHS / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} instances of the batch (every 16th), {len(sample) * NRHS} solves "
                      f"(assembly + FP64 M_L set-up per instance + FGMRES(30) to 1e-8 per right-hand side), "
                      f"one single-threaded oracle process per core; the oracle sets up each instance on its own "
                      f"(the GPU sets up the packed batch)",
            "wall_s": dt, "cpu_seconds": float(sum(t for t, _ in rs)),
            "iterations": {"min": min(its), "mean": float(np.mean(its)), "max": max(its)},
            "cpu": platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def _oracle_sweep_member(k):
    import oracle
    from paper_2206_03203_gb300 import inputs
    oracle.build()
    inst = inputs.random_segments_2d(contrast=inputs.CONTRASTS[k])
    t0 = time.perf_counter()
    res, *_ = oracle.solve(inst, maxit=5000)
    return time.perf_counter() - t0, res.iterations


def cpu_baseline_sweep():
    """The oracle on the whole nine-contrast sweep: nine single-threaded
    processes at once (one per contrast), wall time of the slowest."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = min(os.cpu_count() or 1, 9)
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        rs = pool.map(_oracle_sweep_member, range(9))
        dt = time.perf_counter() - t0
    return {"value": 9 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "the whole sweep (nine contrasts), one single-threaded oracle process per contrast",
            "wall_s": dt, "iterations_per_contrast": [i for _, i in rs]}


def run_reference(args):
    """The reference arm: the CPU oracle on a bounded sample of the batch (16
    instances, every 16th, 4 right-hand sides each), one process per host core;
    each step solves the sample once."""
    rank, _, world = rank_info()
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle
    oracle.build()
    sample = list(range(0, BATCH, 16))
    cores = min(os.cpu_count() or 1, len(sample))
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_batch_instance, sample[:cores])
        t = 0.0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rs = pool.map(_oracle_batch_instance, sample)
            t += time.perf_counter() - t0
    its = [i for _, r in rs for i in r]
    value = len(sample) * NRHS * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)", "parallelism": f"CPU oracle, {cores} processes",
                   "sample_iterations": {"min": min(its), "mean": float(np.mean(its)), "max": max(its)}},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one step = {len(sample)} instances of the batch (every 16th) x 4 right-hand "
                                   "sides, assembly + FP64 M_L set-up + FGMRES(30) to 1e-8, one single-threaded "
                                   "oracle process per core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)



def _timed(fn, flush, warmup=1, steps=1):
    """Device-timed seconds per step of fn() (CUDA events, L2 flushed before
    each step)."""
    import torch
    for _ in range(warmup):
        fn()
    tot = 0.0
    out = None
    for _ in range(steps):
        flush.fill_(0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    return tot / steps, out


def class_rates_every4(ctx, fn, classes=("spmv", "vc_resid", "vc_post", "vc_restrict", "gs_dot", "gs_axpy")):
    """Per-class launch averages of one run of fn() (events around every 4th
    restart cycle): achieved HBM GB/s and FP64 TFLOP/s against the peaks."""
    peak, _ = measured_peaks()
    for c in classes:
        ctx.timing_enable(c, True)
    ctx.timing_sample_every(4)
    ctx.timing_reset()
    fn()
    out = {}
    for c in classes:
        n_t, ms_t, by_t, fl_t = ctx.timing_sampled(c)
        ctx.timing_enable(c, False)
        if n_t and ms_t > 0:
            gbs = by_t / (ms_t / 1e3) / 1e9
            out[c] = {"avg_launch_us": round(ms_t / n_t * 1e3, 3), "algorithmic_bytes_per_launch": by_t / n_t,
                      "hbm_gbs": round(gbs, 1), "hbm_frac_of_measured": round(gbs / peak, 4),
                      "fp64_tflops": round(fl_t / (ms_t / 1e3) / 1e12, 4)}
    return out


def vcycle_rate(ctx, inst, dev, flush, reps: int = 20):
    """One application of M_L (Algorithm 1: V-cycle on S~, A_fm SpMV, V-cycle
    on A_ff) on the contrast-1e4 member, FP64 and FP32 hierarchies: median
    event time over `reps` applications with L2 flushed before each, and the
    algorithmic bytes of the application -- per non-dense level the matrix
    read twice (residual and post-smoothing), about eight vector passes and
    the aggregate map, the dense coarsest inverse once, and the A_fm SpMV."""
    import torch
    peak, _ = measured_peaks()
    s = ctx.assemble(inst, device_arrays=dev)
    n_m, n_f, nnz_fm = s.n_m, s.n_f, s.nnz[2]
    out = {}
    for prec, bv, bx in (("fp64", 8, 8), ("fp32", 4, 4)):
        p = ctx.setup(s, precision=prec, format="auto")
        total = 0.0
        for blk in (0, 1):
            info = p.info(blk)
            last = len(info["n"]) - 1
            for l, (n_l, z_l) in enumerate(zip(info["n"], info["nnz"])):
                if l == last and info["dense"]:
                    total += 8.0 * n_l * n_l + 2 * bx * n_l
                elif l == last and info.get("diagonal"):
                    total += 3 * bx * n_l
                else:
                    total += 2 * ((bv + 4) * z_l + 4 * (n_l + 1)) + 8 * bx * n_l + 4 * n_l
        total += 12.0 * nnz_fm + 4.0 * (n_f + 1) + 8.0 * (n_m + 2 * n_f)
        r = torch.randn(s.N, dtype=torch.float64, device="cuda")
        z = torch.zeros_like(r)
        for _ in range(3):
            ctx.precond_apply(p, r, z)
        ts = []
        for _ in range(reps):
            flush.fill_(0.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.precond_apply(p, r, z)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = float(np.median(ts))
        out[prec] = {"us_per_application": t * 1e6, "algorithmic_bytes": total, "hbm_gbs": total / t / 1e9,
                     "hbm_frac_of_measured": total / t / 1e9 / peak,
                     "levels": [p.info(0)["n"], p.info(1)["n"]]}
        p.close()
    s.close()
    return out


def variants(ctx, insts, dev_arrays, N, flush):
    """Secondary measurements (not the headline): the FP32 V-cycle path on the
    same sweep, the nine-plane 3D instance, and the 256-instance batch."""
    import torch

    from paper_2206_03203_gb300 import inputs, mdsolve, sharding
    out = {}

    def mdsolve_ctx(stream):
        return mdsolve.Context(torch.cuda.current_device(), stream=stream)

    def sweep(prec, krylov="fgmres", form="primal", **setup):
        its = []
        for k, inst in enumerate(insts):
            s = ctx.assemble(inst, device_arrays=dev_arrays[k], form=form)
            p = ctx.setup(s, precision=prec, format="auto", **setup)
            x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
            try:
                code, st = ctx.solve(s, p, None, x, rtol=1e-8, max_iters=5000, krylov=krylov)
                its.append(st[0].iterations if code == 0 else f"{st[0].iterations} (not converged)")
            except Exception as e:  # a variant that breaks down is reported, not fatal
                its.append(f"error: {e}")
            p.close()
            s.close()
        return its

    t, its = _timed(lambda: sweep("fp32"), flush)
    out["seg2d_1024_sweep_fp32_vcycle"] = {"solves_per_s": len(insts) / t, "s_per_step": t, "iterations": its,
                                           "precision": "FP32 V-cycle values/vectors, FP64 FGMRES",
                                           "classes": class_rates_every4(ctx, lambda: sweep("fp32"))}
    t, its = _timed(lambda: sweep("fp64", prolongation="smoothed"), flush)
    out["seg2d_1024_sweep_fp64_smoothed_aggregation"] = {
        "solves_per_s": len(insts) / t, "s_per_step": t, "iterations": its,
        "precision": "FP64 throughout; smoothed-aggregation prolongation instead of piecewise-constant"}
    # the other block preconditioners of Sec. 3.2 on the same sweep (FP64)
    for name, kw in (("block_diagonal_pcg", dict(kind="diag", krylov="pcg")),
                     ("block_diagonal_minres", dict(kind="diag", krylov="minres")),
                     ("block_upper_fgmres", dict(kind="upper", krylov="fgmres"))):
        kry = kw.pop("krylov")
        t, its = _timed(lambda kry=kry, kw=kw: sweep("fp64", krylov=kry, **kw), flush, warmup=0)
        out[f"seg2d_1024_sweep_fp64_{name}"] = {"solves_per_s": len(insts) / t, "s_per_step": t, "iterations": its}
    # the same sweep with the nine solves spread over four library contexts,
    # each on its own CUDA stream and host thread (longest solves first): the
    # latency-bound phases of one solve (coarse levels, host round trips)
    # overlap with the others' kernels
    import queue
    from concurrent.futures import ThreadPoolExecutor
    T = 4
    streams = [torch.cuda.Stream() for _ in range(T)]
    cts = [mdsolve_ctx(s_.cuda_stream) for s_ in streams]
    xs4 = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in N]
    torch.cuda.synchronize()

    def sweep_streams():
        q = queue.Queue()
        for k in sorted(range(len(insts)), key=lambda k: -SWEEP_WORK[k]):
            q.put(k)
        its = {}

        def worker(i):
            while True:
                try:
                    k = q.get_nowait()
                except queue.Empty:
                    return
                c_ = cts[i]
                s = c_.assemble(insts[k], device_arrays=dev_arrays[k])
                p = c_.setup(s, precision="fp64", format="auto")
                xs4[k].zero_()
                code, st = c_.solve(s, p, None, xs4[k], rtol=1e-8, max_iters=5000)
                its[k] = st[0].iterations if code == 0 else f"{st[0].iterations} (status {code})"
                p.close()
                s.close()
        with ThreadPoolExecutor(T) as ex:
            list(ex.map(worker, range(T)))
        for st_ in streams:
            st_.synchronize()
        return [its[k] for k in range(len(insts))]
    sweep_streams()
    ts = []
    for _ in range(2):
        flush.fill_(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = sweep_streams()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out["seg2d_1024_sweep_fp64_4streams"] = {
        "solves_per_s": len(insts) / min(ts), "s_per_step": min(ts), "iterations": its,
        "how": "the headline sweep, nine solves over four contexts / CUDA streams / host threads; host clock"}
    for c_ in cts:
        c_.close()

    # time-to-solution tuning of smoother / sweeps / degree / precision on the
    # contrast-1e4 member (the default candidate set of the binding)
    s = ctx.assemble(insts[-1], device_arrays=dev_arrays[-1])
    best, res = ctx.tune(s, base={"format": "auto"}, rtol=1e-8, max_iters=5000)
    out["seg2d_1024_c1e4_solver_tuning"] = {
        "best": res[best]["candidate"] if best >= 0 else None,
        "candidates": [{"smoother": r["candidate"][0], "sweeps": r["candidate"][1],
                        "cheb_degree": r["candidate"][2], "precision": r["candidate"][3], "status": r["status"],
                        "iterations": r["iterations"], "setup_ms": round(r["setup_ms"], 2),
                        "solve_ms": round(r["solve_ms"], 2)} for r in res]}
    s.close()

    # the paper's own partition (pressures of all cells; interface fluxes)
    for name, kw in (("flux_form_ML_fgmres", dict(kind="lower", krylov="fgmres")),
                     ("flux_form_smoothed_aggregation_ML_fgmres",
                      dict(kind="lower", krylov="fgmres", prolongation="smoothed")),
                     ("flux_form_block_diagonal_minres", dict(kind="diag", krylov="minres"))):
        kry = kw.pop("krylov")
        t, its = _timed(lambda kry=kry, kw=kw: sweep("fp64", krylov=kry, form="flux", **kw), flush, warmup=0)
        out[f"seg2d_1024_sweep_fp64_{name}"] = {
            "solves_per_s": len(insts) / t, "s_per_step": t, "iterations": its,
            "N": [int(n + 2 * inst.n_f) for n, inst in zip(N, insts)]}
    p3 = inputs.planes_3d(128, kf=1e4)

    def one_flux():
        s = ctx.assemble(p3, form="flux", junction="star")
        p = ctx.setup(s, precision="fp64", format="auto")
        x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(s, p, None, x, rtol=1e-8, max_iters=5000)
        n = s.N
        p.close()
        s.close()
        return st[0].iterations, n
    t, (it, nflux) = _timed(one_flux, flush)
    out["planes3d_128_kf1e4_fp64_flux_form_intersection_cells"] = {
        "solves_per_s": 1.0 / t, "s_per_step": t, "iterations": it, "N": nflux,
        "form": "paper's partition: pressures of all cells and 3,456 intersection cells; interface fluxes"}
    for kf, tag in ((1e-4, "kf1e-4"), (1.0, "kf1"), (1e4, "kf1e4")):
        pk = p3 if kf == 1e4 else inputs.planes_3d(128, kf=kf)
        for prec in ("fp64", "fp32"):
            def one(prec=prec, pk=pk):
                s = ctx.assemble(pk)
                p = ctx.setup(s, precision=prec, format="auto")
                x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
                code, st = ctx.solve(s, p, None, x, rtol=1e-8, max_iters=5000)
                p.close()
                s.close()
                return st[0].iterations
            t, it = _timed(one, flush)
            out[f"planes3d_128_{tag}_{prec}"] = {"solves_per_s": 1.0 / t, "s_per_step": t, "iterations": it,
                                                 "N": pk.n_m + pk.n_f}
    # 256^3 with 30 rectangles, 8 random-Dirichlet right-hand sides in lockstep,
    # FP32 finest level and FP16 row-scaled coarse levels under FP64 FGMRES
    big = inputs.large_3d(256)

    def one_big():
        s = ctx.assemble(big)
        p = ctx.setup(s, precision="fp16", format="auto")
        x = torch.zeros(s.N * 8, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(s, p, None, x, nrhs=8, rtol=1e-8, max_iters=5000)
        n = s.N
        p.close()
        s.close()
        return [q.iterations for q in st], n
    t, (its, nbig) = _timed(one_big, flush, warmup=1)
    out["large3d_256_30rects_x8rhs_fp16"] = {
        "solves_per_s": 8.0 / t, "s_per_step": t, "iterations": its, "N": nbig,
        "dof_iter_per_s": nbig * sum(its) / t,
        "precision": "FP32 finest level, FP16 row-scaled coarse levels, FP64 FGMRES; 8 columns in lockstep"}
    batch = inputs.batch_3d(256)
    world = rank_info()[2]
    if world > 1:
        # instances are independent: each rank solves its own share, no exchange
        shard = sharding.shard_by_work([sharding.instance_work(b.n_m, b.n_f) for b in batch], world)
        batch = [batch[i] for i in shard[rank_info()[0]]]

    def batched(prec):
        s = ctx.assemble_batch(batch)
        p = ctx.setup(s, precision=prec, format="auto")
        x = torch.zeros(s.N * 4, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(s, p, None, x, nrhs=4, rtol=1e-8, max_iters=5000)
        assert code == 0
        n = s.N
        p.close()
        s.close()
        return [q.iterations for q in st], n
    for prec, desc in (("bf16", "FP32 fine level, BF16 row-scaled coarse levels, FP64 FGMRES; packed lockstep batch"),
                       ("fp64", "FP64 throughout (the plain GPU solve of the same batch); packed lockstep batch")):
        t, (its, n) = _timed(lambda prec=prec: batched(prec), flush)
        t, total_solves = sharding.reduce_over_ranks(t, len(its))
        out[f"batch3d_256inst_x4rhs_{prec}"] = {
            "solves_per_s": total_solves / t, "s_per_step": t, "solves": total_solves,
            "iterations_min_mean_max": [min(its), float(np.mean(its)), max(its)], "N_packed": n, "precision": desc}
    # the same batch solved instance by instance (4 columns in lockstep each)
    def per_instance():
        its = []
        for inst in batch:
            s = ctx.assemble(inst)
            p = ctx.setup(s, precision="bf16", format="auto")
            x = torch.zeros(s.N * 4, dtype=torch.float64, device="cuda")
            code, st = ctx.solve(s, p, None, x, nrhs=4, rtol=1e-8, max_iters=5000)
            assert code == 0
            its += [q.iterations for q in st]
            p.close()
            s.close()
        return its
    t, its = _timed(per_instance, flush, warmup=0)
    t, total_solves = sharding.reduce_over_ranks(t, len(its))
    out["batch3d_256inst_x4rhs_bf16_per_instance"] = {
        "solves_per_s": total_solves / t, "s_per_step": t, "solves": total_solves,
        "iterations_min_mean_max": [min(its), float(np.mean(its)), max(its)],
        "precision": "as the packed bf16 batch, one instance (4 columns) at a time"}
    # kernel classes of the mixed-precision batch (finest level, 4 interleaved columns)
    out["batch3d_256inst_x4rhs_bf16"]["classes"] = class_rates_every4(ctx, lambda: batched("bf16"))
    return out


def run_profile_case(args):
    """A short fixed run for ncu: the contrast-1e4 member of the 1024^2 sweep
    (or, with --batch-profile K, the first K instances of the 256-instance
    batch with 4 right-hand sides), assembled, set up and solved for
    --max-iters FGMRES iterations."""
    import torch

    from paper_2206_03203_gb300 import build, inputs, mdsolve
    build.build()
    ctx = mdsolve.Context(0)
    if args.batch_profile > 0:
        batch = [inputs.batch_instance(i, BATCH) for i in range(args.batch_profile)]
        s = ctx.assemble_batch(batch)
        p = ctx.setup(s, precision=args.precision, format=args.format)
        x = torch.zeros(s.N * NRHS, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(s, p, None, x, nrhs=NRHS, rtol=1e-8, max_iters=args.max_iters)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": f"batch of {args.batch_profile}", "N": s.N,
                          "iterations_max": max(q.iterations for q in st), "launches": ctx.launch_count()}))
        return
    inst = inputs.random_segments_2d(n=args.n, contrast=1e4)
    s = ctx.assemble(inst)
    p = ctx.setup(s, precision=args.precision, format=args.format)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(s, p, None, x, rtol=1e-8, max_iters=args.max_iters)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": inst.name, "N": s.N, "iterations": st[0].iterations,
                      "relres": st[0].relres_true, "launches": ctx.launch_count()}))


def refinement_growth(columns, its):
    """Per dimension, the ratio of the iteration count on the finest grid to
    that on the coarsest (None where a count is missing), and whether it
    exceeds 2 (the growth the table is meant to flag)."""
    out = {}
    for dim in sorted({c.split()[0] for c in columns}):
        idx = [k for k, c in enumerate(columns) if c.split()[0] == dim]
        first, last = its[idx[0]], its[idx[-1]]
        ok = isinstance(first, int) and isinstance(last, int) and first > 0
        ratio = last / first if ok else None
        out[dim] = {"ratio": ratio, "over_2x": bool(ratio is not None and ratio > 2.0)}
    return out


def run_table1(args):
    """The shape of the paper's Table 1 (Sec. 4): M_L + FGMRES iteration counts
    to a relative residual of 1e-6 over tangential fracture permeability
    K_par in {1e-4, 1, 1e4} x normal permeability kappa (k_n) in {1e-4, 1,
    1e4}, k_m = 1, on three refinements of a 2D and a 3D instance, in the
    paper's partition with intersection cells and in the primal partition.
    Stand-ins for the paper's benchmark geometries: the four-fracture unit
    square (2D, a = 1e-4) and the nine-plane unit cube (3D, a = 1e-3)."""
    import dataclasses

    import torch

    from paper_2206_03203_gb300 import build, inputs, mdsolve
    build.build()
    ctx = mdsolve.Context(0)
    vals = (1e-4, 1.0, 1e4)
    geoms = [("2d", n, lambda n, kf: inputs.fixed_2d(n=n, kf=kf)) for n in (64, 128, 256)] + \
            [("3d", n, lambda n, kf: inputs.planes_3d(n, kf=kf)) for n in (16, 32, 64)]
    out = {}
    for form, junction in (("flux", "star"), ("primal", "pairwise")):
        rows = {}
        for kpar in vals:
            for kap in vals:
                its = []
                for tag, n, make in geoms:
                    inst = make(n, kpar)
                    inst = dataclasses.replace(inst, fc_kn=np.full(inst.n_f, kap))
                    s = ctx.assemble(inst, form=form, junction=junction)
                    try:
                        p = ctx.setup(s, precision="fp64", format="auto", prolongation=args.prolongation)
                    except mdsolve.MDSError as e:  # reported in the table, not fatal
                        its.append(f"set-up: {e}")
                        s.close()
                        continue
                    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
                    code, st = ctx.solve(s, p, None, x, rtol=1e-6, max_iters=5000)
                    its.append(st[0].iterations if code == 0 else None)
                    p.close()
                    s.close()
                rows[f"K_par={kpar:g} kappa={kap:g}"] = its
        cols = [f"{t} n={n}" for t, n, _ in geoms]
        out[form] = {"columns": cols, "rows": rows,
                     "refinement_growth": {k: refinement_growth(cols, v) for k, v in rows.items()}}
    print(json.dumps({"table1_shape": out, "prolongation": args.prolongation}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action="store_true", help="also run the secondary variant measurements")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1024^2 sweep line")
    ap.add_argument("--no-direct", action="store_true", help="skip the host direct solves of the accuracy check")
    ap.add_argument("--profile-case", action="store_true", help="short fixed run for ncu captures")
    ap.add_argument("--table1", action="store_true", help="iteration counts over (K_par, kappa), the shape of "
                                                           "the paper's Table 1")
    ap.add_argument("--prolongation", default="piecewise", help="AMG prolongation of --table1 (piecewise, smoothed)")
    ap.add_argument("--max-iters", type=int, default=60)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--format", default="auto", help="level storage of the profile case (auto, csr, sell)")
    ap.add_argument("--batch-profile", type=int, default=0, help="profile case: a batch of this many instances")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.table1:
        run_table1(args)
        return
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
