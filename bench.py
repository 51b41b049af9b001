"""Benchmark: solves/s of the block-preconditioned FGMRES solver to 1e-8.

Workload (one step): the 2D 1024 x 1024 instance with log-normal k_m
(sigma = 1) and 64 random axis-aligned segments, swept over the nine
contrasts 1e-4 .. 1e4 (even segments k_f = c, odd ones 1/c).  For each
contrast: GPU two-point-flux assembly from device-resident instance arrays,
Schur complement and AMG set-up, and FP64 FGMRES(30) with M_L to a relative
residual of 1e-8.  value = solves per second over the whole step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs an independent replica of the workload (a
single solve is not split across GPUs); value sums the ranks' solves over the
slowest rank's time.  ``--impl reference`` times the CPU oracle on a bounded
sample instead (rank 0 only).

Accuracy: the relative residual of every solve, and for the contrast-1e4
member the relative error of the GPU solution against a sparse direct solve
(SuperLU) of the same assembled FP64 system on the host, computed in a
separate process while the GPU runs.
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

METRIC = "solves/s to 1e-8 rel-res (assemble + set-up + FGMRES, contrast sweep)"
UNIT = "solves/s"
FP64_PEAK_TFLOPS = 1.25
# approximate FGMRES iterations per contrast member: the order (longest
# first) in which the solves are handed to concurrent streams
SWEEP_WORK = [1700, 1420, 1610, 645, 226, 505, 1006, 1180, 1770]
WORKLOAD = ("2D 1024x1024 TPFA, log-normal k_m sigma=1, 64 random segments (k_f = c / 1/c, a = 1e-4), "
            "contrast sweep c = 1e-4..1e4 (9 solves per step), FP64 FGMRES(30) + M_L, rtol 1e-8")


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


def profile_traffic(kernel_class: str, avg_alg_bytes: float):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic.txt lines: '<class> <workload> <dram bytes> <algorithmic
    bytes of that launch>'), scaled to this run's average launch by the ratio
    of algorithmic bytes."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel_class and f[1] == "seg2d-1024":
            try:
                return float(f[2]) / float(f[3]) * avg_alg_bytes
            except (ValueError, ZeroDivisionError):
                return None
    return None


def _direct_solve(indptr, indices, data, b):
    """Sparse LU (SuperLU, COLAMD ordering) of the assembled system on the
    host: the FP64 direct solution the GPU result is compared with."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = sp.csc_matrix(sp.csr_matrix((data, indices, indptr), shape=(len(indptr) - 1,) * 2))
    return spla.spsolve(A, b, permc_spec="COLAMD")


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2206_03203_gb300 import build, inputs, mdsolve, sharding

    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    build.build()
    ctx = mdsolve.Context(local)
    insts = [inputs.random_segments_2d(contrast=c) for c in inputs.CONTRASTS]
    # device-resident instance arrays (inputs in HBM before the timed region)
    dev_arrays = []
    for inst in insts:
        dev_arrays.append(dict(
            km=torch.as_tensor(inst.km, device="cuda"),
            fc_axis=torch.as_tensor(inst.fc_axis, device="cuda"),
            fc_pos=torch.as_tensor(np.ascontiguousarray(inst.fc_pos).reshape(-1), device="cuda"),
            fc_kf=torch.as_tensor(inst.fc_kf, device="cuda"),
            fc_a=torch.as_tensor(inst.fc_a, device="cuda"),
            pD_left=torch.as_tensor(inst.pD_left, device="cuda"),
            pD_right=torch.as_tensor(inst.pD_right, device="cuda")))
    N = [inst.n_m + inst.n_f for inst in insts]
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for n in N]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sopt = dict(rtol=1e-8, max_iters=5000, restart=30)
    stats_last = []

    phase_ev = []  # per member of a timed step: events before assembly, after assembly, set-up, solve

    def step(collect=False):
        its = []
        for k, inst in enumerate(insts):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if collect else None
            if ev:
                ev[0].record()
            s = ctx.assemble(inst, device_arrays=dev_arrays[k])
            if ev:
                ev[1].record()
            p = ctx.setup(s, precision="fp64", format="auto")
            if ev:
                ev[2].record()
            xs[k].zero_()
            code, st = ctx.solve(s, p, None, xs[k], **sopt)
            if ev:
                ev[3].record()
                phase_ev.append(ev)
            if code != 0:
                raise RuntimeError(f"solve failed for contrast {inputs.CONTRASTS[k]}: {st[0]}")
            its.append(st[0].iterations)
            if collect:
                stats_last.append(st[0])
            p.close()
            s.close()
        return its

    # direct reference for the contrast-1e4 member: started now, on the host,
    # in a spawned process, so that it runs while the GPU is timed
    direct = None
    if rank == 0 and not args.no_direct:
        import multiprocessing as mp
        s = ctx.assemble(insts[-1], device_arrays=dev_arrays[-1])
        (_, _, _, _, Ah), bh = s.to_host()
        s.close()
        pool = mp.get_context("spawn").Pool(1)
        direct = (pool, pool.apply_async(_direct_solve, (Ah.indptr, Ah.indices, Ah.data, bh[0])), Ah, bh[0])

    peak, peak_src = measured_peaks()
    # warm-up; the first one also profiles every kernel class (events around
    # the launches of every 4th FGMRES restart cycle) to find the dominant one
    classes = ["spmv", "vc_resid", "vc_post", "vc_restrict", "gs_dot", "gs_axpy"]
    for c in classes:
        ctx.timing_enable(c, True)
    ctx.timing_sample_every(4)
    ctx.timing_reset()
    its = step()
    share, per_class = {}, {}
    for c in classes:
        n_all, _, _, _ = ctx.timing_query(c)
        n_t, ms_t, by_t, fl_t = ctx.timing_sampled(c)
        avg = ms_t / n_t if n_t else 0.0
        share[c] = avg * n_all  # estimated total time of the class
        if n_t and ms_t > 0:
            gbs_c = by_t / (ms_t / 1e3) / 1e9
            tf_c = fl_t / (ms_t / 1e3) / 1e12
            per_class[c] = {"launches_per_step": n_all, "avg_launch_us": round(avg * 1e3, 3),
                            "algorithmic_bytes_per_launch": by_t / n_t, "hbm_gbs": round(gbs_c, 1),
                            "hbm_frac_of_measured": round(gbs_c / peak, 4), "fp64_tflops": round(tf_c, 4),
                            "fp64_frac_of_nominal": round(tf_c / FP64_PEAK_TFLOPS, 4)}
    dominant = max(share, key=share.get)
    for c in classes:
        ctx.timing_enable(c, c == dominant)
    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize()

    # timed region
    flush.fill_(1.0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.timing_reset()
    clocks = ClockSampler(local)
    clocks.start()
    t_total = 0.0
    iters = []
    step_s = []
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps (ncu --nvtx-include timed/)
    for s_ in range(args.steps):
        flush.fill_(float(s_))  # L2 flush between steps (256 MB > 129 MB L2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        iters = step(collect=(s_ == args.steps - 1))
        e1.record()
        torch.cuda.synchronize()
        step_s.append(e0.elapsed_time(e1) / 1e3)
        t_total += step_s[-1]
    torch.cuda.nvtx.range_pop()
    # phases of the last timed step (events on the library's stream)
    ph = np.zeros(3)
    for ev in phase_ev:
        ph += (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]))
    phases = {"assemble_ms": ph[0], "setup_ms": ph[1], "solve_ms": ph[2],
              "solve_only_solves_per_s": len(insts) / (ph[2] / 1e3) if ph[2] > 0 else None,
              "dof_iter_per_s_solve_only": (sum(n * i for n, i in zip(N, iters)) / (ph[2] / 1e3)
                                            if ph[2] > 0 else None)}
    launches = ctx.launch_count()
    kl_all = ctx.timing_query(dominant)[0]
    kl, kms, kbytes, kflops = ctx.timing_sampled(dominant)
    for c in classes:
        ctx.timing_enable(c, False)
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # replicas: every rank ran the whole sweep; slowest rank's time, all ranks' solves
    t_total, solves = sharding.reduce_over_ranks(t_total, len(insts) * args.steps)
    value = solves / t_total
    dof_iter = sum(n * i for n, i in zip(N, iters)) * args.steps * world / t_total

    # accuracy of the timed solves
    accuracy = {"relres_true_per_contrast": [st.relres_true for st in stats_last]}
    if direct is not None:
        pool, job, Ah, bh = direct
        xg = xs[-1].cpu().numpy()
        try:
            xd = job.get(timeout=600)
            accuracy["contrast_1e4_vs_direct"] = {
                "rel_error": float(np.linalg.norm(xg - xd) / np.linalg.norm(xd)),
                "relres_direct": float(np.linalg.norm(bh - Ah @ xd) / np.linalg.norm(bh)),
                "relres_gpu": float(np.linalg.norm(bh - Ah @ xg) / np.linalg.norm(bh)),
                "direct": "scipy spsolve (SuperLU, COLAMD) of the same assembled FP64 system, host"}
        except Exception as e:  # the reference is reported, never fatal
            accuracy["contrast_1e4_vs_direct"] = {"error": str(e)}
        pool.terminate()

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    e2e_t = 0.0
    h2d = 0
    d2h = 0
    import dataclasses

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()
    # the instances' arrays and the solutions in pinned host memory
    insts_h = [dataclasses.replace(i, km=pinned(i.km), fc_axis=pinned(i.fc_axis), fc_pos=pinned(i.fc_pos),
                                   fc_kf=pinned(i.fc_kf), fc_a=pinned(i.fc_a), pD_left=pinned(i.pD_left),
                                   pD_right=pinned(i.pD_right)) for i in insts]
    xh_all = [pinned(np.zeros(n)) for n in N]
    for s_ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, inst in enumerate(insts_h):
            s = ctx.assemble(inst)
            p = ctx.setup(s, precision="fp64", format="auto")
            xh = xh_all[k]
            xh[:] = 0.0
            code, st = ctx.solve(s, p, None, xh, **sopt)
            p.close()
            s.close()
        torch.cuda.synchronize()
        e2e_t += time.perf_counter() - t0
    e2e_steps = max(1, min(args.steps, 2))
    for inst in insts:
        h2d += inst.km.nbytes + inst.fc_axis.nbytes + inst.fc_pos.nbytes + inst.fc_kf.nbytes + inst.fc_a.nbytes \
            + inst.pD_left.nbytes + inst.pD_right.nbytes + 8 * (inst.n_m + inst.n_f)  # and the initial guess
        d2h += 8 * (inst.n_m + inst.n_f)
    e2e_value = len(insts) * e2e_steps / e2e_t * world

    avg_ms = kms / max(kl, 1)
    avg_bytes = kbytes / max(kl, 1)
    avg_flops = kflops / max(kl, 1)
    gbs = avg_bytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else None
    tflops = avg_flops / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else None
    hbm_frac = gbs / peak if gbs else None
    alu_frac = tflops / FP64_PEAK_TFLOPS if tflops else None
    traffic = profile_traffic(dominant, avg_bytes)
    if alu_frac and hbm_frac and alu_frac > hbm_frac:
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s (FP64)",
                "frac": alu_frac, "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (152 SMs x 2070 MHz); "
                "a dependent-FMA probe measured 1.20"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": hbm_frac,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                else "fallback 6.8 TB/s"}
    roof.update({"traffic": traffic, "kernel_class": dominant, "algorithmic_bytes_per_launch": avg_bytes,
                 "algorithmic_flops_per_launch": avg_flops, "launches": kl_all, "launches_timed": kl,
                 "avg_launch_ms": avg_ms,
                 "hbm_gbs": gbs, "hbm_frac_of_measured": hbm_frac, "fp64_tflops": tflops,
                 "fp64_frac_of_nominal": alu_frac,
                 "time_share_warmup": {k: round(v / max(sum(share.values()), 1e-9), 3) for k, v in share.items()},
                 "classes_warmup": per_class})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (assembly, set-up, V-cycle, FGMRES)",
                   "l2": "flushed between steps (256 MB write); per-solve working set > 129 MB L2",
                   "parallelism": f"replicas x{world}", "N_per_solve": N[0],
                   "iterations_per_contrast": iters},
        "dof_iter_per_s": dof_iter,
        "step_s": {"median": float(np.median(step_s)), "min": float(np.min(step_s)), "all": step_s},
        "phases_last_step": phases,
        "vcycle": vcycle_rate(ctx, insts[-1], dev_arrays[-1], flush),
        "accuracy": accuracy,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "host_buffers": "pinned; instance arrays in, solution out, every solve"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_variants:
        line["variants"] = variants(ctx, insts, dev_arrays, N, flush)
        if world > 1:
            line["variants"]["note"] = ("sweep/3D variants: replicas (rank 0's time); batch: instances "
                                        "sharded by unknown count, slowest rank's time")
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


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


def class_rates(ctx, fn, classes=("spmv", "vc_resid", "vc_post", "vc_restrict", "gs_dot", "gs_axpy")):
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
                                           "classes": class_rates(ctx, lambda: sweep("fp32"))}
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
    out["batch3d_256inst_x4rhs_bf16"]["classes"] = class_rates(ctx, lambda: batched("bf16"))
    return out


def _oracle_sample():
    """One oracle solve of the contrast-1 member (assemble, M_L set-up, FGMRES
    to 1e-8); returns the seconds of each phase and the iteration count."""
    import oracle
    from paper_2206_03203_gb300 import inputs
    oracle.build()
    inst = inputs.random_segments_2d(contrast=1.0)
    t0 = time.perf_counter()
    A, b = oracle.assemble(inst)
    t1 = time.perf_counter()
    M = oracle.ML(A, inst.n_m)
    t2 = time.perf_counter()
    res = oracle.fgmres(A, b[0], M, rtol=1e-8, maxit=5000)
    t3 = time.perf_counter()
    assert res.converged
    return t1 - t0, t2 - t1, t3 - t2, res.iterations


def cpu_baseline(samples: int = 1, all_cores: bool = True):
    """The oracle (plain sequential FP64 C) on a bounded sample of the same
    workload: the contrast-1 solve of the sweep, assembled, set up and solved
    to 1e-8 (the cheapest of the nine; about 10-30 s of CPU work), on one
    core; then the same sample as one process per host core at once (the
    host's throughput with the oracle as it stands)."""
    phases = np.zeros(3)
    t0 = time.perf_counter()
    for _ in range(samples):
        a, s_, v, its = _oracle_sample()
        phases += (a, s_, v)
    dt = time.perf_counter() - t0
    out = {"value": samples / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{samples} solve(s) of the contrast-1 member of the sweep (1024x1024, "
                     f"{its} FGMRES iterations), assemble + set-up + solve, single thread",
           "phases_s": {"assemble": phases[0] / samples, "setup": phases[1] / samples,
                        "solve": phases[2] / samples},
           "cpu": platform.processor() or platform.machine(), "nproc": os.cpu_count()}
    if all_cores:
        import multiprocessing as mp
        k = os.cpu_count() or 1
        with mp.get_context("spawn").Pool(k) as pool:
            t0 = time.perf_counter()
            rs = pool.starmap(_oracle_sample, [()] * k)
            dt = time.perf_counter() - t0
        out["all_cores"] = {"value": k / dt, "unit": UNIT, "cores": k,
                            "sample": f"{k} concurrent single-threaded oracle processes, one contrast-1 solve each"}
    return out


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return
    import oracle
    from paper_2206_03203_gb300 import inputs
    oracle.build()
    small = inputs.fixed_2d()
    for _ in range(args.warmup):
        oracle.solve(small)
    inst = inputs.random_segments_2d(contrast=1.0)
    t = 0.0
    its = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res, A, b, M = oracle.solve(inst, maxit=5000)
        t += time.perf_counter() - t0
        its = res.iterations
    value = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64", "parallelism": "CPU oracle, 1 thread",
                   "sample_iterations": its},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one step = the contrast-1 solve of the sweep (assemble + set-up + FGMRES), "
                                   "sequential C oracle; warm-up steps solve the 64x64 instance"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A short fixed run for ncu: the contrast-1e4 member of the sweep,
    assembled, set up and solved for --max-iters FGMRES iterations."""
    import torch

    from paper_2206_03203_gb300 import build, inputs, mdsolve
    build.build()
    ctx = mdsolve.Context(0)
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
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-direct", action="store_true", help="skip the host direct solve of the accuracy check")
    ap.add_argument("--profile-case", action="store_true", help="short fixed run for ncu captures")
    ap.add_argument("--table1", action="store_true", help="iteration counts over (K_par, kappa), the shape of "
                                                           "the paper's Table 1")
    ap.add_argument("--prolongation", default="piecewise", help="AMG prolongation of --table1 (piecewise, smoothed)")
    ap.add_argument("--max-iters", type=int, default=60)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--format", default="auto", help="level storage of the profile case (auto, csr, sell)")
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
