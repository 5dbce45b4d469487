#!/usr/bin/env python
"""Benchmark of the PTROM hot path on GB300.

One step = one implicit trapezoid FOM step (Sec. 2, Eq. linKstep) of the
two-Gaussian-cluster workload (N=16384, delta=0.02, dt=0.005), solved by
Jacobian-free Newton-Krylov: the velocity with self blocks (inexact Jacobian
for the preconditioner), the J v products inside GMRES, the residual and the
FP64 state update -- all in libptrom.so.  The metric is Biot-Savart pair
evaluations per second: (velocity + J v launches) x N^2 pairs per step.

Inputs are synthetic (seeded generator), resident in HBM when the timed
region starts; the 129 MB L2 is flushed (256 MB memset) before every timed
step.  With --impl reference the FP64 CPU oracle is timed instead on the host
cores (a bounded sample of the same workload).

The JSON line also carries the PTROM-vs-GPU-FOM step speed-up on the same
workload ("ptrom"): a model trained by ptrom_build (untimed) is stepped
online for one instance and for a batch of one instance per SM, with its QoI
errors against the GPU FOM.

Multi-GPU: every rank runs an independent replica (the FOM step of one
instance does not shard on this hardware); value = all ranks' pairs / the
slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Biot-Savart pair evals/s"
UNIT = "pairs/s"
WORKLOAD = {
    "workload": "two-cluster FOM implicit trapezoid step, JFNK (GMRES on J v), FP32C pair sums",
    "n_bodies": 16384,
    "delta": 0.02,
    "dt": 0.005,
    "clusters": "2 Gaussian, std 0.1, centres 1.0 apart, circulation ratio 1:1",
    "newton_tol": 1e-8,
    "gmres": "restart 30, rtol 1e-4, block-diagonal right preconditioner",
    "l2": "flushed (256 MB memset) before every timed step",
    "source_split": "autotuned per all-pairs kernel before the warm-up steps (ptrom_tune_pairs)",
}
# Algorithmic work per pair (an FMA counts 2 flops, the reciprocal 1), the
# per-unit figures the roofline is quoted on: velocity = 2 differences +
# |r|^2 + delta (2 FMA) + reciprocal + gamma r^-1 + 2 accumulating FMA = 12;
# the self blocks add 8; J v 26; J^T w with (df/dGamma)^T w 30.  The kernels'
# own pair bodies issue 12, 24, 23 and 31 FP32 flops (OPS_PER_PAIR).
FLOPS_PER_PAIR = {"velocity": 12, "velocity_selfjac": 20, "jvp": 26, "vjp": 30}
OPS_PER_PAIR = {"velocity": 12, "velocity_selfjac": 24, "jvp": 23, "vjp": 31}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count, sm_mhz):
    """FP32 non-tensor peak: SMs x 128 lanes x 2 flop (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    return rank, local, ws


def aggregate_ranks(ms, units, device, ws):
    """Whole-job figures of a replicas run: the slowest rank's timed
    milliseconds and the units every rank processed.  Collective over the
    default process group when ws > 1 (NCCL on GPUs, gloo in the CPU tests)."""
    if ws <= 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


# --------------------------------------------------------------------- oracle
def run_reference(args):
    """The FP64 CPU oracle on the host cores: per step, the pair sums one FOM
    Newton iteration makes (velocity + self blocks, 8 J v products) on a
    bounded sample of 512 target rows against all 16384 sources."""
    import numpy as np

    from oracle import direct
    from paper_2103_01983_gb300 import workloads as W

    n = WORKLOAD["n_bodies"]
    x, G = W.two_cluster(n, seed=0)
    rows = np.random.default_rng(0).choice(n, 512, replace=False)
    idx = np.r_[rows, n + rows]
    v = W.random_vectors(2 * n, 1, seed=1)[0]

    def step():
        direct.velocity(x, G, WORKLOAD["delta"], targets=x[idx], with_selfjac=True)
        for _ in range(8):
            direct.jvp(x, G, WORKLOAD["delta"], v, rows=rows)
        return 9 * rows.size * n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    pairs = 0
    for _ in range(args.steps):
        pairs += step()
    dt = time.perf_counter() - t0
    value = pairs / dt
    cores = direct.num_threads()
    sample = "per step: velocity+self blocks and 8 J v products at 512 sampled targets x 16384 sources (FP64 C loops)"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas x{args.gpus}"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline(budget_s=12.0):
    """Oracle pair throughput on the host cores (bounded sample, FP64)."""
    import numpy as np

    from oracle import direct
    from paper_2103_01983_gb300 import workloads as W

    n = WORKLOAD["n_bodies"]
    x, G = W.two_cluster(n, seed=0)
    v = W.random_vectors(2 * n, 1, seed=1)[0]
    rows = np.random.default_rng(0).choice(n, 1024, replace=False)
    idx = np.r_[rows, n + rows]
    pairs, t0, reps = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s:
        direct.velocity(x, G, WORKLOAD["delta"], targets=x[idx], with_selfjac=True)
        for _ in range(4):
            direct.jvp(x, G, WORKLOAD["delta"], v, rows=rows)
        pairs += 5 * rows.size * n
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": UNIT, "cores": direct.num_threads(), "kind": "oracle",
            "sample": f"{reps} x (velocity+self blocks and 4 J v products) at 1024 sampled targets "
                      f"x {n} sources, FP64, {dt:.1f} s"}


# --------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    rank, local, ws = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2103_01983_gb300 import ptrom
    from paper_2103_01983_gb300 import workloads as W

    n, delta, dt = WORKLOAD["n_bodies"], WORKLOAD["delta"], WORKLOAD["dt"]
    x0, G = W.two_cluster(n, seed=0)
    x = torch.tensor(x0, device=dev)
    Gt = torch.tensor(G, device=dev)
    params = ptrom.fom_params(dt, delta, "jfnk", tol=WORKLOAD["newton_tol"], prec="fp32c",
                              gmres_restart=30, gmres_max_iter=200, gmres_rtol=1e-4)
    f = ptrom.bs_velocity(x, Gt, delta)
    work = ptrom.fom_workspace(params, n, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    ptrom.tune_pairs(n, delta)  # cache the fastest source split of each all-pairs kernel at this size
    for _ in range(args.warmup):
        ptrom.fom_step(params, Gt, x, f, work=work)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)

    clk = Clocks(local)
    clk.start()
    time.sleep(0.25)
    ptrom.timing_read()
    # the timed region brackets only the all-pairs launches with events (the
    # small kernels' events would add gaps of their own); the step breakdown
    # below comes from a separate instrumented pass
    ptrom.timing_enable(True, kinds=list(FLOPS_PER_PAIR))
    l0 = ptrom.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    agg = {"velocity_evals": 0, "jvp_evals": 0, "newton_iters": 0, "linear_iters": 0}
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        st = ptrom.fom_step(params, Gt, x, f, work=work)
        ev[k][1].record(stream)
        for key in agg:
            agg[key] += st[key]
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    launches = ptrom.launch_count() - l0  # the L2-flush memsets are torch's, not counted
    ptrom.timing_enable(False)
    ktimes = ptrom.timing_read()
    clocks = clk.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    pairs = (agg["velocity_evals"] + agg["jvp_evals"]) * n * n

    ms_all, pairs_all = aggregate_ranks(ms, pairs, dev, ws)
    value = pairs_all / (ms_all * 1e-3)

    # roofline of the dominant kernel (largest event-timed total)
    peaks, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_count, sm_mhz)
    dom = max((k for k in ktimes if k in FLOPS_PER_PAIR), key=lambda k: ktimes[k][0])
    dom_ms, dom_cnt = ktimes[dom]
    achieved = FLOPS_PER_PAIR[dom] * n * n * dom_cnt / (dom_ms * 1e-3) / 1e12 if dom_cnt else None
    traffic = _traffic(dom, n)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_source": (f"nominal FP32 non-tensor peak: {sm_count} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz "
                                f"(sm_max_mhz from MEASURED_PEAKS.json, {peak_src}; the file holds no FP32 figure)"),
                "flops_per_pair": FLOPS_PER_PAIR[dom], "ops_issued_per_pair": OPS_PER_PAIR[dom],
                "launches": dom_cnt, "avg_launch_us": 1e3 * dom_ms / dom_cnt if dom_cnt else None}
    kernels = {k: {"launches": c, "avg_us": 1e3 * t / c,
                   "pairs_per_s": n * n * c / (t * 1e-3),
                   "tflops": FLOPS_PER_PAIR[k] * n * n * c / (t * 1e-3) / 1e12}
               for k, (t, c) in ktimes.items() if c and k in FLOPS_PER_PAIR}
    kernels["at_n65536"] = _pairs_leg(ptrom, dev, flush, peak)
    if not args.no_jphi:
        kernels["jphi"] = _jphi_leg(ptrom, dev, flush)
        kernels["jphi_tc"] = _jphi_leg(ptrom, dev, flush, prec="tf32x3")
        kernels["jphi_tc_f16"] = _jphi_leg(ptrom, dev, flush, prec="f16x3")
    other = _step_breakdown(ptrom, params, Gt, x, f, work, stream, flush)

    # end to end: host buffers, H2D of the step's inputs and D2H of its result
    e2e = _e2e(args, ptrom, params, x0, G, dev, stream, n)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair sums (compensated), f64 state",
        "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas x{ws}"),
        "roofline": roofline, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
        "step_stats": {k: v / args.steps for k, v in agg.items()},
        "kernels": kernels,
        "step_breakdown": other,
    }
    if rank == 0 and not args.no_ptrom:
        line["ptrom"] = ptrom_leg(ptrom, dev, ms_all / args.steps)
    if rank == 0 and not args.no_batch:
        line["batched"] = batch_leg(ptrom, dev)
    if rank == 0 and args.vortex_pair:
        line["vortex_pair"] = vortex_pair_leg(ptrom, dev, args.qr_prec)
    if rank == 0 and args.mushroom:
        line["mushroom"] = mushroom_leg(ptrom, dev, args.qr_prec)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def _hamiltonian_gpu(x, G, n):
    """H = 1/(4 pi) sum_j sum_{i != j} Gamma_i Gamma_j log |x_i - x_j| (Sec. 6.1), on the GPU."""
    import torch
    chi, psi = x[:n], x[n:]
    H = torch.zeros((), dtype=torch.float64, device=x.device)
    for a in range(0, n, 4096):
        dx = chi[a:a + 4096, None] - chi[None, :]
        dy = psi[a:a + 4096, None] - psi[None, :]
        r2 = dx * dx + dy * dy
        r2[r2 == 0] = 1.0                      # log 1 = 0 removes i == j
        H = H + (G[a:a + 4096, None] * G[None, :] * 0.5 * torch.log(r2)).sum()
    return float(H) / (4.0 * 3.141592653589793)


# (name, Barnes-Hut theta, least-squares precision): the opening angle of the
# PTROM configuration with FP64 QR, the same with the FP32 QR, and a narrower
# angle whose QoI errors stay below 0.1 %
PTROM_VARIANTS = (("theta0.25_qr_fp64", 0.25, "fp64"), ("theta0.5_qr_fp64", 0.5, "fp64"),
                  ("theta0.25_qr_fp32c", 0.25, "fp32c"), ("theta0.5_qr_fp32c", 0.5, "fp32c"))
QOI_BOUND = 1e-3  # 0.1 % on both QoIs (MAE_D and AE_H), the largest error over the checked steps


def ptrom_leg(ptrom, dev, fom_ms_per_step, steps=200):
    """PTROM-vs-GPU-FOM step speed-up on the benchmarked workload.

    Offline (untimed): ptrom_build trains reproductively on `steps` FOM steps
    (POD rank 20, residual rank 40, 40 sampled bodies, Barnes-Hut clusters at
    each variant's opening angle).  Online (timed): `steps` PTROM steps in one
    launch for one instance, and for a batch of one instance per SM.  QoI
    errors (MAE_D, AE_H of Sec. 6.1) against the GPU FOM every 25th step: the
    maximum and the time average (the paper reports time averages)."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    n, delta, dt = WORKLOAD["n_bodies"], WORKLOAD["delta"], WORKLOAD["dt"]
    x0, G = W.two_cluster(n, seed=0)
    x0d = torch.tensor(x0, device=dev)
    Gd = torch.tensor(G, device=dev)
    fp = ptrom.fom_params(dt, delta, "jfnk", tol=WORKLOAD["newton_tol"], prec="fp32c")
    out = {"workload": f"two-cluster N={n}, reproductive, {steps} steps, k=20, n_s=40, M_r=40, "
                       "Barnes-Hut clusters", "variants": {}}
    # FOM reference states
    x = x0d.clone()
    f = ptrom.bs_velocity(x, Gd, delta)
    work = ptrom.fom_workspace(fp, n, dev)
    ref = {}
    for k in range(1, steps + 1):
        ptrom.fom_step(fp, Gd, x, f, work=work)
        if k % 25 == 0:
            ref[k] = x.clone()
    H_ref = {k: _hamiltonian_gpu(v, Gd, n) for k, v in ref.items()}
    l = float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))
    for name, theta, qr in PTROM_VARIANTS:
        t0 = time.perf_counter()
        model, info = ptrom.ptrom_build(x0d[None], Gd[None], 20, 40, 40, steps, fp, criterion="bh", theta=theta,
                                        tol=1e-4, qr_prec=qr)
        build_s = time.perf_counter() - t0
        M = model.M
        st = model.new_state(dev)
        hist = torch.zeros(steps, M, dtype=torch.float64, device=dev)
        ptrom.ptrom_step([model], [model.new_state(dev)], 5)   # warm-up launch
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ptrom.ptrom_step([model], [st], steps, hist=[hist], want_stats=False)
        e1.record()
        torch.cuda.synchronize(dev)
        us_step = 1e3 * e0.elapsed_time(e1) / steps
        stats = ptrom.ptrom_step([model], [model.new_state(dev)], steps)
        # batched: one instance per SM in one launch
        B = torch.cuda.get_device_properties(dev).multi_processor_count
        sts = [model.new_state(dev) for _ in range(B)]
        ptrom.ptrom_step([model] * B, sts, 5)
        torch.cuda.synchronize(dev)
        e0.record()
        ptrom.ptrom_step([model] * B, sts, steps, want_stats=False)
        e1.record()
        torch.cuda.synchronize(dev)
        batch_ms = e0.elapsed_time(e1)
        mae, aeh = [], []
        for k, xr in ref.items():
            xp = model.reconstruct(hist[k - 1])
            d = torch.sqrt((xp[:n] - xr[:n]) ** 2 + (xp[n:] - xr[n:]) ** 2)
            mae.append(float(d.sum()) / (l * n))
            aeh.append(abs(_hamiltonian_gpu(xp, Gd, n) - H_ref[k]) / abs(H_ref[k]))
        within = max(mae) <= QOI_BOUND and max(aeh) <= QOI_BOUND
        ratio = fom_ms_per_step * 1e3 / us_step
        v = {
            "theta": theta, "qr_prec": qr,
            "build_s": build_s, "N_c": info["N_c"], "mean_clusters_per_sampled_body": info["mean_list"],
            "ptrom_us_per_step": us_step, "fom_ms_per_step": fom_ms_per_step,
            "within_qoi_bound": within,
            # a speed-up only where both QoIs stay within 0.1 %; otherwise the plain time ratio
            ("speedup_vs_gpu_fom_step" if within else "step_time_ratio_vs_gpu_fom_outside_qoi_bound"): ratio,
            "gn_iters_per_step": stats["gn_iters"] / max(stats["steps"], 1), "noconv_steps": stats["noconv"],
            "batched_instances": B, "batched_solves_per_s": B * steps / (batch_ms * 1e-3),
            "gpu_fom_steps_per_s": 1e3 / fom_ms_per_step,
            "qoi_vs_gpu_fom": {"mae_d_max": max(mae), "ae_h_max": max(aeh), "mae_d_mean": float(np.mean(mae)),
                               "ae_h_mean": float(np.mean(aeh)), "steps_checked": sorted(ref)},
        }
        out["variants"][name] = v
        del model
    ok = {k: v for k, v in out["variants"].items() if v["within_qoi_bound"]}
    for tag, pool in (("best", ok), ("best_fp64_qr", {k: v for k, v in ok.items() if v["qr_prec"] == "fp64"})):
        if pool:
            k = max(pool, key=lambda kk: pool[kk]["speedup_vs_gpu_fom_step"])
            out[f"speedup_at_qoi_bound_{tag}"] = {"variant": k, "speedup": pool[k]["speedup_vs_gpu_fom_step"]}
    return out


def vortex_pair_leg(ptrom, dev, qr_prec="fp64"):
    """The paper's vortex-pair parametric experiment (Sec. 6.2); see
    ``parametric_leg``."""
    return parametric_leg(ptrom, dev, "vortex_pair", qr_prec)


def mushroom_leg(ptrom, dev, qr_prec="fp64"):
    """The paper's mushroom-cloud parametric experiment (Sec. 6.3, with the
    superimposed inflow); see ``parametric_leg``."""
    return parametric_leg(ptrom, dev, "mushroom", qr_prec)


def parametric_leg(ptrom, dev, which, qr_prec="fp64"):
    """One of the paper's parametric experiments end to end: PTROM trained at
    4 Latin-hypercube parameters, queried on the 6 x 6 grid; time-averaged
    QoI errors against the GPU FOM at each query, and the PTROM-vs-FOM step
    speed-up (GPU FOM step time / GPU PTROM step time).  qr_prec: the online
    least squares' precision (FP64 Householder QR, or FP32)."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    if which == "vortex_pair":
        V = W.VORTEX_PAIR
        train, query = W.vortex_pair_params(0)
        setup = lambda a, b: (*W.vortex_pair(a, b), None)
        M, Mr, ns = 85, 110, 60
        paper = {"paper_N_c": 233, "paper_mae_d_mean": 0.0136e-2, "paper_ae_h_mean": 6.09e-6,
                 "paper_speedup_mean": 3.94}
        l = float(np.hypot(2 * V["half_width"], 2 * V["half_width"]))
        desc = ("vortex pair, N=500, delta=0.2121, dt=0.01, 500 steps; trained at 4 LHS parameters, "
                "queried on the 6x6 grid; M=85, M_r=110, 60 sampled bodies, neighbour p_c=1")
    else:
        V = W.MUSHROOM
        train, query = W.mushroom_params(0)
        setup = W.mushroom
        M, Mr, ns = 110, 185, 75
        paper = {"paper_N_c": 294, "paper_mae_d_mean": 0.0634e-2, "paper_ae_h_mean": 2.39e-5,
                 "paper_speedup_mean": 1.71}
        l = 2 * V["half_width"]
        desc = ("mushroom cloud, N=500, delta=0.15, dt=0.005, 1000 steps, semicircular inflow; trained at 4 LHS "
                "parameters, queried on the 6x6 grid; M=110, M_r=185, 75 sampled bodies, neighbour p_c=1")
    n, delta, dt, steps = V["n"], V["delta"], V["dt"], V["steps"]
    fp = ptrom.fom_params(dt, delta, "jfnk", tol=1e-12, prec="fp64", gmres_rtol=1e-10, gmres_max_iter=400)
    xs, gs, us = zip(*[setup(a, b) for a, b in train])
    t0 = time.perf_counter()
    model, info = ptrom.ptrom_build(torch.tensor(np.stack(xs), device=dev), torch.tensor(np.stack(gs), device=dev),
                                    M, Mr, ns, steps, fp, criterion="nb", p_c=1.0, tol=1e-4, qr_prec=qr_prec,
                                    u_infs=None if us[0] is None else torch.tensor(np.stack(us), device=dev))
    build_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for g1, gN in query:
        x0, G, u = setup(g1, gN)
        x = torch.tensor(x0, device=dev)
        Gd = torch.tensor(G, device=dev)
        ud = None if u is None else torch.tensor(u, device=dev)
        f = ptrom.bs_velocity(x, Gd, delta, prec="fp64")
        work = ptrom.fom_workspace(fp, n, dev)
        fom = torch.empty(steps, 2 * n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        e0.record()
        for k in range(steps):
            ptrom.fom_step(fp, Gd, x, f, work=work, u_inf=ud)
            fom[k] = x
        e1.record()
        torch.cuda.synchronize(dev)
        fom_ms = e0.elapsed_time(e1)
        model.set_param_full(torch.tensor(x0, device=dev), Gd)
        if ud is not None:
            model.set_inflow_full(ud)
        st = model.new_state(dev)
        hist = torch.zeros(steps, model.M, dtype=torch.float64, device=dev)
        e0.record()
        ptrom.ptrom_step([model], [st], steps, hist=[hist], want_stats=False)
        e1.record()
        torch.cuda.synchronize(dev)
        rom_ms = e0.elapsed_time(e1)
        rec = torch.stack([model.reconstruct(hist[k]) for k in range(steps)])
        mae = float((torch.sqrt((rec[:, :n] - fom[:, :n]) ** 2 + (rec[:, n:] - fom[:, n:]) ** 2).mean(dim=1) / l).mean())
        ks = list(range(0, steps, 25))
        aeh = float(np.mean([abs(_hamiltonian_gpu(rec[k], Gd, n) - _hamiltonian_gpu(fom[k], Gd, n))
                             / abs(_hamiltonian_gpu(fom[k], Gd, n)) for k in ks]))
        rows.append((float(g1), float(gN), mae, aeh, fom_ms / rom_ms))
    r = np.array(rows)
    return {"workload": desc, "qr_prec": qr_prec, "build_s": build_s, "N_c": info["N_c"], "paper_N_c": paper["paper_N_c"],
            "mae_d_mean": float(r[:, 2].mean()), "mae_d_max": float(r[:, 2].max()),
            "paper_mae_d_mean": paper["paper_mae_d_mean"],
            "ae_h_mean": float(r[:, 3].mean()), "ae_h_max": float(r[:, 3].max()),
            "paper_ae_h_mean": paper["paper_ae_h_mean"],
            "speedup_vs_gpu_fom_step_mean": float(r[:, 4].mean()),
            "paper_speedup_mean": paper["paper_speedup_mean"],
            "paper_speedup_note": "pair-loop time ratio, MATLAB on one CPU core",
            "queries": [[round(a, 2), round(b, 2), m, h, sp] for a, b, m, h, sp in rows]}


def _fom_run(ptrom, fp, x0, G, steps, dev, every, keep_all=False):
    """GPU FOM trajectory of `steps` steps: states every `every` steps (and,
    with keep_all, every state as the training snapshots), device ms per step."""
    import torch
    n = G.size
    x = torch.tensor(x0, device=dev)
    Gd = torch.tensor(G, device=dev)
    f = ptrom.bs_velocity(x, Gd, fp.delta)
    work = ptrom.fom_workspace(fp, n, dev)
    allx = torch.empty(steps, 2 * n, dtype=torch.float64, device=dev) if keep_all else None
    ref = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    for k in range(1, steps + 1):
        ptrom.fom_step(fp, Gd, x, f, work=work)
        if keep_all:
            allx[k - 1] = x
        if k % every == 0:
            ref[k] = x.clone()
    e1.record()
    torch.cuda.synchronize(dev)
    return allx, ref, e0.elapsed_time(e1) / steps


def c3_leg(ptrom, dev, n=65536, steps=1000, ks=(20, 40, 60), mults=(2, 4), thetas=(0.5,), every=25):
    """The parametric PTROM configuration: two-cluster bodies with common random
    numbers, separation in [0.8, 1.2] and circulation ratio in [0.5, 2.0];
    trained (offline, untimed) on the GPU FOM at 8 Latin-hypercube parameters
    (seed 1), queried at 4 held-out ones (seed 2); POD rank k, M_r = 2k,
    n_s = mult * k sampled bodies, Barnes-Hut theta (each of thetas), FP64
    least squares.
    Per configuration and held-out parameter: time-averaged MAE_D and AE_H of
    the PTROM against the GPU FOM, of the best point of the trial manifold
    (the basis alone), and of Tier II on the first training parameter (the
    clustered LSPG over all bodies); a speed-up only where both PTROM QoIs
    stay within 0.1 %."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    delta, dt = WORKLOAD["delta"], WORKLOAD["dt"]
    fp = ptrom.fom_params(dt, delta, "jfnk", tol=WORKLOAD["newton_tol"], prec="fp32c")
    train, held = W.param_lhs(8, seed=1), W.param_lhs(4, seed=2)
    t0 = time.perf_counter()
    snaps, x0s, gs, train_ref = [], [], [], None
    for q, (sep, ratio) in enumerate(train):
        x0, G = W.two_cluster(n, seed=0, sep=sep, ratio=ratio)
        allx, ref, _ = _fom_run(ptrom, fp, x0, G, steps, dev, every, keep_all=True)
        snaps.append(allx)
        x0s.append(x0)
        gs.append(G)
        if q == 0:
            train_ref = ref
    S = torch.cat(snaps)
    del snaps
    X0 = torch.tensor(np.stack(x0s), device=dev)
    GS = torch.tensor(np.stack(gs), device=dev)
    held_runs = []
    for sep, ratio in held:
        x0, G = W.two_cluster(n, seed=0, sep=sep, ratio=ratio)
        _, ref, fom_ms = _fom_run(ptrom, fp, x0, G, steps, dev, every)
        Gd = torch.tensor(G, device=dev)
        held_runs.append({"sep": float(sep), "ratio": float(ratio), "x0": x0, "G": G, "Gd": Gd, "ref": ref,
                          "fom_ms": fom_ms, "H": {k: _hamiltonian_gpu(v, Gd, n) for k, v in ref.items()}})
    fom_s = time.perf_counter() - t0
    out = {"workload": (f"two clusters, N={n}, delta={delta}, dt={dt}, {steps} steps; 8 LHS training parameters "
                        f"(seed 1), 4 held-out (seed 2); M_r = 2k; Barnes-Hut theta in {list(thetas)}; FP64 least squares; "
                        f"QoIs time-averaged over every {every}th step against the GPU FOM"),
           "fom_seconds": fom_s, "configs": []}
    l_of = lambda x0: float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))

    def qois(recs, run):
        """time-averaged MAE_D and AE_H of the states recs[k] against run's FOM"""
        l = l_of(run["x0"])
        mae, aeh = [], []
        for k, xr in run["ref"].items():
            xp = recs[k]
            d = torch.sqrt((xp[:n] - xr[:n]) ** 2 + (xp[n:] - xr[n:]) ** 2)
            mae.append(float(d.sum()) / (l * n))
            aeh.append(abs(_hamiltonian_gpu(xp, run["Gd"], n) - run["H"][k]) / abs(run["H"][k]))
        return float(np.mean(mae)), float(np.mean(aeh))

    for theta, k, mult in ((t, k_, m) for t in thetas for k_ in ks for m in mults):
        cfg = {"k": k, "M_r": 2 * k, "n_s": mult * k, "theta": theta}
        t0 = time.perf_counter()
        try:
            model, info = ptrom.ptrom_build(X0, GS, k, 2 * k, mult * k, steps, fp, criterion="bh",
                                            theta=theta, tol=1e-4, qr_prec="fp64", snapshots=S)
        except ptrom.PtromError as e:
            cfg["error"] = str(e)
            out["configs"].append(cfg)
            continue
        cfg.update(build_s=time.perf_counter() - t0, N_c=info["N_c"],
                   mean_clusters_per_sampled_body=info["mean_list"])
        q = model.query()
        Phi = torch.tensor(q["phi"], device=dev)
        t2 = torch.tensor(model.query_training()["tier2"][0], device=dev)
        x0t = torch.tensor(x0s[0], device=dev)
        run0 = {"x0": x0s[0], "Gd": GS[0], "ref": train_ref,
                "H": {kk: _hamiltonian_gpu(v, GS[0], n) for kk, v in train_ref.items()}}
        cfg["tier2_train0"] = qois({kk: x0t + Phi @ t2[kk] for kk in train_ref}, run0)
        rows = []
        for run in held_runs:
            x0d = torch.tensor(run["x0"], device=dev)
            best = {kk: x0d + Phi @ (Phi.T @ (xr - x0d)) for kk, xr in run["ref"].items()}
            model.set_param_full(x0d, run["Gd"])
            st = model.new_state(dev)
            hist = torch.zeros(steps, k, dtype=torch.float64, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record()
            stats = ptrom.ptrom_step([model], [st], steps, hist=[hist])
            e1.record()
            torch.cuda.synchronize(dev)
            rom_us = 1e3 * e0.elapsed_time(e1) / steps
            rec = {kk: model.reconstruct(hist[kk - 1]) for kk in run["ref"]}
            m_p, h_p = qois(rec, run)
            m_b, h_b = qois(best, run)
            within = m_p <= QOI_BOUND and h_p <= QOI_BOUND
            row = {"sep": run["sep"], "ratio": run["ratio"], "mae_d": m_p, "ae_h": h_p,
                   "best_mae_d": m_b, "best_ae_h": h_b, "ptrom_us_per_step": rom_us,
                   "fom_ms_per_step": run["fom_ms"], "gn_iters_per_step": stats["gn_iters"] / steps,
                   "noconv_steps": stats["noconv"], "within_qoi_bound": within}
            row["speedup_vs_gpu_fom_step" if within else "step_time_ratio_vs_gpu_fom_outside_qoi_bound"] = \
                1e3 * run["fom_ms"] / rom_us
            rows.append(row)
        cfg["held_out"] = rows
        out["configs"].append(cfg)
        del model, Phi
    return out


# Sec. 6.4's PTROM hyper-parameters: per neighbourhood width (Tables 2-4) and
# bases case (tolerance 1e-1 .. 1e-4), M and p_c for N = 100 .. 5000, and the
# paper's resulting N_c.  M_r = 2M and n_s = M_r throughout.
SV_NS = (100, 500, 1000, 2000, 3000, 4000, 5000)
SV_TOL = (1e-1, 1e-2, 1e-3, 1e-4)
SV_M = {"narrow": ((13, 21, 21, 21, 23, 23, 23), (14, 22, 22, 22, 23, 23, 24), (14, 23, 23, 23, 25, 25, 26),
                   (16, 24, 24, 26, 26, 26, 26)),
        "moderate": ((13, 21, 21, 21, 23, 23, 23), (14, 22, 22, 22, 23, 23, 24), (14, 23, 23, 23, 25, 25, 26),
                     (18, 24, 24, 26, 26, 26, 26)),
        "wide": ((13, 21, 21, 21, 23, 23, 23), (14, 22, 22, 22, 23, 23, 24), (14, 23, 23, 23, 25, 25, 26),
                 (18, 24, 24, 26, 26, 32, 33))}
SV_PC = {"narrow": ((0,) * 7, (0,) * 7, (0,) * 7, (0, 0, 0, 0, 0.5, 0.5, 0.5)),
         "moderate": ((1,) * 7,) * 4, "wide": ((2,) * 7,) * 4}
SV_NC = {"narrow": ((68, 113, 121, 122, 134, 131, 142), (69, 114, 129, 127, 142, 130, 140),
                    (70, 120, 132, 134, 136, 143, 156), (80, 128, 130, 134, 151, 159, 144)),
         "moderate": ((73, 122, 139, 123, 135, 137, 149), (79, 130, 142, 149, 137, 150, 144),
                      (79, 127, 133, 132, 146, 153, 149), (84, 131, 144, 144, 147, 159, 143)),
         "wide": ((79, 133, 135, 143, 161, 183, 154), (80, 130, 154, 153, 164, 155, 159),
                  (80, 136, 146, 165, 178, 173, 173), (113, 150, 143, 167, 194, 216, 213))}


def single_vortex_leg(ptrom, dev, ns=SV_NS, widths=("narrow", "moderate", "wide"), cases=(0, 1, 2, 3)):
    """Sec. 6.4's reproductive single-vortex experiment (Table 1 conditions,
    delta = 0) for the PTROM settings of Tables 2-4: per N, one FP64 GPU FOM
    trajectory (JFNK) gives the snapshots; per (width, bases case) a PTROM is
    trained on them and run over the same steps.  Reported: N_c beside the
    paper's, time-averaged MAE_D and AE_H against the FOM (the paper reports all
    below 0.1 %), Gauss-Newton iterations and step times."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    out = []
    for n in ns:
        col = SV_NS.index(n)
        x0, G, dt, steps = W.single_vortex(n)
        fp = ptrom.fom_params(dt, 0.0, "jfnk", tol=1e-12, prec="fp64", gmres_rtol=1e-10, gmres_max_iter=400)
        allx, _, fom_ms = _fom_run(ptrom, fp, x0, G, steps, dev, steps, keep_all=True)
        Gd = torch.tensor(G, device=dev)
        xd = torch.tensor(x0, device=dev)
        l = float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))
        chk = list(range(99, steps, 100))
        H = {k: _hamiltonian_gpu(allx[k], Gd, n) for k in chk}
        for width in widths:
            for case in cases:
                M, pc = SV_M[width][case][col], SV_PC[width][case][col]
                row = {"n": n, "width": width, "bases_case": case + 1, "tol": SV_TOL[case], "M": M, "p_c": pc,
                       "paper_N_c": SV_NC[width][case][col]}
                try:
                    model, info = ptrom.ptrom_build(xd[None], Gd[None], M, 2 * M, 2 * M, steps, fp, criterion="nb",
                                                    p_c=pc, tol=SV_TOL[case], qr_prec="fp64", snapshots=allx)
                except ptrom.PtromError as e:
                    row["error"] = str(e)
                    out.append(row)
                    continue
                st = model.new_state(dev)
                hist = torch.zeros(steps, M, dtype=torch.float64, device=dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                stats = ptrom.ptrom_step([model], [st], steps, hist=[hist])
                e1.record()
                torch.cuda.synchronize(dev)
                rec = torch.stack([model.reconstruct(hist[k]) for k in range(steps)])
                mae = float((torch.sqrt((rec[:, :n] - allx[:, :n]) ** 2 + (rec[:, n:] - allx[:, n:]) ** 2)
                             .mean(dim=1) / l).mean())
                aeh = float(np.mean([abs(_hamiltonian_gpu(rec[k], Gd, n) - H[k]) / abs(H[k]) for k in chk]))
                row.update(N_c=info["N_c"], mae_d=mae, ae_h=aeh, gn_iters_per_step=stats["gn_iters"] / steps,
                           noconv_steps=stats["noconv"], ptrom_us_per_step=1e3 * e0.elapsed_time(e1) / steps,
                           fom_ms_per_step=fom_ms)
                out.append(row)
                del model
        del allx
    return out


def batch_leg(ptrom, dev):
    """Batched FOM over 64 instances of uneven N (log-uniform in [4096,
    131072], separation and circulation ratio uniform in their ranges, seed 3):
    aggregate pair evals/s of one batched velocity launch and of one batched
    block-diagonal Newton step, against per-instance launches."""
    import torch

    from paper_2103_01983_gb300 import workloads as W

    ns, seps, ratios = W.batch_instances(64, seed=3)
    xs, Gs = [], []
    for k, (n, sep, ratio) in enumerate(zip(ns, seps, ratios)):
        x, G = W.two_cluster(int(n), seed=k, sep=float(sep), ratio=float(ratio))
        xs.append(torch.tensor(x, device=dev))
        Gs.append(torch.tensor(G, device=dev))
    pairs = float(sum(int(n) * int(n) for n in ns))
    deltas = [WORKLOAD["delta"]] * len(xs)
    fs = [torch.empty_like(x) for x in xs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    t_b = timed(lambda: ptrom.bs_velocity_batched(xs, Gs, deltas, f_outs=fs), 3)
    t_s = timed(lambda: [ptrom.bs_velocity(x, G, WORKLOAD["delta"], f_out=f) for x, G, f in zip(xs, Gs, fs)], 3)
    p = ptrom.fom_params(WORKLOAD["dt"], WORKLOAD["delta"], "blockdiag", prec="fp32c")
    works = [ptrom.fom_workspace(p, G.numel(), dev) for G in Gs]
    xb = [x.clone() for x in xs]
    fb = [ptrom.bs_velocity(x, G, WORKLOAD["delta"]) for x, G in zip(xb, Gs)]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    stats = ptrom.fom_step_batched(p, Gs, xb, fb, works)
    torch.cuda.synchronize(dev)
    tb_step = time.perf_counter() - t0
    xsg = [x.clone() for x in xs]
    fsg = [ptrom.bs_velocity(x, G, WORKLOAD["delta"]) for x, G in zip(xsg, Gs)]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    it_single = 0
    for x, G, f, w in zip(xsg, Gs, fsg, works):
        it_single += ptrom.fom_step(p, G, x, f, work=w)["velocity_evals"]
    torch.cuda.synchronize(dev)
    ts_step = time.perf_counter() - t0
    evals_b = sum(s["velocity_evals"] * int(n) ** 2 for s, n in zip(stats, ns))
    return {
        "workload": "64 two-cluster instances, N log-uniform in [4096, 131072] (seed 3), delta 0.02, dt 0.005",
        "total_bodies": int(sum(ns)), "pairs_per_velocity_eval": pairs,
        "batched_velocity_ms": t_b, "per_instance_velocity_ms": t_s,
        "batched_velocity_pairs_per_s": pairs / (t_b * 1e-3),
        "per_instance_velocity_pairs_per_s": pairs / (t_s * 1e-3),
        "batched_fom_step_s": tb_step, "per_instance_fom_step_s": ts_step,
        "batched_fom_step_pairs_per_s": evals_b / tb_step,
        "fom_mode": "block-diagonal inexact Newton (the paper's), FP32C pair sums",
    }


def c4_leg(ptrom, dev, count=64, steps=100, k=40, theta=0.5):
    """The batching configuration's PTROM half: `count` two-cluster instances of
    uneven N (log-uniform in [4096, 131072], separation and circulation ratio
    uniform in their ranges, seed 3), each with its own PTROM (k = 40,
    M_r = n_s = 2k, Barnes-Hut theta, FP64 least squares) trained reproductively
    on its own `steps`-step GPU FOM trajectory (offline, untimed).  Timed: all
    instances' online solves in one launch against one launch per instance;
    reported as PTROM instance-steps (solves) per second beside the GPU FOM's
    instance-steps per second, with each instance's QoI errors."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    ns, seps, ratios = W.batch_instances(count, seed=3)
    fp = ptrom.fom_params(WORKLOAD["dt"], WORKLOAD["delta"], "jfnk", tol=WORKLOAD["newton_tol"], prec="fp32c")
    models, rows, refs, fom_ms_total = [], [], [], 0.0
    t0 = time.perf_counter()
    for i, (n, sep, ratio) in enumerate(zip(ns, seps, ratios)):
        n = int(n)
        x0, G = W.two_cluster(n, seed=i, sep=float(sep), ratio=float(ratio))
        allx, _, fom_ms = _fom_run(ptrom, fp, x0, G, steps, dev, steps, keep_all=True)
        fom_ms_total += fom_ms
        row = {"n": n, "sep": float(sep), "ratio": float(ratio), "fom_ms_per_step": fom_ms}
        try:
            model, info = ptrom.ptrom_build(torch.tensor(x0, device=dev)[None], torch.tensor(G, device=dev)[None],
                                            k, 2 * k, 2 * k, steps, fp, criterion="bh", theta=theta, tol=1e-4,
                                            qr_prec="fp64", snapshots=allx)
        except ptrom.PtromError as e:
            row["error"] = str(e)
            rows.append(row)
            continue
        row["N_c"] = info["N_c"]
        models.append(model)
        refs.append((x0, allx[-1].clone(), allx[steps // 2 - 1].clone()))
        rows.append(row)
        del allx
    build_s = time.perf_counter() - t0
    B = len(models)
    hists = [torch.zeros(steps, k, dtype=torch.float64, device=dev) for _ in models]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ptrom.ptrom_step(models, [m.new_state(dev) for m in models], 2, want_stats=False)   # warm-up launch
    sts = [m.new_state(dev) for m in models]
    torch.cuda.synchronize(dev)
    e0.record()
    ptrom.ptrom_step(models, sts, steps, hist=hists, want_stats=False)
    e1.record()
    torch.cuda.synchronize(dev)
    batched_ms = e0.elapsed_time(e1)
    sts1 = [m.new_state(dev) for m in models]
    e0.record()
    for m, st in zip(models, sts1):
        ptrom.ptrom_step([m], [st], steps, want_stats=False)
    e1.record()
    torch.cuda.synchronize(dev)
    single_ms = e0.elapsed_time(e1)
    maes = []
    it = iter(r for r in rows if "error" not in r)
    for m, h, (x0, x_end, x_mid), r in zip(models, hists, refs, it):
        n = r["n"]
        l = float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))
        errs = []
        for xr, kk in ((x_mid, steps // 2 - 1), (x_end, steps - 1)):
            xp = m.reconstruct(h[kk])
            errs.append(float(torch.sqrt((xp[:n] - xr[:n]) ** 2 + (xp[n:] - xr[n:]) ** 2).sum()) / (l * n))
        r["mae_d_mid_end"] = errs
        maes.append(max(errs))
    return {
        "workload": (f"{count} two-cluster instances, N log-uniform in [4096, 131072] (seed 3); each a reproductive "
                     f"PTROM, k={k}, M_r=n_s={2 * k}, Barnes-Hut theta={theta}, FP64 least squares, "
                     f"{steps} steps"),
        "instances_built": B, "build_and_fom_s": build_s,
        "batched_launch_ms": batched_ms, "per_instance_launches_ms": single_ms,
        "batched_solves_per_s": B * steps / (batched_ms * 1e-3),
        "per_instance_solves_per_s": B * steps / (single_ms * 1e-3),
        "gpu_fom_instance_steps_per_s": count / (fom_ms_total * 1e-3),
        "mae_d_max": max(maes) if maes else None, "mae_d_mean": float(np.mean(maes)) if maes else None,
        "instances": rows,
    }


def _pairs_leg(ptrom, dev, flush, peak, n=65536, reps=5):
    """The four all-pairs kernels of the FOM step at N = 65536 (two clusters,
    split autotuned for this shape first): library-side events on their
    launches, L2 flushed before each; TFLOP/s at the survey's flops per pair
    and the fraction of the same nominal FP32 peak as the roofline line."""
    import torch

    from paper_2103_01983_gb300 import workloads as W

    x0, G = W.two_cluster(n, seed=0)
    x = torch.tensor(x0, device=dev)
    Gt = torch.tensor(G, device=dev)
    v = torch.tensor(W.random_vectors(2 * n, 1, seed=1)[0], device=dev)
    ptrom.tune_pairs(n, WORKLOAD["delta"])
    calls = {"velocity": lambda: ptrom.bs_velocity(x, Gt, WORKLOAD["delta"]),
             "velocity_selfjac": lambda: ptrom.bs_velocity(x, Gt, WORKLOAD["delta"], selfjac=True),
             "jvp": lambda: ptrom.bs_jvp(x, Gt, WORKLOAD["delta"], v),
             "vjp": lambda: ptrom.bs_vjp(x, Gt, WORKLOAD["delta"], v)}
    out = {}
    for kind, fn in calls.items():
        fn()
        torch.cuda.synchronize(dev)
        ptrom.timing_read()
        ptrom.timing_enable(True, kinds=[kind])
        for _ in range(reps):
            flush.zero_()
            fn()
        torch.cuda.synchronize(dev)
        ptrom.timing_enable(False)
        t, c = ptrom.timing_read()[kind]
        pps = n * n * c / (t * 1e-3)
        tf = FLOPS_PER_PAIR[kind] * pps / 1e12
        out[kind] = {"launches": c, "avg_us": 1e3 * t / c, "pairs_per_s": pps, "tflops": tf,
                     "frac_of_nominal_fp32": tf / peak if peak else None}
    out["n"] = n
    return out


def _jphi_leg(ptrom, dev, flush, n=65536, M=60, reps=5, prec="fp32c"):
    """J Phi (the LSPG basis product) on the two-cluster workload at N = 65536
    with M = 60 random basis columns: library-side events on its launches (the
    source-split sum included), L2 flushed before each.  prec "fp32c": FP32
    pipes; "tf32x3" / "f16x3": tensor cores (TF32 or scaled FP16 hi/lo
    splits, three products)."""
    import numpy as np
    import torch

    from paper_2103_01983_gb300 import workloads as W

    x0, G = W.two_cluster(n, seed=0)
    x = torch.tensor(x0, device=dev)
    Gt = torch.tensor(G, device=dev)
    phi = torch.tensor(np.random.default_rng(5).standard_normal((2 * n, M)) / np.sqrt(2 * n), device=dev)
    for _ in range(2):
        ptrom.bs_jphi(x, Gt, WORKLOAD["delta"], phi, prec=prec)
    torch.cuda.synchronize(dev)
    ptrom.timing_read()
    ptrom.timing_enable(True, kinds=["jphi"])
    for _ in range(reps):
        flush.zero_()
        ptrom.bs_jphi(x, Gt, WORKLOAD["delta"], phi, prec=prec)
    torch.cuda.synchronize(dev)
    ptrom.timing_enable(False)
    t, c = ptrom.timing_read()["jphi"]
    flops = 20 + 8 * M  # per pair: the 2x2 block, then 4 multiply-adds per column
    pps = n * n * c / (t * 1e-3)
    out = {"n": n, "M": M, "prec": prec, "launches": c, "avg_us": 1e3 * t / c, "pairs_per_s": pps,
           "flops_per_pair": flops, "tflops": flops * pps / 1e12}
    if prec in ("tf32x3", "f16x3"):
        npad = 64 * ((M + 63) // 64)
        # per pair: 3 products (hi hi, hi lo, lo hi) of a 2x2 block with N columns
        kind = "kind::tf32, TF32" if prec == "tf32x3" else "kind::f16, power-of-two-scaled FP16"
        out["units"] = (f"tcgen05 {kind} hi/lo splits on pair blocks generated in shared memory, "
                        "FP32 sums in tensor memory folded every 64 MMA steps into compensated totals")
        out["tensor_tflops_issued"] = 24 * npad * pps / 1e12
    else:
        out["units"] = "SIMT FP32 pair blocks, FP32 compensated"
    return out


def _step_breakdown(ptrom, params, Gt, x, f, work, stream, flush, steps=10):
    """Untimed-region diagnostic: every library launch kind event-timed over a
    few steps -> per-step device time of each kind and the rest of the step
    (launch gaps, copies, host waits).  These events add gaps of their own, so
    the step here is longer than in the timed region."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ptrom.timing_read()
    ptrom.timing_enable(True)
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        ptrom.fom_step(params, Gt, x, f, work=work)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ptrom.timing_enable(False)
    kt = ptrom.timing_read()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    out = {k: {"launches_per_step": c / steps, "us_per_step": 1e3 * t / steps}
           for k, (t, c) in kt.items() if c}
    out["rest_us_per_step"] = 1e3 * (ms - sum(t for t, _ in kt.values())) / steps
    out["step_us_instrumented"] = 1e3 * ms / steps
    return out


def _traffic(kind, n):
    """DRAM bytes per launch from the committed ncu capture of this kernel at
    this size; None when there is none or the kernel sources changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in rec["source_files"]:
            with open(os.path.join(ROOT, f), "rb") as src:
                h.update(src.read())
        if h.hexdigest() != rec["source_sha256"] or rec["sizes"].get(kind) != n:
            return None
        return rec.get(kind)
    except (OSError, ValueError, KeyError):
        return None


def _e2e(args, ptrom, params, x0, G, dev, stream, n):
    import torch

    xh = torch.tensor(x0).pin_memory()
    Gh = torch.tensor(G).pin_memory()
    x = torch.empty_like(xh, device=dev)
    Gd = torch.empty_like(Gh, device=dev)
    x.copy_(xh)
    Gd.copy_(Gh)
    fh = ptrom.bs_velocity(x, Gd, params.delta).cpu().pin_memory()
    f = torch.empty_like(fh, device=dev)
    work = ptrom.fom_workspace(params, n, dev)
    steps = max(3, min(args.steps, 20))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    # the same library-side events on the all-pairs launches as the device-timed leg
    ptrom.timing_enable(True, kinds=list(FLOPS_PER_PAIR))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pairs = 0
    for k in range(steps):
        flush.zero_()  # L2 flushed before every step, outside its events, as in the device-timed leg
        ev[k][0].record(stream)
        x.copy_(xh, non_blocking=True)
        f.copy_(fh, non_blocking=True)
        Gd.copy_(Gh, non_blocking=True)
        st = ptrom.fom_step(params, Gd, x, f, work=work)
        xh.copy_(x, non_blocking=True)
        fh.copy_(f, non_blocking=True)
        ev[k][1].record(stream)
        pairs += (st["velocity_evals"] + st["jvp_evals"]) * n * n
    torch.cuda.synchronize(dev)
    ptrom.timing_enable(False)
    ptrom.timing_read()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    nb = xh.numel() * 8
    return {"value": pairs / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 2 * nb + Gh.numel() * 8,
            "d2h_bytes_per_step": 2 * nb, "steps": steps,
            "note": ("public API (ptrom.fom_step) from pinned host buffers; x, f, Gamma H2D and x, f D2H every "
                     "step; L2 flushed before every step; all-pairs launches event-timed as in the device leg")}


def kernel_only(args):
    """Launch one all-pairs kernel `args.steps` times at N = args.n (for ncu;
    J Phi with M = 60 columns);
    with "ptrom", train the PTROM leg's model (theta 0.5, FP32 QR; untimed)
    and launch the online kernel args.warmup + args.steps times, 10 time
    steps per launch."""
    import torch

    from paper_2103_01983_gb300 import ptrom
    from paper_2103_01983_gb300 import workloads as W

    if args.kernel_only == "ptrom":
        x0, G = W.two_cluster(args.n, seed=0)
        fp = ptrom.fom_params(WORKLOAD["dt"], WORKLOAD["delta"], "jfnk", tol=WORKLOAD["newton_tol"], prec="fp32c")
        model, _ = ptrom.ptrom_build(torch.tensor(x0, device="cuda")[None], torch.tensor(G, device="cuda")[None],
                                     20, 40, 40, 200, fp, criterion="bh", theta=0.5, qr_prec="fp32c")
        st = model.new_state()
        for _ in range(args.warmup + args.steps):
            ptrom.ptrom_step([model], [st], 10, want_stats=False)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": "ptrom", "n": args.n, "launches": args.warmup + args.steps}))
        return
    x0, G = W.two_cluster(args.n, seed=0)
    x = torch.tensor(x0, device="cuda")
    Gt = torch.tensor(G, device="cuda")
    v = torch.tensor(W.random_vectors(2 * args.n, 1, seed=1)[0], device="cuda")
    phi = torch.tensor(W.random_vectors(2 * args.n, 60, seed=2).T.copy(), device="cuda") \
        if args.kernel_only.startswith("jphi") else None
    fn = {"velocity": lambda: ptrom.bs_velocity(x, Gt, 0.02),
          "velocity_selfjac": lambda: ptrom.bs_velocity(x, Gt, 0.02, selfjac=True),
          "jvp": lambda: ptrom.bs_jvp(x, Gt, 0.02, v),
          "vjp": lambda: ptrom.bs_vjp(x, Gt, 0.02, v),
          "jphi": lambda: ptrom.bs_jphi(x, Gt, 0.02, phi),
          "jphi_tc": lambda: ptrom.bs_jphi(x, Gt, 0.02, phi, prec="tf32x3"),
          "jphi_tc_f16": lambda: ptrom.bs_jphi(x, Gt, 0.02, phi, prec="f16x3")}[args.kernel_only]
    for _ in range(args.warmup + args.steps):
        fn()
    torch.cuda.synchronize()
    print(json.dumps({"kernel_only": args.kernel_only, "n": args.n, "launches": args.warmup + args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ptrom", action="store_true", help="skip the PTROM speed-up leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances leg")
    ap.add_argument("--no-jphi", action="store_true", help="skip the J Phi kernel legs")
    ap.add_argument("--vortex-pair", action="store_true",
                    help="also run the paper's vortex-pair parametric experiment (about 3 minutes)")
    ap.add_argument("--single-vortex", action="store_true",
                    help="run only the single-vortex leg (Table 1 conditions, Tables 2-4 settings) and print it")
    ap.add_argument("--sv-n", type=str, default=",".join(map(str, SV_NS)), help="bodies of the --single-vortex leg")
    ap.add_argument("--sv-cases", type=str, default="1,2,3,4", help="bases cases of the --single-vortex leg")
    ap.add_argument("--c4", action="store_true",
                    help="run only the batched PTROM leg (64 instances of uneven N, one model each) and print it")
    ap.add_argument("--c3", action="store_true",
                    help="run only the parametric PTROM leg (8 training, 4 held-out parameters) and print it")
    ap.add_argument("--c3-n", type=int, default=65536, help="bodies of the --c3 leg")
    ap.add_argument("--c3-steps", type=int, default=1000, help="time steps of the --c3 leg")
    ap.add_argument("--c3-ks", type=str, default="20,40,60", help="POD ranks k of the --c3 leg")
    ap.add_argument("--c3-mults", type=str, default="2,4", help="n_s / k of the --c3 leg")
    ap.add_argument("--c3-thetas", type=str, default="0.5", help="Barnes-Hut thetas of the --c3 leg")
    ap.add_argument("--mushroom", action="store_true",
                    help="also run the paper's mushroom-cloud parametric experiment (about 5 minutes)")
    ap.add_argument("--qr-prec", choices=["fp64", "fp32c"], default="fp64",
                    help="online least-squares precision of the --vortex-pair / --mushroom legs")
    ap.add_argument("--kernel-only", choices=["velocity", "velocity_selfjac", "jvp", "vjp", "jphi", "jphi_tc",
                                              "jphi_tc_f16", "ptrom"],
                    help="profiling aid: launch only this kernel (no JSON metric line)")
    ap.add_argument("--n", type=int, default=16384, help="bodies for --kernel-only")
    args = ap.parse_args()
    if args.kernel_only:
        kernel_only(args)
        return
    if args.single_vortex:
        import torch
        from paper_2103_01983_gb300 import ptrom
        ns = tuple(int(v) for v in args.sv_n.split(","))
        cases = tuple(int(v) - 1 for v in args.sv_cases.split(","))
        print(json.dumps({"single_vortex": single_vortex_leg(ptrom, torch.device("cuda", 0), ns=ns, cases=cases)}),
              flush=True)
        return
    if args.c4:
        import torch
        from paper_2103_01983_gb300 import ptrom
        print(json.dumps({"c4": c4_leg(ptrom, torch.device("cuda", 0))}), flush=True)
        return
    if args.c3:
        import torch
        from paper_2103_01983_gb300 import ptrom
        lst = lambda t, f: tuple(f(v) for v in t.split(","))
        print(json.dumps({"c3": c3_leg(ptrom, torch.device("cuda", 0), n=args.c3_n, steps=args.c3_steps,
                                       ks=lst(args.c3_ks, int), mults=lst(args.c3_mults, int),
                                       thetas=lst(args.c3_thetas, float))}), flush=True)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        args.steps = min(args.steps, 20)
        print(json.dumps(run_reference(args)), flush=True)
        return
    line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
