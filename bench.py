"""Benchmark of the fused PF-LB-FD time step on GB300.

Workload: the 2-D reactive particle bed, 1024 x 256 D2Q9, 5 species with the
one-step CH4 chemistry, transported solid temperature, 40 seeded ellipses
(synthetic stand-in for the paper's packed beds).  A step is one pass of the
whole hot path: pull collide-stream with drag, FD transport of T / Y / Ts,
Arrhenius source, FP64 P0 / mass reduction; one fused kernel launch.

Prints ONE JSON line (rank 0).  `value` is MLUPS of the FP32 path (the
configuration's mixed-precision leg) with inputs resident in HBM and L2
flushed between steps; the plain FP64 GPU step is timed alongside and the
error of FP32 against it is reported.  `--impl reference` times the FP64 CPU
oracle instead (the reference arm of this project).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_17214_gb300 import inputs as I  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
KERNEL_SRC = os.path.join(ROOT, "paper_2310_17214_gb300", "csrc", "pflb_kernels.cuh")


def alg_bytes_per_cell(prob, precision):
    """Algorithmic bytes per cell update: populations read + write, T r/w,
    Y r/w, phi read, Ts r/w (derived fields excluded)."""
    Q = 9 if prob["dim"] == 2 else 19
    b_g = {"fp64": 8, "fp32": 4, "fp32_fp16": 2}[precision]
    b = 8 if precision == "fp64" else 4
    K = prob.get("K", 0)
    ts = 2 * b if prob.get("Ts_field") else 0
    return 2 * Q * b_g + 2 * b + 2 * K * b + b + ts


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_hash():
    """Identity of the step kernel's build: its source and the compiler flags."""
    from paper_2310_17214_gb300 import build as B
    h = hashlib.sha256()
    with open(KERNEL_SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(B.ARCH + B.FLAGS[:-2]).encode())  # the include path is machine-specific
    return h.hexdigest()[:16]


def recorded_fp64_flops(workload):
    """FP64 flops per cell of the FP64 step from the committed ncu count, if
    it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_fp64_flops.txt")
    if not os.path.exists(path):
        return None
    h = kernel_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == workload and parts[1] == "fp64" and parts[2] == h:
            return float(parts[3])
    return None


def recorded_traffic(workload, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == workload and parts[1] == precision and parts[2] == h:
            return float(parts[3])
    return None


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle arm
def time_oracle(prob, fields, budget_s=12.0, max_steps=None, min_steps=2):
    """Time the FP64 CPU oracle on the full grid (single thread) for about
    budget_s seconds.  Returns (MLUPS, steps, seconds)."""
    from oracle import oracle as O
    s = O.OracleState(prob, fields["phi"], fields["T"], fields["Y"], fields["Ts"])
    N = fields["phi"].size
    n, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        n += 1
        el = time.perf_counter() - t0
        if (el >= budget_s and n >= min_steps) or (max_steps and n >= max_steps):
            break
    return N * n / el / 1e6, n, el


def crop_problem(prob, fields, ncols):
    """The first `ncols` columns of the workload (same physics, inlet and
    outlet kept), for bounded CPU samples."""
    q = dict(prob)
    q["nx"] = ncols
    nx, ny = prob["nx"], prob["ny"]
    cut = lambda a, k=1: None if a is None else \
        np.ascontiguousarray(np.asarray(a).reshape(k, ny, nx)[:, :, :ncols]).reshape(-1)
    f = {"phi": cut(fields["phi"]), "T": cut(fields["T"]), "Ts": cut(fields["Ts"]),
         "Y": cut(fields["Y"], prob.get("K", 1)) if fields["Y"] is not None else None}
    return q, f


def run_reference(args, prob, fields, world, rank, pg):
    """Reference arm: the FP64 CPU oracle on the host, each step a bounded
    sample (a column crop of the workload) so that warm-up plus timed steps
    take about two and a half minutes in total."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    ny = prob["ny"]
    q, f = crop_problem(prob, fields, 64)
    s = O.OracleState(q, f["phi"], f["T"], f["Y"], f["Ts"])
    t0 = time.perf_counter()
    s.step(2)
    rate = 2 * 64 * ny / (time.perf_counter() - t0)  # cells per second
    budget = 150.0 / (args.steps + args.warmup)
    ncols = int(max(8, min(prob["nx"], budget * rate / ny)))
    q, f = crop_problem(prob, fields, ncols)
    s = O.OracleState(q, f["phi"], f["T"], f["Y"], f["Ts"])
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    el = time.perf_counter() - t0
    N = ncols * ny
    mlups = N * args.steps / el / 1e6
    sample = (f"first {ncols} of {prob['nx']} columns x {ny} rows of the workload, "
              f"{args.steps} steps after {args.warmup} warm-up steps, single-threaded FP64 C")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"reactive_bed_{prob['nx']}x{ny}_d2q9_k5", "nx": prob["nx"],
                       "ny": ny, "lattice": "D2Q9", "species": prob["K"]},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "MLUPS of the fused PF-LB-FD step (2-D reactive bed 1024x256 D2Q9)"


# --------------------------------------------------------------------- GPU arm
def time_gpu(prob, fields, precision, steps, warmup, dev, flush, pg=None, clocks=False):
    import torch
    from paper_2310_17214_gb300._native import Domain
    st = torch.cuda.current_stream(dev)
    dom = Domain(prob, precision, stream=st.cuda_stream, device=dev.index)
    dom.set_phase_field(fields["phi"], fields["Ts"])
    dom.set_fields(fields["T"], fields["Y"])
    for _ in range(warmup):
        flush.zero_()
        dom.step(1)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    barrier(pg)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index) if clocks else None
    if sampler:
        sampler.__enter__()
    w0 = time.perf_counter()
    for e0, e1 in evs:
        flush.zero_()
        e0.record(st)
        dom.step(1)
        e1.record(st)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    barrier(pg)
    if sampler:
        sampler.__exit__()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    sc = dom.scalars()
    return dom, ms, wall, (sampler.summary() if sampler else None), sc


def e2e_measure(prob, fields, precision, steps, dev):
    """Public-API round trip per step with HOST buffers: upload the step's
    input state from pinned host memory (pflb_set_state), one step, read the
    result state back into pinned host memory (pflb_get_state)."""
    import torch
    from paper_2310_17214_gb300._native import Domain
    st = torch.cuda.current_stream(dev)
    dom = Domain(prob, precision, stream=st.cuda_stream, device=dev.index)
    dom.set_phase_field(fields["phi"], fields["Ts"])
    dom.set_fields(fields["T"], fields["Y"])
    nb = dom.state_bytes()
    h_in = torch.empty(nb, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nb, dtype=torch.uint8).pin_memory()
    dom.get_state(h_in)
    for _ in range(3):
        dom.set_state(h_in)
        dom.step(1)
        dom.get_state(h_out)
        h_in.copy_(h_out)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        dom.set_state(h_in)
        dom.step(1)
        dom.get_state(h_out)
        h_in, h_out = h_out, h_in
    el = time.perf_counter() - t0
    dom.close()
    return fields["phi"].size * steps / el / 1e6, nb


def error_vs_fp64(prob, fields, steps, dev):
    """L2 relative error of the FP32 path against the FP64 GPU path after
    `steps` steps (u and T - T_in over the whole grid)."""
    import torch
    from paper_2310_17214_gb300._native import Domain
    st = torch.cuda.current_stream(dev)
    out = {}
    for prec in ("fp64", "fp32"):
        dom = Domain(prob, prec, stream=st.cuda_stream, device=dev.index)
        dom.set_phase_field(fields["phi"], fields["Ts"])
        dom.set_fields(fields["T"], fields["Y"])
        dom.step(steps)
        out[prec] = dom.get("T", "u")
        dom.close()
    l2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"steps": steps,
            "u_l2_rel": l2(out["fp32"]["u"], out["fp64"]["u"]),
            "T_l2_rel": l2(out["fp32"]["T"] - prob["T_in"], out["fp64"]["T"] - prob["T_in"])}


def _ms_per_step(dom, steps, flush, st):
    """Mean device time of one step (CUDA events, L2 flushed between steps)."""
    import torch
    for _ in range(3):
        flush.zero_()
        dom.step(1)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dom.step(1)
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def surrogate_leg(dev, flush, steps=2000, samples=1_000_000, epochs=40, tol=1e-6):
    """The learned chemistry on the two-step bed (2048 x 512, six species):
    sample the Newton run (FP32 transport), train on the GPU, run the
    surrogate from the same initial state, and compare it with the Newton
    run after `steps` steps; then time the plain FP64 step (FP64 transport
    and Newton), the FP32 + Newton step and the FP32 + surrogate step."""
    import torch
    from paper_2310_17214_gb300 import surrogate as S
    from paper_2310_17214_gb300._native import Domain
    st = torch.cuda.current_stream(dev)
    p = I.config4(precision="fp32")
    f = I.config4_fields(p)

    def dom_of(chem, prec):
        d = Domain(dict(p, chem=chem), prec, stream=st.cuda_stream, device=dev.index)
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"], f["Y"])
        return d

    ref = dom_of("implicit", "fp32")
    t0 = time.perf_counter()
    X, D = S.collect(ref, f["phi"], samples, 8, steps // 8, seed=0)
    t_collect = time.perf_counter() - t0
    ref.step(steps - 7 * (steps // 8))
    theta = S.theta_scale(p)
    stats, Xn, Yn = S.normalisation(X, D, theta)
    t0 = time.perf_counter()
    net, loss = S.train(Xn, Yn, epochs=epochs, batch=8192, seed=0, device=dev.index)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    sur = dom_of("surrogate", "fp32")
    sur.set_surrogate(net, S.make_surrogate(stats, X, theta, p["species"], tol))
    sur.step(steps)
    err = S.flame_errors(sur.get("T"), ref.get("T"), f["phi"], p)
    fb, ev = sur.chem_stats()
    t_newton32 = _ms_per_step(ref, 30, flush, st)
    t_sur = _ms_per_step(sur, 100, flush, st)
    d64 = dom_of("implicit", "fp64")
    t_plain64 = _ms_per_step(d64, 20, flush, st)
    for d in (ref, sur, d64):
        d.close()
    net.close()
    N = f["phi"].size
    return {"workload": f"two_step_bed_{p['nx']}x{p['ny']}_d2q9_k6",
            "plain_fp64_ms_per_step": t_plain64, "fp32_newton_ms_per_step": t_newton32,
            "fp32_surrogate_ms_per_step": t_sur,
            "surrogate_mlups": N / t_sur / 1e3, "plain_fp64_mlups": N / t_plain64 / 1e3,
            "speedup_vs_plain_fp64": t_plain64 / t_sur,
            "speedup_vs_fp32_newton": t_newton32 / t_sur,
            "error_after_steps": steps, "error_vs": "FP32 + Newton run from the same state",
            **err, "fallback_frac": fb / ev if ev else None, "residual_tol": tol,
            "samples": int(len(X)), "sample_s": t_collect, "train_epochs": epochs,
            "train_s": t_train, "train_loss": loss}


def batch_leg(dev, steps=200):
    """48 uneven 2-D beds without species (8.5 M cells, FP32): aggregate
    MLUPS of the batched persistent kernel (tile shape and grid from the
    autotuner, graph replay) against the same domains advanced by 48
    separate launches per step.  Inputs exceed L2 (no flush needed)."""
    import torch
    from paper_2310_17214_gb300._native import Batch, Domain
    st = torch.cuda.current_stream(dev)
    probs = I.config5()
    doms, N = [], 0
    for p in probs:
        f = I.config5_fields(p)
        d = Domain(p, "fp32", stream=st.cuda_stream, device=dev.index)
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"])
        doms.append(d)
        N += f["phi"].size

    def timed(fn, k):
        fn(2)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn(k)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    def separate(k):
        for _ in range(k):
            for d in doms:
                d.step(1)

    ms_sep = timed(separate, max(10, steps // 4))
    b = Batch(doms)
    cfg, table = b.autotune(steps=5)
    ms_batch = timed(b.step, steps)
    peaks, kind = measured_peaks()
    bpc = 2 * 9 * 4 + 2 * 4 + 4
    achieved = bpc * N / (ms_batch * 1e-3) / 1e9
    out = {"workload": f"batched_beds_48_domains_{N}_cells_d2q9_k0", "cells": N,
           "domains": len(doms), "batch_mlups": N / ms_batch / 1e3,
           "batch_ms_per_step": ms_batch, "separate_launches_mlups": N / ms_sep / 1e3,
           "separate_ms_per_step": ms_sep, "speedup_vs_separate": ms_sep / ms_batch,
           "config": cfg, "autotune_us_per_step": {f"{t}/{k}": v for (t, k), v in table.items()},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                        "alg_bytes_per_cell": bpc, "peak_kind": kind},
           "gpu_launches_per_step": 1}
    b.close()
    for d in doms:
        d.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_fp16"])
    ap.add_argument("--quick", action="store_true", help="skip the FP64, e2e and CPU legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local, pg = dist_setup(args.gpus)
    prob = I.config2(precision=args.precision)
    fields = I.config2_fields(prob)
    porosity = fields["info"]["porosity_bed"]

    if args.impl == "reference":
        run_reference(args, prob, fields, world, rank, pg)
        return

    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    N = fields["phi"].size

    dom, ms, wall, clk, sc = time_gpu(prob, fields, args.precision, args.steps, args.warmup,
                                      dev, flush, pg, clocks=(rank == 0))
    dom.close()
    t_sum = sum(ms) / 1e3
    t_max = max_over_ranks(pg, t_sum)
    value = world * N * args.steps / t_max / 1e6
    peaks, peak_kind = measured_peaks()
    bpc = alg_bytes_per_cell(prob, args.precision)
    per_launch = t_sum / args.steps
    achieved = bpc * N / per_launch / 1e9
    workload = f"reactive_bed_{prob['nx']}x{prob['ny']}_d2q9_k5"
    traffic = recorded_traffic(workload, args.precision)

    extra = {}
    if not args.quick and rank == 0:
        d64, ms64, wall64, _, _ = time_gpu(prob, fields, "fp64", max(20, args.steps // 4),
                                           args.warmup, dev, flush)
        d64.close()
        t64 = sum(ms64) / len(ms64) / 1e3
        extra["fp64_step"] = {"value": N / t64 / 1e6, "unit": "MLUPS",
                              "ms_per_step": t64 * 1e3, "steps": len(ms64),
                              "alg_bytes_per_cell": alg_bytes_per_cell(prob, "fp64"),
                              "achieved_gbs": alg_bytes_per_cell(prob, "fp64") * N / t64 / 1e9}
        # the FP64 step is bound by the FP64 pipe: its roofline is the probed FMA rate
        from paper_2310_17214_gb300._native import probe_fp64_tflops
        peak64 = probe_fp64_tflops(dev.index)
        fpc = recorded_fp64_flops(workload)
        ach64 = fpc * N / t64 / 1e12 if fpc else None
        extra["fp64_step"]["roofline"] = {
            "bound": "alu", "unit": "TFLOP/s", "peak": peak64,
            "peak_kind": "measured FP64 FMA rate (pflb_probe_fp64_fma)",
            "flops_per_cell": fpc, "achieved": ach64,
            "frac": ach64 / peak64 if ach64 else None}
        extra["speedup_vs_fp64"] = t64 / per_launch
        extra["error_vs_fp64"] = error_vs_fp64(prob, fields, 500, dev)
        extra["surrogate"] = surrogate_leg(dev, flush)
        extra["batch"] = batch_leg(dev)
        e2e_v, nb = e2e_measure(prob, fields, args.precision, 30, dev)
        e2e = {"value": e2e_v, "unit": "MLUPS", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb,
               "what": "pflb_set_state from pinned host + pflb_step(1) + pflb_get_state to "
                       "pinned host, per step"}
        from oracle import oracle as O
        O.build()
        cv, cn, ce = time_oracle(prob, fields, budget_s=12.0)
        cpu = {"value": cv, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"full {prob['nx']}x{prob['ny']} grid, {cn} steps ({ce:.1f} s, "
                         f"single-threaded FP64 C)"}
    else:
        e2e, cpu = None, None

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp32_fp16": "f32 (f16-stored populations)"}[
            args.precision],
        "data": "synthetic (seeded ellipse packing, porosity %.3f in the bed)" % porosity,
        "config": {"workload": workload, "nx": prob["nx"], "ny": prob["ny"], "lattice": "D2Q9",
                   "species": prob["K"], "precision": args.precision,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_kind": peak_kind + " (copy burst)",
                     "alg_bytes_per_cell": bpc, "kernel": "step_kernel<2,5,float,float>"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clk, "wall_s_timed": wall, "final_step": sc["step"],
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
