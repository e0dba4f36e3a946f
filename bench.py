"""Benchmark of the fused PF-LB-FD time step on GB300.

Headline workload: the 3-D reactive particle bed, 256 x 128 x 128 D3Q19,
5 species with the one-step CH4 chemistry, transported solid temperature,
138 seeded ellipsoids (synthetic stand-in for the paper's packed beds), FP32
compute and storage by default (--precision selects FP16-stored residuals or
FP64); the step kernel is the one the library's autotuner picks for the
domain.  A step is one
pass of the whole hot path: pull collide-stream with drag, FD transport of
T / Y / Ts, Arrhenius source, FP64 P0 / mass reduction -- one fused kernel
launch.  The working set (>= 0.5 GB) is larger than the 129 MB L2, so no flush
is needed between steps.

Prints ONE JSON line (rank 0).  `value` is MLUPS with inputs resident in HBM;
legs beside it: the plain FP64 GPU step of the same bed, the other FP32
storage mode, the error of FP32 and FP16-stored runs against the FP64 run per
field after 2000 steps, the 2-D reactive bed (1024 x 256), the learned
chemistry surrogate, the batch of 48 beds, the end-to-end call with host
buffers and the oracle on the host cores.  `--impl reference` times the FP64
CPU oracle on the same workload (the reference arm of this project).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision fp32|fp32_fp16|fp64] [--quick]
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_17214_gb300 import inputs as I  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
KERNEL_SRC = [os.path.join(ROOT, "paper_2310_17214_gb300", "csrc", f)
              for f in ("pflb_kernels.cuh", "pflb_step3d.cuh")]
DEFAULT_PRECISION = "fp32"
METRIC = "MLUPS of the fused PF-LB-FD step (3-D D3Q19 reactive bed 256x128x128)"


def alg_bytes_per_cell(prob, precision):
    """Algorithmic bytes per cell update: populations read + write (with the
    FP16-stored mode, the FP16 residuals plus the cell's FP32 moments), T r/w,
    Y r/w, phi read, Ts r/w (derived fields excluded)."""
    Q = 9 if prob["dim"] == 2 else 19
    b = 8 if precision == "fp64" else 4
    if precision == "fp32_fp16":
        pops = 2 * Q * 2 + 2 * 4 * (prob["dim"] + 1)
    else:
        pops = 2 * Q * b
    K = prob.get("K", 0)
    ts = 2 * b if prob.get("Ts_field") else 0
    return pops + 2 * b + 2 * K * b + b + ts


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_hash():
    """Identity of the step kernels' build: their sources and the compiler flags."""
    from paper_2310_17214_gb300 import build as B
    h = hashlib.sha256()
    for src in KERNEL_SRC:
        with open(src, "rb") as f:
            h.update(f.read())
    h.update(" ".join(B.ARCH + B.FLAGS[:-2]).encode())  # the include path is machine-specific
    return h.hexdigest()[:16]


def _recorded(fname, workload, precision):
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    h = kernel_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == workload and parts[1] == precision and parts[2] == h:
            return float(parts[3])
    return None


def recorded_fp64_flops(workload):
    """FP64 flops per cell of the FP64 step from the committed ncu count, if it
    was taken on the current kernel source (else None)."""
    return _recorded("step_kernel_fp64_flops.txt", workload, "fp64")


def recorded_traffic(workload, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    return _recorded("step_kernel_traffic.txt", workload, precision)


class ClockSampler:
    """SM clock and clock-event reasons sampled through NVML (ctypes, read
    only) every millisecond while the timed region runs."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index):
        self.dev = device_index
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._nvml = None
        self._h = None

    def _open(self):
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if nv.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.dev)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok and nv.nvmlDeviceGetHandleByIndex_v2(self.dev, ctypes.byref(h)) != 0:
            return False
        self._nvml, self._h = nv, h
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = mx.value
        return True

    def _run(self):
        nv, h = self._nvml, self._h
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0:
                r = rs.value if nv.nvmlDeviceGetCurrentClocksEventReasons(
                    h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((mhz.value, r))
            time.sleep(0.001)

    def __enter__(self):
        if self._open():
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._nvml is not None:
            self._t.join(timeout=2)

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "NVML, 1 ms period, timed region"}


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


def workload_name(prob):
    if prob["dim"] == 3:
        return f"reactive_bed_{prob['nx']}x{prob['ny']}x{prob['nz']}_d3q19_k{prob['K']}"
    return f"reactive_bed_{prob['nx']}x{prob['ny']}_d2q9_k{prob['K']}"


def config_of(prob, fields, precision, world=1):
    """The workload's config, identical in both arms of the benchmark."""
    return {"parallelism": f"replicas x{world}" if world > 1 else "single device",
            "workload": workload_name(prob), "nx": prob["nx"], "ny": prob["ny"],
            "nz": prob.get("nz", 1), "lattice": "D3Q19" if prob["dim"] == 3 else "D2Q9",
            "species": prob["K"], "particles": fields["info"]["placed"],
            "porosity_bed": round(fields["info"]["porosity_bed"], 3),
            "precision": precision,
            "l2": "not flushed: the working set is larger than the 129 MB L2"}


# ------------------------------------------------------------------ oracle arm
def oracle_mlups(prob, fields, steps, threads):
    """FP64 CPU oracle on the given grid: (MLUPS, seconds, threads used)."""
    from oracle import oracle as O
    used = O.set_threads(threads)
    s = O.OracleState(prob, fields["phi"], fields["T"], fields["Y"], fields["Ts"])
    t0 = time.perf_counter()
    s.step(steps)
    el = time.perf_counter() - t0
    return fields["phi"].size * steps / el / 1e6, el, used


def cpu_baseline():
    """The oracle on the 64^3 crop of the headline bed: all host cores, and
    one core, each a sample of about 6-10 s."""
    p = I.config3_crop(64)
    f = I.config3_fields(p)
    v_all, el_all, cores = oracle_mlups(p, f, 40, 0)
    v_one, el_one, _ = oracle_mlups(p, f, 8, 1)
    try:
        model = next(ln.split(":", 1)[1].strip() for ln in open("/proc/cpuinfo")
                     if ln.lower().startswith(("model name", "cpu part")))
    except Exception:
        model = None
    return {"value": v_all, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"64^3 crop of the 3-D bed recipe (one-step chemistry, solid field), "
                      f"40 steps on {cores} threads ({el_all:.1f} s); FP64 C with OpenMP "
                      f"over the independent per-cell loops",
            "single_thread": {"value": v_one, "sample": f"8 steps ({el_one:.1f} s)"},
            "host_cpu": model, "nproc": os.cpu_count()}


def run_reference(args, prob, fields, world, rank, pg):
    """Reference arm: the FP64 CPU oracle on the host cores on the headline
    workload, each step a bounded sample (a column crop when the whole grid
    would not fit about two and a half minutes in all)."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    cores = O.set_threads(0)
    nx, ny, nz = prob["nx"], prob["ny"], prob.get("nz", 1)
    plane = ny * nz
    q, f = crop_problem(prob, fields, 16)
    s = O.OracleState(q, f["phi"], f["T"], f["Y"], f["Ts"])
    t0 = time.perf_counter()
    s.step(2)
    rate = 2 * 16 * plane / (time.perf_counter() - t0)  # cells per second
    budget = 150.0 / (args.steps + args.warmup)
    ncols = int(max(8, min(nx, budget * rate / plane)))
    q, f = crop_problem(prob, fields, ncols)
    s = O.OracleState(q, f["phi"], f["T"], f["Y"], f["Ts"])
    for _ in range(args.warmup):
        s.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1)
    el = time.perf_counter() - t0
    N = ncols * plane
    mlups = N * args.steps / el / 1e6
    sample = (f"first {ncols} of {nx} columns of the workload ({N} cells), {args.steps} steps "
              f"after {args.warmup} warm-up steps, FP64 C on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(prob, fields, args.precision, world),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def crop_problem(prob, fields, ncols):
    """The first `ncols` x-columns of the workload (same physics, inlet and
    outlet kept), for bounded CPU samples."""
    q = dict(prob)
    q["nx"] = ncols
    shape = (prob.get("nz", 1), prob["ny"], prob["nx"]) if prob["dim"] == 3 else \
        (prob["ny"], prob["nx"])

    def cut(a, k=1):
        if a is None:
            return None
        return np.ascontiguousarray(np.asarray(a).reshape((k,) + shape)[..., :ncols]).reshape(-1)
    f = {"phi": cut(fields["phi"]), "T": cut(fields["T"]), "Ts": cut(fields["Ts"]),
         "Y": cut(fields["Y"], prob.get("K", 1)) if fields["Y"] is not None else None}
    return q, f


# --------------------------------------------------------------------- GPU arm
KERNEL_FN = {"tiled": "step_kernel", "march": "step3d_march_kernel<prefetch=false>",
             "march_prefetch": "step3d_march_kernel<prefetch=true>", "tma": "step_tma_kernel",
             "persistent": "step_persistent_kernel<32x8>",
             "persistent_32x16": "step_persistent_kernel<32x16>"}


def make_domain(prob, fields, precision, dev, stream, tune=False):
    """A domain of the workload with its fields set; with `tune`, the step
    kernel the library's autotuner picks (state restored afterwards)."""
    from paper_2310_17214_gb300._native import Domain
    dom = Domain(prob, precision, stream=stream, device=dev.index)
    dom.set_phase_field(fields["phi"], fields["Ts"])
    dom.set_fields(fields["T"], fields["Y"])
    dom.tuned = None
    if tune:
        chosen, table = dom.autotune(10)
        dom.tuned = {"chosen": chosen, "us_per_step": table}
    return dom


def time_steps(dom, steps, warmup, dev, st, flush=None, pg=None, clocks=False):
    """CUDA-event time of each of `steps` single steps (after `warmup`)."""
    import torch
    for _ in range(warmup):
        if flush is not None:
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
        if flush is not None:
            flush.zero_()
        e0.record(st)
        dom.step(1)
        e1.record(st)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    barrier(pg)
    if sampler:
        sampler.__exit__()
    return [e0.elapsed_time(e1) for e0, e1 in evs], wall, (sampler.summary() if sampler else None)


def e2e_measure(prob, fields, precision, steps, dev):
    """Public-API round trip per step with HOST buffers: upload the step's
    input state from pinned host memory (pflb_set_state), one step, read the
    result state back into pinned host memory (pflb_get_state)."""
    import torch
    st = torch.cuda.current_stream(dev)
    dom = make_domain(prob, fields, precision, dev, st.cuda_stream)
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


def errors_vs_fp64(prob, fields, steps, dev, precisions):
    """L2 relative error per field (u, T - T_in, Y, Ts - T_in over the whole
    grid) of each FP32 mode against the FP64 GPU run after `steps` steps."""
    import torch
    st = torch.cuda.current_stream(dev)
    out = {}
    for prec in ("fp64",) + tuple(precisions):
        dom = make_domain(prob, fields, prec, dev, st.cuda_stream, tune=True)
        dom.step(steps)
        out[prec] = dom.get("T", "Y", "Ts", "u")
        dom.close()
    l2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    T_in = prob["T_in"]
    ref = out["fp64"]
    res = {"steps": steps, "against": "FP64 GPU run of the same bed"}
    for prec in precisions:
        g = out[prec]
        res[prec] = {"u": l2(g["u"], ref["u"]), "T": l2(g["T"] - T_in, ref["T"] - T_in),
                     "Y": l2(g["Y"], ref["Y"]), "Ts": l2(g["Ts"] - T_in, ref["Ts"] - T_in)}
    return res


def _ms_per_call(dom, nsteps, calls, flush, st):
    """Mean device time of one dom.step(nsteps) call (CUDA events, L2 flushed
    before each call)."""
    import torch
    tot = 0.0
    for _ in range(calls):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dom.step(nsteps)
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / calls


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


def bed2d_leg(dev, flush, peaks, steps=50):
    """The 2-D reactive bed (1024 x 256 D2Q9, 35 MB in FP32: L2-resident, so
    the L2 is flushed between steps) in FP32."""
    import torch
    st = torch.cuda.current_stream(dev)
    p = I.config2(precision="fp32")
    f = I.config2_fields(p)
    dom = make_domain(p, f, "fp32", dev, st.cuda_stream)
    ms = _ms_per_step(dom, steps, flush, st)
    dom.close()
    N = f["phi"].size
    bpc = alg_bytes_per_cell(p, "fp32")
    ach = bpc * N / (ms * 1e-3) / 1e9
    return {"workload": workload_name(p), "precision": "fp32", "ms_per_step": ms,
            "mlups": N / ms / 1e3, "l2": "flushed between steps (256 MiB write)",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                         "alg_bytes_per_cell": bpc}}


def moving_bed_leg(dev, prob, fields, static_ms, steps=20):
    """The headline 3-D bed with its particles translating along the
    periodic y axis (u_s = 0.002 lattice units): per step the z-march step
    plus the kernel that writes the displaced phase field."""
    import torch
    st = torch.cuda.current_stream(dev)
    p = dict(prob, u_s=[0.0, 0.002, 0.0])
    dom = make_domain(p, fields, "fp32", dev, st.cuda_stream)
    dom.select_kernel("march")
    times, _, _ = time_steps(dom, steps, 3, dev, st)
    dom.close()
    ms = float(np.mean(times))
    N = fields["phi"].size
    return {"workload": workload_name(prob) + "_moving_particles", "u_s": p["u_s"],
            "ms_per_step": ms, "mlups": N / ms / 1e3, "kernels_per_step": 2,
            "overhead_vs_static": ms / static_ms - 1.0}


def flame2d_leg(dev, flush, precisions=("fp32", "fp64"), settle=400, steps=200):
    """The 2-D wall-bounded flame (480 x 120 D2Q9, five species, one-step
    chemistry, isothermal walls) held by the inlet feedback: per step the fused
    step kernel plus the two feedback kernels (consumption sum, inlet speed).
    6 MB of state: L2-resident, so the L2 is flushed between steps; the
    launch latency of three small kernels bounds it, not HBM.  Also timed:
    calls of 200 steps (the library replays step pairs from a CUDA graph),
    the L2 flushed before each call."""
    import torch
    st = torch.cuda.current_stream(dev)
    out = {}
    for prec in precisions:
        p = I.config6(precision=prec)
        f = I.config6_fields(p)
        dom = make_domain(p, f, prec, dev, st.cuda_stream)
        dom.step(settle)
        ms = _ms_per_step(dom, steps, flush, st)
        ms_long = _ms_per_call(dom, 200, 5, flush, st) / 200
        sc = dom.scalars()
        dom.close()
        N = f["phi"].size
        out[prec] = {"ms_per_step": ms, "mlups": N / ms / 1e3, "kernels_per_step": 3,
                     "ms_per_step_200_step_calls": ms_long, "mlups_200_step_calls": N / ms_long / 1e3,
                     "u_in_m_s": sc["u_in"] * p["dx"] / p["dt"],
                     "steps_before": settle + steps + 3 + 1000}
    q = I.config6()
    return {"workload": f"wall_bounded_flame_{q['nx']}x{q['ny']}_d2q9_k{q['K']}",
            "l2": "flushed between steps (256 MiB write)",
            **out}


def calibration_leg(dev, values=(25, 50, 75, 100, 145, 200, 300, 450), steps=15000):
    """The A_u calibration sweep of Sec. 4.1 (diffuse vs sharp channel,
    L = 50, eta = 8, Re = 100, characteristic outlet): one library run per
    A_u, each on its own stream; wall time of the whole sweep and the A_u
    that minimises the velocity MSE (the paper's 145 is context: its outlet
    scheme and numerics differ)."""
    import time
    import torch
    from paper_2310_17214_gb300 import calibration
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r = calibration.sweep_A_u(values, steps=steps, precision="fp64", device=dev.index)
    torch.cuda.synchronize(dev)
    r["wall_s"] = time.perf_counter() - t0
    r["runs"] = len(values) + 1
    return r


def surrogate_leg(dev, flush, steps=2000, samples=1_000_000, epochs=40, tol=1e-6):
    """The learned chemistry on the two-step bed (2048 x 512, six species):
    sample the Newton run (FP32 transport), train on the GPU, run the
    surrogate from the same initial state, and compare it with the Newton
    run and with the plain FP64 run after `steps` steps; then time the plain
    FP64 step (FP64 transport and Newton), the FP32 + Newton step and the
    FP32 + surrogate step, the latter also with cold tiles skipping the
    network (skip_eps)."""
    import torch
    from paper_2310_17214_gb300 import surrogate as S
    st = torch.cuda.current_stream(dev)
    p = I.config4(precision="fp32")
    f = I.config4_fields(p)

    def dom_of(chem, prec):
        return make_domain(dict(p, chem=chem), f, prec, dev, st.cuda_stream)

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
    T_sur = sur.get("T")
    err = S.flame_errors(T_sur, ref.get("T"), f["phi"], p)
    d64 = dom_of("implicit", "fp64")
    d64.step(steps)
    err64 = S.flame_errors(T_sur, d64.get("T"), f["phi"], p)
    d64.close()
    # the same network with cold tiles skipping it (increment bound 1e-12)
    skip_eps = 1e-12
    sk = dom_of("surrogate", "fp32")
    rec_skip = S.make_surrogate(stats, X, theta, p["species"], tol, skip_eps=skip_eps)
    T_skip = S.skip_temperature(net.get_params(), rec_skip, p["M"])
    sk.set_surrogate(net, rec_skip)
    sk.step(steps)
    err_skip = S.flame_errors(sk.get("T"), ref.get("T"), f["phi"], p)
    fb, ev = sur.chem_stats()
    t_newton32 = _ms_per_step(ref, 30, flush, st)
    t_sur = _ms_per_step(sur, 100, flush, st)
    # the same network on the tcgen05 engine, same state
    from paper_2310_17214_gb300._native import MLP_ENGINES
    rec = S.make_surrogate(stats, X, theta, p["species"], tol)
    rec.engine = MLP_ENGINES["tcgen05"]
    sw = dom_of("surrogate", "fp32")
    sw.set_surrogate(net, rec)
    sw.set_state(sur.get_state())
    t_tc = _ms_per_step(sw, 100, flush, st)
    sw.close()
    sk.set_state(sur.get_state())
    t_skip = _ms_per_step(sk, 100, flush, st)
    sk.close()
    d64 = dom_of("implicit", "fp64")
    t_plain64 = _ms_per_step(d64, 20, flush, st)
    for d in (ref, sur, d64):
        d.close()
    net.close()
    N = f["phi"].size
    return {"workload": f"two_step_bed_{p['nx']}x{p['ny']}_d2q9_k6",
            "plain_fp64_ms_per_step": t_plain64, "fp32_newton_ms_per_step": t_newton32,
            "fp32_surrogate_ms_per_step": t_sur,
            "network_engine": "warp-level mma.sync (32 cells per warp)",
            "fp32_surrogate_tcgen05_ms_per_step": t_tc,
            "fp32_surrogate_cold_skip_ms_per_step": t_skip, "cold_skip_eps": skip_eps,
            "cold_skip_T_K": T_skip,
            "error_vs_fp32_newton_cold_skip": err_skip,
            "surrogate_mlups": N / t_sur / 1e3, "plain_fp64_mlups": N / t_plain64 / 1e3,
            "speedup_vs_plain_fp64": t_plain64 / t_sur,
            "speedup_vs_fp32_newton": t_newton32 / t_sur,
            "error_after_steps": steps,
            "error_vs_fp32_newton": err, "error_vs_plain_fp64": err64,
            "fallback_frac": fb / ev if ev else None, "residual_tol": tol,
            "samples": int(len(X)), "sample_s": t_collect, "train_epochs": epochs,
            "train_s": t_train, "train_loss": loss}


def batch_leg(dev, peaks, steps=200):
    """48 uneven 2-D beds without species (8.5 M cells, FP32): aggregate
    MLUPS of the batched persistent kernel (tile shape and grid from the
    autotuner, graph replay) against the same domains advanced by 48
    separate launches per step.  Inputs exceed L2 (no flush needed)."""
    import torch
    from paper_2310_17214_gb300._native import Batch
    st = torch.cuda.current_stream(dev)
    doms, N = [], 0
    for p in I.config5():
        f = I.config5_fields(p)
        doms.append(make_domain(p, f, "fp32", dev, st.cuda_stream))
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
    bpc = 2 * 9 * 4 + 2 * 4 + 4
    achieved = bpc * N / (ms_batch * 1e-3) / 1e9
    out = {"workload": f"batched_beds_48_domains_{N}_cells_d2q9_k0", "cells": N,
           "domains": len(doms), "batch_mlups": N / ms_batch / 1e3,
           "batch_ms_per_step": ms_batch, "separate_launches_mlups": N / ms_sep / 1e3,
           "separate_ms_per_step": ms_sep, "speedup_vs_separate": ms_sep / ms_batch,
           "config": cfg, "autotune_us_per_step": {f"{t}/{k}": v for (t, k), v in table.items()},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                        "alg_bytes_per_cell": bpc},
           "gpu_launches_per_step": 1}
    b.close()
    for d in doms:
        d.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=DEFAULT_PRECISION,
                    choices=["fp32", "fp64", "fp32_fp16"])
    ap.add_argument("--quick", action="store_true", help="the headline only, no legs")
    ap.add_argument("--kernel", default=None,
                    help="step kernel of the headline (tiled, march, ...) instead of the "
                         "autotuner's choice (for profiler runs, where the autotuner's own "
                         "timings are distorted)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world, rank, local, pg = dist_setup(args.gpus)
    prob = I.config3(precision=args.precision)
    fields = I.config3_fields(prob)

    if args.impl == "reference":
        run_reference(args, prob, fields, world, rank, pg)
        return

    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    N = fields["phi"].size
    peaks, peak_kind = measured_peaks()

    dom = make_domain(prob, fields, args.precision, dev, st.cuda_stream, tune=args.kernel is None)
    if args.kernel is not None:
        dom.select_kernel(args.kernel)
        dom.tuned = {"chosen": args.kernel, "us_per_step": None}
    tuned = dom.tuned
    ms, wall, clk = time_steps(dom, args.steps, args.warmup, dev, st, pg=pg, clocks=(rank == 0))
    final_step = dom.scalars()["step"]
    dom.close()
    t_sum = sum(ms) / 1e3
    t_max = max_over_ranks(pg, t_sum)
    value = world * N * args.steps / t_max / 1e6
    bpc = alg_bytes_per_cell(prob, args.precision)
    per_launch = t_sum / args.steps
    achieved = bpc * N / per_launch / 1e9
    workload = workload_name(prob)
    kname = {"fp32": "float,float", "fp32_fp16": "float,__half", "fp64": "double,double"}
    kernel = f"{KERNEL_FN[tuned['chosen']]} (3-D, K=5, {kname[args.precision]})"

    extra = {}
    if not args.quick and rank == 0:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        legs = {}
        for prec in ("fp32", "fp32_fp16", "fp64"):
            if prec == args.precision:
                continue
            d = make_domain(prob, fields, prec, dev, st.cuda_stream, tune=True)
            n = 10 if prec == "fp64" else 50
            m, _, _ = time_steps(d, n, 3, dev, st)
            tl = d.tuned
            d.close()
            t = sum(m) / len(m) / 1e3
            b = alg_bytes_per_cell(prob, prec)
            legs[prec] = {"ms_per_step": t * 1e3, "mlups": N / t / 1e6,
                          "alg_bytes_per_cell": b, "achieved_gbs": b * N / t / 1e9,
                          "hbm_frac": b * N / t / 1e9 / peaks["hbm_gbs"], "autotune": tl}
        legs[args.precision] = {"ms_per_step": per_launch * 1e3, "mlups": N / per_launch / 1e6,
                                "alg_bytes_per_cell": bpc, "achieved_gbs": achieved,
                                "hbm_frac": achieved / peaks["hbm_gbs"], "autotune": tuned}
        # the FP64 step is bound by the FP64 pipe: its roofline is the probed FMA rate
        from paper_2310_17214_gb300._native import probe_fp64_tflops
        peak64 = probe_fp64_tflops(dev.index)
        fpc = recorded_fp64_flops(workload)
        t64 = legs["fp64"]["ms_per_step"] / 1e3
        ach64 = fpc * N / t64 / 1e12 if fpc else None
        legs["fp64"]["roofline"] = {
            "bound": "alu", "unit": "TFLOP/s", "peak": peak64,
            "peak_kind": "measured FP64 FMA rate (pflb_probe_fp64_fma)",
            "flops_per_cell": fpc, "achieved": ach64, "frac": ach64 / peak64 if ach64 else None}
        extra["precision_legs"] = legs
        extra["speedup_vs_fp64"] = {p_: t64 / (legs[p_]["ms_per_step"] / 1e3)
                                    for p_ in ("fp32", "fp32_fp16")}
        extra["error_vs_fp64"] = errors_vs_fp64(prob, fields, 2000, dev, ("fp32", "fp32_fp16"))
        extra["bed_2d"] = bed2d_leg(dev, flush, peaks)
        extra["flame_2d"] = flame2d_leg(dev, flush)
        extra["moving_bed"] = moving_bed_leg(dev, prob, fields, legs["fp32"]["ms_per_step"])
        extra["calibration_A_u"] = calibration_leg(dev)
        extra["surrogate"] = surrogate_leg(dev, flush)
        extra["batch"] = batch_leg(dev, peaks)
        e2e_v, nb = e2e_measure(prob, fields, args.precision, 10, dev)
        e2e = {"value": e2e_v, "unit": "MLUPS", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb,
               "what": "pflb_set_state from pinned host + pflb_step(1) + pflb_get_state to "
                       "pinned host, per step"}
        from oracle import oracle as O
        O.build()
        cpu = cpu_baseline()
    else:
        e2e, cpu = None, None

    if rank != 0:
        return
    cfg = config_of(prob, fields, args.precision, world)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp32_fp16": "f32 (f16-stored populations)"}[
            args.precision],
        "data": "synthetic (seeded ellipsoid packing, porosity %.3f in the bed)" %
                fields["info"]["porosity_bed"],
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "traffic": recorded_traffic(workload, args.precision),
                     "peak_kind": peak_kind + " (copy burst)",
                     "alg_bytes_per_cell": bpc, "kernel": kernel},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clk, "wall_s_timed": wall, "final_step": final_step,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
