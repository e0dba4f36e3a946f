"""Small, self-contained workloads for profiler captures.

    python -m paper_2310_17214_gb300.profile_cases surrogate [nx ny]
    python -m paper_2310_17214_gb300.profile_cases batch [n_domains tile]

Each case sets up its workload, warms up, and brackets a few steps with
cudaProfilerStart / cudaProfilerStop (torch.cuda.profiler), so that a capture
with `ncu --profile-from-start off` sees only those steps.

surrogate: the two-step six-species bed (FP32 transport); samples the Newton
run (200k rows), trains the network for 30 epochs, copies the Newton run's
state into a surrogate-mode domain, then profiles three surrogate steps and
two Newton steps.
batch: the first n of the 48 batched beds (FP32, K = 0) with one tile shape
at the most resident blocks; profiles two batch steps.
step3d: the 3-D D3Q19 reactive bed (256 x 128 x 128, or its first ncols
columns) in one precision; times 20 steps with CUDA events, then profiles
two steps.
step2d: the 2-D reactive bed (1024 x 256 D2Q9) in one precision with one
kernel; times 50 steps with CUDA events (L2 flushed between steps), then
profiles two steps.
"""
from __future__ import annotations

import sys

from . import inputs as I
from . import surrogate as S
from ._native import Batch, Domain


def surrogate_case(nx=2048, ny=512, precision="fp32"):
    """The two-step bed with the trained surrogate on both network engines
    (tcgen05 and warp-level mma.sync, the latter also with cold tiles
    skipping the network) beside the Newton run: CUDA-event time per step of
    each, then two profiled steps of each."""
    import torch
    from ._native import MLP_ENGINES
    p = I.config4(nx=nx, ny=ny, precision=precision)
    f = I.config4_fields(p)

    def dom_of(chem):
        d = Domain(dict(p, chem=chem), precision)
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"], f["Y"])
        return d

    d = dom_of("implicit")
    X, D = S.collect(d, f["phi"], 200_000, 4, 500, seed=0)
    theta = S.theta_scale(p)
    stats, Xn, Yn = S.normalisation(X, D, theta)
    net, _ = S.train(Xn, Yn, epochs=30, batch=8192)
    rec = S.make_surrogate(stats, X, theta, p["species"], 1e-6)
    doms = {}
    for name in ("tcgen05", "warp_mma", "warp_mma_cold_skip"):
        rec.engine = MLP_ENGINES["tcgen05" if name == "tcgen05" else "warp_mma"]
        rec.skip_eps = 1e-12 if name.endswith("cold_skip") else 0.0
        sd = dom_of("surrogate")
        sd.set_surrogate(net, rec)
        sd.set_state(d.get_state())
        sd.step(5)
        doms[name] = sd
    d.step(5)
    for name, sd in list(doms.items()) + [("newton", d)]:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sd.step(20)
        e1.record()
        torch.cuda.synchronize()
        print(f"{name}: {e0.elapsed_time(e1) / 20:.4f} ms per step", flush=True)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for sd in doms.values():
        sd.step(2)
    d.step(2)
    for sd in list(doms.values()) + [d]:
        sd.scalars()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("fallback/evaluated", {k: v.chem_stats() for k, v in doms.items()})


def batch_case(n=48, tile="32x16"):
    import torch
    doms = []
    for p in I.config5(n=n):
        f = I.config5_fields(p)
        d = Domain(p, "fp32")
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"])
        doms.append(d)
    b = Batch(doms)
    b.set_config(tile, 0)
    b.step(4)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    b.step(2)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(b.config(), sum(p["nx"] * p["ny"] for p in I.config5(n=n)))


def step3d_case(precision="fp32_fp16", ncols=256, kernel="tiled"):
    import time

    import numpy as np
    import torch
    p = I.config3(precision=precision)
    f = I.config3_fields(p)
    if ncols < p["nx"]:
        nx, ny, nz = p["nx"], p["ny"], p["nz"]
        cut = lambda a, k=1: np.ascontiguousarray(
            np.asarray(a).reshape(k, nz, ny, nx)[..., :ncols]).reshape(-1)
        f = {"phi": cut(f["phi"]), "T": cut(f["T"]), "Ts": cut(f["Ts"]),
             "Y": cut(f["Y"], p["K"])}
        p = dict(p, nx=ncols)
    d = Domain(p, precision)
    d.set_phase_field(f["phi"], f["Ts"])
    d.set_fields(f["T"], f["Y"])
    d.select_kernel(kernel)
    d.step(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    d.step(20)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / 20
    N = f["phi"].size
    print(f"step3d {precision} {p['nx']}x{p['ny']}x{p['nz']} kernel {kernel}: "
          f"{ms * 1e3:.1f} us/step, {N / ms / 1e3:.0f} MLUPS", flush=True)
    torch.cuda.profiler.start()
    d.step(2)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("scalars", d.scalars())


def step2d_case(precision="fp32", kernel="tiled", steps=50):
    import torch
    p = I.config2(precision=precision)
    f = I.config2_fields(p)
    d = Domain(p, precision)
    d.set_phase_field(f["phi"], f["Ts"])
    d.set_fields(f["T"], f["Y"])
    d.select_kernel(kernel)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    d.step(5)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        d.step(1)
        e1.record()
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / steps
    N = f["phi"].size
    print(f"step2d {precision} {p['nx']}x{p['ny']} kernel {kernel}: "
          f"{ms * 1e3:.1f} us/step, {N / ms / 1e3:.0f} MLUPS", flush=True)
    torch.cuda.profiler.start()
    d.step(2)
    d.scalars()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


if __name__ == "__main__":
    case = sys.argv[1] if len(sys.argv) > 1 else "surrogate"
    if case == "surrogate":
        args = [int(a) for a in sys.argv[2:4]]
        surrogate_case(*args)
    elif case == "batch":
        batch_case(int(sys.argv[2]) if len(sys.argv) > 2 else 48,
                   sys.argv[3] if len(sys.argv) > 3 else "32x16")
    elif case == "step3d":
        step3d_case(sys.argv[2] if len(sys.argv) > 2 else "fp32_fp16",
                    int(sys.argv[3]) if len(sys.argv) > 3 else 256,
                    sys.argv[4] if len(sys.argv) > 4 else "tiled")
    elif case == "step2d":
        step2d_case(sys.argv[2] if len(sys.argv) > 2 else "fp32",
                    sys.argv[3] if len(sys.argv) > 3 else "tiled")
    else:
        raise SystemExit(f"unknown case {case}")
