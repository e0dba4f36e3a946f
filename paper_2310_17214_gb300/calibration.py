"""Calibration sweeps of the diffuse-interface couplings A_u (Sec. 4.1) and
A_T (Sec. 4.2).

The paper tunes A_u so that the velocity profile of a channel whose walls are
diffuse solid layers (eq. def-phi) matches the sharp-interface channel: the
mean standard error of eq. mean-standard-error-f across the section at 0.9 H
has a minimum at A_u*.  A_T is tuned the same way on the temperature profile
of the channel with hot walls (T_w, gas entering at 300 K).  Each value is an
independent run of the library on the GPU; every run gets its own CUDA
stream, so the runs of a sweep overlap on the device.  The setup (width
L = 50, eta = 8, Re = 100, H = 5 L, characteristic outlet) is the one of Figs.
A_u-vs-MSE and A_T-vs-MSE; the inlet is uniform (times the fluid fraction in
the diffuse channel) in both sweeps.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I


def _run_all(probs, steps, precision, device, chunk, field="u"):
    """Step every problem `steps` times, each domain on its own stream,
    round-robin in chunks; returns the streamwise velocity (field "u") or the
    temperature (field "T") of each."""
    import torch
    from ._native import Domain
    dev = torch.device("cuda", device)
    doms, streams = [], []
    for p in probs:
        st = torch.cuda.Stream(device=dev)
        f = I.di_channel_fields(p)
        d = Domain(p, precision, stream=st.cuda_stream, device=device)
        d.set_phase_field(f["phi"])
        d.set_fields(f["T"], None)
        doms.append(d)
        streams.append(st)
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        for d in doms:
            d.step(n)
        done += n
    torch.cuda.synchronize(dev)
    out = []
    for d in doms:
        out.append(d.get("u")[0] if field == "u" else d.get("T"))
        d.close()
    return out


def _minimum(values, mse):
    """The sampled minimiser and the minimiser of a parabola through the three
    samples around it in (log value, log MSE)."""
    k = int(np.argmin(mse))
    refined = values[k]
    if 0 < k < len(values) - 1:
        x = np.log(values[k - 1:k + 2])
        y = np.log(mse[k - 1:k + 2])
        c2, c1, _ = np.polyfit(x, y, 2)
        if c2 > 0:
            refined = float(math.exp(-c1 / (2 * c2)))
    return values[k], refined


def sweep_A_u(values, L=50, eta=8, solid=8, Re=100.0, u_in=0.05, H=None, steps=15000,
              precision="fp64", device=0, chunk=1000, run=None):
    """MSE(A_u) of the diffuse channel against the sharp one.  Returns the
    values, the MSE of each, the sampled minimiser and the minimiser of a
    parabola through the three samples around it in (log A_u, log MSE).
    `run` (a function from the list of problems to their streamwise
    velocities) replaces the library runs, e.g. by another implementation of
    the same steps."""
    values = [float(a) for a in values]
    p_si = I.di_channel(L=L, eta=eta, solid=solid, Re=Re, u_in=u_in, H=H, sharp=True)
    p_di = [I.di_channel(L=L, eta=eta, solid=solid, Re=Re, u_in=u_in, H=H, A_u=a)
            for a in values]
    if run is None:
        def run(probs):
            return _run_all(probs, steps, precision, device, chunk)
    us = run([p_si] + p_di)
    mse = [I.channel_mse(us[0], u, p_si, p) for u, p in zip(us[1:], p_di)]
    sampled, refined = _minimum(values, mse)
    return {"A_u": values, "mse": mse, "A_u_star_sampled": sampled,
            "A_u_star": refined, "steps": steps, "precision": precision,
            "setup": {"L": L, "eta": eta, "Re": Re, "H": p_si["nx"], "u_in": u_in,
                      "outlet": "characteristic", "section": "0.9 H"}}


def sweep_A_T(values, L=50, eta=8, solid=8, Re=100.0, u_in=0.05, H=None, T_w=400.0,
              A_u=145.0, steps=15000, precision="fp64", device=0, chunk=1000, run=None):
    """MSE(A_T) of the hot-wall diffuse channel against the sharp one (Sec.
    4.2, Fig. A_T-vs-MSE): the temperature across the section at 0.9 H, eq.
    mean-standard-error-f with f = T.  `run` (a function from the list of
    problems to their temperature fields) replaces the library runs, e.g. by
    another implementation of the same steps.  Returns the values, the MSE
    of each, the sampled and refined minimisers, and the paper's fit
    A_T* = 24.24 + 33.81 T_w / T_in as context."""
    values = [float(a) for a in values]
    p_si = I.di_channel(L=L, eta=eta, solid=solid, Re=Re, u_in=u_in, H=H, sharp=True, T_w=T_w)
    p_di = [I.di_channel(L=L, eta=eta, solid=solid, Re=Re, u_in=u_in, H=H, A_u=A_u,
                         T_w=T_w, A_T=a) for a in values]
    if run is None:
        def run(probs):
            return _run_all(probs, steps, precision, device, chunk, field="T")
    Ts = run([p_si] + p_di)
    mse = [I.channel_mse(Ts[0], T, p_si, p) for T, p in zip(Ts[1:], p_di)]
    sampled, refined = _minimum(values, mse)
    return {"A_T": values, "mse": mse, "A_T_star_sampled": sampled, "A_T_star": refined,
            "paper_fit_A_T_star": 24.24 + 33.81 * T_w / p_si["T_in"], "steps": steps,
            "precision": precision,
            "setup": {"L": L, "eta": eta, "Re": Re, "H": p_si["nx"], "u_in": u_in, "T_w": T_w,
                      "T_in": p_si["T_in"], "A_u": A_u, "outlet": "characteristic",
                      "section": "0.9 H"}}
