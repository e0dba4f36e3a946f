"""Calibrate the one-step CH4 pre-exponential factor with 1-D oracle flames.

The paper does not print its rate constants (BFER, Sec. 4.4); the reactive
workloads use a project-chosen one-step rate Q = A exp(-15000/T)[CH4][O2] with
A chosen so that a 1-D lean (phi = 0.7) flame runs at about 0.2 m/s.  This
script measures the laminar burning speed S_F of the oracle's own scheme
(dx = 25 um, dt = 0.25 us, Sec. 4.4.2) for a few A and prints the A that gives
the target by log-log interpolation (S_F ~ sqrt(A) in the thin-flame limit).

S_F is taken as the paper does for its stationary flame (Sec. 4.4.1): the
inlet speed is driven by the mass-flow feedback, so that the fuel entering
equals the fuel consumed, and once the front no longer moves the inlet speed
is the burning velocity.  The mean front drift over the measuring window is
printed beside it.

Uses only the oracle and the input generators.  Run:
    python oracle/calibrate_one_step.py
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import oracle as O  # noqa: E402
from paper_2310_17214_gb300 import inputs as I  # noqa: E402


def flame_speed(A, nx=480, settle=16000, window=8000):
    """(S_F in m/s, front drift in cells/step over the window, T_ad)."""
    p = I.config2(nx=nx, ny=1)
    p["reactions"] = I.one_step_mechanism(A)
    p["bc"] = ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"]
    p["u_in"] = 0.0
    p["inlet_feedback"] = 0  # CH4
    p["Ts_field"] = 0
    p["A_T"] = 0.0
    p["A_u"] = 0.0
    x = np.arange(nx)
    Yin = np.asarray(p["Y_in"])
    Yb = np.asarray(I.burnt_composition(p["Y_in"], p["species"], p["M"]))
    cp_b = float(np.dot(Yb, p["cp"]))
    q = -float(np.dot(np.asarray(p["hf"]), Yb - Yin))
    Tad = 300.0 + q / cp_b
    w = 0.5 * (1 + np.tanh((x - int(nx * 0.6)) / 4.0))
    T = 300.0 + (Tad - 300.0) * w
    Y = (Yin[:, None] * (1 - w) + Yb[:, None] * w).reshape(-1)
    s = O.OracleState(p, np.zeros(nx), T, Y)

    def front():
        Tm = 0.5 * (300.0 + Tad)
        i = np.where(s.T > Tm)[0].min()
        return i - 1 + (Tm - s.T[i - 1]) / (s.T[i] - s.T[i - 1])

    s.step(settle)
    x0, u = front(), 0.0
    n = 0
    while n < window:
        s.step(500)
        n += 500
        u += s.u_in
    u /= window // 500
    return u * p["dx"] / p["dt"], (front() - x0) / window, Tad


def main():
    target = 0.2
    As = [3e8, 4e8, 5e8]
    res = []
    for A in As:
        sf, drift, Tad = flame_speed(A)
        res.append((A, sf))
        print(f"A = {A:.3e}  S_F = {sf:.4f} m/s  front drift {drift:+.2e} cells/step "
              f"(T_ad = {Tad:.1f} K)", flush=True)
    a = np.log([r[0] for r in res])
    s = np.log([max(r[1], 1e-6) for r in res])
    k, c = np.polyfit(s, a, 1)
    A_star = math.exp(k * math.log(target) + c)
    sf, drift, _ = flame_speed(A_star)
    print(f"calibrated A = {A_star:.4e}  ->  S_F = {sf:.4f} m/s  (drift {drift:+.2e})")


if __name__ == "__main__":
    main()
