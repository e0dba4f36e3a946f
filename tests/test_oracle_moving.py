"""Pins of the oracle's moving solid (interface velocity v_I = u_s != 0).

The indicator of the solid is carried with the interface velocity (Sec. 2:
d_t chi + v_I . grad chi = 0), the drag of Sec. 3.2.1 acts on the velocity
relative to the solid, u - u_s, and the solid carries its temperature.  What
the physics fixes:
* the phase field of step n is the initial one displaced by n u_s;
* a fluid moving with the solid feels no drag and stays uniform;
* Galilean invariance: a disc moving at -U through fluid at rest sees the
  flow of a resting disc in a stream of speed U.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_17214_gb300 import inputs as I


@pytest.fixture(autouse=True)
def _threads():
    O.set_threads(0)
    yield


def _box(nx=128, ny=64, u_s=None, U=0.0):
    p = I._base(2, nx, ny)
    I.lattice_air(p, 0.05)
    p["bc"] = ["periodic"] * 6
    p.update({"A_u": 145.0, "eta": 4.0})
    if u_s is not None:
        p["u_s"] = list(u_s) + [0.0]
    phi = I.disc_phi(nx, ny, 48.0, 32.0, 8.0, 4.0).reshape(-1)
    u = np.zeros((2, nx * ny))
    u[0] = U
    return p, O.OracleState(p, phi, np.full(nx * ny, 300.0), u=u)


def test_phase_field_is_displaced_by_the_solid_velocity():
    """u_s = (0.5, -0.25): after 4 steps the field is the initial one moved
    by (+2, -1) cells exactly; after 1 step it lies halfway and a quarter of
    the way between the neighbouring cells (linear interpolation)."""
    p, s = _box(u_s=(0.5, -0.25))
    phi0 = s.phi.reshape(64, 128)
    s.step(1)
    half = s.phase().reshape(64, 128)
    a = 0.5 * (phi0 + np.roll(phi0, 1, axis=1))       # x shifted by 0.5
    ref = 0.75 * a + 0.25 * np.roll(a, -1, axis=0)    # y shifted by -0.25
    assert np.max(np.abs(half - ref)) <= 1e-15
    s.step(3)
    assert np.max(np.abs(s.phase().reshape(64, 128) - np.roll(np.roll(phi0, 2, axis=1), -1,
                                                                 axis=0))) <= 1e-15


def test_fluid_moving_with_the_solid_feels_no_drag():
    """Fluid and disc both at u_s: the drag vanishes and the uniform state
    stays uniform to round-off while the disc moves."""
    us = (0.02, 0.01)
    p, s = _box(u_s=us)
    u0 = np.zeros((2, s.N))
    u0[0], u0[1] = us
    s = O.OracleState(p, s.phi, np.full(s.N, 300.0), u=u0)
    s.step(300)
    u, _, _ = s.moments()
    assert np.max(np.abs(u[0] - us[0])) <= 1e-12
    assert np.max(np.abs(u[1] - us[1])) <= 1e-12
    assert np.max(np.abs(s.diagnostics()["drag"])) <= 1e-12


def test_moving_disc_sees_the_flow_of_a_resting_disc():
    """Galilean invariance: the drag on a disc moving at -U through fluid at
    rest follows the drag on the resting disc in a stream of speed U (both in
    a periodic box, the fluid inside the disc included) to 5 % over 600 steps
    (the lattice scheme is Galilean invariant to O(U^3), and the moving
    disc's phase field is interpolated between cells)."""
    U = 0.02
    _, a = _box(U=U)
    _, b = _box(u_s=(-U, 0.0))
    for _ in range(6):
        a.step(100)
        b.step(100)
        fa, fb = a.diagnostics()["drag"][0], b.diagnostics()["drag"][0]
        assert fa > 0
        assert abs(fb / fa - 1) <= 0.05, (fa, fb)


def test_moving_solid_carries_its_temperature():
    """A solid filling a periodic box, no conduction: a warm spot in the
    solid temperature moves with u_s.  The upwind transport conserves the
    heat content and moves the spot's centroid by exactly u_s per step."""
    nx, ny = 96, 8
    p = I._base(2, nx, ny)
    I.lattice_air(p, 0.05)
    p["bc"] = ["periodic"] * 6
    p.update({"Ts_field": 1, "rhocp_s": 1.0, "lambda_s": 0.0, "u_s": [0.1, 0.0, 0.0]})
    x = np.broadcast_to(np.arange(nx, dtype=np.float64), (ny, nx)).reshape(-1)
    Ts = 300.0 + 50.0 * np.exp(-((x - 30.0) / 4.0) ** 2)
    s = O.OracleState(p, np.ones(nx * ny), Ts.copy(), Ts=Ts.copy())
    s.step(200)
    w0, w1 = Ts - 300.0, s.Ts - 300.0
    assert abs(w1.sum() / w0.sum() - 1) <= 1e-12
    c0, c1 = (x * w0).sum() / w0.sum(), (x * w1).sum() / w1.sum()
    assert abs((c1 - c0) - 20.0) <= 1e-9
