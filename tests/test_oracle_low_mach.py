"""Pins of the oracle's low-Mach coupling and of the inlet feedback against
what the conservation laws fix.

* Mass: with rho from the EOS at uniform P0 (Sec. 3, eq.
  rho-in-terms-of-P0-and-T) the continuity equation becomes the divergence
  constraint div u = (1/T) DT/Dt + Mw sum_k (1/M_k) DY_k/Dt - (1/P0) dP0/dt
  that the LB source carries (Sec. 3.3, eq. body-force).  In a steady heated
  stream the mass entering must then leave: the inflow and outflow of
  phi_f rho u balance and the fluid mass stops changing.  A divergence built
  from the Eulerian increment alone (no convection), or a P_h that takes only
  half of rho cs^2 D and not half of the whole zeroth moment of the source,
  leaves a defect of several per cent of the throughput.
* Inlet feedback (Sec. 4.4.1): when the inlet speed carries in exactly the
  fuel that the flame consumes, the flame front stays where it is.
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


def test_heated_channel_closes_the_mass_balance():
    """Channel with the disc held at 2 T_in (the Cd/Nu workload): once the
    heated wake is steady, the fluid mass no longer changes and the summed
    outflow equals the summed inflow to 1e-3 of the throughput."""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    s = O.OracleState(p, f["phi"], f["T"], u=f["u"])
    d0 = s.diagnostics()
    s.step(6000)
    d1 = s.diagnostics()
    s.step(2000)
    d2 = s.diagnostics()

    def residual(d):
        return (d["mass"] - d0["mass"]) - (d["flux_in_total"] - d["flux_out_total"])

    throughput = d2["flux_in_total"] - d1["flux_in_total"]
    assert throughput > 0
    # the heated wake is lighter: the fluid mass fell, and now holds
    assert d1["mass"] < d0["mass"]
    assert abs(d2["mass"] - d1["mass"]) <= 1e-4 * d2["mass"]
    # steady: inflow and outflow balance over the last 2000 steps
    assert abs(residual(d2) - residual(d1)) <= 1e-3 * throughput


def _flame_1d(nx=480, feedback=True):
    p = I.config2(nx=nx, ny=1)
    p["bc"] = ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"]
    p["u_in"], p["Ts_field"], p["A_T"], p["A_u"] = 0.0, 0, 0.0, 0.0
    if feedback:
        p["inlet_feedback"] = 0  # CH4
    x = np.arange(nx)
    Yin = np.asarray(p["Y_in"])
    Yb = np.asarray(I.burnt_composition(p["Y_in"], p["species"], p["M"]))
    Tad = 300.0 - float(np.dot(np.asarray(p["hf"]), Yb - Yin)) / float(np.dot(Yb, p["cp"]))
    w = 0.5 * (1 + np.tanh((x - int(nx * 0.6)) / 4.0))
    T = 300.0 + (Tad - 300.0) * w
    Y = (Yin[:, None] * (1 - w) + Yb[:, None] * w).reshape(-1)
    return p, O.OracleState(p, np.zeros(nx), T, Y), Tad


def _front(T, Tad):
    Tm = 0.5 * (300.0 + Tad)
    i = np.where(T > Tm)[0].min()
    return i - 1 + (Tm - T[i - 1]) / (T[i] - T[i - 1])


def test_inlet_feedback_holds_a_one_dimensional_flame_in_place():
    """1-D lean CH4 flame (phi = 0.7, one-step rate) with the feedback on the
    fuel: the inlet speed settles and the front moves by less than a tenth of
    the distance the inflow travels meanwhile.  A feedback off by a constant
    factor (a wrong density, fuel fraction or inlet area) moves the front by
    that factor's deviation times the inflow's travel."""
    p, s, Tad = _flame_1d()
    assert s.u_in == 0.0
    s.step(16000)
    x0, u0 = _front(s.T, Tad), s.u_in
    us = []
    for _ in range(16):
        s.step(500)
        us.append(s.u_in)
    x1, u1 = _front(s.T, Tad), float(np.mean(us))
    travel = u1 * 8000
    assert u1 > 0 and abs(u1 / u0 - 1) <= 0.02
    assert abs(x1 - x0) <= 0.1 * travel, (x1 - x0, travel)


def test_inlet_feedback_off_keeps_the_set_inlet_speed():
    p, s, _ = _flame_1d(nx=64, feedback=False)
    s.step(20)
    assert s.u_in == p["u_in"] == 0.0


# ------------------------------------------------ characteristic outlet
def _pulse_channel(outlet, nx=400, steps=700):
    """A right-going plane acoustic pulse (P_h = rho cs u) in a 1-D channel
    with a closed inlet; returns the acoustic energy before and after the
    pulse has met the outlet."""
    p = I._base(2, nx, 1)
    I.lattice_air(p, 0.01)
    p["bc"] = ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"]
    p["u_in"] = 0.0
    if outlet == "nscbc":
        p["outlet"] = "nscbc"
    x = np.arange(nx)
    Ph = 1e-3 * np.exp(-((x - nx // 2) / 10.0) ** 2)
    cs = 3.0 ** -0.5
    u = np.zeros((2, nx))
    u[0] = Ph / cs
    s = O.OracleState(p, np.zeros(nx), np.full(nx, 300.0), u=u, Ph=Ph)

    def energy():
        uu, rho, ph = s.moments()
        return float(np.sum(0.5 * ph ** 2 / (rho * cs * cs) + 0.5 * rho * uu[0] ** 2))

    E0 = energy()
    s.step(steps)
    return E0, energy()


def test_characteristic_outlet_absorbs_a_plane_pulse():
    """Sec. 4.1 uses the non-reflecting outlet of Poinsot and Lele because a
    fixed-pressure outlet reflects sound: a plane pulse leaving through a
    P_h = 0 outlet comes back with almost all its energy (amplitude
    reflection about 0.93 after viscous loss), through the characteristic
    outlet with less than 2 % of it (reflection below 0.15)."""
    E0, E1 = _pulse_channel("fixed")
    assert np.sqrt(E1 / E0) > 0.9
    E0, E1 = _pulse_channel("nscbc")
    assert np.sqrt(E1 / E0) < 0.15


def test_characteristic_outlet_keeps_the_steady_channel_flow():
    """In a steady channel flow the outlet condition must not change the flow:
    the velocity field with the characteristic outlet matches the one with
    P_h = 0 to 2e-3 of the peak speed (only the pressure level moves: the
    boundary pressure settles where the incoming wave balances the outgoing
    one), and it no longer changes."""
    res = {}
    for outlet in ("fixed", "nscbc"):
        p = I._base(2, 160, 24)
        I.lattice_air(p, 0.05)
        p["bc"] = ["inlet", "outlet", "wall", "wall", "periodic", "periodic"]
        p.update({"u_in": 0.04, "inlet_parabolic": 1})
        if outlet == "nscbc":
            p["outlet"] = "nscbc"
        s = O.OracleState(p, np.zeros(160 * 24), np.full(160 * 24, 300.0))
        s.step(8000)
        res[outlet] = (s.moments()[0][0], s)
    ref = res["fixed"][0]
    got, s = res["nscbc"]
    assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max()
    pb = s.outlet_pressure
    assert np.all(pb == pb[0]) and pb[0] > 0
    s.step(1000)
    assert np.abs(s.moments()[0][0] - got).max() <= 2e-4 * np.abs(ref).max()


def test_diffuse_channel_inlet_carries_the_sharp_channel_flux():
    """Inlet profile 2 (uniform speed times the fluid fraction) over the
    diffuse walls of eq. def-phi carries u_in times the channel width: the
    fluid fractions of a wall interface sum to the sharp wall position."""
    q = I.di_channel(L=50, eta=8, solid=8)
    phi = I.di_channel_fields(q)["phi"].reshape(q["ny"], q["nx"])[:, 0]
    assert abs(np.sum(1.0 - phi) - 50.0) <= 1e-12
    assert phi[0] == 1.0 and phi[q["ny"] // 2] == 0.0
