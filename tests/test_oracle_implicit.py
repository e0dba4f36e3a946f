"""Pins of the oracle's backward-Euler Newton chemistry (two-step mechanism,
reversible CO/CO2 step) against closed forms and an independent ODE solve."""
import math

import numpy as np

from oracle import oracle as O
from paper_2310_17214_gb300 import inputs as I

ELEM = {"CH4": (1, 4, 0, 0), "O2": (0, 0, 2, 0), "CO": (1, 0, 1, 0), "CO2": (1, 0, 2, 0),
        "H2O": (0, 2, 1, 0), "N2": (0, 0, 0, 2)}


def reactor(chem="implicit"):
    p = I.config4(nx=1, ny=1, chem=chem)
    p["bc"] = ["periodic"] * 6
    p["p0_mode"] = "fixed"
    p["Ts_field"] = 0
    p["A_T"] = p["A_u"] = 0.0
    return p


def test_linear_decay_is_the_backward_euler_closed_form():
    """A -> B, first order, isothermal: Y^{n+1} = Y^n / (1 + k dt) exactly."""
    p = reactor()
    p["hf"] = [0.0] * 6
    p["reactions"] = [{"A": 4e6, "b": 0.0, "EaR": 0.0, "order": [1, 0, 0, 0, 0, 0],
                       "stoich": [-1, 0, 0, 0, 0, 0]}]
    p["M"] = list(p["M"])
    # make the decay mass-conserving by producing an equal-mass species
    p["reactions"][0]["stoich"] = [-1, 0, p["M"][0] / p["M"][2], 0, 0, 0]
    Y = np.array(I.lean_ch4_air(0.7, I.SPECIES6))
    rho = 1.0
    dY, dT, rc = O.chem_implicit(p, 1000.0, Y, rho)
    assert rc == 0
    k = 4e6  # first order in CH4: dY/dt = -k Y
    ref = Y[0] / (1 + k * p["dt"]) - Y[0]
    assert abs(dY[0] - ref) < 1e-15
    assert dT == 0.0


def test_reversible_step_reaches_its_equilibrium_constant():
    """CO + 1/2 O2 <-> CO2 alone at fixed T: many backward-Euler steps settle
    at [CO2]/([CO][O2]^(1/2)) = K_c(T) = exp(dS/R - dH/RT) (p0/RT)^(-1/2)."""
    p = reactor()
    p["hf"] = [0.0] * 6
    p["reactions"] = [I.two_step_mechanism()[1]]
    p["dt"] = 1e-4
    T = 2400.0
    M = np.array(p["M"])
    Y = np.array([0.0, 0.10, 0.05, 0.05, 0.10, 0.70])
    rho = 0.15
    for _ in range(400):
        dY, dT, rc = O.chem_implicit(p, T, Y, rho / p["rho_ref"])
        assert rc == 0
        Y = Y + dY
    C = rho * Y / M
    R = 8.314
    Kc = math.exp(-86.5 / R + 283.0e3 / (R * T)) * (101325.0 / (R * T)) ** (-0.5)
    assert abs(C[3] / (C[2] * math.sqrt(C[1])) / Kc - 1) < 1e-8


def test_two_step_reactor_conserves_elements_and_mass():
    p = reactor()
    p["p0_mode"] = "closed"
    Y0 = np.array(I.lean_ch4_air(0.7, I.SPECIES6))
    s = O.OracleState(p, np.zeros(1), np.array([1600.0]), Y0)
    M = np.asarray(p["M"])
    A = np.array([ELEM[sp] for sp in p["species"]], dtype=float)
    e0 = (Y0 / M) @ A
    for _ in range(30):
        s.step(20)
        assert abs(s.Y.sum() - 1) < 1e-13
        assert np.allclose((s.Y / M) @ A, e0, rtol=1e-12, atol=1e-15)
    assert s.T[0] > 1900.0  # it burnt


def test_implicit_reactor_matches_ode_integration():
    """Constant-volume reactor with the two-step mechanism: the oracle's
    backward Euler (implicit chemistry, lagged dP0/dt) against an adaptive
    stiff ODE solve of the same equations, within O(dt)."""
    from scipy.integrate import solve_ivp

    p = reactor()
    p["p0_mode"] = "closed"
    Y0 = np.array(I.lean_ch4_air(0.7, I.SPECIES6))
    T0 = 1500.0
    s = O.OracleState(p, np.zeros(1), np.array([T0]), Y0)
    n = 1500
    s.step(n)
    M = np.asarray(p["M"])
    cpk = np.asarray(p["cp"])
    hf = np.asarray(p["hf"])
    R = 8.314
    rho = p["P0"] / (R * T0) / np.sum(Y0 / M)

    def omega(T, Y):
        C = rho * np.maximum(Y, 0) / M
        w = np.zeros(6)
        for r in p["reactions"]:
            kf = r["A"] * math.exp(-r["EaR"] / T)
            q = kf * np.prod([C[k] ** o for k, o in enumerate(r["order"]) if o])
            if "reverse" in r:
                dn = sum(r["stoich"])
                Kc = math.exp(r["reverse"]["dS"] / R - r["reverse"]["dH"] / (R * T)) * \
                    (101325.0 / (R * T)) ** dn
                q -= kf / Kc * np.prod([C[k] ** o for k, o in enumerate(r["reverse"]["order"]) if o])
            w += M * np.asarray(r["stoich"], dtype=float) * q
        return w

    def rhs(t, z):
        T, Y = z[0], z[1:]
        w = omega(T, Y)
        dY = w / rho
        invMw = np.sum(Y / M)
        dinvMw = np.sum(dY / M)
        cp = np.sum(Y * cpk)
        dT = (R * rho * T * dinvMw - np.sum(hf * w)) / (rho * cp - R * rho * invMw)
        return np.concatenate([[dT], dY])

    sol = solve_ivp(rhs, [0, n * p["dt"]], np.concatenate([[T0], Y0]), method="LSODA",
                    rtol=1e-9, atol=1e-12)
    assert abs(s.T[0] - sol.y[0, -1]) < 3.0, (s.T[0], sol.y[0, -1])
    assert np.max(np.abs(s.Y - sol.y[1:, -1])) < 5e-4
    assert abs(sol.y[0, -1] - T0) > 300.0
