"""Brute-force transcription of one full step on tiny grids, checked against the
oracle on random states.

The transcription below is written from the scheme's definition (Sec. 3.3
plus the readings listed in the design notes) in a different shape from the
oracle: dictionaries of per-cell values, explicit neighbour lookups, the
lattice generated from its velocity set rather than tabulated.  It catches
index, ordering and boundary-rule mistakes in the oracle's C code.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_17214_gb300 import inputs as I

R = 8.314
CS2 = 1.0 / 3.0


def gen_lattice(dim):
    """D2Q9 / D3Q19 generated from the speed shells, ordered like the oracle
    (the test only relies on the set; order is taken from the oracle)."""
    c_or, w_or = O.lattice(dim)
    vel = [tuple(int(v) for v in ci[:dim]) for ci in c_or]
    w = {}
    for v in vel:
        n2 = sum(a * a for a in v)
        if dim == 2:
            w[v] = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[n2]
        else:
            w[v] = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[n2]
    # sanity: the set is the full shell structure
    expect = [v for v in itertools.product([-1, 0, 1], repeat=dim)
              if sum(a * a for a in v) <= 2]
    assert sorted(vel) == sorted(expect)
    return vel, w


def brute_step(p, phi, g, T, Y, Ts, P0, P0p, m0):
    dim, nx, ny = p["dim"], p["nx"], p["ny"]
    nz = p["nz"] if dim == 3 else 1
    K = p.get("K", 0)
    vel, W = gen_lattice(dim)
    Q = len(vel)
    shape = (nx, ny, nz)
    cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    idx = {c: i for i, c in enumerate(cells)}
    bc = p["bc"]
    dx, dt, rr = p["dx"], p["dt"], p["rho_ref"]

    def Mw_of(Yc):
        return p["M0"] if K == 0 else 1.0 / sum(Yc[k] / p["M"][k] for k in range(K))

    def cp_of(Yc):
        return p["cp0"] if K == 0 else sum(Yc[k] * p["cp"][k] for k in range(K))

    def rho_of(Tc, Yc):
        return P0 * Mw_of(Yc) / (R * Tc * rr)

    def mu_of(Tc):
        mu = p["mu_ref"]
        if p.get("sutherland"):
            Ts_, S = p["suth_T"], p["suth_S"]
            mu = p["mu_ref"] * (Tc / Ts_) ** 1.5 * (Ts_ + S) / (Tc + S)
        return mu * dt / (rr * dx * dx)

    def D_of(Tc):
        out = []
        for k in range(K):
            D = p["Dref"][k] * ((Tc / p["D_Tref"]) ** p["D_exp"] if p["D_exp"] else 1.0)
            out.append(D * dt / (dx * dx))
        return out

    def cellval(c):
        i = idx[c]
        return {"T": T[i], "Y": [Y[k][i] for k in range(K)], "phi": phi[i],
                "Ts": Ts[i] if Ts is not None else p["Ts_uniform"]}

    def nbval(c, a, s):
        q = list(c)
        q[a] += s
        face = 2 * a + (1 if s > 0 else 0)
        if 0 <= q[a] < shape[a]:
            return cellval(tuple(q))
        if bc[face] == "periodic":
            q[a] %= shape[a]
            return cellval(tuple(q))
        v = dict(cellval(c))
        if bc[face] == "inlet":
            v["T"] = p["T_in"]
            v["Y"] = list(p["Y_in"])
        elif bc[face] == "wall" and p["wall_T"][face] > 0:
            v["T"] = p["wall_T"][face]
        return v

    # ---- per-cell EOS and properties at step n
    rho = {c: rho_of(T[idx[c]], [Y[k][idx[c]] for k in range(K)]) for c in cells}
    mu = {c: mu_of(T[idx[c]]) for c in cells}
    Kd = {c: p["A_u"] * mu[c] * (1 - phi[idx[c]]) * phi[idx[c]] ** 2 / p["eta"] ** 2
          for c in cells}
    Yin = list(p["Y_in"])
    rho_in = P0 * Mw_of(Yin) / (R * p["T_in"] * rr)

    def inlet_u(c):
        u = p["u_in"]
        if p.get("inlet_parabolic"):
            for a in range(1, dim):
                if bc[2 * a] == "wall":
                    n, s = shape[a], c[a] + 0.5
                    u *= 4 * s * (n - s) / (n * n)
        return u

    # ---- streaming with boundary rules
    def pulled(c, uw):
        out = {}
        for v in vel:
            src = [c[a] - v[a] for a in range(dim)]
            kinds = []
            for a in range(dim):
                if src[a] < 0 or src[a] >= shape[a]:
                    face = 2 * a + (1 if src[a] >= shape[a] else 0)
                    if bc[face] == "periodic":
                        src[a] %= shape[a]
                    else:
                        kinds.append((bc[face], face))
            opp = tuple(-a for a in v)
            own_opp = g[vel.index(opp)][idx[c]]
            walls = [f for k_, f in kinds if k_ == "wall"]
            if walls:
                uwall = p["wall_u"][walls[0]]
                out[v] = own_opp + 2 * W[v] * rho[c] * sum(v[a] * uwall[a] for a in range(dim))
            elif any(k_ == "inlet" for k_, _ in kinds):
                out[v] = own_opp + 2 * W[v] * rho_in * v[0] * inlet_u(c)
            elif any(k_ == "outlet" for k_, _ in kinds):
                cu = sum(v[a] * uw[a] for a in range(dim))
                uu = sum(x * x for x in uw)
                out[v] = -own_opp + W[v] * rho[c] * (cu * cu / CS2 - uu)
            else:
                full = tuple(src) + (0,) * (3 - dim)
                out[v] = g[vel.index(v)][idx[full]]
        return out

    gin, u = {}, {}
    for c in cells:
        uw = [0.0] * dim
        npass = 2 if (bc[1] == "outlet" and c[0] == nx - 1) else 1
        for _ in range(npass):
            gi = pulled(c, uw)
            uc = []
            for a in range(dim):
                m = sum(v[a] * gi[v] for v in vel) / CS2
                uc.append((m + 0.5 * p["Fb"][a]) / (rho[c] + 0.5 * Kd[c]))
            uw = uc
        gin[c], u[c] = gi, uc

    # ---- FD transport
    Tn, Yn, Tsn = {}, {}, {}
    for c in cells:
        v0 = cellval(c)
        phif, phis = 1 - v0["phi"], v0["phi"]
        cp0 = cp_of(v0["Y"])
        lam0 = mu[c] * cp0 / p["Pr"]
        D0 = D_of(v0["T"])
        fluid = phif >= p["phi_min"]
        solid = (phis >= p["phi_min"]) if p.get("Ts_field") else True
        SI = (p["A_T"] * lam0 * phif * phis ** 2 / p["eta"] ** 2 * (v0["Ts"] - v0["T"])
              if fluid and solid else 0.0)
        om, omT = [0.0] * K, 0.0
        if p.get("chem") == "explicit" and K:
            rho_phys = rho[c] * rr
            Cc = [rho_phys * max(v0["Y"][k], 0.0) / p["M"][k] for k in range(K)]
            for rx in p["reactions"]:
                q = rx["A"] * math.exp(-rx["EaR"] / v0["T"]) * v0["T"] ** rx.get("b", 0.0)
                for k in range(K):
                    if rx["order"][k]:
                        q *= Cc[k] ** rx["order"][k]
                for k in range(K):
                    om[k] += p["M"][k] * rx["stoich"][k] * q
            om = [o * dt / rr for o in om]
            omT = -sum(p["hf"][k] * om[k] for k in range(K))
        nbs = [(nbval(c, a, -1), nbval(c, a, +1)) for a in range(dim)]
        Yn[c] = []
        for k in range(K):
            if not fluid:
                Yn[c].append(v0["Y"][k])
                continue
            kap0 = phif * rho[c] * D0[k]
            adv = dif = 0.0
            for a, (vm, vp) in enumerate(nbs):
                ua = u[c][a]
                adv += ua * (v0["Y"][k] - vm["Y"][k]) if ua > 0 else ua * (vp["Y"][k] - v0["Y"][k])
                km = 0.5 * (kap0 + (1 - vm["phi"]) * rho_of(vm["T"], vm["Y"]) * D_of(vm["T"])[k])
                kp = 0.5 * (kap0 + (1 - vp["phi"]) * rho_of(vp["T"], vp["Y"]) * D_of(vp["T"])[k])
                dif += kp * (vp["Y"][k] - v0["Y"][k]) - km * (v0["Y"][k] - vm["Y"][k])
            Yn[c].append(v0["Y"][k] + (-phif * rho[c] * adv + dif + phif * om[k]) / (phif * rho[c]))
        if fluid:
            adv = dif = cross = 0.0
            for a, (vm, vp) in enumerate(nbs):
                ua = u[c][a]
                adv += ua * (v0["T"] - vm["T"]) if ua > 0 else ua * (vp["T"] - v0["T"])
                lm = mu_of(vm["T"]) * cp_of(vm["Y"]) / p["Pr"]
                lp = mu_of(vp["T"]) * cp_of(vp["Y"]) / p["Pr"]
                km = 0.5 * (phif * lam0 + (1 - vm["phi"]) * lm)
                kp = 0.5 * (phif * lam0 + (1 - vp["phi"]) * lp)
                dif += kp * (vp["T"] - v0["T"]) - km * (v0["T"] - vm["T"])
                for k in range(K):
                    cross += (p["cp"][k] * D0[k] * 0.5 * (vp["Y"][k] - vm["Y"][k]) *
                              0.5 * (vp["T"] - vm["T"]))
            rhs = (-phif * rho[c] * cp0 * adv + dif +
                   phif * (rho[c] * cross + (P0 - P0p) / rr + omT + SI))
            Tn[c] = v0["T"] + rhs / (phif * rho[c] * cp0)
        else:
            Tn[c] = v0["Ts"]
        if p.get("Ts_field"):
            if phis >= p["phi_min"]:
                Ls = p["lambda_s"] * dt / (rr * dx * dx)
                dif = 0.0
                for vm, vp in nbs:
                    dif += (0.5 * (phis + vp["phi"]) * Ls * (vp["Ts"] - v0["Ts"]) -
                            0.5 * (phis + vm["phi"]) * Ls * (v0["Ts"] - vm["Ts"]))
                Tsn[c] = v0["Ts"] + (dif - phif * SI) / (phis * p["rhocp_s"] / rr)
            else:
                Tsn[c] = v0["Ts"]

    # ---- divergence, source, collision
    gnew = [np.zeros(len(cells)) for _ in range(Q)]
    for c in cells:
        v0 = cellval(c)
        Mw = Mw_of(v0["Y"])
        # material derivative over the step, DT/Dt = d_t T + u.grad T: the
        # Eulerian increment plus the convection with central differences
        # (none in frozen cells)
        fluid = (1 - v0["phi"]) >= p["phi_min"]
        nbs = [(nbval(c, a, -1), nbval(c, a, +1)) for a in range(dim)]
        cT = sum(u[c][a] * 0.5 * (vp["T"] - vm["T"]) for a, (vm, vp) in enumerate(nbs))
        cY = [sum(u[c][a] * 0.5 * (vp["Y"][k] - vm["Y"][k]) for a, (vm, vp) in enumerate(nbs))
              for k in range(K)]
        if not fluid:
            cT, cY = 0.0, [0.0] * K
        D = (Tn[c] - v0["T"] + cT) / v0["T"]
        D += Mw * sum((Yn[c][k] - v0["Y"][k] + cY[k]) / p["M"][k] for k in range(K))
        D -= (P0 - P0p) / P0
        r, uc = rho[c], u[c]
        G = []
        for a in range(dim):
            vm, vp = nbval(c, a, -1), nbval(c, a, +1)
            G.append(CS2 * 0.5 * (rho_of(vp["T"], vp["Y"]) - rho_of(vm["T"], vm["Y"])))
        F = [p["Fb"][a] - Kd[c] * uc[a] for a in range(dim)]
        tau = 0.5 + mu[c] / (r * CS2)
        uu = sum(x * x for x in uc)
        feqs, xis = {}, {}
        for v in vel:
            cu = sum(v[a] * uc[a] for a in range(dim))
            feqs[v] = r * W[v] * (1 + cu / CS2 + cu * cu / (2 * CS2 ** 2) - uu / (2 * CS2))
            xis[v] = sum((v[a] - uc[a]) * (G[a] * (feqs[v] / r - W[v]) + F[a] * feqs[v] / r)
                         for a in range(dim)) + r * CS2 * W[v] * D
        # P_h: the pulled zeroth moment plus half the source's zeroth moment
        Ph = sum(gin[c].values()) + 0.5 * sum(xis.values())
        for i, v in enumerate(vel):
            geq = CS2 * feqs[v] + W[v] * (Ph - r * CS2)
            gi = gin[c][v]
            gnew[i][idx[c]] = gi - (gi - geq) / tau + (1 - 1 / (2 * tau)) * xis[v]

    Tout = np.array([Tn[c] for c in cells])
    Yout = np.array([[Yn[c][k] for c in cells] for k in range(K)]) if K else None
    Tsout = np.array([Tsn[c] for c in cells]) if p.get("Ts_field") else None
    I_ = sum((1 - phi[idx[c]]) * Mw_of([Yout[k][idx[c]] for k in range(K)] if K else []) /
             Tout[idx[c]] for c in cells)
    P0n = P0 if p["p0_mode"] == "fixed" else m0 * R * rr / I_
    return np.concatenate(gnew), Tout, Yout, Tsout, P0n


CASES = {
    "2d_channel_reactive": dict(dim=2, nx=5, ny=4, bc=["inlet", "outlet", "wall", "wall",
                                                      "periodic", "periodic"], react=True),
    "2d_periodic_closed": dict(dim=2, nx=4, ny=4, bc=["periodic"] * 6, react=True,
                               p0="closed"),
    "2d_walls_dirichlet": dict(dim=2, nx=4, ny=3, bc=["wall", "wall", "wall", "periodic",
                                                     "periodic", "periodic"][:2] +
                               ["wall", "wall", "periodic", "periodic"], react=False),
    "3d_channel": dict(dim=3, nx=4, ny=3, nz=3, bc=["inlet", "outlet", "periodic", "periodic",
                                                   "wall", "wall"], react=True),
    "3d_periodic_closed": dict(dim=3, nx=3, ny=3, nz=3, bc=["periodic"] * 6, react=False,
                               p0="closed"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_bruteforce_one_step(name):
    cs = CASES[name]
    if cs["react"]:
        p = I.config2(nx=cs["nx"], ny=cs["ny"])
        p["dim"], p["nz"] = cs["dim"], cs.get("nz", 1)
        p["reactions"] = I.one_step_mechanism(3.3e8)
    else:
        p = I._base(cs["dim"], cs["nx"], cs["ny"], cs.get("nz", 1))
        I.lattice_air(p, 0.01)
        p["sutherland"] = 1
        p["A_u"], p["A_T"], p["Ts_uniform"] = 60.0, 50.0, 450.0
        p["Fb"] = [1e-5, -2e-5, 3e-6]
    p["bc"] = cs["bc"]
    p["p0_mode"] = cs.get("p0", "fixed")
    p["inlet_parabolic"] = 1
    p["u_in"] = 0.03
    p["eta"] = 2.5
    p["wall_u"] = [[0, 0, 0], [0, 0, 0], [0.01, 0, 0], [0, -0.005, 0.002], [0, 0, 0], [0, 0, 0]]
    p["wall_T"] = [350.0, 0.0, 0.0, 420.0, 0.0, 380.0]
    f = I.random_state(p, seed=11, T_range=(320.0, 900.0), u_amp=0.03)
    # cover pure-fluid cells and frozen-fluid cells (phi_f < phi_min)
    idx = np.arange(f["phi"].size)
    f["phi"] = np.where(idx % 5 == 0, 0.0, np.where(idx % 7 == 3, 1.0, f["phi"]))
    s = O.OracleState(p, f["phi"], f["T"], f["Y"], f["Ts"], u=f["u"], Ph=f["Ph"])
    # make the state less trivial: one oracle step, then perturb P0 history
    s.step(1)
    s.scal[1] = s.scal[0] * (1 - 3e-5) if p["p0_mode"] == "closed" else s.scal[0]
    K = p.get("K", 0)
    N = O.ncells(p)
    g0, T0 = s.g.copy(), s.T.copy()
    Y0 = s.Y.reshape(K, N).copy() if K else None
    Ts0 = s.Ts.copy() if s.Ts is not None else None
    P0, P0p, m0 = s.scal[0], s.scal[1], s.scal[2]
    Q = s.Q
    gb, Tb, Yb, Tsb, P0b = brute_step(p, f["phi"], [g0[i * N:(i + 1) * N] for i in range(Q)],
                                      T0, Y0, Ts0, P0, P0p, m0)
    s.step(1)
    assert np.max(np.abs(s.T - Tb)) < 1e-10
    assert np.max(np.abs(s.g - gb)) < 1e-14
    if K:
        assert np.max(np.abs(s.Y - Yb.reshape(-1))) < 1e-13
    if Tsb is not None:
        assert np.max(np.abs(s.Ts - Tsb)) < 1e-10
    assert abs(s.P0 / P0b - 1) < 1e-14
