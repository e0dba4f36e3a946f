"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds none of the scheme's arithmetic.  It only states the
workloads (lattice shape, boundary kinds, physical constants in SI units) as
plain dictionaries and builds the static phase field phi_s and the initial
T, Y, Ts fields, byte-identical for every consumer.  Each solver converts the
physical constants to its own lattice units itself.

The paper's particle assemblies (packed beds of cylinders, grain-growth
particles; Sec. 4.4.3-4.4.4) are not public data: seeded random ellipses and
ellipsoids with a diffuse tanh profile stand in for them.

Constants that are not printed in the paper are chosen here and documented:
species molar masses and standard formation enthalpies are textbook values
(CH4 -74.87, CO2 -393.52, H2O(g) -241.83 kJ/mol); the constant species heat
capacities, reference diffusivities and the one-step pre-exponential factor
are project choices.  Sutherland constants (T* = 273 K, S = 110.5 K,
mu* = 1.68e-5 Pa s) follow Sec. 4, eq. muT.
"""
from __future__ import annotations

import math

import numpy as np

R_GAS = 8.314

# molar masses from standard atomic weights (kg/mol), so that every reaction
# conserves mass exactly: sum_k M_k s_kj = 0
_AW = {"C": 12.011e-3, "H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}
_COMP = {"CH4": {"C": 1, "H": 4}, "O2": {"O": 2}, "CO": {"C": 1, "O": 1},
         "CO2": {"C": 1, "O": 2}, "H2O": {"H": 2, "O": 1}, "N2": {"N": 2}}


def molar_mass(sp):
    return sum(n * _AW[e] for e, n in _COMP[sp].items())


def element_matrix(species, elements=("C", "H", "O", "N")):
    """Atoms of each element in each species ([E][K]) and element molar masses."""
    return ([[float(_COMP[sp].get(e, 0)) for sp in species] for e in elements],
            [_AW[e] for e in elements])


# Sutherland laws of the pure gases (mu_ref in Pa s at T_ref, T_ref, S in K):
# values of the standard viscosity tables, used by the mixture-averaged
# transport option; steam is referred to 350 K.
SUTHERLAND = {"N2": (1.663e-5, 273.0, 107.0), "O2": (1.919e-5, 273.0, 139.0),
              "CO2": (1.370e-5, 273.0, 222.0), "CO": (1.657e-5, 273.0, 136.0),
              "CH4": (1.030e-5, 273.0, 198.0), "H2O": (1.120e-5, 350.0, 1064.0)}


def mixture_transport(p):
    """Switch a reactive problem to mixture-averaged viscosity and
    conductivity (Sec. 4.4, eqs. muT_mix, phi_mix, conduct_mix) with the
    species' Sutherland laws; the single-gas mu_ref, Sutherland constants and
    Pr are then unused."""
    p["transport"] = "mixture"
    p["mu_k"] = [SUTHERLAND[s][0] for s in p["species"]]
    p["suth_Tk"] = [SUTHERLAND[s][1] for s in p["species"]]
    p["suth_Sk"] = [SUTHERLAND[s][2] for s in p["species"]]
    return p


# one-step CH4 mechanism species order
SPECIES5 = ["CH4", "O2", "CO2", "H2O", "N2"]
M5 = [molar_mass(s) for s in SPECIES5]
HF_MOL5 = [-74.87e3, 0.0, -393.52e3, -241.83e3, 0.0]
CP5 = [2700.0, 1100.0, 1200.0, 2300.0, 1200.0]
DREF5 = [2.2e-5, 2.1e-5, 1.6e-5, 2.5e-5, 2.0e-5]

# two-step mechanism species order
SPECIES6 = ["CH4", "O2", "CO", "CO2", "H2O", "N2"]
M6 = [molar_mass(s) for s in SPECIES6]
HF_MOL6 = [-74.87e3, 0.0, -110.53e3, -393.52e3, -241.83e3, 0.0]
CP6 = [2700.0, 1100.0, 1200.0, 1200.0, 2300.0, 1200.0]
DREF6 = [2.2e-5, 2.1e-5, 2.0e-5, 1.6e-5, 2.5e-5, 2.0e-5]

# one-step pre-exponential factor (m^3/(mol s)); Ea/R = 15000 K, first order
# in CH4 and O2 (project-chosen, see the design notes for its calibration).
A_ONE_STEP = 3.68e8


def lean_ch4_air(phi_eq: float, species):
    """Mass fractions of a CH4/air mixture at equivalence ratio phi_eq."""
    n_o2 = 2.0 / phi_eq
    moles = {"CH4": 1.0, "O2": n_o2, "N2": 3.76 * n_o2}
    mm = dict(zip(SPECIES6, M6))
    mass = {s: moles.get(s, 0.0) * mm[s] for s in species}
    tot = sum(mass.values())
    return [mass[s] / tot for s in species]


def _mixture_M(Y, M):
    return 1.0 / sum(y / m for y, m in zip(Y, M))


# ----------------------------------------------------------------- phase field
def tanh_profile(dist, eta):
    """phi_s = 0.5 (1 - tanh(2 d / eta)) for signed distance d (d < 0 inside)."""
    return 0.5 * (1.0 - np.tanh(2.0 * dist / eta))


def disc_phi(nx, ny, cx, cy, radius, eta):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return tanh_profile(r - radius, eta)


def _ellipse_dist(X, Y, cx, cy, a, b, th):
    """Signed-distance surrogate of an ellipse, (sqrt(F) - 1) min(a, b).

    It is 1-Lipschitz like the exact distance (sqrt(F) is a norm with
    Lipschitz constant 1/min(a, b)), so the tanh profile changes phi_f by at
    most a factor exp(4/eta) between neighbouring cells.  The first-order
    form (F - 1)/|grad F| is not, and inside elongated particles it produces
    neighbour ratios that make the phi_f-weighted explicit diffusion blow up."""
    ct, st = math.cos(th), math.sin(th)
    xr = (X - cx) * ct + (Y - cy) * st
    yr = -(X - cx) * st + (Y - cy) * ct
    F = (xr / a) ** 2 + (yr / b) ** 2
    return (np.sqrt(F) - 1.0) * min(a, b)


def _rot3(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipse_assembly(nx, ny, count, amin, amax, porosity, eta, seed, x0, periodic_y=True,
                     gap=None, max_attempts=200000, per_particle=None):
    """Seeded non-overlapping ellipses in a bed region starting at x0.

    The bed's length is chosen so that the solid area of the drawn particles
    gives the target porosity inside it; particles keep a gap of at least eta
    (checked on the grid).  With `per_particle`, a particle that finds no
    place in that many draws makes the bed 10 % longer (dense targets jam
    random sequential addition).  Returns (phi_s [ny, nx], info)."""
    rng = np.random.default_rng(seed)
    gap = eta if gap is None else gap
    axes = rng.uniform(amin, amax, size=(count, 2))
    axes.sort(axis=1)
    axes = axes[:, ::-1]
    angles = rng.uniform(0, math.pi, size=count)
    area = float(np.sum(math.pi * axes[:, 0] * axes[:, 1]))
    length = min(nx - x0 - 8, int(math.ceil(area / (1.0 - porosity) / ny)))
    occ = np.zeros((ny, nx), dtype=bool)
    phi = np.zeros((ny, nx))
    placed = []
    order = np.argsort(-axes[:, 0] * axes[:, 1])
    attempts = 0
    for idx in order:
        a, b = axes[idx]
        th = angles[idx]
        ok = False
        tries = 0
        while attempts < max_attempts and not ok:
            attempts += 1
            tries += 1
            if per_particle and tries > per_particle:
                grown = min(nx - x0 - 8, int(length * 1.1) + 1)
                if grown == length:
                    break
                length, tries = grown, 0
            cx = rng.uniform(x0 + a, x0 + length - a)
            cy = rng.uniform(0, ny) if periodic_y else rng.uniform(b, ny - b)
            r = int(math.ceil(a + gap + eta)) + 1
            xs = np.arange(int(cx) - r, int(cx) + r + 1)
            ys = np.arange(int(cy) - r, int(cy) + r + 1)
            if xs[0] < 0 or xs[-1] >= nx:
                continue
            ysw = ys % ny if periodic_y else ys
            if not periodic_y and (ys[0] < 0 or ys[-1] >= ny):
                continue
            X, Y = np.meshgrid(xs.astype(float), ys.astype(float))
            d = _ellipse_dist(X, Y, cx, cy, a, b, th)
            grow = d <= gap
            if np.any(occ[np.ix_(ysw, xs)] & grow):
                continue
            ok = True
            inside = d <= 0.0
            sub = occ[np.ix_(ysw, xs)]
            occ[np.ix_(ysw, xs)] = sub | inside
            prof = tanh_profile(d, eta)
            cur = phi[np.ix_(ysw, xs)]
            phi[np.ix_(ysw, xs)] = np.maximum(cur, prof)
            placed.append((cx, cy, a, b, th))
        if not ok:
            break
    bed = phi[:, x0:x0 + length]
    info = {"placed": len(placed), "requested": count, "bed_x0": x0, "bed_len": length,
            "porosity_bed": float(1.0 - bed.mean()), "attempts": attempts}
    return phi, info


def _ellipsoid_surface(c, axes, Rm, n, inflate):
    """n quasi-uniform points on an ellipsoid surface pushed out by `inflate`."""
    i = np.arange(n) + 0.5
    th = np.arccos(1 - 2 * i / n)
    ph = np.pi * (1 + 5 ** 0.5) * i
    unit = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], axis=1)
    pts = unit * (np.asarray(axes) + inflate)
    return c + pts @ Rm.T


def _inside_ellipsoid(pts, c, axes, Rm, period):
    d = pts - c
    for a in (1, 2):
        d[:, a] -= period[a] * np.round(d[:, a] / period[a])
    q = d @ Rm
    return np.any((q[:, 0] / axes[0]) ** 2 + (q[:, 1] / axes[1]) ** 2 + (q[:, 2] / axes[2]) ** 2
                  <= 1.0)


def ellipsoid_assembly(nx, ny, nz, count, amin, amax, porosity, eta, seed, x0, gap=None,
                       per_particle=150, n_surface=300):
    """Seeded non-overlapping ellipsoids (periodic in y and z) in a bed region.

    Random sequential addition with a bounding-sphere pre-check and a
    surface-sample overlap test (surfaces inflated by the gap).  A particle
    that cannot be placed is retried after the bed grows by 10 %; the bed
    length starts from the target porosity.  Returns (phi_s, info)."""
    rng = np.random.default_rng(seed)
    gap = eta if gap is None else gap
    axes = np.sort(rng.uniform(amin, amax, size=(count, 3)), axis=1)[:, ::-1]
    rots = [_rot3(rng) for _ in range(count)]
    vol = float(np.sum(4.0 / 3.0 * math.pi * np.prod(axes, axis=1)))
    length = int(math.ceil(vol / (1.0 - porosity) / (ny * nz)))
    period = np.array([0.0, ny, nz], dtype=float)
    placed = []  # (center, idx)
    centers = np.zeros((count, 3))
    radii = np.zeros(count)
    surf = {}
    pending = list(np.argsort(-np.prod(axes, axis=1)))
    attempts = 0
    for _round in range(20):
        lim = min(nx - x0 - 8, length)
        left = []
        for idx in pending:
            a = axes[idx]
            if lim < 2 * a[0] + 1:
                left.append(idx)
                continue
            ok = False
            for _ in range(per_particle):
                attempts += 1
                c = np.array([rng.uniform(x0 + a[0], x0 + lim - a[0]), rng.uniform(0, ny),
                              rng.uniform(0, nz)])
                n = len(placed)
                if n:
                    d = c[None, :] - centers[:n]
                    d[:, 1:] -= period[1:] * np.round(d[:, 1:] / period[1:])
                    near = np.nonzero(np.sqrt((d * d).sum(1)) < a[0] + radii[:n] + gap)[0]
                else:
                    near = []
                if len(near):
                    pts = _ellipsoid_surface(c, a, rots[idx], n_surface, gap)
                    bad = False
                    for m in near:
                        cj, j = placed[m]
                        if _inside_ellipsoid(pts, cj, axes[j], rots[j], period) or \
                                _inside_ellipsoid(surf[j], c, a, rots[idx], period):
                            bad = True
                            break
                    if bad:
                        continue
                ok = True
                centers[len(placed)] = c
                radii[len(placed)] = a[0]
                surf[idx] = _ellipsoid_surface(c, a, rots[idx], n_surface, gap)
                placed.append((c, idx))
                break
            if not ok:
                left.append(idx)
        if not left:
            break
        pending = left
        length = int(length * 1.15) + 2
    # rasterise
    phi = np.zeros((nz, ny, nx), dtype=np.float64)
    for (c, idx) in placed:
        a, Rm = axes[idx], rots[idx]
        r = int(math.ceil(a[0] + 2 * eta)) + 1
        xs = np.arange(max(0, int(c[0]) - r), min(nx, int(c[0]) + r + 1))
        ys = np.arange(int(c[1]) - r, int(c[1]) + r + 1)
        zs = np.arange(int(c[2]) - r, int(c[2]) + r + 1)
        Z, Y, X = np.meshgrid(zs.astype(float), ys.astype(float), xs.astype(float), indexing="ij")
        P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ Rm
        F = (P[..., 0] / a[0]) ** 2 + (P[..., 1] / a[1]) ** 2 + (P[..., 2] / a[2]) ** 2
        sel = np.ix_(zs % nz, ys % ny, xs)
        # 1-Lipschitz signed-distance surrogate (see _ellipse_dist)
        phi[sel] = np.maximum(phi[sel], tanh_profile((np.sqrt(F) - 1.0) * a.min(), eta))
    bed_len = min(nx - x0 - 8, length)
    bed = phi[:, :, x0:x0 + bed_len]
    info = {"placed": len(placed), "requested": count, "bed_x0": x0, "bed_len": bed_len,
            "porosity_bed": float(1.0 - bed.mean()), "attempts": attempts}
    return phi, info


# ------------------------------------------------------------------ problems
def _base(dim, nx, ny, nz=1):
    return {"dim": dim, "nx": nx, "ny": ny, "nz": nz,
            "bc": ["inlet", "outlet", "wall", "wall", "periodic", "periodic"],
            "wall_u": [[0.0, 0.0, 0.0]] * 6, "wall_T": [0.0] * 6,
            "dx": 1.0, "dt": 1.0, "rho_ref": 1.0, "K": 0, "M0": 0.02897, "cp0": 1006.0,
            "mu_ref": 0.0, "sutherland": 0, "suth_T": 273.0, "suth_S": 110.5, "Pr": 0.71,
            "A_u": 0.0, "A_T": 0.0, "eta": 4.0, "Fb": [0.0, 0.0, 0.0],
            "inlet_parabolic": 0, "u_in": 0.0, "T_in": 300.0, "Y_in": [],
            "p0_mode": "fixed", "P0": 101325.0, "Ts_field": 0, "Ts_uniform": 300.0,
            "rhocp_s": 1.0, "lambda_s": 0.0, "phi_min": 1e-6, "chem": "none",
            "reactions": [], "D_Tref": 300.0, "D_exp": 0.0}


def lattice_air(prob, nu_lattice, T_ref=300.0):
    """Lattice-unit air (dx = dt = 1): rho_ref = inlet density so rho* = 1."""
    rho = prob["P0"] * prob["M0"] / (R_GAS * T_ref)
    prob["rho_ref"] = rho
    prob["mu_ref"] = nu_lattice * rho  # mu* = mu dt / (rho_ref dx^2) = nu
    return prob


def config1(nx=128, ny=64, steps=5000):
    """128x64 D2Q9 FP64 channel, parabolic inlet u_max = 0.05, disc D = 16 at
    (32, 32) with tanh width 4, A_u = 1, particle held at 2 T_in via A_T,
    Re = 20 on u_mean = 2/3 u_max."""
    p = _base(2, nx, ny)
    p["bc"] = ["inlet", "outlet", "wall", "wall", "periodic", "periodic"]
    nu = (2.0 / 3.0) * 0.05 * 16.0 / 20.0
    lattice_air(p, nu)
    p.update({"A_u": 1.0, "A_T": 24.24 + 33.81 * 2.0, "eta": 4.0, "inlet_parabolic": 1,
              "u_in": 0.05, "T_in": 300.0, "Ts_uniform": 600.0, "p0_mode": "fixed",
              "steps": steps, "name": "cfg1_channel_disc_128x64_d2q9"})
    return p


def config1_fields(p):
    phi = disc_phi(p["nx"], p["ny"], 32.0, 32.0, 8.0, p["eta"]).reshape(-1)
    T = (1.0 - phi) * p["T_in"] + phi * p["Ts_uniform"]
    return {"phi": phi, "T": T, "Y": None, "Ts": None, "u": None}


def config5(n=48, seed=5, precision="fp32", steps=2000, base=(256, 128)):
    """n independent 2-D channel beds without species, advanced as a batch:
    sizes log-uniform from 256x128 to 1024x512 (aspect 2:1, ragged), bed
    porosity uniform in 0.4-0.8, parabolic inlet u_max uniform in 0.02-0.08,
    lattice air (nu = 0.05) at 300 K over particles held at 600 K, ellipse
    semi-axes growing with the domain, bed from x = nx/8 over about half
    the channel.  Sizes, porosities and speeds come from one seeded PCG64;
    `base` is the smallest size (tests use smaller beds)."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        s = 2.0 ** rng.uniform(0.0, 2.0)
        por = float(rng.uniform(0.4, 0.8))
        umax = float(rng.uniform(0.02, 0.08))
        nx, ny = int(round(base[0] * s)), int(round(base[1] * s))
        g = s * base[0] / 256.0  # particle size scale
        p = _base(2, nx, ny)
        p["bc"] = ["inlet", "outlet", "wall", "wall", "periodic", "periodic"]
        lattice_air(p, 0.05)
        p.update({"A_u": 145.0, "A_T": 70.0, "eta": 4.0, "inlet_parabolic": 1, "u_in": umax,
                  "T_in": 300.0, "Ts_uniform": 600.0, "p0_mode": "fixed",
                  "precision": precision, "steps": steps, "seed": seed * 1000 + i,
                  "bed": {"count": max(4, int(round(65.5 * (1.0 - por)))), "amin": 6.0 * g,
                          "amax": 14.0 * g, "porosity": por, "x0": nx // 8},
                  "name": f"cfg5_bed_{i}_{nx}x{ny}_d2q9_{precision}"})
        probs.append(p)
    return probs


def config5_fields(p):
    b = p["bed"]
    phi, info = ellipse_assembly(p["nx"], p["ny"], b["count"], b["amin"], b["amax"],
                                 b["porosity"], p["eta"], p["seed"], b["x0"], periodic_y=False,
                                 per_particle=200)
    phi = phi.reshape(-1)
    T = (1.0 - phi) * p["T_in"] + phi * p["Ts_uniform"]
    return {"phi": phi, "T": T, "Y": None, "Ts": None, "u": None, "info": info}


def _reactive_gas(p, species, M, cp, hf_mol, dref):
    p["K"] = len(species)
    p["species"] = list(species)
    p["M"] = list(M)
    p["cp"] = list(cp)
    p["hf"] = [h / m for h, m in zip(hf_mol, M)]
    p["Dref"] = list(dref)
    p["D_Tref"], p["D_exp"] = 300.0, 1.7
    p["sutherland"] = 1
    p["mu_ref"] = 1.68e-5
    p["suth_T"], p["suth_S"] = 273.0, 110.5
    return p


def one_step_mechanism(A=A_ONE_STEP):
    # CH4 + 2 O2 -> CO2 + 2 H2O ; Q = A exp(-15000/T) [CH4][O2]
    return [{"A": A, "b": 0.0, "EaR": 15000.0, "order": [1, 1, 0, 0, 0],
             "stoich": [-1, -2, 1, 2, 0]}]


def config2(nx=1024, ny=256, precision="fp64", steps=20000, seed=2):
    """2-D reactive bed: lean (phi = 0.7) CH4/O2/N2 at 300 K, 5 species with
    constant cp_k and D_k = D_ref (T/300)^1.7, one-step Arrhenius chemistry,
    40 seeded ellipses (semi-axes 8-20, porosity ~0.6 in the bed), solid
    rho cp 1000x and conductivity 10x the inlet gas, ignition by a 1500 K
    slab of burnt gas near the inlet (48 cells = 1.2 mm: a 16-cell slab
    quenches with the calibrated rate)."""
    p = _base(2, nx, ny)
    p["bc"] = ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"]
    _reactive_gas(p, SPECIES5, M5, CP5, HF_MOL5, DREF5)
    p["dx"], p["dt"] = 2.5e-5, 2.5e-7
    Y_in = lean_ch4_air(0.7, SPECIES5)
    Mw = _mixture_M(Y_in, M5)
    p["rho_ref"] = p["P0"] * Mw / (R_GAS * 300.0)
    cp_in = sum(y * c for y, c in zip(Y_in, CP5))
    lam_in = 1.68e-5 * (300.0 / 273.0) ** 1.5 * (273.0 + 110.5) / (300.0 + 110.5) * cp_in / 0.71
    p.update({"A_u": 145.0, "A_T": 70.0, "eta": 4.0, "u_in": 0.1 * p["dt"] / p["dx"],
              "T_in": 300.0, "Y_in": Y_in, "p0_mode": "fixed", "chem": "explicit",
              "reactions": one_step_mechanism(), "Ts_field": 1, "Ts_uniform": 300.0,
              "rhocp_s": 1000.0 * p["rho_ref"] * cp_in, "lambda_s": 10.0 * lam_in,
              "precision": precision, "steps": steps, "seed": seed,
              "ignite": [16, 64, 1500.0], "bed": {"count": 40, "amin": 8, "amax": 20,
                                                 "porosity": 0.6, "x0": 96},
              # hottest temperature for the create-time stability check: above
              # the adiabatic flame temperature of the inlet mixture (1822 K)
              "T_max": 1900.0,
              "name": f"cfg2_reactive_bed_{nx}x{ny}_d2q9_{precision}"})
    return p


def burnt_composition(Y_in, species, M):
    """Complete combustion of the CH4 in Y_in to CO2 and H2O (lean mixture)."""
    Y = dict(zip(species, Y_in))
    mm = dict(zip(species, M))
    if "CO" in Y:
        Y["CO"] = Y.get("CO", 0.0)
    n = Y["CH4"] / mm["CH4"]
    Y["O2"] -= 2.0 * n * mm["O2"]
    Y["CO2"] += n * mm["CO2"]
    Y["H2O"] += 2.0 * n * mm["H2O"]
    Y["CH4"] = 0.0
    return [Y[s] for s in species]


def reactive_fields(p, phi):
    """Fresh inlet mixture everywhere except an ignition slab of hot burnt
    products (complete combustion) at the given temperature; the temperature
    blends to the solid temperature inside the particles."""
    N = phi.size
    K = p["K"]
    T = np.full(N, p["T_in"])
    shape = (p["ny"], p["nx"]) if p["dim"] == 2 else (p["nz"], p["ny"], p["nx"])
    xs = np.broadcast_to(np.arange(p["nx"]), shape).reshape(-1)
    lo, hi, Tig = p.get("ignite", [0, 0, p["T_in"]])
    slab = (xs >= lo) & (xs < hi)
    T[slab] = Tig
    Y = np.repeat(np.asarray(p["Y_in"], dtype=np.float64)[:, None], N, axis=1)
    if slab.any():
        Yb = np.asarray(burnt_composition(p["Y_in"], p["species"], p["M"]))
        Y[:, slab] = Yb[:, None]
    Y = Y.reshape(-1)
    Ts = np.full(N, p["Ts_uniform"]) if p.get("Ts_field") else None
    # inside the particles the temperature starts at the solid temperature
    phi = phi.reshape(-1)
    T = (1.0 - phi) * T + phi * p["Ts_uniform"]
    return {"phi": phi, "T": T, "Y": Y, "Ts": Ts, "u": None}


def config2_fields(p):
    b = p["bed"]
    phi, info = ellipse_assembly(p["nx"], p["ny"], b["count"], b["amin"], b["amax"],
                                 b["porosity"], p["eta"], p["seed"], b["x0"],
                                 periodic_y=p["bc"][2] == "periodic")
    f = reactive_fields(p, phi)
    f["info"] = info
    return f


def two_step_mechanism(A1=3.31e8, A2=1.0e8):
    """Project-chosen two-step CH4 mechanism on (CH4, O2, CO, CO2, H2O, N2):
    R1  CH4 + 1.5 O2 -> CO + 2 H2O,  Q1 = A1 exp(-15000/T) [CH4][O2];
    R2  CO + 0.5 O2 <-> CO2,         Q2 = A2 exp(-12000/T) ([CO][O2]^0.5 - [CO2]/K_c),
    K_c from the standard reaction enthalpy and entropy of CO + 1/2 O2 -> CO2
    (-283.0 kJ/mol, -86.5 J/(mol K)).  The rate constants of the paper's
    mechanism are not printed in the paper and are not used here."""
    return [{"A": A1, "b": 0.0, "EaR": 15000.0, "order": [1, 1, 0, 0, 0, 0],
             "stoich": [-1, -1.5, 1, 0, 2, 0]},
            {"A": A2, "b": 0.0, "EaR": 12000.0, "order": [0, 0.5, 1, 0, 0, 0],
             "stoich": [0, -0.5, -1, 1, 0, 0],
             "reverse": {"dH": -283.0e3, "dS": -86.5, "order": [0, 0, 0, 1, 0, 0]}}]


def config4(nx=2048, ny=512, precision="fp64", steps=2000, seed=4, chem="implicit"):
    """2-D bed with the two-step six-species mechanism integrated per cell by
    backward Euler with Newton iterations (FP64), 60 seeded ellipses."""
    p = config2(nx, ny, precision=precision, steps=steps, seed=seed)
    p["K"] = 6
    p["species"], p["M"] = list(SPECIES6), list(M6)
    p["cp"], p["Dref"] = list(CP6), list(DREF6)
    p["hf"] = [h / m for h, m in zip(HF_MOL6, M6)]
    p["Y_in"] = lean_ch4_air(0.7, SPECIES6)
    p["chem"] = chem
    p["reactions"] = two_step_mechanism()
    p["bed"] = {"count": 60, "amin": 8, "amax": 20, "porosity": 0.6, "x0": 160}
    # the two-step mechanism releases part of its heat later, through CO: a
    # 1500 K slab quenches within 2000 steps, one near T_ad (1822 K) lights
    p["ignite"] = [16, 64, 1800.0]
    p["name"] = f"cfg4_two_step_bed_{nx}x{ny}_d2q9_{precision}"
    return p


def config4_fields(p):
    return config2_fields(p)


def config3(nx=256, ny=128, nz=128, precision="fp32_fp16", steps=2000, seed=3):
    """3-D D3Q19 reactive bed: 150 seeded ellipsoids (semi-axes 6-16, porosity
    ~0.5), the one-step mechanism and transport of the 2-D reactive bed,
    periodic in y and z."""
    p = config2(nx, ny, precision=precision, steps=steps, seed=seed)
    p["dim"], p["nz"] = 3, nz
    p["bc"] = ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"]
    # 3-D explicit diffusion needs a smaller step than 2-D at the same grid
    p["dt"] = 1.5e-7
    p["u_in"] = 0.1 * p["dt"] / p["dx"]
    p["bed"] = {"count": 150, "amin": 6, "amax": 16, "porosity": 0.5, "x0": 52}
    p["ignite"] = [8, 44, 1500.0]
    p["name"] = f"cfg3_reactive_bed_{nx}x{ny}x{nz}_d3q19_{precision}"
    return p


def config3_crop(n=64, precision="fp32_fp16", seed=3):
    """The 3-D bed recipe on an n^3 lattice, for comparisons with the oracle:
    same physics, mechanism, time step and inlet, the particle count scaled
    with the volume (150 ellipsoids in 256 x 128 x 128 -> about 10 in 64^3),
    semi-axes 6-16 cells, the bed from x = 3n/8 and an ignition slab over
    [n/8, 5n/8) at 1500 K."""
    p = config3(nx=n, ny=n, nz=n, precision=precision, seed=seed)
    vol = n ** 3 / (256 * 128 * 128)
    p["bed"] = {"count": max(1, int(round(150 * vol))), "amin": 6, "amax": 16,
                "porosity": 0.5, "x0": 3 * n // 8}
    p["ignite"] = [n // 8, 5 * n // 8, 1500.0]
    p["name"] = f"cfg3_crop_reactive_bed_{n}^3_d3q19_{precision}"
    return p


def config3_fields(p):
    b = p["bed"]
    phi, info = ellipsoid_assembly(p["nx"], p["ny"], p["nz"], b["count"], b["amin"], b["amax"],
                                   b["porosity"], p["eta"], p["seed"], b["x0"])
    f = reactive_fields(p, phi)
    f["info"] = info
    return f


def adiabatic_temperature(p):
    """Adiabatic flame temperature of the inlet mixture (complete combustion,
    constant cp_k): T_in + q / cp_burnt."""
    Yin = np.asarray(p["Y_in"])
    Yb = np.asarray(burnt_composition(p["Y_in"], p["species"], p["M"]))
    q = -float(np.dot(np.asarray(p["hf"]), Yb - Yin))
    return p["T_in"] + q / float(np.dot(Yb, p["cp"]))


def config6(nx=480, ny=120, precision="fp64", steps=20000, width=None):
    """2-D wall-bounded flame (the straight-channel flame of Sec. 4.4.2): the
    lean one-step CH4 mixture of the reactive bed, a channel ny cells wide
    (120 cells = 3 mm at dx = 25 um) between isothermal walls at 300 K
    (half-way bounce-back with the wall temperature, the sharp-interface
    form), parabolic inlet profile, no solid.  The first quarter of the channel
    holds the fresh mixture at 300 K, the rest the burnt products at the
    adiabatic flame temperature; the inlet feedback on CH4 (Sec. 4.4.1) keeps
    the flame near x = nx/4.  The first inlet speed is the calibrated burning
    velocity as a mean (peak 1.5 S_F)."""
    p = config2(nx=nx, ny=ny, precision=precision, steps=steps)
    p.pop("bed", None)
    p.pop("ignite", None)
    p["bc"] = ["inlet", "outlet", "wall", "wall", "periodic", "periodic"]
    p["wall_T"] = [0.0, 0.0, 300.0, 300.0, 0.0, 0.0]
    p.update({"A_u": 0.0, "A_T": 0.0, "Ts_field": 0, "inlet_parabolic": 1,
              "u_in": 1.5 * 0.2 * p["dt"] / p["dx"], "inlet_feedback": 0,
              "name": f"cfg6_wall_bounded_flame_{nx}x{ny}_d2q9_{precision}"})
    return p


def config6_fields(p, blend=4.0):
    """Fresh mixture up to x = nx/4, burnt products at T_ad beyond (tanh blend
    of `blend` cells)."""
    nx, ny = p["nx"], p["ny"]
    x = np.broadcast_to(np.arange(nx, dtype=np.float64), (ny, nx)).reshape(-1)
    w = 0.5 * (1.0 + np.tanh((x - nx / 4.0) / blend))
    Tad = adiabatic_temperature(p)
    T = p["T_in"] + (Tad - p["T_in"]) * w
    Yin = np.asarray(p["Y_in"])
    Yb = np.asarray(burnt_composition(p["Y_in"], p["species"], p["M"]))
    Y = (Yin[:, None] * (1.0 - w) + Yb[:, None] * w).reshape(-1)
    return {"phi": np.zeros(nx * ny), "T": T, "Y": Y, "Ts": None, "u": None}


def wall_phi(d, eta):
    """Solid fraction at signed distance d from a wall (d > 0 in the fluid),
    Sec. 4, eq. def-phi: 1/2 [1 - sin(pi d / eta)] across |d| < eta/2."""
    d = np.asarray(d, dtype=np.float64)
    return np.where(d <= -eta / 2, 1.0,
                    np.where(d >= eta / 2, 0.0, 0.5 * (1.0 - np.sin(np.pi * d / eta))))


def di_channel(L=50, eta=8, solid=8, Re=100.0, u_in=0.05, H=None, A_u=145.0, sharp=False,
               T_w=None, A_T=0.0):
    """Isothermal channel of Sec. 4.1 (Fig. A_u-vs-MSE): width L cells between
    two planar walls, inlet-outlet distance H = 5 L, uniform inlet speed,
    characteristic (non-reflecting) outlet, Re = u_in L / nu = 100, air at
    300 K everywhere.  Diffuse form: solid layers `solid` cells thick on both
    sides with eq. def-phi interfaces of width eta centred on the walls, the
    inlet speed weighted by the fluid fraction, drag A_u.  Sharp form
    (sharp=True): the same channel with the walls as half-way bounce-back
    lattice walls and no phase field (the coupling of Sec. 4 switched off).
    With T_w (Sec. 4.2, Fig. A_T-vs-MSE) the walls are hot: the gas enters at
    300 K, the sharp walls hold T_w, the diffuse walls are solid layers at
    T_w (uniform solid temperature) that exchange heat with the gas through
    the interface coupling A_T."""
    H = 5 * L if H is None else H
    ny = L if sharp else L + 2 * solid
    p = _base(2, H, ny)
    lattice_air(p, u_in * L / Re)
    p["bc"] = ["inlet", "outlet", "wall", "wall", "periodic", "periodic"]
    p.update({"u_in": u_in, "inlet_parabolic": 0 if sharp else 2, "outlet": "nscbc",
              "A_u": 0.0 if sharp else A_u, "A_T": 0.0, "eta": float(eta), "T_in": 300.0,
              "Ts_uniform": 300.0, "p0_mode": "fixed", "L": L, "solid": 0 if sharp else solid,
              "name": f"channel_{'si' if sharp else 'di'}_L{L}_eta{eta}_Re{Re:g}"})
    if T_w is not None:
        p["wall_T"] = [0.0, 0.0, float(T_w), float(T_w), 0.0, 0.0]
        p["Ts_uniform"] = float(T_w)
        p["A_T"] = 0.0 if sharp else float(A_T)
        p["name"] += f"_Tw{T_w:g}"
    return p


def di_channel_fields(p):
    """Phase field of the channel walls (zero in the sharp form); gas at
    T_in, and the solid layers (phi_f below phi_min) at the solid
    temperature, which they take from the first step on anyway."""
    nx, ny, s, L = p["nx"], p["ny"], p["solid"], p["L"]
    yc = np.arange(ny) + 0.5
    d = np.minimum(yc - s, (s + L) - yc)
    col = wall_phi(d, p["eta"]) if s > 0 else np.zeros(ny)
    phi = np.repeat(col[:, None], nx, axis=1).reshape(-1)
    T = np.full(nx * ny, float(p["T_in"]))
    T[1.0 - phi < p.get("phi_min", 1e-6)] = p["Ts_uniform"]
    return {"phi": phi, "T": T, "Y": None, "Ts": None, "u": None}


def channel_mse(u_si, u_di, p_si, p_di, at=0.9):
    """Mean standard error of Sec. 4.1, eq. mean-standard-error-f: the
    streamwise velocity across the cross-section at x = at H of the diffuse
    run against the sharp run, over the bulk fluid eta/2 <= y <= L - eta/2
    (y from the wall), normalised by the sharp profile's maximum."""
    L, eta, s = p_si["L"], p_di["eta"], p_di["solid"]
    xs = int(round(at * p_si["nx"])) - 1
    f_si = np.asarray(u_si).reshape(p_si["ny"], p_si["nx"])[:, xs]
    f_di = np.asarray(u_di).reshape(p_di["ny"], p_di["nx"])[s:s + L, xs]
    y = np.arange(L) + 0.5
    m = (y >= eta / 2) & (y <= L - eta / 2)
    return float(np.mean(((f_si[m] - f_di[m]) / np.max(f_si)) ** 2))


def with_initial_u(p, fields):
    """Initial velocity: the inlet profile times the fluid fraction."""
    N = fields["phi"].size
    u = np.zeros((p["dim"], N))
    u[0] = p["u_in"] * (1.0 - fields["phi"])
    if p.get("inlet_parabolic"):
        ny = p["ny"]
        y = np.broadcast_to(np.arange(ny)[:, None], (ny, p["nx"])).reshape(-1) + 0.5
        u[0] *= 4.0 * y * (ny - y) / (ny * ny)
    fields["u"] = u
    return fields


def smooth_field(shape, seed, modes=5):
    """Seeded smooth periodic field in [0, 1] (a few low Fourier modes)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(modes):
        k = rng.integers(0, 3, size=len(shape))
        ph = rng.uniform(0, 2 * math.pi)
        f += rng.uniform(0.5, 1.0) * np.cos(2 * math.pi * sum(ki * g for ki, g in zip(k, grids)) + ph)
    f -= f.min()
    return f / max(f.max(), 1e-300)


def random_state(p, seed, T_range=(300.0, 600.0), u_amp=0.02, phi_kind="smooth", phi_max=0.6):
    """Seeded smooth random fields for parity cases.  Phase fields stay smooth
    (cell-to-cell ratios of phi_f bounded) because the phi_f-weighted explicit
    diffusion is only stable for profiles resolved on the grid."""
    rng = np.random.default_rng(seed)
    shape = (p["nz"], p["ny"], p["nx"]) if p["dim"] == 3 else (p["ny"], p["nx"])
    N = int(np.prod(shape))
    sf = lambda k: smooth_field(shape, seed * 97 + k).reshape(-1)
    if phi_kind == "smooth":
        phi = phi_max * sf(1)
    elif phi_kind == "zero":
        phi = np.zeros(N)
    else:
        phi = np.asarray(phi_kind, dtype=np.float64).reshape(-1)
    T = T_range[0] + (T_range[1] - T_range[0]) * sf(2)
    K = p.get("K", 0)
    Y = None
    if K:
        Y0 = np.asarray(p["Y_in"], dtype=np.float64)
        Y = Y0[:, None] * (0.8 + 0.4 * np.stack([sf(10 + k) for k in range(K)]))
        Y /= Y.sum(axis=0, keepdims=True)
        Y = Y.reshape(-1)
    u = u_amp * (2 * np.stack([sf(20 + a) for a in range(p["dim"])]) - 1)
    Ph = 1e-3 * (2 * sf(30) - 1)
    Ts = T_range[0] + (T_range[1] - T_range[0]) * sf(31) if p.get("Ts_field") else None
    return {"phi": phi, "T": T, "Y": Y, "Ts": Ts, "u": u, "Ph": Ph}
