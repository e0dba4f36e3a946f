"""ctypes wrapper around the plain FP64 CPU oracle (``pflb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the product path never does.
It imports nothing from the product package.  Parameters arrive as the plain
problem dictionary produced by the input generators (physical quantities plus
the lattice shape); the conversion to the oracle's own struct happens here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pflb_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")
KMAX, JMAX = 8, 4
BC = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
P0MODE = {"fixed": 0, "closed": 1}
CHEM = {"none": 0, "explicit": 1, "implicit": 2}

_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int * 6),
        ("wall_u", (C.c_double * 3) * 6),
        ("wall_T", C.c_double * 6),
        ("dx", C.c_double), ("dt", C.c_double), ("rho_ref", C.c_double),
        ("K", C.c_int),
        ("M0", C.c_double), ("cp0", C.c_double),
        ("M", C.c_double * KMAX), ("cp", C.c_double * KMAX), ("hf", C.c_double * KMAX),
        ("Dref", C.c_double * KMAX),
        ("D_Tref", C.c_double), ("D_exp", C.c_double),
        ("mu_ref", C.c_double), ("sutherland", C.c_int),
        ("suth_T", C.c_double), ("suth_S", C.c_double), ("Pr", C.c_double),
        ("A_u", C.c_double), ("A_T", C.c_double), ("eta", C.c_double),
        ("Fb", C.c_double * 3),
        ("inlet_parabolic", C.c_int),
        ("u_in", C.c_double), ("T_in", C.c_double), ("Y_in", C.c_double * KMAX),
        ("p0_mode", C.c_int),
        ("Ts_field", C.c_int),
        ("Ts_uniform", C.c_double), ("rhocp_s", C.c_double), ("lambda_s", C.c_double),
        ("phi_min", C.c_double),
        ("chem_mode", C.c_int), ("J", C.c_int),
        ("A", C.c_double * JMAX), ("b", C.c_double * JMAX), ("EaR", C.c_double * JMAX),
        ("order", (C.c_double * KMAX) * JMAX), ("stoich", (C.c_double * KMAX) * JMAX),
        ("rev", C.c_int * JMAX), ("dH", C.c_double * JMAX), ("dS", C.c_double * JMAX),
        ("rorder", (C.c_double * KMAX) * JMAX), ("p_ref", C.c_double),
        ("transport_mix", C.c_int), ("mu_k", C.c_double * KMAX),
        ("suth_Tk", C.c_double * KMAX), ("suth_Sk", C.c_double * KMAX),
        ("feedback", C.c_int), ("fb_k", C.c_int),
        ("nscbc", C.c_int), ("nscbc_K", C.c_double), ("ob", C.POINTER(C.c_double)),
        ("moving", C.c_int), ("u_s", C.c_double * 3),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE double arithmetic (no contraction);
    its independent per-cell loops run on OpenMP host threads."""
    with _lock:
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                                   "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"])
            os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        P = C.POINTER(OrcParams)
        L.orc_params_size.restype = C.c_int
        assert L.orc_params_size() == C.sizeof(OrcParams), "OrcParams layout mismatch"
        L.orc_lattice.argtypes = [C.c_int, np.ctypeslib.ndpointer(dtype=np.int32), dp]
        L.orc_lattice.restype = C.c_int
        L.orc_equilibrium.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
        L.orc_source.argtypes = [C.c_int, C.c_double, dp, dp, dp, C.c_double, dp]
        L.orc_chem_rates.argtypes = [P, C.c_double, dp, C.c_double, dp, C.POINTER(C.c_double)]
        L.orc_chem_implicit.argtypes = [P, C.c_double, dp, C.c_double, dp,
                                        C.POINTER(C.c_double)]
        L.orc_chem_implicit.restype = C.c_int
        L.orc_fd_phase.argtypes = [P, dp, dp, dp, C.c_void_p, dp, C.c_double, C.c_double,
                                   dp, dp, C.c_void_p, C.c_void_p]
        L.orc_init.argtypes = [P, dp, dp, dp, dp, C.c_void_p, C.c_void_p, C.c_double, dp]
        L.orc_moments.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [P, dp, dp, dp, dp, C.c_void_p, dp, C.c_void_p]
        L.orc_run.argtypes = [P, dp, dp, dp, dp, C.c_void_p, dp, C.c_int]
        L.orc_diagnostics.argtypes = [P, dp, dp, dp, dp, C.c_void_p, dp, dp]
        L.orc_phase_at.argtypes = [P, dp, C.c_double, dp]
        L.orc_mixture_transport.argtypes = [P, C.c_double, dp, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's per-cell loops (0: all cores); returns
    the number in effect.  Results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(prob: dict) -> OrcParams:
    """Fill the oracle's struct from a problem dictionary (see the input module)."""
    p = OrcParams()
    p.dim = prob["dim"]
    p.nx, p.ny = prob["nx"], prob["ny"]
    p.nz = prob.get("nz", 1) if p.dim == 3 else 1
    for f, name in enumerate(prob["bc"]):
        p.bc[f] = BC[name]
    for f, v in enumerate(prob.get("wall_u", [[0, 0, 0]] * 6)):
        for a in range(3):
            p.wall_u[f][a] = v[a]
    for f, v in enumerate(prob.get("wall_T", [0.0] * 6)):
        p.wall_T[f] = v
    p.dx, p.dt, p.rho_ref = prob["dx"], prob["dt"], prob["rho_ref"]
    K = prob.get("K", 0)
    p.K = K
    p.M0, p.cp0 = prob.get("M0", 0.02897), prob.get("cp0", 1006.0)
    for k in range(K):
        p.M[k] = prob["M"][k]
        p.cp[k] = prob["cp"][k]
        p.hf[k] = prob["hf"][k]
        p.Dref[k] = prob["Dref"][k]
    p.D_Tref, p.D_exp = prob.get("D_Tref", 300.0), prob.get("D_exp", 0.0)
    p.mu_ref, p.sutherland = prob["mu_ref"], int(prob.get("sutherland", 0))
    p.suth_T, p.suth_S, p.Pr = prob.get("suth_T", 273.0), prob.get("suth_S", 110.5), prob["Pr"]
    p.A_u, p.A_T, p.eta = prob["A_u"], prob["A_T"], prob["eta"]
    for a, v in enumerate(prob.get("Fb", [0, 0, 0])):
        p.Fb[a] = v
    p.inlet_parabolic = int(prob.get("inlet_parabolic", 0))
    p.u_in, p.T_in = prob.get("u_in", 0.0), prob.get("T_in", 300.0)
    for k in range(K):
        p.Y_in[k] = prob["Y_in"][k]
    p.p0_mode = P0MODE[prob.get("p0_mode", "fixed")]
    p.Ts_field = int(prob.get("Ts_field", 0))
    p.Ts_uniform = prob.get("Ts_uniform", 300.0)
    p.rhocp_s, p.lambda_s = prob.get("rhocp_s", 1.0), prob.get("lambda_s", 0.0)
    p.phi_min = prob.get("phi_min", 1e-6)
    p.chem_mode = CHEM[prob.get("chem", "none")]
    rx = prob.get("reactions", [])
    p.J = len(rx)
    for j, r in enumerate(rx):
        p.A[j], p.b[j], p.EaR[j] = r["A"], r.get("b", 0.0), r["EaR"]
        for k in range(K):
            p.order[j][k] = r["order"][k]
            p.stoich[j][k] = r["stoich"][k]
        if r.get("reverse"):
            p.rev[j] = 1
            p.dH[j], p.dS[j] = r["reverse"]["dH"], r["reverse"]["dS"]
            for k in range(K):
                p.rorder[j][k] = r["reverse"]["order"][k]
    p.p_ref = prob.get("p_ref", 101325.0)
    if prob.get("inlet_feedback") is not None:
        p.feedback, p.fb_k = 1, int(prob["inlet_feedback"])
    us = prob.get("u_s")
    if us is not None and any(float(v) != 0.0 for v in us):
        p.moving = 1
        for a in range(3):
            p.u_s[a] = float(us[a]) if a < len(us) else 0.0
    if prob.get("outlet") == "nscbc":
        # K = sigma cs (1 - Ma^2) / l with l the domain length (Ma^2 << 1 dropped)
        p.nscbc = 1
        p.nscbc_K = prob.get("nscbc_sigma", 0.25) * (1.0 / 3.0) ** 0.5 / prob["nx"]
    if prob.get("transport") == "mixture":
        p.transport_mix = 1
        for k in range(K):
            p.mu_k[k], p.suth_Tk[k], p.suth_Sk[k] = prob["mu_k"][k], prob["suth_Tk"][k], \
                prob["suth_Sk"][k]
    return p


def ncells(prob):
    return prob["nx"] * prob["ny"] * (prob.get("nz", 1) if prob["dim"] == 3 else 1)


def nq(prob):
    return 9 if prob["dim"] == 2 else 19


class OracleState:
    """Host state of one oracle run (all float64, SoA)."""

    def __init__(self, prob, phi, T, Y=None, Ts=None, u=None, Ph=None, P0=None):
        self.prob = prob
        self.p = make_params(prob)
        N, Q, K = ncells(prob), nq(prob), prob.get("K", 0)
        self.N, self.Q, self.K = N, Q, K
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(N)
        self.T = np.ascontiguousarray(T, dtype=np.float64).reshape(N).copy()
        self.Y = (np.ascontiguousarray(Y, dtype=np.float64).reshape(K * N).copy()
                  if K > 0 else np.zeros(1))
        self.Ts = (np.ascontiguousarray(Ts, dtype=np.float64).reshape(N).copy()
                   if Ts is not None else None)
        self.g = np.zeros(Q * N)
        self.scal = np.zeros(12)
        # outlet state of the characteristic outlet: P_b, then P_h, u_x of the
        # columns nx-1 and nx-2 (5 x ny nz); the params hold a pointer to it
        nf = prob["ny"] * (prob.get("nz", 1) if prob["dim"] == 3 else 1)
        self.ob = np.zeros(6 * nf)
        self.p.ob = self.ob.ctypes.data_as(C.POINTER(C.c_double))
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        pp = None if Ph is None else np.ascontiguousarray(Ph, dtype=np.float64).reshape(-1)
        lib().orc_init(C.byref(self.p), self.phi, self.g, self.T, self.Y, _ptr(uu), _ptr(pp),
                       float(prob["P0"] if P0 is None else P0), self.scal)

    def step(self, n=1):
        L = lib()
        if n == 1:
            L.orc_step(C.byref(self.p), self.phi, self.g, self.T, self.Y, _ptr(self.Ts),
                       self.scal, None)
        else:
            L.orc_run(C.byref(self.p), self.phi, self.g, self.T, self.Y, _ptr(self.Ts),
                      self.scal, int(n))

    def step_diag(self):
        """One step; returns (u[dim,N], rho, P_h, D) of the step."""
        dim = self.prob["dim"]
        diag = np.zeros((dim + 3) * self.N)
        lib().orc_step(C.byref(self.p), self.phi, self.g, self.T, self.Y, _ptr(self.Ts),
                       self.scal, _ptr(diag))
        d = diag.reshape(dim + 3, self.N)
        return d[:dim].copy(), d[dim].copy(), d[dim + 1].copy(), d[dim + 2].copy()

    def moments(self):
        """(u[dim,N], rho[N], sum g[N]) that the next step will see."""
        dim = self.prob["dim"]
        u = np.zeros(dim * self.N)
        rho = np.zeros(self.N)
        ph = np.zeros(self.N)
        lib().orc_moments(C.byref(self.p), self.phi, self.g, self.T, self.Y, self.scal, u, rho, ph)
        return u.reshape(dim, self.N), rho, ph

    def phase(self):
        """Solid fraction of the step the state is at (a moving solid is
        displaced by steps x u_s from the field it was created with)."""
        out = np.zeros(self.N)
        lib().orc_phase_at(C.byref(self.p), self.phi, float(self.scal[6]), out)
        return out

    def diagnostics(self):
        """Drag force (dim), heat from the solid, fluid mass, outlet mixing-cup
        sums (rho u cp T, rho u cp) and the summed inlet / outlet fluxes."""
        out = np.zeros(7)
        lib().orc_diagnostics(C.byref(self.p), self.phi, self.g, self.T, self.Y, _ptr(self.Ts),
                              self.scal, out)
        dim = self.prob["dim"]
        Tm = out[5] / out[6] if out[6] != 0 else 0.0
        return {"drag": out[:dim].copy(), "heat": out[3], "mass": out[4], "outlet_Tm": Tm,
                "flux_in_total": self.scal[7], "flux_out_total": self.scal[8]}

    @property
    def P0(self):
        return self.scal[0]

    @property
    def outlet_pressure(self):
        """Boundary pressure P_b of the next step per outlet cell
        (characteristic outlet; one value over the face)."""
        nf = self.ob.size // 6
        return self.ob[:nf].copy()

    @property
    def u_in(self):
        """Inlet peak speed of the next step (lattice units)."""
        return self.scal[9]


def lattice(dim):
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    Q = lib().orc_lattice(dim, c, w)
    return c.reshape(19, 3)[:Q].copy(), w[:Q].copy()


def equilibrium(dim, Ph, rho, u):
    Q = 9 if dim == 2 else 19
    out = np.zeros(Q)
    lib().orc_equilibrium(dim, float(Ph), float(rho), np.ascontiguousarray(u, dtype=np.float64), out)
    return out


def source(dim, rho, G, u, F, D):
    Q = 9 if dim == 2 else 19
    out = np.zeros(Q)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    lib().orc_source(dim, float(rho), f64(G), f64(u), f64(F), float(D), out)
    return out


def chem_rates(prob, T, Y, rho_lat):
    p = make_params(prob)
    om = np.zeros(KMAX)
    wT = C.c_double()
    lib().orc_chem_rates(C.byref(p), float(T), np.ascontiguousarray(Y, dtype=np.float64),
                         float(rho_lat), om, C.byref(wT))
    return om[: prob["K"]].copy(), wT.value


def fd_phase(prob, phi, T, Y, Ts, u, P0, P0prev):
    """Run only the FD transport phase with a prescribed velocity field."""
    p = make_params(prob)
    N, K = ncells(prob), prob.get("K", 0)
    Tn = np.zeros(N)
    Yn = np.zeros(max(K, 1) * N)
    Tsn = np.zeros(N) if Ts is not None else None
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    Yin = f64(Y) if K > 0 else np.zeros(1)
    lib().orc_fd_phase(C.byref(p), f64(phi), f64(T), Yin, _ptr(None if Ts is None else f64(Ts)),
                       f64(u), float(P0), float(P0prev), Tn, Yn, _ptr(Tsn), None)
    return Tn, (Yn[: K * N] if K > 0 else None), Tsn


def mixture_transport(prob, T, Y):
    """(mu, lambda) in SI units of a gas of composition Y at T, mixture rules."""
    p = make_params(prob)
    mu, lam = C.c_double(), C.c_double()
    Yp = np.zeros(KMAX)
    Yp[: prob["K"]] = Y
    lib().orc_mixture_transport(C.byref(p), float(T), Yp, C.byref(mu), C.byref(lam))
    return mu.value, lam.value


def chem_implicit(prob, T, Y, rho_lat):
    """Backward-Euler chemistry increments (dY[K], dT) over one step."""
    p = make_params(prob)
    dY = np.zeros(KMAX)
    dT = C.c_double()
    rc = lib().orc_chem_implicit(C.byref(p), float(T), np.ascontiguousarray(Y, dtype=np.float64),
                                 float(rho_lat), dY, C.byref(dT))
    return dY[: prob["K"]].copy(), dT.value, rc
