"""ctypes binding of libpflb.so (include/pflb.h).  Argument marshalling only:
every step of the time-step path runs in the library's CUDA kernels.  There is
no CPU fallback: if the library cannot be loaded this module raises."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KMAX, JMAX = 8, 4
BC = {"periodic": 0, "wall": 1, "inlet": 2, "outlet": 3}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_fp16": 2}
P0MODE = {"fixed": 0, "closed": 1}
CHEM = {"none": 0, "explicit": 1, "implicit": 2, "surrogate": 3}
MLP_PARAMS = 9286
FIELD = {"T": 1, "Y": 2, "Ts": 4, "u": 8, "rho": 16, "Ph": 32, "g": 64}
FIELD_ORDER = ["T", "Y", "Ts", "u", "rho", "Ph", "g"]
HOST, DEVICE = 0, 1
F64, F32 = 0, 1


class Desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("precision", C.c_int), ("bc", C.c_int * 6),
        ("wall_u", (C.c_double * 3) * 6), ("wall_T", C.c_double * 6),
        ("dx", C.c_double), ("dt", C.c_double), ("rho_ref", C.c_double),
        ("M0", C.c_double), ("cp0", C.c_double),
        ("mu_ref", C.c_double), ("sutherland", C.c_int),
        ("suth_T", C.c_double), ("suth_S", C.c_double), ("Pr", C.c_double),
        ("A_u", C.c_double), ("A_T", C.c_double), ("eta", C.c_double),
        ("Fb", C.c_double * 3),
        ("inlet_parabolic", C.c_int), ("u_in", C.c_double), ("T_in", C.c_double),
        ("p0_mode", C.c_int), ("P0", C.c_double),
        ("Ts_field", C.c_int), ("Ts_uniform", C.c_double),
        ("rhocp_s", C.c_double), ("lambda_s", C.c_double), ("phi_min", C.c_double),
        ("T_max", C.c_double), ("outlet_nscbc", C.c_int), ("nscbc_sigma", C.c_double),
        ("u_s", C.c_double * 3),
        ("stream", C.c_void_p), ("device", C.c_int),
    ]


class Mechanism(C.Structure):
    _fields_ = [
        ("K", C.c_int), ("J", C.c_int), ("chem_mode", C.c_int),
        ("M", C.c_double * KMAX), ("cp", C.c_double * KMAX), ("hf", C.c_double * KMAX),
        ("Dref", C.c_double * KMAX), ("D_Tref", C.c_double), ("D_exp", C.c_double),
        ("Y_in", C.c_double * KMAX),
        ("A", C.c_double * JMAX), ("b", C.c_double * JMAX), ("EaR", C.c_double * JMAX),
        ("order", (C.c_double * KMAX) * JMAX), ("stoich", (C.c_double * KMAX) * JMAX),
        ("rev", C.c_int * JMAX), ("dH", C.c_double * JMAX), ("dS", C.c_double * JMAX),
        ("rorder", (C.c_double * KMAX) * JMAX), ("p_ref", C.c_double),
        ("transport", C.c_int), ("mu_k", C.c_double * KMAX), ("suth_Tk", C.c_double * KMAX),
        ("suth_Sk", C.c_double * KMAX),
        ("inlet_feedback", C.c_int),
    ]


class Scalars(C.Structure):
    _fields_ = [("P0", C.c_double), ("P0_prev", C.c_double), ("mass", C.c_double),
                ("I", C.c_double), ("flux_in", C.c_double), ("flux_out", C.c_double),
                ("step", C.c_longlong), ("status", C.c_int), ("u_in", C.c_double),
                ("fuel", C.c_double), ("outlet_pb", C.c_double)]


class Diagnostics(C.Structure):
    _fields_ = [("drag", C.c_double * 3), ("heat", C.c_double), ("mass", C.c_double),
                ("outlet_Tm", C.c_double), ("flux_in_total", C.c_double),
                ("flux_out_total", C.c_double), ("step", C.c_longlong)]


class Surrogate(C.Structure):
    _fields_ = [
        ("x_mean", C.c_double * 8), ("x_std", C.c_double * 8),
        ("y_mean", C.c_double * 6), ("y_std", C.c_double * 6),
        ("theta_s", C.c_double),
        ("lo", C.c_double * 8), ("hi", C.c_double * 8),
        ("n_elem", C.c_int), ("elem", (C.c_double * KMAX) * 4), ("elem_mass", C.c_double * 4),
        ("tol", C.c_double), ("engine", C.c_int), ("skip_eps", C.c_double),
    ]


MLP_ENGINES = {"warp_mma": 0, "tcgen05": 1}


_lib = None


def lib():
    """Load libpflb.so (building it first when sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpflb.so is missing; run __graft_entry__.build()")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.pflb_create_domain.argtypes = [C.POINTER(Desc), C.POINTER(vp)]
        L.pflb_validate.argtypes = [C.POINTER(Desc), C.POINTER(Mechanism)]
        L.pflb_set_phase_field.argtypes = [vp, vp, vp, C.c_int, C.c_int]
        L.pflb_set_mechanism.argtypes = [vp, C.POINTER(Mechanism)]
        L.pflb_set_fields.argtypes = [vp, C.c_uint, vp, C.c_int, C.c_int]
        L.pflb_step.argtypes = [vp, C.c_int]
        L.pflb_get_fields.argtypes = [vp, C.c_uint, vp, C.c_size_t, C.c_int, C.c_int]
        L.pflb_get_scalars.argtypes = [vp, C.POINTER(Scalars)]
        L.pflb_get_diagnostics.argtypes = [vp, C.POINTER(Diagnostics)]
        L.pflb_lattice.argtypes = [C.c_int, vp, vp]
        L.pflb_state_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.pflb_get_state.argtypes = [vp, vp, C.c_size_t, C.c_int]
        L.pflb_set_state.argtypes = [vp, vp, C.c_size_t, C.c_int]
        L.pflb_step_noalloc.argtypes = [C.POINTER(Desc), C.POINTER(Mechanism), vp, vp, vp,
                                        vp, vp, vp, vp, vp, vp, C.POINTER(Scalars)]
        L.pflb_select_kernel.argtypes = [vp, C.c_int]
        L.pflb_set_wait_limit.argtypes = [vp, C.c_longlong]
        L.pflb_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), vp]
        L.pflb_destroy.argtypes = [vp]
        L.pflb_mlp_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
        L.pflb_mlp_set_params.argtypes = [vp, vp]
        L.pflb_mlp_get_params.argtypes = [vp, vp]
        L.pflb_mlp_forward.argtypes = [vp, vp, vp, C.c_longlong]
        L.pflb_mlp_gradient.argtypes = [vp, vp, vp, C.c_longlong, vp, C.POINTER(C.c_double)]
        L.pflb_mlp_train.argtypes = [vp, vp, vp, C.c_longlong, C.c_int, C.c_int, C.c_float,
                                     C.POINTER(C.c_double)]
        L.pflb_mlp_destroy.argtypes = [vp]
        L.pflb_set_surrogate.argtypes = [vp, vp, C.POINTER(Surrogate)]
        L.pflb_chem_increments.argtypes = [vp, vp, C.c_size_t, C.c_int, C.c_int]
        L.pflb_chem_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.pflb_create_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
        L.pflb_batch_step.argtypes = [vp, C.c_int]
        L.pflb_batch_set_config.argtypes = [vp, C.c_int, C.c_int]
        L.pflb_batch_get_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(C.c_int)]
        L.pflb_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]
        L.pflb_batch_destroy.argtypes = [vp]
        L.pflb_batch_last_error.argtypes = [vp]
        L.pflb_batch_last_error.restype = C.c_char_p
        L.pflb_probe_fp64_fma.argtypes = [C.c_int, C.POINTER(C.c_double)]
        L.pflb_last_error.argtypes = [vp]
        L.pflb_last_error.restype = C.c_char_p
        _lib = L
    return _lib


class PflbError(RuntimeError):
    """A failed library call; `code` is the PFLB_ERR_* status."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


def _check(rc, handle=None):
    if rc != 0:
        msg = lib().pflb_last_error(handle)
        raise PflbError(f"pflb error {rc}: {msg.decode() if msg else ''}", rc)


def make_desc(prob: dict, precision: str = "fp64", stream: int = 0, device: int = 0) -> Desc:
    d = Desc()
    d.dim, d.nx, d.ny = prob["dim"], prob["nx"], prob["ny"]
    d.nz = prob.get("nz", 1) if d.dim == 3 else 1
    d.precision = PRECISION[precision]
    for f, name in enumerate(prob["bc"]):
        d.bc[f] = BC[name]
    for f, v in enumerate(prob.get("wall_u", [[0, 0, 0]] * 6)):
        for a in range(3):
            d.wall_u[f][a] = v[a]
    for f, v in enumerate(prob.get("wall_T", [0.0] * 6)):
        d.wall_T[f] = v
    d.dx, d.dt, d.rho_ref = prob["dx"], prob["dt"], prob["rho_ref"]
    d.M0, d.cp0 = prob.get("M0", 0.02897), prob.get("cp0", 1006.0)
    d.mu_ref, d.sutherland = prob["mu_ref"], int(prob.get("sutherland", 0))
    d.suth_T, d.suth_S, d.Pr = prob.get("suth_T", 273.0), prob.get("suth_S", 110.5), prob["Pr"]
    d.A_u, d.A_T, d.eta = prob["A_u"], prob["A_T"], prob["eta"]
    for a, v in enumerate(prob.get("Fb", [0, 0, 0])):
        d.Fb[a] = v
    d.inlet_parabolic = int(prob.get("inlet_parabolic", 0))
    d.u_in, d.T_in = prob.get("u_in", 0.0), prob.get("T_in", 300.0)
    d.p0_mode = P0MODE[prob.get("p0_mode", "fixed")]
    d.P0 = prob["P0"]
    d.Ts_field = int(prob.get("Ts_field", 0))
    d.Ts_uniform = prob.get("Ts_uniform", 300.0)
    d.rhocp_s, d.lambda_s = prob.get("rhocp_s", 1.0), prob.get("lambda_s", 0.0)
    d.phi_min = prob.get("phi_min", 1e-6)
    d.T_max = prob.get("T_max", 0.0)
    if prob.get("outlet") == "nscbc":
        d.outlet_nscbc, d.nscbc_sigma = 1, float(prob.get("nscbc_sigma", 0.25))
    for a, v in enumerate(prob.get("u_s", [])[:3]):
        d.u_s[a] = float(v)
    d.stream = stream
    d.device = device
    return d


def make_mechanism(prob: dict) -> Mechanism:
    m = Mechanism()
    K = prob.get("K", 0)
    m.K = K
    rx = prob.get("reactions", []) if K else []
    m.J = len(rx)
    m.chem_mode = CHEM[prob.get("chem", "none")] if K else 0
    for k in range(K):
        m.M[k], m.cp[k], m.hf[k] = prob["M"][k], prob["cp"][k], prob["hf"][k]
        m.Dref[k], m.Y_in[k] = prob["Dref"][k], prob["Y_in"][k]
    m.D_Tref, m.D_exp = prob.get("D_Tref", 300.0), prob.get("D_exp", 0.0)
    for j, r in enumerate(rx):
        m.A[j], m.b[j], m.EaR[j] = r["A"], r.get("b", 0.0), r["EaR"]
        for k in range(K):
            m.order[j][k] = r["order"][k]
            m.stoich[j][k] = r["stoich"][k]
        if r.get("reverse"):
            m.rev[j] = 1
            m.dH[j], m.dS[j] = r["reverse"]["dH"], r["reverse"]["dS"]
            for k in range(K):
                m.rorder[j][k] = r["reverse"]["order"][k]
    m.p_ref = prob.get("p_ref", 101325.0)
    if K and prob.get("transport") == "mixture":
        m.transport = 1
        for k in range(K):
            m.mu_k[k], m.suth_Tk[k], m.suth_Sk[k] = prob["mu_k"][k], prob["suth_Tk"][k], \
                prob["suth_Sk"][k]
    if prob.get("inlet_feedback") is not None:
        m.inlet_feedback = int(prob["inlet_feedback"]) + 1  # species index + 1
    return m


def validate(prob: dict, precision: str = "fp64"):
    """(status, message) of the description and mechanism checks that
    pflb_create_domain and pflb_set_mechanism make; no CUDA call."""
    d = make_desc(prob, precision)
    m = make_mechanism(prob) if prob.get("K", 0) else None
    rc = lib().pflb_validate(C.byref(d), C.byref(m) if m is not None else None)
    msg = lib().pflb_last_error(None)
    return rc, (msg.decode() if msg else "")


def lattice(dim):
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    Q = lib().pflb_lattice(dim, c.ctypes.data, w.ctypes.data)
    return c.reshape(19, 3)[:Q].copy(), w[:Q].copy()


def _arg(a, dtype):
    """(pointer, where, dtype code, keepalive) for a numpy array or torch tensor."""
    code = F64 if dtype == np.float64 else F32
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        t = a.contiguous().to(torch.float64 if code == F64 else torch.float32)
        return t.data_ptr(), (DEVICE if t.is_cuda else HOST), code, t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, HOST, code, arr


class Domain:
    """One simulation domain living on one GPU (handle of the C ABI)."""

    def __init__(self, prob: dict, precision: str = "fp64", stream: int = 0, device: int = 0):
        self.prob = prob
        self.precision = precision
        self.dim = prob["dim"]
        self.N = prob["nx"] * prob["ny"] * (prob.get("nz", 1) if self.dim == 3 else 1)
        self.Q = 9 if self.dim == 2 else 19
        self.K = prob.get("K", 0)
        self._h = C.c_void_p()
        self._desc = make_desc(prob, precision, stream, device)
        _check(lib().pflb_create_domain(C.byref(self._desc), C.byref(self._h)), None)
        if self.K:
            self._mech = make_mechanism(prob)
            _check(lib().pflb_set_mechanism(self._h, C.byref(self._mech)), self._h)

    def set_phase_field(self, phi, Ts=None, dtype=np.float64):
        p, where, code, k1 = _arg(phi, dtype)
        ts = None
        if Ts is not None:
            ts, where2, _, k2 = _arg(Ts, dtype)
            assert where2 == where, "phi and Ts must live on the same side"
        _check(lib().pflb_set_phase_field(self._h, p, ts, code, where), self._h)

    def set_fields(self, T, Y=None, u=None, dtype=np.float64):
        parts, mask = [T], FIELD["T"]
        if self.K:
            parts.append(Y)
            mask |= FIELD["Y"]
        if u is not None:
            parts.append(u)
            mask |= FIELD["u"]
        if hasattr(T, "data_ptr"):
            import torch
            buf = torch.cat([torch.as_tensor(x).reshape(-1) for x in parts])
        else:
            buf = np.concatenate([np.asarray(x, dtype=dtype).reshape(-1) for x in parts])
        p, where, code, keep = _arg(buf, dtype)
        _check(lib().pflb_set_fields(self._h, mask, p, code, where), self._h)

    def step(self, n: int = 1):
        _check(lib().pflb_step(self._h, int(n)), self._h)

    def _sizes(self):
        return {"T": self.N, "Y": self.K * self.N, "Ts": self.N, "u": self.dim * self.N,
                "rho": self.N, "Ph": self.N, "g": self.Q * self.N}

    def get(self, *names, dtype=np.float64, out=None):
        """Fields as numpy arrays (host), or written into a packed device tensor `out`."""
        mask = 0
        for n in names:
            mask |= FIELD[n]
        sizes = self._sizes()
        order = [n for n in FIELD_ORDER if mask & FIELD[n]]
        total = sum(sizes[n] for n in order)
        if out is not None:
            p, where, code, keep = _arg(out, dtype)
            _check(lib().pflb_get_fields(self._h, mask, out.data_ptr(), out.numel() *
                                         out.element_size(), code, DEVICE), self._h)
            return out
        buf = np.empty(total, dtype=dtype)
        code = F64 if dtype == np.float64 else F32
        _check(lib().pflb_get_fields(self._h, mask, buf.ctypes.data, buf.nbytes, code, HOST),
               self._h)
        res, off = {}, 0
        for n in order:
            res[n] = buf[off:off + sizes[n]]
            off += sizes[n]
        if "u" in res:
            res["u"] = res["u"].reshape(self.dim, self.N)
        if "Y" in res:
            res["Y"] = res["Y"].reshape(self.K, self.N)
        if "g" in res:
            res["g"] = res["g"].reshape(self.Q, self.N)
        return res if len(names) > 1 else res[names[0]]

    def scalars(self) -> dict:
        s = Scalars()
        _check(lib().pflb_get_scalars(self._h, C.byref(s)), self._h)
        return {f: getattr(s, f) for f, _ in Scalars._fields_}

    def diagnostics(self) -> dict:
        """Drag force (dim), heat from the solid, fluid mass, outlet mixing-cup
        temperature and the summed inlet / outlet fluxes (lattice units)."""
        s = Diagnostics()
        _check(lib().pflb_get_diagnostics(self._h, C.byref(s)), self._h)
        return {"drag": np.array(s.drag[:self.dim]), "heat": s.heat, "mass": s.mass,
                "outlet_Tm": s.outlet_Tm, "flux_in_total": s.flux_in_total,
                "flux_out_total": s.flux_out_total, "step": s.step}

    KERNELS = {"tiled": 0, "tma": 1, "persistent": 2, "persistent_32x16": 3, "march": 4,
               "march_prefetch": 5}

    def select_kernel(self, name: str):
        _check(lib().pflb_select_kernel(self._h, self.KERNELS[name]), self._h)

    def set_wait_limit(self, cycles: int):
        """Bound of the device-side waits in SM clock cycles (0: one probe)."""
        _check(lib().pflb_set_wait_limit(self._h, int(cycles)), self._h)

    def autotune(self, steps: int = 20):
        """Time each step kernel (state restored afterwards), keep the fastest.
        Returns (chosen name, {name: us per step or None})."""
        ch = C.c_int()
        us = np.zeros(len(self.KERNELS))
        _check(lib().pflb_autotune(self._h, int(steps), C.byref(ch), us.ctypes.data), self._h)
        names = {v: k for k, v in self.KERNELS.items()}
        return names[ch.value], {names[i]: (float(us[i]) if us[i] > 0 else None)
                                 for i in range(len(self.KERNELS))}

    def set_surrogate(self, net: "Mlp", surr: Surrogate):
        """Attach a trained network (chem mode "surrogate", six species)."""
        self._net = net  # the network must outlive its use by this domain
        self._surr = surr
        _check(lib().pflb_set_surrogate(self._h, net._h, C.byref(surr)), self._h)

    def chem_increments(self):
        """(dY [K, N], dT [N]) of one chemistry step of the current state."""
        buf = np.empty((self.K + 1) * self.N)
        _check(lib().pflb_chem_increments(self._h, buf.ctypes.data, buf.nbytes, F64, HOST),
               self._h)
        buf = buf.reshape(self.K + 1, self.N)
        return buf[:self.K], buf[self.K]

    def chem_stats(self):
        """(cells that fell back to the integrator, cells the network evaluated)."""
        fb, ev = C.c_double(), C.c_double()
        _check(lib().pflb_chem_stats(self._h, C.byref(fb), C.byref(ev)), self._h)
        return fb.value, ev.value

    def state_bytes(self) -> int:
        n = C.c_size_t()
        _check(lib().pflb_state_bytes(self._h, C.byref(n)), self._h)
        return n.value

    def get_state(self, out=None):
        """Serialised checkpoint into `out` (uint8 numpy array or torch tensor,
        host or device) or a new host numpy array."""
        nb = self.state_bytes()
        if out is None:
            out = np.empty(nb, dtype=np.uint8)
        if hasattr(out, "data_ptr"):
            where = DEVICE if out.is_cuda else HOST
            ptr, size = out.data_ptr(), out.numel() * out.element_size()
        else:
            where, ptr, size = HOST, out.ctypes.data, out.nbytes
        _check(lib().pflb_get_state(self._h, ptr, size, where), self._h)
        return out

    def set_state(self, buf):
        if hasattr(buf, "data_ptr"):
            where = DEVICE if buf.is_cuda else HOST
            ptr, size = buf.data_ptr(), buf.numel() * buf.element_size()
        else:
            buf = np.ascontiguousarray(buf)
            where, ptr, size = HOST, buf.ctypes.data, buf.nbytes
        _check(lib().pflb_set_state(self._h, ptr, size, where), self._h)

    def close(self):
        if self._h:
            lib().pflb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_noalloc(prob, precision, arrays, scalars, stream=0, device=0):
    """One step through pflb_step_noalloc on caller-owned CUDA tensors.

    For callers that cannot allocate device memory (host frameworks that own
    all device memory through their own pool, loops that forbid allocator
    calls after start-up): the library allocates nothing here; its reduction
    scratch is a fixed device array.
    `arrays` maps phi, g_in, g_out, T_in, T_out, Y_in, Y_out, Ts_in, Ts_out to
    contiguous CUDA tensors in the compute precision (Y/Ts may be absent);
    `scalars` is a dict with P0, P0_prev, mass, step, status and is returned
    updated."""
    d = make_desc(prob, precision, stream, device)
    m = make_mechanism(prob) if prob.get("K", 0) else None
    sc = Scalars()
    for k in ("P0", "P0_prev", "mass", "I", "flux_in", "flux_out"):
        setattr(sc, k, float(scalars.get(k, 0.0)))
    sc.step, sc.status = int(scalars.get("step", 0)), int(scalars.get("status", 0))
    ptr = lambda k: (arrays[k].data_ptr() if arrays.get(k) is not None else None)
    rc = lib().pflb_step_noalloc(C.byref(d), C.byref(m) if m is not None else None,
                                 ptr("phi"), ptr("g_in"), ptr("g_out"), ptr("T_in"),
                                 ptr("T_out"), ptr("Y_in"), ptr("Y_out"), ptr("Ts_in"),
                                 ptr("Ts_out"), C.byref(sc))
    if rc != 0:
        msg = lib().pflb_last_error(None)
        raise PflbError(f"pflb_step_noalloc error {rc}: {msg.decode() if msg else ''}", rc)
    return {f: getattr(sc, f) for f, _ in Scalars._fields_}


def _dev_f32(t, cols):
    """Pointer of a contiguous float32 CUDA tensor with `cols` columns."""
    import torch
    if not (hasattr(t, "data_ptr") and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and t.dim() == 2 and t.shape[1] == cols):
        raise ValueError(f"expected a contiguous float32 CUDA tensor [n, {cols}]")
    return t.data_ptr()


class Mlp:
    """The chemistry-surrogate network (8 -> 64 -> 64 -> 64 -> 6) on one GPU:
    BF16 tensor-core forward, backward and Adam kernels with FP32 master
    parameters.  Inputs and targets are float32 CUDA tensors."""

    def __init__(self, device: int = 0, stream: int = 0):
        self._h = C.c_void_p()
        rc = lib().pflb_mlp_create(device, stream, C.byref(self._h))
        if rc != 0:
            raise PflbError(f"pflb_mlp_create error {rc}")

    def _rc(self, rc, what):
        if rc != 0:
            raise PflbError(f"{what} error {rc}")

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == MLP_PARAMS
        self._rc(lib().pflb_mlp_set_params(self._h, th.ctypes.data), "pflb_mlp_set_params")

    def get_params(self):
        th = np.empty(MLP_PARAMS, dtype=np.float32)
        self._rc(lib().pflb_mlp_get_params(self._h, th.ctypes.data), "pflb_mlp_get_params")
        return th

    def forward(self, X, out=None):
        import torch
        n = X.shape[0]
        if out is None:
            out = torch.empty((n, 6), dtype=torch.float32, device=X.device)
        self._rc(lib().pflb_mlp_forward(self._h, _dev_f32(X, 8), _dev_f32(out, 6), n),
                 "pflb_mlp_forward")
        return out

    def gradient(self, X, Y):
        """(mean squared error, flat FP32 gradient) over all rows."""
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = C.c_double()
        self._rc(lib().pflb_mlp_gradient(self._h, _dev_f32(X, 8), _dev_f32(Y, 6), X.shape[0],
                                         g.ctypes.data, C.byref(loss)), "pflb_mlp_gradient")
        return loss.value, g

    def train(self, X, Y, batch: int, steps: int, lr: float) -> float:
        """`steps` Adam steps over consecutive mini-batches; last mini-batch loss."""
        loss = C.c_double()
        self._rc(lib().pflb_mlp_train(self._h, _dev_f32(X, 8), _dev_f32(Y, 6), X.shape[0],
                                      int(batch), int(steps), float(lr), C.byref(loss)),
                 "pflb_mlp_train")
        return loss.value

    def close(self):
        if self._h:
            lib().pflb_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many 2-D domains without species advanced together: one persistent
    kernel per step over all their tiles, replayed from a CUDA graph."""

    TILES = {"32x8": 0, "32x16": 1, "64x4": 2}

    def __init__(self, domains):
        self.domains = list(domains)  # kept alive as long as the batch
        arr = (C.c_void_p * len(self.domains))(*[d._h.value for d in self.domains])
        self._h = C.c_void_p()
        rc = lib().pflb_create_batch(arr, len(self.domains), C.byref(self._h))
        if rc != 0:
            msg = lib().pflb_batch_last_error(None)
            raise PflbError(f"pflb_create_batch error {rc}: {msg.decode() if msg else ''}")

    def _check(self, rc):
        if rc != 0:
            msg = lib().pflb_batch_last_error(self._h)
            raise PflbError(f"pflb batch error {rc}: {msg.decode() if msg else ''}")

    def step(self, n: int = 1):
        self._check(lib().pflb_batch_step(self._h, int(n)))

    def set_config(self, tile: str = "32x8", blocks_per_sm: int = 0):
        self._check(lib().pflb_batch_set_config(self._h, self.TILES[tile], int(blocks_per_sm)))

    def config(self):
        t, b, g = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().pflb_batch_get_config(self._h, C.byref(t), C.byref(b), C.byref(g)))
        names = {v: k for k, v in self.TILES.items()}
        return {"tile": names[t.value], "blocks_per_sm": b.value, "grid": g.value}

    def autotune(self, steps: int = 5):
        """Time every (tile shape, blocks per SM), keep the fastest; the
        domains' states are put back.  Returns (config, {(tile, bps): us})."""
        t, b = C.c_int(), C.c_int()
        us = np.zeros(3 * 8)
        self._check(lib().pflb_batch_autotune(self._h, int(steps), C.byref(t), C.byref(b),
                                              us.ctypes.data))
        names = {v: k for k, v in self.TILES.items()}
        table = {(names[i // 8], i % 8 + 1): float(us[i]) for i in range(24) if us[i] > 0}
        return self.config(), table

    def close(self):
        if self._h:
            lib().pflb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fp64_tflops(device: int = 0) -> float:
    """Measured FP64 FMA rate of the GPU (TFLOP/s), the FP64 paths' ceiling."""
    t = C.c_double()
    rc = lib().pflb_probe_fp64_fma(int(device), C.byref(t))
    if rc != 0:
        raise PflbError(f"pflb_probe_fp64_fma error {rc}")
    return t.value
