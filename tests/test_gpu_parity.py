"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by
element, on the same seeded inputs.

Bars: FP64 path max relative error <= 1e-10 per field (max|a-b| / max|b|);
FP32 path L2 relative error <= 1e-4 in u and T; FP16-stored populations as
stated in the test.  Sizes span several 256-cell blocks with a ragged tail.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300._native import Domain

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def maxrel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def l2rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_pair(p, f, nsteps, precision="fp64", chunks=1):
    ora = O.OracleState(p, f["phi"], f["T"], f["Y"], f["Ts"], u=f.get("u"))
    dom = Domain(p, precision)
    dom.set_phase_field(f["phi"], f["Ts"])
    dom.set_fields(f["T"], f["Y"], f.get("u"))
    per = nsteps // chunks
    for _ in range(chunks):
        ora.step(per)
        dom.step(per)
    names = ["T", "g", "u", "rho", "Ph"] + (["Y"] if p.get("K") else []) + \
        (["Ts"] if p.get("Ts_field") else [])
    got = dom.get(*names)
    u, rho, ph = ora.moments()
    ref = {"T": ora.T, "g": ora.g.reshape(ora.Q, ora.N), "u": u, "rho": rho, "Ph": ph}
    if p.get("K"):
        ref["Y"] = ora.Y.reshape(ora.K, ora.N)
    if p.get("Ts_field"):
        ref["Ts"] = ora.Ts
    sc = dom.scalars()
    dom.close()
    return got, ref, sc, ora


def small_case(dim, nx, ny, nz=1, **kw):
    p = I._base(dim, nx, ny, nz)
    I.lattice_air(p, kw.pop("nu", 0.04))
    p.update(kw)
    return p


def assert_fp64(got, ref, sc, ora, tol=FP64_TOL):
    for k in ref:
        e = maxrel(got[k], ref[k])
        assert e <= tol, f"{k}: max rel err {e:.3e}"
    assert abs(sc["P0"] / ora.P0 - 1) <= tol
    assert sc["step"] == ora.scal[6]


# ----------------------------------------------------------------- FP64 parity
def test_fp64_config1_channel_disc_full_size():
    """The 128x64 channel with the heated disc (drag A_u = 1, A_T from the
    wall-temperature fit), 400 steps from a developed inlet profile."""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    assert_fp64(*run_pair(p, f, 400, chunks=2))


def test_fp64_config1_5000_steps_drag_nusselt_mass_balance():
    """The 128x64 channel with the heated disc over the configuration's 5000
    steps: fields within 1e-10 of the oracle, and the diagnostics -- drag on
    the disc, heat from the disc, fluid mass, summed boundary fluxes, outlet
    mixing-cup temperature -- within 1e-10, hence the drag coefficient
    Cd = 2 F_x / (rho u_mean^2 D), the Nusselt number Nu = Q / (pi lambda
    (T_s - T_in)) and the mass-balance residual (mass change minus net
    inflow) of the GPU run equal the oracle's."""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    O.set_threads(0)
    ora = O.OracleState(p, f["phi"], f["T"], u=f["u"])
    dom = Domain(p, "fp64")
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], None, f["u"])
    d0, o0 = dom.diagnostics(), ora.diagnostics()
    for _ in range(5):
        ora.step(1000)
        dom.step(1000)
    got = dom.get("T", "g", "u")
    u, _, _ = ora.moments()
    for k, ref in (("T", ora.T), ("g", ora.g.reshape(9, -1)), ("u", u)):
        assert maxrel(got[k], ref) <= FP64_TOL, k
    dg, do = dom.diagnostics(), ora.diagnostics()
    assert dg["step"] == 5000
    for k in ("heat", "mass", "outlet_Tm", "flux_in_total", "flux_out_total"):
        assert abs(dg[k] - do[k]) <= FP64_TOL * abs(do[k]), k
    assert np.max(np.abs(dg["drag"] - do["drag"])) <= FP64_TOL * np.max(np.abs(do["drag"]))
    u_mean, D, lam = 2.0 / 3.0 * p["u_in"], 16.0, (p["mu_ref"] / p["rho_ref"]) * p["cp0"] / p["Pr"]
    res = {}
    for name, d, d_0 in (("gpu", dg, d0), ("oracle", do, o0)):
        res[name] = {"Cd": 2.0 * d["drag"][0] / (u_mean ** 2 * D),
                     "Nu": d["heat"] / (np.pi * lam * (p["Ts_uniform"] - p["T_in"])),
                     "mass_residual": (d["mass"] - d_0["mass"]) -
                                      (d["flux_in_total"] - d["flux_out_total"])}
    print("config1 after 5000 steps:", res)
    for k in ("Cd", "Nu"):
        assert res["gpu"][k] > 0 and abs(res["gpu"][k] / res["oracle"][k] - 1) <= FP64_TOL
    assert abs(res["gpu"]["mass_residual"] - res["oracle"]["mass_residual"]) <= \
        FP64_TOL * do["mass"]


def test_fp64_ragged_2d_walls_random_state():
    p = small_case(2, 61, 37, bc=["inlet", "outlet", "wall", "wall", "periodic", "periodic"],
                   A_u=80.0, A_T=60.0, eta=3.0, inlet_parabolic=1, u_in=0.03,
                   Ts_uniform=520.0, sutherland=1, wall_T=[0, 0, 410.0, 0, 0, 0],
                   wall_u=[[0, 0, 0], [0, 0, 0], [0, 0, 0], [0.01, 0, 0], [0, 0, 0], [0, 0, 0]])
    f = I.random_state(p, 21, T_range=(300.0, 500.0), u_amp=0.01)
    assert_fp64(*run_pair(p, f, 60))


def test_fp64_reactive_bed_small():
    """Reactive 2-D bed (5 species, one-step chemistry, transported solid
    temperature) on a reduced lattice, 300 steps through ignition."""
    p = I.config2(nx=160, ny=48)
    p["bed"] = {"count": 6, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 40}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    p["ignite"] = [8, 32, 1500.0]
    f = I.config2_fields(p)
    f["T"][(np.arange(f["T"].size) % p["nx"] > 8) & (np.arange(f["T"].size) % p["nx"] < 32)] = 1800.0
    assert_fp64(*run_pair(p, f, 300, chunks=3))


def test_fp64_closed_box_p0_closure():
    """Closed periodic box with heat release: P0 follows the closure."""
    p = I.config2(nx=33, ny=9)
    p["bc"] = ["periodic"] * 6
    p["p0_mode"] = "closed"
    p["Ts_field"] = 0
    p["reactions"] = I.one_step_mechanism(3.3e8)
    rng = np.random.default_rng(5)
    f = I.reactive_fields(p, rng.uniform(0, 0.3, 33 * 9))
    f["T"] = 1200.0 + 400.0 * rng.uniform(0, 1, 33 * 9)
    got, ref, sc, ora = run_pair(p, f, 150)
    assert_fp64(got, ref, sc, ora)
    assert abs(ora.P0 / p["P0"] - 1) > 1e-3  # the closure really moved P0


@pytest.mark.parametrize("bc", [
    ["inlet", "outlet", "periodic", "periodic", "wall", "wall"],
    ["periodic", "periodic", "periodic", "periodic", "periodic", "periodic"],
])
def test_fp64_3d_small(bc):
    p = small_case(3, 19, 11, 7, bc=bc, A_u=60.0, A_T=50.0, eta=2.5, inlet_parabolic=1,
                   u_in=0.02, Ts_uniform=480.0, nu=0.05)
    f = I.random_state(p, 31, T_range=(300.0, 450.0), u_amp=0.01)
    assert_fp64(*run_pair(p, f, 40))


def test_fp64_3d_reactive_crop():
    """A 64^3 crop of the 3-D reactive bed (one-step chemistry, solid field)."""
    p = I.config3(nx=64, ny=32, nz=32, precision="fp64")
    p["bed"] = {"count": 6, "amin": 5, "amax": 8, "porosity": 0.5, "x0": 24}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    f = I.config3_fields(p)
    assert_fp64(*run_pair(p, f, 12, chunks=2))


def test_fp64_six_species_no_chemistry():
    p = I.config2(nx=70, ny=20)
    p["K"] = 6
    p["species"], p["M"] = I.SPECIES6, I.M6
    p["cp"], p["Dref"] = I.CP6, I.DREF6
    p["hf"] = [h / m for h, m in zip(I.HF_MOL6, I.M6)]
    p["Y_in"] = I.lean_ch4_air(0.7, I.SPECIES6)
    p["chem"], p["reactions"] = "none", []
    p["Ts_field"] = 0
    f = I.random_state(p, 41, T_range=(300.0, 900.0), u_amp=0.002)
    assert_fp64(*run_pair(p, f, 50))


def test_fp64_degenerate_shapes():
    # one-cell-thick periodic direction and the smallest x extent
    p = small_case(2, 2, 1, bc=["periodic"] * 6, Fb=[1e-5, 0, 0])
    f = I.random_state(p, 51, T_range=(300.0, 320.0), u_amp=0.005)
    assert_fp64(*run_pair(p, f, 30))
    p = small_case(2, 257, 1, bc=["inlet", "outlet", "periodic", "periodic", "periodic",
                                  "periodic"], u_in=0.01)
    f = I.random_state(p, 52, T_range=(300.0, 320.0), u_amp=0.005, phi_kind="zero")
    assert_fp64(*run_pair(p, f, 30))


def test_fp64_full_size_reactive_bed_first_steps():
    """The 1024x256 reactive bed in the configuration the benchmark times:
    the first steps agree with the oracle everywhere."""
    p = I.config2()
    f = I.config2_fields(p)
    assert_fp64(*run_pair(p, f, 6, chunks=2))


# ---------------------------------------------------------- mixed precision
def test_fp32_config1_error_after_2000_steps():
    """FP32 compute and storage on the 128x64 channel: L2 relative error of u
    and T after 2000 steps <= 1e-4 (P0 reduction stays FP64)."""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    got, ref, sc, ora = run_pair(p, f, 2000, precision="fp32", chunks=4)
    eu = l2rel(got["u"], ref["u"])
    eT = l2rel(got["T"] - 300.0, ref["T"] - 300.0)
    print(f"fp32 cfg1 2000 steps: L2 rel u {eu:.3e}, T-T_in {eT:.3e}")
    assert eu <= 1e-4 and eT <= 1e-4


def test_fp16_storage_config1_error_after_2000_steps():
    """FP16 residuals from the first-order equilibrium with FP32 cell moments
    on the 128x64 channel: L2 relative error of u and T after 2000 steps
    <= 1e-4, the bar of the FP32 path."""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    got, ref, sc, ora = run_pair(p, f, 2000, precision="fp32_fp16", chunks=4)
    eu = l2rel(got["u"], ref["u"])
    eT = l2rel(got["T"] - 300.0, ref["T"] - 300.0)
    print(f"fp16-stored cfg1 2000 steps: L2 rel u {eu:.3e}, T-T_in {eT:.3e}")
    assert eu <= 1e-4 and eT <= 1e-4


def test_fp16_storage_decodes_populations():
    """get_fields(G) of an FP16-stored domain returns the populations of the
    documented storage format, g_i = w_i (P + 3 c_i . j) + h_i w_i / S, with
    h_i the FP16 residuals and (P, j) the FP32 cell moments of the checkpoint
    (header 64 bytes, scalars 104 bytes, residuals Q*N halves, moments
    (dim+1)*N floats); and an FP16-stored run stays within 2e-4 of the FP32
    run in u after 20 steps through the expansion that ignition drives."""
    p = I.config2(nx=96, ny=40, precision="fp32_fp16")
    p["bed"] = {"count": 4, "amin": 5, "amax": 9, "porosity": 0.6, "x0": 30}
    f = I.config2_fields(p)
    out = {}
    for prec in ("fp32", "fp32_fp16"):
        d = Domain(p, prec)
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"], f["Y"])
        d.step(20)
        out[prec] = d.get("g", "u")
        if prec == "fp32_fp16":
            st = d.get_state()
        d.close()
    N, Q = p["nx"] * p["ny"], 9
    # from the end: Ts, Y (5 species), T (floats), moments, residuals
    off = st.nbytes - 4 * N * (1 + 5 + 1) - 4 * 3 * N - 2 * Q * N
    h = np.frombuffer(st[off:off + 2 * Q * N].tobytes(), dtype=np.float16).astype(np.float64)
    off += 2 * Q * N
    M = np.frombuffer(st[off:off + 4 * 3 * N].tobytes(), dtype=np.float32).astype(np.float64)
    h, M = h.reshape(Q, N), M.reshape(3, N)
    c, w = O.lattice(2)
    g = w[:, None] * (M[0][None, :] + 3.0 * (c[:, 0, None] * M[1][None, :] +
                                             c[:, 1, None] * M[2][None, :]))
    g += h * w[:, None] / 16384.0
    assert maxrel(out["fp32_fp16"]["g"], g) <= 1e-6
    assert l2rel(out["fp32_fp16"]["u"], out["fp32"]["u"]) <= 2e-4


@pytest.mark.parametrize("precision", ["fp32", "fp32_fp16"])
def test_fp32_reactive_bed_2000_steps(precision):
    """The reduced reactive bed (160 x 48, one-step chemistry through
    ignition, transported solid temperature) after 2000 steps against the
    oracle: L2 relative error of T - T_in and Y <= 1e-4, of u <= 1.5e-4.
    The velocity bar is looser than 1e-4 on this case because the FP32 path
    itself sits at 1.0e-4 there -- with exact exp / div / sqrt as well as with
    the fast approximations -- the ignition transient spreading rounding
    differences over the whole channel as a pressure wave; the FP16-stored
    residuals must stay within 10 % of that.  (The 1e-4 bar in u holds on the
    channel after 2000 steps and on the 3-D crop.)"""
    p = I.config2(nx=160, ny=48, precision=precision)
    p["bed"] = {"count": 6, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 40}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    f = I.config2_fields(p)
    O.set_threads(0)
    got, ref, sc, ora = run_pair(p, f, 2000, precision=precision, chunks=2)
    err = {"u": l2rel(got["u"], ref["u"]), "T": l2rel(got["T"] - 300.0, ref["T"] - 300.0),
           "Y": l2rel(got["Y"], ref["Y"])}
    print(f"{precision} 160x48 reactive, 2000 steps: " +
          ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    assert err["T"] <= 1e-4 and err["Y"] <= 1e-4
    assert err["u"] <= (1.5e-4 if precision == "fp32" else 1.1 * 1.5e-4)


# ------------------------------------------------------- kernel variants
def _two_kernels(p, f, precision, nsteps):
    out = {}
    for kern in ("tiled", "tma"):
        dom = Domain(p, precision)
        dom.set_phase_field(f["phi"], f["Ts"])
        dom.set_fields(f["T"], f["Y"], f.get("u"))
        dom.select_kernel(kern)
        dom.step(nsteps)
        out[kern] = dom.get(*(["T", "g", "u"] + (["Y"] if p.get("K") else [])))
        out[kern]["P0"] = dom.scalars()["P0"]
        dom.close()
    return out


@pytest.mark.parametrize("precision", ["fp32"])
def test_tma_kernel_agrees_with_tiled_kernel(precision):
    """The TMA-pipelined kernel runs the same per-cell arithmetic on staged
    copies of the same data: results agree to FP32 rounding.  (FP16 storage
    carries per-cell moments that the TMA stage does not fetch: that kernel
    runs FP32 storage only.)"""
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    out = _two_kernels(p, f, precision, 300)
    for k in ("T", "g", "u"):
        assert maxrel(out["tma"][k], out["tiled"][k]) <= 1e-6, k
    p = I.config2(nx=160, ny=48, precision=precision)
    p["bed"] = {"count": 6, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 40}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    f = I.config2_fields(p)
    out = _two_kernels(p, f, precision, 200)
    for k in ("T", "g", "u", "Y"):
        assert maxrel(out["tma"][k], out["tiled"][k]) <= 1e-6, k


def test_tma_kernel_against_oracle_fp32():
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    ora = O.OracleState(p, f["phi"], f["T"], u=f["u"])
    ora.step(1000)
    u_ref, _, _ = ora.moments()
    dom = Domain(p, "fp32")
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], None, f["u"])
    dom.select_kernel("tma")
    dom.step(1000)
    got = dom.get("T", "u")
    dom.close()
    assert l2rel(got["u"], u_ref) <= 1e-4
    assert l2rel(got["T"] - 300.0, ora.T - 300.0) <= 1e-4


def test_autotune_keeps_the_physics():
    p = I.config2(nx=256, ny=64, precision="fp32")
    p["bed"] = {"count": 8, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 80}
    f = I.config2_fields(p)
    ref = Domain(p, "fp32")
    ref.set_phase_field(f["phi"], f["Ts"])
    ref.set_fields(f["T"], f["Y"])
    ref.step(50)
    a = ref.get("T", "g")
    ref.close()
    dom = Domain(p, "fp32")
    dom.set_phase_field(f["phi"], f["Ts"])
    dom.set_fields(f["T"], f["Y"])
    chosen, times = dom.autotune(10)
    assert chosen in Domain.KERNELS and times["tiled"] is not None
    assert times["persistent"] is not None and times["persistent_32x16"] is not None
    assert dom.scalars()["step"] == 0
    dom.select_kernel("tiled")
    dom.step(50)
    b = dom.get("T", "g")
    dom.close()
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["g"], b["g"])
    # a lattice whose rows are not 16-byte multiples cannot use the TMA kernel
    q = I.config2(nx=250, ny=40, precision="fp32")
    q["bed"] = {"count": 4, "amin": 6, "amax": 9, "porosity": 0.6, "x0": 80}
    g = I.config2_fields(q)
    d2 = Domain(q, "fp32")
    d2.set_phase_field(g["phi"], g["Ts"])
    d2.set_fields(g["T"], g["Y"])
    chosen, times = d2.autotune(5)
    assert chosen != "tma" and times["tma"] is None
    d2.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fp16"])
def test_persistent_kernels_equal_the_tiled_kernel(precision):
    """The persistent kernels run the same per-tile code over the same tiles
    (32 x 8) or taller ones (32 x 16): every field bit for bit, and kernels
    may be switched between steps (the deferred reduction of the last step
    is combined over the block count of the launch that wrote it).  FP64
    fields agree to 1e-13 relative instead: the compiler may fuse a multiply
    and an add into an FMA in one tile-height instantiation and not in the
    other, which moves the last bit."""
    p = I.config2(nx=200, ny=72, precision=precision)
    p["bed"] = {"count": 6, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 50}
    f = I.config2_fields(p)
    runs = {}
    for plan in (["tiled"], ["persistent"], ["persistent_32x16"],
                 ["tiled", "persistent_32x16", "persistent", "tiled"]):
        dom = Domain(p, precision)
        dom.set_phase_field(f["phi"], f["Ts"])
        dom.set_fields(f["T"], f["Y"])
        for kern in plan * (4 // len(plan)):
            dom.select_kernel(kern)
            dom.step(15)
        runs["/".join(plan)] = (dom.get("T", "g", "Y"), dom.scalars())
        dom.close()
    ref, sref = runs["tiled"]
    for name, (got, sc) in runs.items():
        for k in ref:
            if precision == "fp64":
                err = np.max(np.abs(got[k] - ref[k])) / np.max(np.abs(ref[k]))
                print(f"{name} {k}: max relative difference {err:.2e}")
                assert err <= 1e-13, (name, k, err)
            else:
                assert np.array_equal(got[k], ref[k]), (name, k)
        assert sc["step"] == sref["step"] == 60
        tol = 1e-12 if precision == "fp64" else 1e-6
        for k in ("I", "mass", "flux_in", "flux_out"):
            assert abs(sc[k] - sref[k]) <= tol * max(abs(sref[k]), 1e-300), (name, k)


# ------------------------------------------------------ implicit chemistry
def _two_step_case(nx=96, ny=40, precision="fp64"):
    p = I.config4(nx=nx, ny=ny, precision=precision)
    p["bed"] = {"count": 4, "amin": 5, "amax": 8, "porosity": 0.6, "x0": 40}
    p["ignite"] = [8, 32, 1800.0]
    return p, I.config4_fields(p)


def test_fp64_implicit_two_step_chemistry():
    """Two-step six-species mechanism (reversible CO/CO2 step) integrated per
    cell by backward Euler + Newton on the GPU (pre-pass kernel) against the
    oracle's integrator, through ignition."""
    p, f = _two_step_case()
    got, ref, sc, ora = run_pair(p, f, 90, chunks=3)
    assert_fp64(got, ref, sc, ora)
    Y = ora.Y.reshape(6, -1)
    assert Y[2].max() > 1e-3  # CO was produced: both reactions are active


def test_fp32_transport_with_fp64_implicit_chemistry():
    p, f = _two_step_case(precision="fp32")
    got, ref, sc, ora = run_pair(p, f, 200, precision="fp32", chunks=2)
    assert l2rel(got["T"] - 300.0, ref["T"] - 300.0) <= 1e-4
    assert l2rel(got["Y"], ref["Y"]) <= 1e-4


# ---------------------------------------------- mixture-averaged transport
@pytest.mark.parametrize("kern", ["tiled", "persistent"])
def test_fp64_reactive_bed_mixture_transport(kern):
    """The reduced reactive bed with mixture-averaged viscosity and
    conductivity (Sec. 4.4, eqs. muT_mix, phi_mix, conduct_mix; species
    Sutherland laws, modified Eucken conductivities) through ignition: FP64
    max relative error <= 1e-10 against the oracle, and the flow differs from
    the single-gas run (the option is live)."""
    p = I.config2(nx=160, ny=48)
    p["bed"] = {"count": 6, "amin": 6, "amax": 10, "porosity": 0.6, "x0": 40}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    I.mixture_transport(p)
    f = I.config2_fields(p)
    O.set_threads(0)
    ora = O.OracleState(p, f["phi"], f["T"], f["Y"], f["Ts"])
    dom = Domain(p, "fp64")
    dom.set_phase_field(f["phi"], f["Ts"])
    dom.set_fields(f["T"], f["Y"])
    dom.select_kernel(kern)
    ora.step(200)
    dom.step(200)
    got = dom.get("T", "g", "u", "Y", "Ts")
    u, _, _ = ora.moments()
    ref = {"T": ora.T, "g": ora.g.reshape(9, -1), "u": u, "Y": ora.Y.reshape(5, -1), "Ts": ora.Ts}
    for k in ref:
        assert maxrel(got[k], ref[k]) <= FP64_TOL, k
    dom.close()
    q = dict(p)
    q.pop("transport")
    single = O.OracleState(q, f["phi"], f["T"], f["Y"], f["Ts"])
    single.step(200)
    assert maxrel(single.T, ora.T) > 1e-4


def test_3d_mixture_transport_march_fp64_and_fp32():
    """The 3-D crop with mixture transport: the z-march kernel in FP64 within
    1e-10 of the oracle after 20 steps, FP32 within 1e-4 (L2, u and T)."""
    p = I.config3_crop(32)
    I.mixture_transport(p)
    f = I.config3_fields(p)
    O.set_threads(0)
    ora = O.OracleState(p, f["phi"], f["T"], f["Y"], f["Ts"])
    ora.step(20)
    u, _, _ = ora.moments()
    for prec in ("fp64", "fp32"):
        dom = Domain(p, prec)
        dom.set_phase_field(f["phi"], f["Ts"])
        dom.set_fields(f["T"], f["Y"])
        dom.select_kernel("march")
        dom.step(20)
        got = dom.get("T", "u")
        dom.close()
        if prec == "fp64":
            assert maxrel(got["T"], ora.T) <= FP64_TOL and maxrel(got["u"], u) <= FP64_TOL
        else:
            assert l2rel(got["u"], u) <= 1e-4 and l2rel(got["T"] - 300.0, ora.T - 300.0) <= 1e-4


# ------------------------------------------------------ inlet feedback
@pytest.mark.parametrize("precision,kern", [("fp64", "tiled"), ("fp64", "persistent"),
                                            ("fp32", "tiled")])
def test_inlet_feedback_wall_bounded_flame(precision, kern):
    """2-D wall-bounded flame (isothermal walls, parabolic inlet, fresh
    mixture in the first quarter) with the inlet speed fed back from the CH4
    consumption of every step (Sec. 4.4.1), against the oracle: the inlet
    speed after each 250 steps and the fields after 1000 steps within 1e-10
    (FP64; FP32: 1e-4 L2 in the fields and 1e-4 in the inlet speed).  The
    feedback moves the inlet speed: it must not stay at its start value."""
    p = I.config6(nx=192, ny=64)
    f = I.config6_fields(p)
    ora = O.OracleState(p, f["phi"], f["T"], f["Y"])
    dom = Domain(p, precision)
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], f["Y"])
    dom.select_kernel(kern)
    assert dom.scalars()["u_in"] == pytest.approx(p["u_in"], rel=1e-15)
    tol = FP64_TOL if precision == "fp64" else 1e-4
    for _ in range(4):
        ora.step(250)
        dom.step(250)
        sc = dom.scalars()
        assert abs(sc["u_in"] / ora.u_in - 1) <= tol, (sc["u_in"], ora.u_in)
        assert abs(sc["fuel"] / ora.scal[10] - 1) <= tol
    assert abs(ora.u_in / p["u_in"] - 1) > 1e-3
    got = dom.get("T", "u", "Y")
    u, _, _ = ora.moments()
    ref = {"T": ora.T, "u": u, "Y": ora.Y.reshape(ora.K, ora.N)}
    for k in ref:
        if precision == "fp64":
            assert maxrel(got[k], ref[k]) <= FP64_TOL, k
        else:
            r = ref[k] - (p["T_in"] if k == "T" else 0.0)
            assert l2rel(got[k] - (p["T_in"] if k == "T" else 0.0), r) <= 1e-4, k
    dom.close()


def test_inlet_feedback_is_refused_where_unsupported():
    """A feedback species without an inlet face, or on a closed domain, is
    refused at set_mechanism."""
    from paper_2310_17214_gb300._native import PflbError
    p = I.config6(nx=64, ny=32)
    p["p0_mode"] = "closed"
    with pytest.raises(PflbError, match="feedback"):
        Domain(p, "fp64")


# ------------------------------------------------ characteristic outlet
@pytest.mark.parametrize("precision,kern", [("fp64", "tiled"), ("fp64", "persistent"),
                                            ("fp32", "tiled")])
def test_characteristic_outlet_diffuse_channel(precision, kern):
    """Diffuse-wall channel of Sec. 4.1 (eq. def-phi walls, fluid-fraction
    inlet, drag A_u) with the characteristic outlet, against the oracle after
    1200 steps (the start-up pressure wave has met the outlet): fields and the
    boundary pressure within 1e-10 (FP64).  FP32: 1e-4 L2 in u, and P_b within
    1e-5 lattice pressure units (3e-5 of the pressure scale rho cs^2; P_b
    integrates 1200 FP32 differences of the outlet columns)."""
    p = I.di_channel(L=20, eta=4, solid=4, H=100, A_u=145.0)
    f = I.di_channel_fields(p)
    ora = O.OracleState(p, f["phi"], f["T"])
    dom = Domain(p, precision)
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], None)
    dom.select_kernel(kern)
    for _ in range(4):
        ora.step(300)
        dom.step(300)
    pb_ref = ora.outlet_pressure[0]
    pb = dom.scalars()["outlet_pb"]
    assert pb_ref != 0.0
    got = dom.get("u", "g")
    u, _, _ = ora.moments()
    if precision == "fp64":
        assert abs(pb - pb_ref) <= FP64_TOL * abs(pb_ref)
        assert maxrel(got["u"], u) <= FP64_TOL
        assert maxrel(got["g"], ora.g.reshape(ora.Q, ora.N)) <= FP64_TOL
    else:
        assert abs(pb - pb_ref) <= 1e-5
        assert l2rel(got["u"], u) <= 1e-4
    dom.close()


def test_characteristic_outlet_3d_march_fp64():
    """The characteristic outlet on the 3-D z-march kernel: a wall-bounded
    3-D channel (ragged 37 x 12 x 10) against the oracle, 400 steps."""
    p = small_case(3, 37, 12, 10, bc=["inlet", "outlet", "wall", "wall", "wall", "wall"],
                   u_in=0.04, inlet_parabolic=1, outlet="nscbc", nu=0.05)
    N = 37 * 12 * 10
    f = {"phi": np.zeros(N), "T": np.full(N, 300.0), "Y": None, "Ts": None}
    ora = O.OracleState(p, f["phi"], f["T"])
    dom = Domain(p, "fp64")
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], None)
    dom.select_kernel("march")
    ora.step(400)
    dom.step(400)
    assert ora.outlet_pressure[0] != 0.0
    assert abs(dom.scalars()["outlet_pb"] / ora.outlet_pressure[0] - 1) <= FP64_TOL
    u, _, _ = ora.moments()
    assert maxrel(dom.get("u"), u) <= FP64_TOL
    dom.close()


# ------------------------------------------------ moving solid
def _moving_box(dim=2, ts_field=False):
    if dim == 2:
        nx, ny, nz = 96, 48, 1
        p = small_case(2, nx, ny, bc=["periodic"] * 6, nu=0.05)
        phi = I.disc_phi(nx, ny, 40.0, 24.0, 8.0, 4.0).reshape(-1)
        p["u_s"] = [-0.013, 0.007, 0.0]
    else:
        nx, ny, nz = 36, 24, 20
        p = small_case(3, nx, ny, nz, bc=["periodic"] * 6, nu=0.05)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r = np.sqrt((x - 18.0) ** 2 + (y - 12.0) ** 2 + (z - 10.0) ** 2)
        phi = (0.5 * (1.0 - np.tanh(2.0 * (r - 6.0) / 4.0))).reshape(-1)
        p["u_s"] = [0.011, -0.006, 0.004]
    p.update({"A_u": 145.0, "A_T": 70.0, "eta": 4.0, "Ts_uniform": 600.0})
    N = nx * ny * nz
    Ts = None
    if ts_field:
        # solid heat capacity and conductivity twice the air's (physical units)
        lam_air = p["mu_ref"] * p["cp0"] / p["Pr"]
        p.update({"Ts_field": 1, "rhocp_s": 2.0 * p["rho_ref"] * p["cp0"],
                  "lambda_s": 2.0 * lam_air})
        Ts = np.full(N, 600.0)
    T = (1.0 - phi) * 300.0 + phi * 600.0
    return p, {"phi": phi, "T": T, "Y": None, "Ts": Ts}


@pytest.mark.parametrize("precision,kern", [("fp64", "tiled"), ("fp64", "persistent"),
                                            ("fp32", "tiled")])
def test_moving_disc_against_oracle(precision, kern):
    """A heated disc translating at a fractional velocity through a periodic
    box of resting air (phase field displaced each step, drag on u - u_s,
    exchange with the moving solid), against the oracle after 300 steps:
    fields and the drag within 1e-10 (FP64; FP32 1e-4 L2)."""
    p, f = _moving_box()
    ora = O.OracleState(p, f["phi"], f["T"])
    dom = Domain(p, precision)
    dom.set_phase_field(f["phi"])
    dom.set_fields(f["T"], None)
    dom.select_kernel(kern)
    ora.step(300)
    dom.step(300)
    u, _, _ = ora.moments()
    got = dom.get("u", "T", "g")
    if precision == "fp64":
        assert maxrel(got["u"], u) <= FP64_TOL
        assert maxrel(got["T"], ora.T) <= FP64_TOL
        assert maxrel(got["g"], ora.g.reshape(ora.Q, ora.N)) <= FP64_TOL
        dg, do = dom.diagnostics(), ora.diagnostics()
        assert np.max(np.abs(dg["drag"] - do["drag"])) <= FP64_TOL * np.max(np.abs(do["drag"]))
    else:
        assert l2rel(got["u"], u) <= 1e-4
        assert l2rel(got["T"] - 300.0, ora.T - 300.0) <= 1e-4
    dom.close()


def test_moving_sphere_3d_march_with_solid_temperature():
    """3-D: a sphere moving obliquely, its transported solid temperature
    carried along, on the z-march kernel in FP64 against the oracle."""
    p, f = _moving_box(dim=3, ts_field=True)
    ora = O.OracleState(p, f["phi"], f["T"], Ts=f["Ts"])
    dom = Domain(p, "fp64")
    dom.set_phase_field(f["phi"], f["Ts"])
    dom.set_fields(f["T"], None)
    dom.select_kernel("march")
    ora.step(200)
    dom.step(200)
    u, _, _ = ora.moments()
    got = dom.get("u", "T", "Ts")
    assert maxrel(got["u"], u) <= FP64_TOL
    assert maxrel(got["T"], ora.T) <= FP64_TOL
    assert maxrel(got["Ts"], ora.Ts) <= FP64_TOL
    dom.close()


def test_moving_solid_state_restores_its_position():
    """A checkpoint of a moving-solid domain carries the step count: a
    domain restored from it continues with the phase field of that step,
    bit for bit like the domain that wrote it."""
    p, f = _moving_box()
    a = Domain(p, "fp64")
    a.set_phase_field(f["phi"])
    a.set_fields(f["T"], None)
    a.step(120)
    st = a.get_state()
    a.step(60)
    b = Domain(p, "fp64")
    b.set_phase_field(f["phi"])
    b.set_fields(f["T"], None)
    b.set_state(st)
    b.step(60)
    ga, gb = a.get("g", "T"), b.get("g", "T")
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    a.close()
    b.close()
