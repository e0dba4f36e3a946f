"""The surrogate network's kernels (forward, backward, Adam) against the FP64
reference MLP, and the surrogate chemistry mode against the Newton
integrator it falls back to.

Bars: forward and per-tensor gradients within 2e-2 relative of the FP64
reference evaluated at the BF16-rounded parameters (BF16 operands, FP32
accumulation); the first Adam step moves each parameter by -lr sign(g)
exactly where the gradient is clearly non-zero; a surrogate that rejects
every cell reproduces the Newton chemistry bit for bit in FP64 and to the
FP32 resolution of the fields in FP32 (where the fallback has its own FP32
integrator, checked cell by cell against the oracle); a surrogate whose
network predicts no change reproduces the run without chemistry."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300 import surrogate as S
from paper_2310_17214_gb300._native import Domain, Mlp, MLP_PARAMS, PflbError

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def l2rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def tensors(flat):
    """Per-tensor slices (W1, b1, ..., W4, b4) of a flat parameter vector."""
    out, o = [], 0
    for a, b in zip(M.DIMS[:-1], M.DIMS[1:]):
        out += [flat[o:o + a * b], flat[o + a * b:o + a * b + b]]
        o += a * b + b
    return out


def case(n, seed):
    rng = np.random.default_rng(seed)
    theta = (M.init(seed) + rng.normal(0, 0.02, M.n_params())).astype(np.float32)
    X = rng.normal(0, 1, (n, 8)).astype(np.float32)
    Y = (np.tanh(X[:, :6] * 0.8) + 0.2 * X[:, 2:8]).astype(np.float32)
    return theta, X, Y


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 16, 1000, 4133])
def test_mlp_forward_matches_reference(n):
    theta, X, _ = case(n, 1)
    net = Mlp()
    net.set_params(theta)
    got = net.forward(dev(X)).cpu().numpy().astype(np.float64)
    ref, _ = M.forward(bf16_round(theta), bf16_round(X))
    assert np.max(np.abs(got - ref)) <= 2e-2 * np.max(np.abs(ref))
    assert np.array_equal(net.get_params(), theta)
    net.close()


@pytest.mark.parametrize("n", [37, 4096, 20011])
def test_mlp_gradient_matches_reference(n):
    theta, X, Y = case(n, 2)
    net = Mlp()
    net.set_params(theta)
    loss, g = net.gradient(dev(X), dev(Y))
    Lr, gr = M.gradient(bf16_round(theta), bf16_round(X), Y.astype(np.float64))
    assert abs(loss - Lr) <= 1e-2 * Lr
    for t, (a, b) in enumerate(zip(tensors(g.astype(np.float64)), tensors(gr))):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 2e-2, (t, rel)
    net.close()


def test_first_adam_step_moves_by_signed_learning_rate():
    """Adam's first bias-corrected step is lr g / (|g| + eps): -lr sign(g)
    wherever |g| is well above eps and the BF16 gradient has the sign of the
    FP64 one."""
    theta, X, Y = case(2048, 3)
    lr = 1e-3
    net = Mlp()
    net.set_params(theta)
    net.train(dev(X), dev(Y), batch=2048, steps=1, lr=lr)
    step = net.get_params().astype(np.float64) - theta.astype(np.float64)
    _, gr = M.gradient(bf16_round(theta), bf16_round(X), Y.astype(np.float64))
    for a, b in zip(tensors(step), tensors(gr)):
        clear = np.abs(b) > 0.2 * np.max(np.abs(b))
        assert clear.sum() > 0
        assert np.allclose(a[clear], -lr * np.sign(b[clear]), rtol=1e-3, atol=0)
    net.close()


def test_adam_steps_match_reference():
    """Four library Adam steps on one fixed batch against the FP64 reference
    Adam fed, at each step, the FP64 gradient at the BF16-rounded parameters:
    this checks the second moment and the bias corrections of steps 2-4, not
    only the first step.  Parameters whose gradient is clearly non-zero move
    as the reference says to 1e-2; every tensor's displacement within 5e-2."""
    theta, X, Y = case(2048, 8)
    lr = 1e-3
    net = Mlp()
    net.set_params(theta)
    net.train(dev(X), dev(Y), batch=2048, steps=4, lr=lr)
    got = net.get_params().astype(np.float64) - theta.astype(np.float64)
    net.close()
    th = theta.astype(np.float64)
    m, v = np.zeros_like(th), np.zeros_like(th)
    g0 = None
    for t in range(1, 5):
        _, g = M.gradient(bf16_round(th.astype(np.float32)), bf16_round(X), Y.astype(np.float64))
        g0 = g if g0 is None else g0
        th, m, v = M.adam(th, g, m, v, t, lr)
    ref = th - theta.astype(np.float64)
    for t, (a, b, gg) in enumerate(zip(tensors(got), tensors(ref), tensors(g0))):
        clear = np.abs(gg) > 0.2 * np.max(np.abs(gg))
        assert clear.sum() > 0
        assert np.allclose(a[clear], b[clear], rtol=1e-2, atol=0), t
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b), t


def test_training_reduces_the_loss():
    theta, X, Y = case(65536, 4)
    net = Mlp()
    net.set_params(M.init(5).astype(np.float32))
    Xd, Yd = dev(X), dev(Y)
    L0, _ = net.gradient(Xd, Yd)
    net.train(Xd, Yd, batch=4096, steps=400, lr=3e-3)
    L1, _ = net.gradient(Xd, Yd)
    assert L1 < 0.1 * L0
    # the trained network's loss agrees with the reference at its own parameters
    Lr = M.loss(bf16_round(net.get_params()), bf16_round(X), Y.astype(np.float64))
    assert abs(L1 - Lr) <= 0.05 * Lr
    net.close()


# --------------------------------------------------- surrogate chemistry mode
def _flame_case(nx=128, ny=40, chem="implicit", precision="fp32"):
    p = I.config4(nx=nx, ny=ny, precision=precision, chem=chem)
    p["bed"] = {"count": 4, "amin": 5, "amax": 8, "porosity": 0.6, "x0": nx // 2}
    p["ignite"] = [8, 40, 1800.0]
    return p, I.config4_fields(p)


def _domain(p, f, precision):
    d = Domain(p, precision)
    d.set_phase_field(f["phi"], f["Ts"])
    d.set_fields(f["T"], f["Y"])
    return d


def _surrogate_record(p, theta_s=0.0, tol=1e-6):
    X = np.array([[300.0] + list(p["Y_in"]) + [p["P0"]]] * 2)
    X[1, 0] = 2500.0
    stats = (X.mean(axis=0), X.std(axis=0), np.zeros(6), np.zeros(6))
    s = S.make_surrogate(stats, X, theta_s, p["species"], tol)
    return s


def _all_fallback(p, f, precision):
    """A surrogate-mode domain whose network is rejected in every fluid cell
    (tolerance -1): every cell goes through the fallback integrator."""
    dom = _domain(dict(p, chem="surrogate"), f, precision)
    net = Mlp()
    net.set_params(np.zeros(MLP_PARAMS, dtype=np.float32))
    dom.set_surrogate(net, _surrogate_record(p, tol=-1.0))
    return dom, net


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_surrogate_rejecting_every_cell_equals_newton(precision):
    """Tolerance -1 sends every fluid cell through the fallback list.  FP64:
    the fallback is the Newton pre-pass's integrator and the run is the Newton
    run bit for bit.  FP32: the fallback integrator is the FP32 one (increment
    form, stopped at a few units in the last place of the field), the Newton
    pre-pass keeps the FP64 residual; after 60 steps through ignition the two
    runs agree to the FP32 resolution of the fields."""
    p, f = _flame_case(precision=precision)
    ref = _domain(p, f, precision)
    ref.step(60)
    a = ref.get("T", "Y", "g")
    dom, net = _all_fallback(p, f, precision)
    dom.step(60)
    b = dom.get("T", "Y", "g")
    if precision == "fp64":
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    else:
        dT = np.abs(a["T"] - b["T"])
        dYm = np.abs(a["Y"] - b["Y"])
        print("fp32 fallback vs Newton run: max dT", dT.max(), "max dY", dYm.max(),
              "L2 T", l2rel(b["T"] - 300.0, a["T"] - 300.0))
        assert np.max(a["T"]) > 1500.0
        assert l2rel(b["T"] - 300.0, a["T"] - 300.0) <= 1e-5
        assert dT.max() <= 0.05 and dYm.max() <= 2e-5
    fb, ev = dom.chem_stats()
    assert ev > 0 and fb == ev
    dom.close()
    ref.close()
    net.close()


def test_fp32_fallback_integrator_matches_one_step():
    """The FP32 fallback integrator against the oracle's FP64 backward-Euler
    step, cell by cell, on an FP32 state after ignition: the increment form
    holds the increments to 1e-4 of themselves or a few units in the last
    place of the field they are added to."""
    from oracle import oracle as O
    p, f = _flame_case(nx=96, ny=24, precision="fp32")
    dom, net = _all_fallback(p, f, "fp32")
    dom.step(5)
    dY, dT = dom.chem_increments()
    g = dom.get("T", "Y")
    P0 = dom.scalars()["P0"]
    rng = np.random.default_rng(0)
    fluid = np.flatnonzero(1.0 - f["phi"] >= 1e-6)
    cells = np.concatenate([rng.choice(fluid, 40, replace=False),
                            fluid[np.argsort(-np.abs(dT[fluid]))[:20]]])
    assert np.max(np.abs(dT[cells])) > 0.1  # reacting cells are in the sample
    eT, eY = 0.0, 0.0
    for c in cells:
        T, Y = float(g["T"][c]), g["Y"][:, c].astype(np.float64)
        rho_lat = P0 / (I.R_GAS * T * np.sum(Y / np.asarray(p["M"]))) / p["rho_ref"]
        ry, rt, rc = O.chem_implicit(p, T, Y, rho_lat)
        assert rc == 0
        eT = max(eT, abs(dT[c] - rt) / (1e-4 * abs(rt) + 4e-6 * T))
        eY = max(eY, np.max(np.abs(dY[:, c] - ry) / (1e-4 * np.abs(ry) + 4e-6 * np.abs(Y) + 1e-12)))
    print("fp32 fallback vs oracle, error / bar: T", eT, "Y", eY)
    assert eT <= 1.0 and eY <= 1.0
    dom.close()
    net.close()


def test_surrogate_predicting_no_change_equals_no_chemistry():
    p, f = _flame_case(precision="fp64")
    ref = _domain(dict(p, chem="none"), f, "fp64")
    ref.step(40)
    a = ref.get("T", "Y", "u")
    dom = _domain(dict(p, chem="surrogate"), f, "fp64")
    net = Mlp()
    net.set_params(np.zeros(MLP_PARAMS, dtype=np.float32))
    rec = _surrogate_record(p)
    rec.lo[0], rec.hi[0] = 0.0, 1e4
    for k in range(1, 7):
        rec.lo[k], rec.hi[k] = -1.0, 2.0
    dom.set_surrogate(net, rec)
    dom.step(40)
    b = dom.get("T", "Y", "u")
    for k in a:
        assert np.max(np.abs(a[k] - b[k])) <= 1e-13 * max(np.max(np.abs(a[k])), 1.0), k
    fb, ev = dom.chem_stats()
    assert fb == 0 and ev > 0
    dom.close()
    ref.close()
    net.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cold_skip_is_exact_for_a_network_that_predicts_no_change(precision):
    """skip_eps > 0 with a network whose output bound is zero: every tile
    skips the network (T_skip is infinite), and the run equals the run that
    evaluates the network everywhere bit for bit, with the same counts (the
    cells outside the narrow training box still fall back)."""
    p, f = _flame_case(precision=precision)
    runs = []
    for eps in (0.0, 1e-12):
        dom = _domain(dict(p, chem="surrogate"), f, precision)
        net = Mlp()
        net.set_params(np.zeros(MLP_PARAMS, dtype=np.float32))
        rec = _surrogate_record(p, theta_s=12000.0)
        rec.skip_eps = eps
        dom.set_surrogate(net, rec)
        dom.step(40)
        runs.append((dom.get("T", "Y", "g"), dom.chem_stats()))
        dom.close()
        net.close()
    (a, sa), (b, sb) = runs
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert sa == sb and sa[0] > 0 and sa[1] > sa[0]


def test_cold_skip_arguments():
    """A negative or NaN skip_eps, or skip_eps without the temperature
    scaling (theta_s = 0), is refused."""
    p, f = _flame_case(precision="fp32")
    dom = _domain(dict(p, chem="surrogate"), f, "fp32")
    net = Mlp()
    net.set_params(np.zeros(MLP_PARAMS, dtype=np.float32))
    for theta_s, eps in ((12000.0, -1.0), (12000.0, float("nan")), (0.0, 1e-12)):
        rec = _surrogate_record(p, theta_s=theta_s)
        rec.skip_eps = eps
        with pytest.raises(PflbError):
            dom.set_surrogate(net, rec)
    dom.close()
    net.close()


def test_chem_increments_of_newton_mode_match_one_step():
    """pflb_chem_increments in the Newton mode against the oracle's
    backward-Euler integrator, cell by cell, on a state after ignition."""
    from oracle import oracle as O
    p, f = _flame_case(nx=96, ny=24, precision="fp64")
    dom = _domain(p, f, "fp64")
    dom.step(5)
    dY, dT = dom.chem_increments()
    g = dom.get("T", "Y")
    P0 = dom.scalars()["P0"]
    rng = np.random.default_rng(0)
    fluid = np.flatnonzero(1.0 - f["phi"] >= 1e-6)
    cells = np.concatenate([rng.choice(fluid, 40, replace=False),
                            fluid[np.argsort(-np.abs(dT[fluid]))[:20]]])
    for c in cells:
        T, Y = g["T"][c], g["Y"][:, c]
        rho_lat = P0 / (I.R_GAS * T * np.sum(Y / np.asarray(p["M"]))) / p["rho_ref"]
        ry, rt, rc = O.chem_implicit(p, T, Y, rho_lat)
        assert rc == 0
        assert abs(dT[c] - rt) <= 1e-9 * max(abs(rt), 1e-3)
        assert np.max(np.abs(dY[:, c] - ry)) <= 1e-9 * max(np.max(np.abs(ry)), 1e-12)
    dom.close()


def _ms_per_step(dom, steps=40):
    dom.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    dom.step(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def test_trained_surrogate_tracks_the_flame_and_beats_newton():
    """What the trained network gains: on a 1024 x 256 two-step bed, a network
    trained by the library's kernels on samples of the Newton run reproduces
    that run after 2000 steps (flame front within one cell, temperature
    within 20 K over fluid cells), with few fallback cells, and its
    chemistry step is several times faster than the Newton step."""
    p = I.config4(nx=1024, ny=256, precision="fp32")
    f = I.config4_fields(p)
    steps = 2000
    ref = _domain(p, f, "fp32")
    X, D = S.collect(ref, f["phi"], 400_000, 8, steps // 8, seed=1)
    ref.step(steps - 7 * (steps // 8))
    theta = S.theta_scale(p)
    stats, Xn, Yn = S.normalisation(X, D, theta)
    net, loss = S.train(Xn, Yn, epochs=40, batch=8192, seed=1)
    assert loss < 1e-3
    sur = _domain(dict(p, chem="surrogate"), f, "fp32")
    sur.set_surrogate(net, S.make_surrogate(stats, X, theta, p["species"], 1e-6))
    sur.step(steps)
    Ta, Tb = sur.get("T"), ref.get("T")
    err = S.flame_errors(Ta, Tb, f["phi"], p)
    assert err["rows_with_front"] > 200 and err["rows_front_mismatch"] == 0
    assert err["front_max_diff_cells"] <= 1.0
    assert err["T_max_abs_diff_K"] <= 20.0
    fb, ev = sur.chem_stats()
    assert fb / ev < 0.02
    # cold tiles skipping the network (increment bound 1e-12 per step): the
    # same flame against the Newton run, and next to the full evaluation
    sk = _domain(dict(p, chem="surrogate"), f, "fp32")
    sk.set_surrogate(net, S.make_surrogate(stats, X, theta, p["species"], 1e-6,
                                           skip_eps=1e-12))
    sk.step(steps)
    Tk = sk.get("T")
    err_k = S.flame_errors(Tk, Tb, f["phi"], p)
    assert err_k["rows_front_mismatch"] == 0 and err_k["front_max_diff_cells"] <= 1.0
    assert err_k["T_max_abs_diff_K"] <= 20.0
    err_ks = S.flame_errors(Tk, Ta, f["phi"], p)
    print("cold skip vs full evaluation:", err_ks)
    assert err_ks["front_max_diff_cells"] <= 0.1 and err_ks["T_max_abs_diff_K"] <= 1.0
    t_newton, t_sur = _ms_per_step(ref), _ms_per_step(sur)
    assert t_sur * 3.0 < t_newton, (t_sur, t_newton)
    sk.close()
    sur.close()
    ref.close()
    net.close()


def _raw_inputs(dom, p):
    g = dom.get("T", "Y")
    P0 = dom.scalars()["P0"]
    N = g["T"].size
    return np.column_stack([g["T"], g["Y"].T, np.full(N, P0)])


def test_network_engines_match_the_reference_mlp():
    """The surrogate's network on tcgen05 (tensor-memory accumulators, 128
    cells per MMA) and on warp-level mma.sync, through the chemistry
    increments of a domain whose record accepts every cell unchanged
    (no element test or projection, unit output scale): each engine within
    2e-2 of the FP64 reference MLP at the BF16-rounded parameters and
    inputs (the forward bar), and the two engines within 2e-3 of each
    other (same BF16 operands, FP32 accumulation in a different order)."""
    from paper_2310_17214_gb300._native import MLP_ENGINES
    p, f = _flame_case(nx=200, ny=40, chem="surrogate", precision="fp32")
    theta, _, _ = case(1, 3)
    net = Mlp()
    net.set_params(theta)
    dom = _domain(p, f, "fp32")
    rec = _surrogate_record(p, tol=-1.0)
    dom.set_surrogate(net, rec)
    dom.step(20)  # every cell by Newton: a state through ignition
    X = _raw_inputs(dom, p)
    fluid = np.flatnonzero(1.0 - f["phi"] >= 1e-6)
    mean, std = X[fluid].mean(axis=0), X[fluid].std(axis=0)
    std[std == 0] = 1.0
    out = {}
    for name in ("tcgen05", "warp_mma"):
        r = _surrogate_record(p)
        for k in range(8):
            r.x_mean[k], r.x_std[k] = mean[k], std[k]
            r.lo[k], r.hi[k] = -1e30, 1e30
        for k in range(6):
            r.y_mean[k], r.y_std[k] = 0.0, 1.0
        r.theta_s, r.n_elem, r.tol = 0.0, 0, 1e30
        r.engine = MLP_ENGINES[name]
        dom.set_surrogate(net, r)
        dY, _ = dom.chem_increments()
        out[name] = dY[:, fluid]
    xn = (X[fluid] - mean) / std
    ref, _ = M.forward(bf16_round(theta), bf16_round(xn.astype(np.float32)))
    ref = ref[:, :6].T
    scale = np.max(np.abs(ref))
    for name, got in out.items():
        assert np.max(np.abs(got - ref)) <= 2e-2 * scale, name
    assert np.max(np.abs(out["tcgen05"] - out["warp_mma"])) <= 2e-3 * scale
    dom.close()
    net.close()
