"""Host-side logic of the surrogate driver (no GPU): the element table, the
sample selection and the normalisation."""
import numpy as np

from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300 import surrogate as S


def test_element_matrix_annihilates_every_reaction():
    """Each reaction conserves every element: sum_k a_ek s_kj = 0.  A wrong
    atom count in the table breaks one of these sums."""
    elem, emass = I.element_matrix(I.SPECIES6)
    for r in I.two_step_mechanism():
        for e in range(4):
            assert abs(sum(a * s for a, s in zip(elem[e], r["stoich"]))) < 1e-12
    # element masses rebuild the species molar masses
    for k in range(6):
        assert abs(sum(elem[e][k] * emass[e] for e in range(4)) - I.M6[k]) < 1e-15


def test_residual_weights_vanish_on_reaction_increments():
    """dY_k = M_k s_kj xi is an exact reaction increment: its element
    residual sum_k a_ek M_e / M_k dY_k is zero."""
    elem, emass = I.element_matrix(I.SPECIES6)
    for r in I.two_step_mechanism():
        dY = np.array([m * s for m, s in zip(I.M6, r["stoich"])]) * 1e-4
        for e in range(4):
            res = sum(elem[e][k] * emass[e] / I.M6[k] * dY[k] for k in range(6))
            assert abs(res) < 1e-18


def test_selection_keeps_active_cells_and_a_uniform_rest():
    rng = np.random.default_rng(0)
    n = 10000
    dT = np.zeros(n)
    act = rng.choice(n, 300, replace=False)
    dT[act] = rng.uniform(0.5, 1.0, 300)
    fluid = np.ones(n, bool)
    fluid[:100] = False
    dY = np.zeros((6, n))
    sel = S.select_samples(dY, dT, fluid, rng, 1000, active_frac=0.5)
    assert len(sel) == 1000 and len(np.unique(sel)) == 1000
    assert np.all(fluid[sel])
    n_act = np.isin(sel, act[fluid[act]]).sum()
    assert n_act == min(500, fluid[act].sum())


def test_normalisation_round_trips_and_marks_constants():
    rng = np.random.default_rng(1)
    X = np.column_stack([rng.uniform(300, 2200, 500), rng.uniform(0, 0.2, (500, 6)),
                         np.full(500, 101325.0)])
    theta = 12000.0
    # increments shaped like Arrhenius rates: exp(-theta / T) times O(1e-2)
    D = np.exp(-theta / X[:, :1]) * rng.normal(0, 1e-2, (500, 6))
    D[:, 5] = 0.0
    (xm, xs, ym, ys), Xn, Yn = S.normalisation(X, D, theta)
    assert xs[7] == 0.0 and np.all(Xn[:, 7] == 0.0)
    assert ys[5] == 0.0 and ym[5] == 0.0
    rebuilt = np.exp(-theta / X[:, 0])[:, None] * (ym + ys * Yn.astype(np.float64))
    assert np.max(np.abs(rebuilt - D)) <= 1e-6 * np.max(np.abs(D))
    assert np.allclose(Xn[:, :7].mean(axis=0), 0, atol=1e-5)


def test_surrogate_record_layout():
    p = I.config4(nx=64, ny=32)
    X = np.array([[300.0] + list(p["Y_in"]) + [p["P0"]], [2000.0] + list(p["Y_in"]) + [p["P0"]]])
    stats = (X.mean(0), X.std(0), np.zeros(6), np.ones(6))
    s = S.make_surrogate(stats, X, 12000.0, p["species"], 1e-6)
    assert s.n_elem == 4 and s.tol == 1e-6 and s.theta_s == 12000.0
    assert s.lo[0] == 300.0 - 17.0 and s.hi[0] == 2000.0 + 17.0
    assert s.lo[7] < p["P0"] < s.hi[7] and s.hi[7] - s.lo[7] < 1e-5 * p["P0"]
    assert s.elem[1][0] == 4.0 and s.elem[3][5] == 2.0


def test_adiabatic_temperature_closes_the_energy_balance():
    """Complete combustion at constant c_p: sum_k hf_k (Yb - Yin) + cp_b
    (T_ad - T_in) = 0, and the lean mixture has O2 left and no CH4."""
    p = I.config4(nx=64, ny=32)
    Tad = S.adiabatic_temperature(p)
    Yin = np.array(p["Y_in"])
    Yb = np.array(I.burnt_composition(list(Yin), p["species"], p["M"]))
    assert Yb[0] == 0.0 and Yb[1] > 0.0
    assert abs(np.sum(np.array(p["hf"]) * (Yb - Yin)) +
               np.sum(np.array(p["cp"]) * Yb) * (Tad - p["T_in"])) < 1e-6
    assert 1700.0 < Tad < 1950.0


def test_front_positions_interpolate_a_linear_ramp_exactly():
    nx = 50
    x = np.arange(nx, dtype=float)
    T = np.tile(np.clip(300.0 + 100.0 * (x - 10.0), 300.0, 2300.0), (3, 1))
    T = np.minimum(T, np.tile(np.clip(300.0 + 100.0 * (40.0 - x), 300.0, 2300.0), (3, 1)))
    f = S.front_positions(T, 1050.0)
    assert np.allclose(f[:, 0], 17.5) and np.allclose(f[:, 1], 32.5)


def test_flame_errors_see_a_shift_of_a_third_of_a_cell():
    p = I.config4(nx=64, ny=4)
    x = np.arange(64, dtype=float)
    ref = np.tile(300.0 + 1500.0 / (1.0 + np.exp((x - 30.0) / 2.0)), (4, 1)).reshape(-1)
    test = np.tile(300.0 + 1500.0 / (1.0 + np.exp((x - 30.0 - 1.0 / 3.0) / 2.0)), (4, 1)).reshape(-1)
    e = S.flame_errors(test, ref, np.zeros(64 * 4), p)
    assert abs(e["front_max_diff_cells"] - 1.0 / 3.0) < 0.02
    assert e["rows_with_front"] == 4 and e["rows_front_mismatch"] == 0


def _record(y_mean, y_std, theta_s, skip_eps):
    X = np.array([[300.0] + [0.1] * 6 + [1e5], [2000.0] + [0.2] * 6 + [1e5]])
    stats = (X.mean(axis=0), X.std(axis=0), np.asarray(y_mean), np.asarray(y_std))
    return S.make_surrogate(stats, X, theta_s, I.SPECIES6, 1e-6, skip_eps=skip_eps)


def test_skip_temperature_meets_its_bound():
    """T_skip of the cold-tile option: with an output layer of constant
    weights w (|tanh| <= 1 bounds each output by 64 |w| (1 + 2^-7) + |b|),
    the projected increment exp(-theta_s / T) ||P||_inf max_k(|ybar_k| +
    s_k max|out_k|) equals skip_eps at T = T_skip.  ||P||_inf is taken here
    from an orthonormal basis of the element-conserving subspace (an
    independent route to the same projection)."""
    import scipy.linalg as sl
    theta = np.zeros(9286, dtype=np.float32)
    theta[-6 - 384:-6] = 0.01
    theta[-6:] = [0.0, 0.1, -0.2, 0.0, 0.05, 0.0]
    y_mean = [0.0, 1e-3, 0.0, -2e-3, 0.0, 0.0]
    y_std = [1.0, 0.5, 2.0, 1.0, 1.0, 0.0]
    rec = _record(y_mean, y_std, 12000.0, 1e-12)
    T_skip = S.skip_temperature(theta, rec, I.M6)
    elem, _ = I.element_matrix(I.SPECIES6)
    B = np.array(elem) / np.asarray(I.M6)[None, :]
    Nb = sl.null_space(B)
    P = Nb @ Nb.T
    out = 64 * float(np.float32(0.01)) * 1.0078125 + np.abs(theta[-6:].astype(np.float64))
    bound = np.max(np.abs(y_mean) + np.asarray(y_std) * out) * np.abs(P).sum(axis=1).max()
    assert T_skip > 0
    assert abs(np.exp(-12000.0 / T_skip) * bound / 1e-12 - 1.0) < 1e-9
    # colder cells are below the bound, hotter ones above it
    assert np.exp(-12000.0 / (0.99 * T_skip)) * bound < 1e-12 < np.exp(-12000.0 / (1.01 * T_skip)) * bound


def test_skip_temperature_edge_cases():
    """No skipping without skip_eps; every temperature skips when the
    network's bound is already below skip_eps."""
    theta = np.zeros(9286, dtype=np.float32)
    assert S.skip_temperature(theta, _record([0.0] * 6, [1.0] * 6, 12000.0, 0.0), I.M6) == 0.0
    assert S.skip_temperature(theta, _record([0.0] * 6, [0.0] * 6, 12000.0, 1e-12),
                              I.M6) == float("inf")
