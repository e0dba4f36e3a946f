"""Training driver of the learned chemistry surrogate.

Pipeline: a plain run (backward-Euler Newton chemistry) provides samples of
(T, Y_1..Y_6, P0) and the increments dY_k over one step; the network
8 -> 64 -> 64 -> 64 -> 6 is trained on them by the library's own forward,
backward and Adam kernels (BF16 tensor cores, FP32 master weights); the
trained network is then attached to domains in surrogate chemistry mode,
where cells outside the training bounding box or with an element residual
above the tolerance fall back to the Newton integrator.

Targets are scaled by the Arrhenius factor exp(-theta_s / T), theta_s the
smallest activation temperature of the mechanism, so that the network fits
a smooth function of the composition and the change in cold gas vanishes
with the true one.  Sample selection and normalisation statistics are host
bookkeeping; every per-cell evaluation runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import _native as N


def theta_scale(prob) -> float:
    """Smallest activation temperature E_a/R of the mechanism's reactions."""
    return float(min(r["EaR"] for r in prob["reactions"]))


def select_samples(dY, dT, fluid, rng, n_keep, active_frac=0.5, rel=1e-3):
    """Indices of the cells to keep from one snapshot: cells whose |dT| is
    above `rel` times the snapshot's largest form `active_frac` of the draw,
    the rest is drawn uniformly from the other fluid cells."""
    idx = np.flatnonzero(fluid)
    if idx.size == 0 or n_keep <= 0:
        return idx[:0]
    a = np.abs(dT[idx])
    amax = a.max()
    act = idx[a > rel * amax] if amax > 0 else idx[:0]
    rest = np.setdiff1d(idx, act, assume_unique=True)
    n_act = min(act.size, int(round(n_keep * active_frac)))
    n_rest = min(rest.size, n_keep - n_act)
    pick = [rng.choice(act, n_act, replace=False) if n_act else act[:0],
            rng.choice(rest, n_rest, replace=False) if n_rest else rest[:0]]
    return np.concatenate(pick)


def collect(dom, phi, n_samples, snapshots, steps_between, seed=0, phi_min=1e-6):
    """Advance `dom` (implicit chemistry) and gather about `n_samples` rows of
    raw inputs X = (T, Y_1..Y_6, P0) and targets dY (one step) over
    `snapshots` snapshots `steps_between` steps apart."""
    rng = np.random.default_rng(seed)
    fluid = (1.0 - np.asarray(phi).reshape(-1)) >= phi_min
    per = max(1, n_samples // snapshots)
    Xs, Ds = [], []
    for s in range(snapshots):
        if s:
            dom.step(steps_between)
        dY, dT = dom.chem_increments()
        f = dom.get("T", "Y")
        P0 = dom.scalars()["P0"]
        sel = select_samples(dY, dT, fluid, rng, per)
        X = np.empty((sel.size, 8))
        X[:, 0] = f["T"][sel]
        X[:, 1:7] = f["Y"][:, sel].T
        X[:, 7] = P0
        Xs.append(X)
        Ds.append(dY[:, sel].T.copy())
    return np.concatenate(Xs), np.concatenate(Ds)


def normalisation(X, D, theta_s):
    """Input/output mean and std (std 0 where a column is constant: the
    feature is ignored, or the output is that constant) and the scaled,
    normalised training arrays."""
    x_mean, x_std = X.mean(axis=0), X.std(axis=0)
    x_std[x_std < 1e-12 * np.maximum(np.abs(x_mean), 1e-300)] = 0.0
    scale = np.exp(-theta_s / X[:, 0]) if theta_s > 0 else np.ones(len(X))
    Z = D / scale[:, None]
    y_mean, y_std = Z.mean(axis=0), Z.std(axis=0)
    const = np.all(D == 0.0, axis=0)
    y_mean[const], y_std[const] = 0.0, 0.0
    xs = np.where(x_std > 0, x_std, 1.0)
    ys = np.where(y_std > 0, y_std, 1.0)
    Xn = np.where(x_std > 0, (X - x_mean) / xs, 0.0)
    Yn = np.where(y_std > 0, (Z - y_mean) / ys, 0.0)
    return (x_mean, x_std, y_mean, y_std), Xn.astype(np.float32), Yn.astype(np.float32)


def make_surrogate(stats, X, theta_s, species, tol=1e-6, pad=0.01, skip_eps=0.0):
    """The pflb_surrogate record: normalisation, bounding box of the raw
    training inputs, element matrix and residual tolerance.  The box is
    widened by `pad` times each feature's range (1e-6 of the value for a
    constant feature): the fresh and the burnt gas, where most cells sit,
    are corners of the box, and round-off would otherwise put them just
    outside it.  skip_eps > 0 lets tiles of cold cells skip the network
    where its increment is bounded by skip_eps (pflb_surrogate.skip_eps)."""
    from .inputs import element_matrix
    x_mean, x_std, y_mean, y_std = stats
    s = N.Surrogate()
    lo, hi = X.min(axis=0), X.max(axis=0)
    width = np.where(hi > lo, pad * (hi - lo), 1e-6 * np.abs(hi))
    lo, hi = lo - width, hi + width
    for f in range(8):
        s.x_mean[f], s.x_std[f] = x_mean[f], x_std[f]
        s.lo[f], s.hi[f] = lo[f], hi[f]
    for k in range(6):
        s.y_mean[k], s.y_std[k] = y_mean[k], y_std[k]
    s.theta_s = theta_s
    elem, emass = element_matrix(species)
    s.n_elem = len(elem)
    for e in range(len(elem)):
        s.elem_mass[e] = emass[e]
        for k in range(len(species)):
            s.elem[e][k] = elem[e][k]
    s.tol = tol
    s.skip_eps = skip_eps
    return s


def skip_temperature(theta, rec, M):
    """T_skip of a record with skip_eps > 0 for the network parameters theta
    (flat FP32 vector) and molar masses M: the bound the library derives in
    pflb_set_surrogate, restated here for reports."""
    eps = float(rec.skip_eps)
    if not eps > 0.0:
        return 0.0
    th = np.asarray(theta, dtype=np.float64)
    b4, W4 = th[-6:], th[-6 - 64 * 6:-6].reshape(64, 6)
    out = np.abs(b4) + 1.0078125 * np.abs(W4).sum(axis=0)
    bound = max(abs(rec.y_mean[k]) + abs(rec.y_std[k]) * out[k] for k in range(6))
    B = np.array([[rec.elem[e][k] / M[k] for k in range(6)] for e in range(rec.n_elem)])
    Pj = np.eye(6) - B.T @ np.linalg.solve(B @ B.T, B) if rec.n_elem else np.eye(6)
    bound *= np.abs(Pj).sum(axis=1).max()
    return rec.theta_s / np.log(bound / eps) if bound > eps else float("inf")


def glorot(seed):
    """Seeded Glorot-uniform weights and zero biases in the flat order."""
    rng = np.random.default_rng(seed)
    dims = [8, 64, 64, 64, 6]
    parts = []
    for a, b in zip(dims[:-1], dims[1:]):
        lim = np.sqrt(6.0 / (a + b))
        parts += [rng.uniform(-lim, lim, a * b), np.zeros(b)]
    return np.concatenate(parts).astype(np.float32)


def train(Xn, Yn, device=0, epochs=20, batch=8192, lr=(3e-3, 1e-4), seed=0, net=None,
          log=None):
    """Train a network on the normalised arrays with the library's kernels;
    a fresh permutation per epoch, learning rate decayed geometrically from
    lr[0] to lr[1].  Returns (network, last mini-batch loss)."""
    import torch
    rng = np.random.default_rng(seed)
    if net is None:
        net = N.Mlp(device)
        net.set_params(glorot(seed))
    n = len(Xn)
    nb = max(1, (n + batch - 1) // batch)
    dev = torch.device("cuda", device)
    Xd = torch.empty((n, 8), dtype=torch.float32, device=dev)
    Yd = torch.empty((n, 6), dtype=torch.float32, device=dev)
    loss = float("nan")
    for ep in range(epochs):
        perm = rng.permutation(n)
        Xd.copy_(torch.from_numpy(np.ascontiguousarray(Xn[perm])))
        Yd.copy_(torch.from_numpy(np.ascontiguousarray(Yn[perm])))
        a = lr[0] * (lr[1] / lr[0]) ** (ep / max(1, epochs - 1))
        loss = net.train(Xd, Yd, batch, nb, a)
        if log:
            log(ep, a, loss)
    return net, loss


def build(prob, dom, phi, n_samples=1_000_000, snapshots=8, steps_between=100, epochs=20,
          batch=8192, tol=1e-6, seed=0, device=0, log=None):
    """Sample a plain run in `dom`, train, and return (network, pflb_surrogate,
    report dict)."""
    theta_s = theta_scale(prob)
    X, D = collect(dom, phi, n_samples, snapshots, steps_between, seed=seed)
    stats, Xn, Yn = normalisation(X, D, theta_s)
    net, loss = train(Xn, Yn, device=device, epochs=epochs, batch=batch, seed=seed, log=log)
    surr = make_surrogate(stats, X, theta_s, prob["species"], tol)
    return net, surr, {"samples": len(X), "loss": loss, "theta_s": theta_s}


# ------------------------------------------------------------ error measures
def adiabatic_temperature(prob) -> float:
    """T_in plus the heat of complete combustion of the inlet mixture over
    the burnt mixture's heat capacity (constant c_p,k)."""
    from .inputs import burnt_composition
    Yin = np.asarray(prob["Y_in"])
    Yb = np.asarray(burnt_composition(list(Yin), prob["species"], prob["M"]))
    hf, cp = np.asarray(prob["hf"]), np.asarray(prob["cp"])
    return float(prob["T_in"] - np.sum(hf * (Yb - Yin)) / np.sum(cp * Yb))


def front_positions(T, level):
    """Per row of a [ny, nx] temperature field, the first and the last x
    where T crosses `level`, linearly interpolated (NaN where it does not)."""
    ny, nx = T.shape
    out = np.full((ny, 2), np.nan)
    for r in range(ny):
        hot = np.flatnonzero(T[r] >= level)
        if hot.size == 0:
            continue
        x0, x1 = hot.min(), hot.max()
        if x0 > 0:
            out[r, 0] = x0 - (T[r, x0] - level) / (T[r, x0] - T[r, x0 - 1])
        if x1 < nx - 1:
            out[r, 1] = x1 + (T[r, x1] - level) / (T[r, x1] - T[r, x1 + 1])
    return out


def flame_errors(T_test, T_ref, phi, prob):
    """Flame-front shift (cells; the progress variable (T - T_in) / (T_ad -
    T_in) crossing 1/2, per row, both edges, maximum over rows) and the
    temperature error over fluid cells (phi_f > 1/2) of a run against a
    reference run."""
    ny, nx = prob["ny"], prob["nx"]
    level = prob["T_in"] + 0.5 * (adiabatic_temperature(prob) - prob["T_in"])
    fa = front_positions(np.asarray(T_test).reshape(ny, nx), level)
    fb = front_positions(np.asarray(T_ref).reshape(ny, nx), level)
    both = ~np.isnan(fa) & ~np.isnan(fb)
    one = np.isnan(fa) != np.isnan(fb)
    fluid = (1.0 - np.asarray(phi).reshape(-1)) > 0.5
    d = np.abs(np.asarray(T_test) - np.asarray(T_ref))[fluid]
    ref = np.asarray(T_ref)[fluid] - prob["T_in"]
    return {"front_max_diff_cells": float(np.max(np.abs(fa - fb)[both])) if both.any() else None,
            "rows_with_front": int(both[:, 1].sum()),
            "rows_front_mismatch": int(one.sum()),
            "T_max_abs_diff_K": float(d.max()),
            "T_l2_rel": float(np.linalg.norm(d) / np.linalg.norm(ref))}
