"""The A_u and A_T calibrations of Secs. 4.1 and 4.2 (Figs. A_u-vs-MSE and
A_T-vs-MSE) on the oracle at a reduced size: the channel (for A_T with gas
entering at 300 K between walls at 400 K) in its diffuse form against its
sharp form.  What the paper's procedure needs and what the physics fixes:

* the sharp channel's temperature across the sampled section is symmetric
  about the centreline and lies between the inlet and wall temperatures,
  hotter at the walls than at the centre;
* the mean standard error of eq. mean-standard-error-f (f = T) has an
  interior minimum in A_T: too weak a coupling leaves the gas near the
  diffuse walls cold, too strong a one heats it ahead of the sharp wall;
* likewise f = u in A_u: too weak a drag lets the gas slip through the
  diffuse walls, too strong a one stops it ahead of the sharp wall.

The sweep drivers (calibration.sweep_A_u, sweep_A_T) take the oracle as
their runner here; on the GPU they run the library with one stream per
value.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_17214_gb300 import calibration as C
from paper_2310_17214_gb300 import inputs as I

SIZE = {"L": 20, "eta": 4, "solid": 4, "H": 60}
STEPS = 3000  # about 2.5 transits of the channel: the section at 0.9 H is steady


@pytest.fixture(autouse=True)
def _threads():
    O.set_threads(0)
    yield


def _oracle_run(probs, field="T"):
    out = []
    for p in probs:
        f = I.di_channel_fields(p)
        s = O.OracleState(p, f["phi"], f["T"])
        s.step(STEPS)
        out.append(s.T.copy() if field == "T" else s.moments()[0][0].copy())
    return out


def test_sharp_hot_wall_channel_profile():
    p = I.di_channel(sharp=True, T_w=400.0, **SIZE)
    T = _oracle_run([p])[0].reshape(p["ny"], p["nx"])
    col = T[:, int(round(0.9 * p["nx"])) - 1]
    assert np.max(np.abs(col - col[::-1])) <= 1e-9 * 400.0
    assert np.all(col > 300.0) and np.all(col < 400.0)
    assert col[0] > col[p["ny"] // 2] + 1.0


def test_A_T_sweep_has_an_interior_minimum():
    r = C.sweep_A_T([8, 30, 100, 300, 1000], T_w=400.0, A_u=145.0, steps=STEPS,
                    run=_oracle_run, **SIZE)
    mse = np.asarray(r["mse"])
    k = int(np.argmin(mse))
    assert 0 < k < len(mse) - 1, mse
    assert mse[k] < 1e-2 * mse[0] and mse[k] < 0.1 * mse[-1], mse
    lo, hi = r["A_T"][k - 1], r["A_T"][k + 1]
    assert lo < r["A_T_star"] < hi
    assert r["paper_fit_A_T_star"] == pytest.approx(24.24 + 33.81 * 400.0 / 300.0)


def test_A_u_sweep_has_an_interior_minimum():
    r = C.sweep_A_u([10, 30, 100, 300, 1000, 3000], steps=STEPS,
                    run=lambda probs: _oracle_run(probs, "u"), **SIZE)
    mse = np.asarray(r["mse"])
    k = int(np.argmin(mse))
    assert 0 < k < len(mse) - 1, mse
    assert mse[k] < 0.05 * mse[0] and mse[k] < 0.05 * mse[-1], mse
    assert r["A_u"][k - 1] < r["A_u_star"] < r["A_u"][k + 1]


def test_refined_minimiser_is_the_vertex_of_the_log_parabola():
    """The refinement fits a parabola through the three samples around the
    sampled minimum in (log value, log MSE): for samples of an exact such
    parabola it returns the vertex; at the end of the range it keeps the
    sampled value."""
    a_star = 137.0
    values = [10.0, 40.0, 100.0, 250.0, 900.0]
    mse = [float(np.exp(0.7 * (np.log(v) - np.log(a_star)) ** 2 - 9.0)) for v in values]
    sampled, refined = C._minimum(values, mse)
    assert sampled == 100.0
    assert refined == pytest.approx(a_star, rel=1e-9)
    sampled, refined = C._minimum(values, sorted(mse))
    assert sampled == refined == 10.0
