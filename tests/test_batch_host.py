"""The batched-bed workload generator (no GPU)."""
import numpy as np

from paper_2310_17214_gb300 import inputs as I


def test_batched_beds_follow_their_recipe():
    probs = I.config5()
    assert len(probs) == 48
    nx = np.array([p["nx"] for p in probs])
    ny = np.array([p["ny"] for p in probs])
    assert nx.min() >= 256 and nx.max() <= 1024 and np.all(np.abs(nx - 2 * ny) <= 1)
    assert len(set(nx.tolist())) > 40  # uneven sizes
    por = np.array([p["bed"]["porosity"] for p in probs])
    u = np.array([p["u_in"] for p in probs])
    assert por.min() >= 0.4 and por.max() <= 0.8
    assert u.min() >= 0.02 and u.max() <= 0.08
    assert all(p["K"] == 0 and p["dim"] == 2 and p["p0_mode"] == "fixed" for p in probs)
    # seeded: the same draw twice, a different one for another seed
    again = I.config5()
    assert [p["nx"] for p in again] == nx.tolist()
    assert [p["nx"] for p in I.config5(seed=6)] != nx.tolist()


def test_small_batched_bed_fields():
    (p,) = I.config5(n=1, seed=7, base=(64, 32))
    f = I.config5_fields(p)
    phi = f["phi"]
    assert phi.shape == (p["nx"] * p["ny"],)
    assert 0.0 <= phi.min() and phi.max() <= 1.0 and phi.max() > 0.99
    assert f["info"]["placed"] >= 4
    # temperature blends from the gas to the particles' 600 K
    assert np.allclose(f["T"], 300.0 + 300.0 * phi)
