"""A pflb_step call of 32 steps or more replays pairs of steps from a CUDA
graph; the same steps launched one call at a time must give the same state
bit for bit.  Cases cover the launch sequences that differ: the feedback
and characteristic-outlet kernels, the persistent tiles with their tile
counters, the 3-D z-march, and the surrogate pre-pass with its fallback
list (every cell rejected, so no network training is needed)."""
import numpy as np
import pytest

from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300 import surrogate as S
from paper_2310_17214_gb300._native import Domain, Mlp, MLP_PARAMS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STEPS = 40  # two plain steps, then 19 replayed pairs


def _compare(make, names, steps=STEPS):
    a, b = make(), make()
    a.step(steps)
    for _ in range(steps):
        b.step(1)
    ga, gb = a.get(*names), b.get(*names)
    for k in names:
        assert np.array_equal(ga[k], gb[k]), k
    sa, sb = a.scalars(), b.scalars()
    for k in ("P0", "step", "u_in", "fuel", "outlet_pb"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    assert sa["step"] == steps
    a.close()
    b.close()


def _domain(p, f, precision, kernel=None, Ts=False):
    d = Domain(p, precision)
    if Ts:
        d.set_phase_field(f["phi"], f["Ts"])
    else:
        d.set_phase_field(f["phi"])
    d.set_fields(f["T"], f["Y"] if p.get("K", 0) > 0 else None)
    if kernel:
        d.select_kernel(kernel)
    return d


@pytest.mark.parametrize("precision,kernel", [("fp64", "tiled"), ("fp32", "persistent")])
def test_graph_replay_flame_with_feedback(precision, kernel):
    p = I.config6(nx=96, ny=32, precision=precision)
    f = I.config6_fields(p)
    _compare(lambda: _domain(p, f, precision, kernel), ("T", "Y", "u", "g"))


def test_graph_replay_characteristic_outlet():
    p = I.di_channel(L=20, eta=4, solid=4, A_u=145.0)
    f = I.di_channel_fields(p)
    _compare(lambda: _domain(p, f, "fp64"), ("T", "u", "g"))


def test_graph_replay_3d_march():
    p = I.config3_crop(32, precision="fp32")
    f = I.config3_fields(p)
    _compare(lambda: _domain(p, f, "fp32", "march", Ts=True), ("T", "Y", "u", "g", "Ts"))


def test_graph_replay_surrogate_fallback():
    p = I.config4(nx=128, ny=40, precision="fp32", chem="surrogate")
    p["bed"] = {"count": 4, "amin": 5, "amax": 8, "porosity": 0.6, "x0": 64}
    p["ignite"] = [8, 40, 1800.0]
    f = I.config4_fields(p)
    X = np.array([[300.0] + list(p["Y_in"]) + [p["P0"]]] * 2)
    X[1, 0] = 2500.0
    stats = (X.mean(axis=0), X.std(axis=0), np.zeros(6), np.zeros(6))
    rec = S.make_surrogate(stats, X, 0.0, p["species"], -1.0)  # every cell falls back
    nets = []

    def make():
        d = _domain(p, f, "fp32", Ts=True)
        net = Mlp()
        net.set_params(np.zeros(MLP_PARAMS, dtype=np.float32))
        nets.append(net)
        d.set_surrogate(net, rec)
        return d

    _compare(make, ("T", "Y", "u", "g"))
    for net in nets:
        net.close()
