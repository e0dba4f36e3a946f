"""Checkpoint / resume through pflb_get_state / pflb_set_state: 2N steps in
one go equal N steps + save + restore into a fresh domain + N steps, bit for
bit (the P0 reduction is deterministic)."""
import numpy as np
import pytest

from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300._native import Domain, PflbError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fp16"])
def test_resume_is_bitwise(precision):
    p = I.config2(nx=96, ny=40)
    p["bed"] = {"count": 4, "amin": 5, "amax": 9, "porosity": 0.6, "x0": 30}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    f = I.config2_fields(p)

    def fresh():
        d = Domain(p, precision)
        d.set_phase_field(f["phi"], f["Ts"])
        d.set_fields(f["T"], f["Y"])
        return d

    a = fresh()
    a.step(80)
    ref = a.get_state()
    b = fresh()
    b.step(40)
    mid = b.get_state()
    b.close()
    c = fresh()
    c.set_state(mid)
    c.step(40)
    got = c.get_state()
    assert got.nbytes == ref.nbytes
    assert np.array_equal(got, ref)
    # a state from another shape is rejected
    q = dict(p)
    q["nx"] = 97
    d = Domain(q, precision)
    d.set_phase_field(np.zeros(97 * 40), np.full(97 * 40, 300.0))
    d.set_fields(np.full(97 * 40, 300.0), np.tile(np.asarray(p["Y_in"])[:, None], 97 * 40))
    with pytest.raises(PflbError):
        d.set_state(mid)
