"""Failure detection on the GPU without a GPU fault: states poisoned on the
host latch PFLB_ERR_UNSTABLE, and a device wait given a zero bound latches
PFLB_ERR_TIMEOUT; in every case the context stays usable and a fresh domain
steps to the same answer as before."""
import numpy as np
import pytest

from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300._native import Domain, PflbError

pytestmark = pytest.mark.gpu

UNSTABLE, TIMEOUT = -5, -6


def channel(precision="fp64"):
    p = I.config1()
    f = I.with_initial_u(p, I.config1_fields(p))
    return p, f


def fresh(p, f, precision):
    d = Domain(p, precision)
    d.set_phase_field(f["phi"])
    d.set_fields(f["T"], None, f["u"])
    return d


def reference_T(p, f, precision, steps=20):
    d = fresh(p, f, precision)
    d.step(steps)
    T = d.get("T")
    d.close()
    return T


def test_nan_temperature_latches_unstable():
    p, f = channel()
    ref = reference_T(p, f, "fp64")
    T = f["T"].copy()
    T[p["nx"] * 30 + 70] = np.nan
    d = Domain(p, "fp64")
    d.set_phase_field(f["phi"])
    d.set_fields(T, None, f["u"])
    d.step(1)
    with pytest.raises(PflbError) as e:
        d.scalars()
    assert e.value.code == UNSTABLE
    d.close()
    assert np.array_equal(reference_T(p, f, "fp64"), ref)  # the context is fine


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_in_one_population_latches_unstable(precision):
    """A NaN confined to one stored population (written through the state
    round trip) reaches the step's reduction at once."""
    p, f = channel(precision)
    d = fresh(p, f, precision)
    d.step(3)
    d.scalars()
    st = d.get_state()
    N, Q = p["nx"] * p["ny"], 9
    esz = 8 if precision == "fp64" else 4
    # layout: header, scalars, populations (Q*N, storage type), T (N)
    g0 = st.nbytes - N * esz - Q * N * esz
    cell, i = p["nx"] * 40 + 90, 6
    off = g0 + (i * N + cell) * esz
    st[off:off + esz] = np.frombuffer(np.array([np.nan], dtype=np.float64 if esz == 8
                                               else np.float32).tobytes(), dtype=np.uint8)
    d.set_state(st)
    d.step(1)
    with pytest.raises(PflbError) as e:
        d.scalars()
    assert e.value.code == UNSTABLE
    d.close()


def test_tma_wait_timeout_latches_timeout_and_context_survives():
    """The TMA kernel's wait for a staged tile given a zero bound (one
    non-blocking probe, issued right after the copies) runs out: the step
    latches PFLB_ERR_TIMEOUT; each block drains its copies before it stops,
    so the next domain on the same context runs normally."""
    p, f = channel("fp32")
    ref = reference_T(p, f, "fp32")
    d = fresh(p, f, "fp32")
    d.select_kernel("tma")
    d.set_wait_limit(0)
    d.step(2)
    with pytest.raises(PflbError) as e:
        d.scalars()
    assert e.value.code == TIMEOUT
    # restoring the bound and the fields gives a working domain again
    d.set_wait_limit(1 << 31)
    d.set_fields(f["T"], None, f["u"])
    d.step(20)
    T = d.get("T")
    d.close()
    assert np.max(np.abs(T - ref)) <= 1e-6 * np.max(np.abs(ref))
    assert np.array_equal(reference_T(p, f, "fp32"), ref)
