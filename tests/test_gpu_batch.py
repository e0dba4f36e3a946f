"""Batched stepping (one persistent kernel over the tiles of many domains)
against the same domains stepped one by one, and against the oracle.

Bars: every field bit for bit equal to single-domain stepping (the per-cell
arithmetic does not depend on the tile shape; a fixed P0 does not depend on
the reduction); the reduction scalars within 1e-6 relative in FP32 (a
thread adds its cells in the compute precision before the compensated warp
sums, so the grouping, which follows the tile shape, moves the FP32
partials by a rounding or two); the FP64 batch within 1e-10 of the
oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300._native import Batch, Domain, PflbError

pytestmark = pytest.mark.gpu

TILES = ["32x8", "32x16", "64x4"]


def beds(n=4, seed=7, precision="fp32", base=(64, 32)):
    probs = I.config5(n=n, seed=seed, precision=precision, base=base)
    return [(p, I.config5_fields(p)) for p in probs]


def make(p, f, precision):
    d = Domain(p, precision)
    d.set_phase_field(f["phi"], f["Ts"])
    d.set_fields(f["T"])
    return d


def fields(d):
    return d.get("T", "g", "u")


@pytest.mark.parametrize("tile", TILES)
def test_batch_equals_one_by_one(tile):
    cases = beds()
    single = [make(p, f, "fp32") for p, f in cases]
    batched = [make(p, f, "fp32") for p, f in cases]
    b = Batch(batched)
    b.set_config(tile)
    # an odd count, single steps in between, then an even count
    for d in single:
        d.step(7)
    b.step(7)
    for d, e in zip(single, batched):
        d.step(3)
        e.step(3)
    for d in single:
        d.step(4)
    b.step(4)
    for d, e in zip(single, batched):
        a, c = fields(d), fields(e)
        for k in a:
            assert np.array_equal(a[k], c[k]), (tile, k)
        sa, sc = d.scalars(), e.scalars()
        assert sa["step"] == sc["step"] == 14
        for k in ("P0", "mass", "I", "flux_in", "flux_out"):
            assert abs(sa[k] - sc[k]) <= 1e-6 * max(abs(sa[k]), 1e-300), (tile, k)
    b.close()
    for d in single + batched:
        d.close()


def test_batch_fp64_matches_oracle():
    cases = beds(n=2, seed=11, precision="fp64", base=(48, 24))
    doms = [make(p, f, "fp64") for p, f in cases]
    b = Batch(doms)
    b.set_config("64x4")
    b.step(25)
    for (p, f), d in zip(cases, doms):
        ora = O.OracleState(p, f["phi"], f["T"], None, f["Ts"])
        ora.step(25)
        got = d.get("T", "g")
        assert np.max(np.abs(got["T"] - ora.T)) <= 1e-10 * np.max(np.abs(ora.T))
        ref_g = ora.g.reshape(ora.Q, ora.N)
        assert np.max(np.abs(got["g"] - ref_g)) <= 1e-10 * np.max(np.abs(ref_g))
        assert d.scalars()["step"] == 25
    b.close()
    for d in doms:
        d.close()


def _closed_box(nx, ny, seed):
    p = I._base(2, nx, ny)
    p["bc"] = ["wall"] * 4 + ["periodic"] * 2
    I.lattice_air(p, 0.05)
    p.update({"A_u": 145.0, "A_T": 70.0, "eta": 4.0, "T_in": 300.0, "Ts_uniform": 600.0,
              "p0_mode": "closed", "seed": seed})
    phi = I.disc_phi(nx, ny, nx / 2.0, ny / 2.0, ny / 4.0, 4.0).reshape(-1)
    T = np.full(nx * ny, 300.0)
    return p, {"phi": phi, "T": T, "Ts": None}


def test_batch_with_a_closed_domain_tracks_its_pressure():
    """A closed box heated by a hot particle: its P0 rises each step, and the
    batch's immediate per-domain combine gives the single-domain P0."""
    cases = [_closed_box(70, 40, 1)] + beds(n=2, seed=3)
    for tile in ("32x8", "64x4"):
        single = [make(p, f, "fp32") for p, f in cases]
        batched = [make(p, f, "fp32") for p, f in cases]
        b = Batch(batched)
        b.set_config(tile)
        b.step(30)
        for d in single:
            d.step(30)
        P0a, P0b = single[0].scalars()["P0"], batched[0].scalars()["P0"]
        assert P0a > 101325.0 * (1 + 1e-6)
        assert abs(P0a - P0b) <= 1e-6 * P0a
        for d, e in zip(single, batched):
            a, c = d.get("T"), e.get("T")
            assert np.max(np.abs(a - c)) <= 1e-5 * np.max(np.abs(a))
        b.close()
        for d in single + batched:
            d.close()


def test_autotune_keeps_the_states():
    cases = beds(n=3, seed=5)
    doms = [make(p, f, "fp32") for p, f in cases]
    for d in doms:
        d.step(2)
    before = [d.get_state().copy() for d in doms]
    b = Batch(doms)
    cfg, table = b.autotune(steps=2)
    assert cfg["tile"] in TILES and cfg["blocks_per_sm"] >= 1 and cfg["grid"] >= 1
    assert len(table) >= 3 and all(v > 0 for v in table.values())
    after = [d.get_state() for d in doms]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    b.step(2)
    assert all(d.scalars()["step"] == 4 for d in doms)
    b.close()
    for d in doms:
        d.close()


def test_batch_rejects_what_it_cannot_run():
    (p, f), = beds(n=1, seed=9)
    d32 = make(p, f, "fp32")
    d64 = make(p, f, "fp64")
    with pytest.raises(PflbError):
        Batch([d32, d64])
    q = I.config4(nx=64, ny=32, precision="fp32")
    q["bed"] = {"count": 2, "amin": 4, "amax": 6, "porosity": 0.6, "x0": 24}
    g = I.config4_fields(q)
    dk = Domain(q, "fp32")
    dk.set_phase_field(g["phi"], g["Ts"])
    dk.set_fields(g["T"], g["Y"])
    with pytest.raises(PflbError):
        Batch([d32, dk])
    for d in (d32, d64, dk):
        d.close()
