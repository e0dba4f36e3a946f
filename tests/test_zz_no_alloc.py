"""pflb_step_noalloc, the allocation-free variant of the fused step, against
pflb_step on the same inputs, two calls in a row.

It exists for callers that cannot allocate device memory -- plug-ins whose
host framework owns every device allocation through its own pool, loops that
forbid allocator calls after start-up.  They pass their own state arrays; the
library's reduction scratch is a fixed device array.  This file is collected
last on purpose."""
import numpy as np
import pytest

from paper_2310_17214_gb300 import inputs as I
from paper_2310_17214_gb300._native import Domain, PflbError, step_noalloc

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def reactive_case():
    p = I.config2(nx=80, ny=36)
    p["bed"] = {"count": 4, "amin": 5, "amax": 8, "porosity": 0.6, "x0": 24}
    p["reactions"] = I.one_step_mechanism(3.3e8)
    return p, I.config2_fields(p)


def inert_case():
    p = I.config1(nx=70, ny=30)
    phi = I.disc_phi(70, 30, 20.0, 15.0, 5.0, p["eta"]).reshape(-1)
    T = (1 - phi) * p["T_in"] + phi * p["Ts_uniform"]
    return p, {"phi": phi, "T": T, "Y": None, "Ts": None}


@pytest.mark.parametrize("case,precision,tol", [
    ("reactive", "fp64", 1e-10), ("inert", "fp64", 1e-10),
    ("reactive", "fp32", 1e-6), ("inert", "fp32", 1e-6)])
def test_noalloc_matches_step_two_calls(case, precision, tol):
    import torch
    p, f = reactive_case() if case == "reactive" else inert_case()
    dom = Domain(p, precision)
    dom.set_phase_field(f["phi"], f["Ts"])
    dom.set_fields(f["T"], f["Y"])
    names = ["T", "g"] + (["Y"] if p.get("K") else []) + (["Ts"] if p.get("Ts_field") else [])
    npdt = np.float64 if precision == "fp64" else np.float32
    tdt = torch.float64 if precision == "fp64" else torch.float32
    start = dom.get(*names, dtype=npdt)
    sc = dom.scalars()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=tdt, device="cuda").contiguous()
    arr = {"phi": dev(f["phi"])}
    for k, n in (("T", "T"), ("g", "g"), ("Y", "Y"), ("Ts", "Ts")):
        if n in start:
            arr[k + "_in"] = dev(start[n])
            arr[k + "_out"] = torch.empty_like(arr[k + "_in"])
    for _ in range(2):
        sc = step_noalloc(p, precision, arr, sc)
        for k in ("T", "g", "Y", "Ts"):
            if k + "_in" in arr:
                arr[k + "_in"], arr[k + "_out"] = arr[k + "_out"], arr[k + "_in"]
    torch.cuda.synchronize()
    dom.step(2)
    ref = dom.get(*names)
    rs = dom.scalars()
    dom.close()
    for k in ("T", "g", "Y", "Ts"):
        if k in ref:
            got = arr[k + "_in"].cpu().numpy().reshape(ref[k].shape)
            assert maxrel(got, ref[k]) <= tol, k
    assert sc["step"] == rs["step"] == 2
    assert abs(sc["P0"] / rs["P0"] - 1) <= tol
    assert abs(sc["I"] / rs["I"] - 1) <= tol


def test_noalloc_rejects_oversized_and_unsupported():
    import torch
    p, f = inert_case()
    q = dict(p)
    q["nx"], q["ny"] = 4096, 2048  # 2^23 cells > the scratch limit; no array is touched
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    arr = {k: t for k in ("phi", "g_in", "g_out", "T_in", "T_out")}
    with pytest.raises(PflbError):
        step_noalloc(q, "fp64", arr, {"P0": p["P0"], "P0_prev": p["P0"]})
    q = dict(p)
    q["dim"], q["nz"] = 3, 4
    with pytest.raises(PflbError):
        step_noalloc(q, "fp64", arr, {"P0": p["P0"], "P0_prev": p["P0"]})


def test_noalloc_validates_the_description_like_create():
    """The description checks of pflb_create_domain run here too, before any
    launch (the arrays are full-size, so nothing could go out of bounds
    regardless): a bad boundary pairing, a P0 that is not positive and an
    unstable description are refused with the reason in pflb_last_error."""
    import torch
    p, f = inert_case()
    N = p["nx"] * p["ny"]
    t = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")
    arr = {"phi": t(N), "g_in": t(9 * N), "g_out": t(9 * N), "T_in": t(N) + 300.0,
           "T_out": t(N)}
    sc = {"P0": p["P0"], "P0_prev": p["P0"]}
    q = dict(p)
    q["bc"] = ["inlet", "outlet", "periodic", "wall", "periodic", "periodic"]
    with pytest.raises(PflbError) as e:
        step_noalloc(q, "fp64", arr, sc)
    assert e.value.code == -1 and "pairs" in str(e.value)
    with pytest.raises(PflbError) as e:
        step_noalloc(p, "fp64", arr, {"P0": 0.0, "P0_prev": 0.0})
    assert e.value.code == -1 and "P0" in str(e.value)
    q = dict(p)
    q["A_T"] = 1e4
    with pytest.raises(PflbError) as e:
        step_noalloc(q, "fp64", arr, sc)
    assert e.value.code == -5 and "exchange" in str(e.value)
