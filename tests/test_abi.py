"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import numpy as np

from oracle import oracle as O
from paper_2310_17214_gb300 import _native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pflb_[a-z0-9_]+)\s*\(", text):
            syms.add(m.group(1))
    return syms


def test_library_exports_every_declared_symbol():
    L = nat.lib()
    syms = declared_symbols()
    assert "pflb_step" in syms and "pflb_create_domain" in syms
    for s in sorted(syms):
        assert hasattr(L, s), f"{s} declared in include/ but not exported"
        assert ctypes.cast(getattr(L, s), ctypes.c_void_p).value


def test_lattice_tables_match_oracle_order():
    for dim in (2, 3):
        c1, w1 = nat.lattice(dim)
        c2, w2 = O.lattice(dim)
        assert np.array_equal(c1, c2)
        assert np.array_equal(w1, w2)


def test_struct_layouts_are_plain_c(tmp_path):
    """The ctypes mirrors of the binding match the header: a C program
    compiled against include/pflb.h prints the size of each struct and the
    offset of each field the mirror names."""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pflb_domain_desc": nat.Desc, "pflb_mechanism": nat.Mechanism,
               "pflb_scalars": nat.Scalars, "pflb_diagnostics": nat.Diagnostics,
               "pflb_surrogate": nat.Surrogate}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pflb.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        cname, field, value = line.split()
        py = mirrors[cname]
        got = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert got == int(value), (cname, field, got, value)


def test_create_rejects_bad_descriptions_without_touching_the_gpu():
    from paper_2310_17214_gb300 import inputs as I
    p = I.config1()
    d = nat.make_desc(p)
    d.bc[0] = nat.BC["outlet"]  # outlet on x-lo is invalid
    h = ctypes.c_void_p()
    rc = nat.lib().pflb_create_domain(ctypes.byref(d), ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"inlet only" in nat.lib().pflb_last_error(None)
    d = nat.make_desc(p)
    d.bc[2], d.bc[3] = nat.BC["periodic"], nat.BC["wall"]
    assert nat.lib().pflb_create_domain(ctypes.byref(d), ctypes.byref(h)) == -1
    d = nat.make_desc(p)
    d.dim = 4
    assert nat.lib().pflb_create_domain(ctypes.byref(d), ctypes.byref(h)) == -7


def test_added_entry_points_reject_null_arguments_without_touching_the_gpu():
    """The surrogate, batch and probe calls check their arguments before any
    CUDA call: NULL handles and outputs give PFLB_ERR_ARG (-1)."""
    L = nat.lib()
    h = ctypes.c_void_p()
    assert L.pflb_create_batch(None, 0, ctypes.byref(h)) == -1 and not h.value
    assert L.pflb_create_batch(None, 3, None) == -1
    assert L.pflb_batch_step(None, 1) == -1
    assert L.pflb_batch_set_config(None, 0, 0) == -1
    assert L.pflb_batch_get_config(None, None, None, None) == -1
    assert L.pflb_batch_autotune(None, 1, None, None, None) == -1
    assert L.pflb_batch_destroy(None) == 0
    assert L.pflb_mlp_create(0, None, None) == -1
    assert L.pflb_mlp_set_params(None, None) == -1
    assert L.pflb_mlp_get_params(None, None) == -1
    assert L.pflb_mlp_forward(None, None, None, 0) == -1
    assert L.pflb_mlp_destroy(None) == 0
    assert L.pflb_set_surrogate(None, None, None) == -1
    assert L.pflb_chem_stats(None, None, None) == -1
    assert L.pflb_probe_fp64_fma(0, None) == -1


def test_every_workload_passes_the_stability_checks():
    """The descriptions of the five workloads (and the 3-D comparison crop)
    pass the create / set_mechanism checks, including T_max."""
    from paper_2310_17214_gb300 import inputs as I
    probs = [I.config1(), I.config2(), I.config2(precision="fp32"), I.config3(),
             I.config3_crop(64), I.config4(), I.config4(chem="surrogate"),
             I.mixture_transport(I.config2()), I.mixture_transport(I.config3()), I.config6(),
             I.di_channel(), I.di_channel(sharp=True),
             I.di_channel(T_w=400.0, A_T=1000.0), I.di_channel(sharp=True, T_w=400.0)] + I.config5()
    for p in probs:
        rc, msg = nat.validate(p, p.get("precision", "fp64"))
        assert rc == 0, (p.get("name"), rc, msg)


def test_create_rejects_unstable_descriptions_without_touching_the_gpu():
    """PFLB_ERR_UNSTABLE (-5) before any allocation: tau not above 1/2, a
    thermal diffusion number above 1/6 in 3-D (the 3-D bed at the 2-D time
    step, at its hottest temperature), a species diffusion number above the
    limit (checked with the mechanism), a solid diffusion number above the
    limit, the interface exchange number above 1, a sonic inlet, the solid
    side of the exchange above 2."""
    from paper_2310_17214_gb300 import inputs as I
    L = nat.lib()
    h = ctypes.c_void_p()

    def create(p):
        d = nat.make_desc(p, p.get("precision", "fp64"))
        rc = L.pflb_create_domain(ctypes.byref(d), ctypes.byref(h))
        assert not h.value
        return rc, L.pflb_last_error(None).decode()

    p = I.config1()
    p["mu_ref"] = 1e-300
    rc, msg = create(p)
    assert rc == -5 and "relaxation time" in msg
    p = I.config3()
    p["dt"] = 2.5e-7
    rc, msg = create(p)
    assert rc == -5 and "thermal diffusion number" in msg, msg
    p["T_max"] = 0.0  # at T_in and the solid temperature the 2-D step is still stable
    assert nat.validate(p)[0] == 0
    p = I.config2()
    p["Dref"] = [d * 20 for d in p["Dref"]]
    rc, msg = nat.validate(p)
    assert rc == -5 and "species" in msg, msg
    p = I.config2()
    p["lambda_s"] *= 1e4
    rc, msg = create(p)
    assert rc == -5 and "solid diffusion" in msg, msg
    p = I.config1()
    p["A_T"] = 1e4
    rc, msg = create(p)
    assert rc == -5 and "exchange" in msg, msg
    p = I.config1()
    p["u_in"] = 0.6
    rc, msg = create(p)
    assert rc == -5 and "sound speed" in msg, msg
    p = I.config2()
    p["rhocp_s"] *= 1e-6  # a solid that the exchange would overshoot
    p["lambda_s"] *= 1e-6  # (same solid diffusion number)
    rc, msg = create(p)
    assert rc == -5 and "solid-side exchange" in msg, msg
