"""The values the paper prints (tests/golden/paper_constants.txt, each with
its citation) are the ones the input generators, the oracle and the library
use."""
import os
import re

import pytest

from paper_2310_17214_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, value, cite = line.split(None, 2)
            assert cite.strip().startswith("Sec."), key
            out[key] = float(value)
    return out


G = golden()


def test_gas_constant_everywhere():
    assert I.R_GAS == G["R_gas_J_per_mol_K"]
    src = open(os.path.join(ROOT, "oracle", "pflb_oracle.c")).read()
    assert re.search(r"#define ORC_R 8\.314\b", src)
    lib = open(os.path.join(ROOT, "paper_2310_17214_gb300", "csrc", "pflb_launch.cuh")).read()
    assert re.search(r"R_GAS = 8\.314;", lib)


def test_sutherland_constants_of_the_reactive_workloads():
    for p in (I.config2(), I.config3(), I.config6()):
        assert p["suth_T"] == G["sutherland_T_star_K"]
        assert p["suth_S"] == G["sutherland_S_K"]
        assert p["mu_ref"] == G["sutherland_mu_star_Pa_s"]
        assert p["sutherland"] == 1


def test_channel_disc_takes_the_printed_A_T_fit():
    p = I.config1()
    ratio = p["Ts_uniform"] / p["T_in"]
    assert p["A_T"] == pytest.approx(G["A_T_fit_intercept"] + G["A_T_fit_slope"] * ratio,
                                     rel=1e-15)


def test_calibration_channel_is_the_printed_setup():
    p = I.di_channel()
    assert p["L"] == G["A_u_test_L_cells"] and p["eta"] == G["A_u_test_eta_cells"]
    assert p["nx"] == G["A_u_test_H_over_L"] * p["L"]
    nu = p["mu_ref"] / p["rho_ref"]
    assert p["u_in"] * p["L"] / nu == pytest.approx(G["A_u_test_Re"], rel=1e-12)
    import inspect
    assert inspect.signature(I.channel_mse).parameters["at"].default == G["mse_section_over_H"]
    # the bench's sweep samples the paper's optimum among its values
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == "calibration_leg")
    values = ast.literal_eval(fn.args.defaults[0])
    assert G["A_u_star"] in values


def test_flame_workload_uses_the_printed_grid():
    p = I.config6()
    assert p["dx"] == G["flame_dx_m"] and p["dt"] == G["flame_dt_s"]
    assert p["ny"] * p["dx"] * 1e3 == pytest.approx(G["flame_channel_width_mm"], rel=1e-12)
    assert p["wall_T"][2] == p["wall_T"][3] == G["flame_wall_T_K"]
    assert p["T_in"] == G["flame_inlet_T_K"]
