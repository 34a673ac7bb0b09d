"""The seeded generators reproduce the paper's printed inputs (Tables 1, 2, 4)
and are deterministic."""

import json
import os

import numpy as np
import pytest

from scenarios import generate as G

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_table1_inputs():
    t = GOLD["table1_1d"]
    sc = G.scenario_1d_table1()
    ph = sc["physics"]
    assert sc["nx"] == t["blocks"]
    assert ph["rho_w"] == t["water_density_kg_m3"] and ph["rho_o"] == t["oil_density_kg_m3"]
    assert ph["c_w"] * G.BAR == pytest.approx(t["water_compressibility_per_bar"])
    assert ph["c_o"] * G.BAR == pytest.approx(t["oil_compressibility_per_bar"])
    assert ph["mu_w"] / G.CP == t["water_viscosity_cp"] and ph["mu_o"] / G.CP == t["oil_viscosity_cp"]
    assert ph["ipv"] == t["ipv"] and ph["rrf"] == t["rrf"]
    assert np.all(sc["phi"] == t["porosity"]) and np.allclose(sc["kx"] / G.MD, t["permeability_md"])
    assert np.all(sc["S0"] == t["initial_water_saturation"]) and np.all(sc["C0"] == t["initial_polymer_kg_m3"])
    assert sc["dx"] == t["grid_size_m"]


def test_table2_inputs():
    t = GOLD["table2_2d"]
    sc = G.scenario_2d_table2()
    ph = sc["physics"]
    lbm_ft3 = 0.45359237 / 0.3048 ** 3
    assert ph["rho_w"] == pytest.approx(t["water_density_lbm_ft3"] * lbm_ft3)
    assert ph["rho_o"] == pytest.approx(t["oil_density_lbm_ft3"] * lbm_ft3)
    assert ph["mu_o"] / G.CP == t["oil_viscosity_cp"]
    assert sc["dx"] == pytest.approx(t["grid_size_ft"] * 0.3048)
    ctl = sc["schedule"][0]["controls"]
    assert ctl[0]["limit"] == pytest.approx(t["injector_bhp_cap_psia"] * G.PSI)
    assert ctl[1]["target"] == pytest.approx(t["producer_bhp_psia"] * G.PSI)


def test_table4_layers():
    sc = G.scenario_layered_table4(nx=4, ny=3)
    n2 = 12
    for (layer, por, kx, ky, kz) in GOLD["table4_layers"]["layers"]:
        sl = slice((layer - 1) * n2, layer * n2)
        assert np.all(sc["phi"][sl] == por)
        assert np.allclose(sc["kx"][sl] / G.MD, kx) and np.allclose(sc["ky"][sl] / G.MD, ky)
        assert np.allclose(sc["kz"][sl] / G.MD, kz)


def test_generators_deterministic_and_shaped():
    a, b = G.scenario_c1(), G.scenario_c1()
    assert np.array_equal(a["kx"], b["kx"])
    assert a["kx"].shape == (300,)
    # lognormal with arithmetic mean 100 mD (sigma 1): sample mean within a loose band
    k = G.scenario_c2(nx=40, ny=40, nz=10)["kx"] / G.MD
    assert 40.0 < np.exp(np.log(k).mean()) * np.exp(0.5 * 1.5 ** 2) < 250.0
    u = G.uniform01(5, 0, 100000)
    assert 0.0 < u.min() and u.max() <= 1.0 and abs(u.mean() - 0.5) < 0.01
    z = G.normal(5, 1, 100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (state += golden gamma, then the mix function).
    z = G.splitmix64(np.array([0x9E3779B97F4A7C15, 2 * 0x9E3779B97F4A7C15 % 2 ** 64], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
