"""Analysis utilities pinned by the numbers the paper prints.

Golden values (tests/golden/table1_geometry.txt): Sec. 3 Table
porous_structure_properties and the acceleration of Sec. 4.2.  Experimental
numbers from Sec. 4.1 (water at SATP, Table experimental_parameters; pore radii
5-25 micrometres; pressure Bond number 0.01).
"""
import math
import os

import numpy as np
import pytest

from paper_2608_15781_b300 import analysis as A
from paper_2608_15781_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_geometry.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_table1_arithmetic():
    g = _golden()
    av = g["surface_area"] / g["volume"]
    assert abs(av - g["area_to_volume"]) < 5e-4                         # 0.17238 printed as 0.172
    eta = A.reactor_efficiency(g["permeability"], av)
    assert abs(eta - g["efficiency"]) < 5e-4                            # 0.18221 printed as 0.182


def test_acceleration_mapping():
    g = _golden()
    a = A.acceleration_for_bond(g["bond_pressure"], g["sigma"], 1.0, g["pore_radius"])
    assert abs(a - g["accel"]) / g["accel"] < 1e-3                      # 3.6156e-5 printed as 3.616e-5


def test_experimental_scales():
    sigma_w, rho_w, g = 0.0721, 997.0, 9.81
    lo = A.pressure_gradient_for_bond(0.01, 25e-6, sigma_w) / 1e5      # bar / m
    hi = A.pressure_gradient_for_bond(0.01, 5e-6, sigma_w) / 1e5
    assert abs(hi - 288) < 1.0 and abs(lo - 11.5) < 0.1                 # printed as 288 and ~12 bar/m
    assert A.bond_number(rho_w, g, 25e-6, sigma_w) < 1e-4               # Bo < 1e-4 for all pore radii
    assert abs(A.laplace_pressure(sigma_w, 5e-6) / 1e5 - 0.288) < 1e-3  # 2 sigma / R (the paper prints 0.280)


def test_damkohler_round_trip():
    kappa, V, L, a, xi, A_r = 6.132, 256 ** 3, 256, 3.616e-5, 1.0, 64
    for Da in (0.1, 1.0, 10.0):
        nu = A.viscosity_for_damkohler(Da, xi, A_r, L, kappa, V, a)
        assert abs(A.damkohler(xi, A_r, nu, L, kappa, V, a) - Da) < 1e-12
        assert abs(A.flow_timescale(nu, L, kappa, a) / A.reactive_timescale(V, xi, A_r) - Da) < 1e-12
        assert A.tau_for_viscosity(nu) > 0.5
    assert abs(A.kinematic_viscosity(A.tau_for_viscosity(0.1)) - 0.1) < 1e-15


def test_morphology_on_known_mask():
    s = np.zeros((10, 12, 14), bool)
    s[:, :, :7] = True          # half the box solid, one flat interface pair in x (periodic)
    m = A.morphology(s)
    assert m["porosity"] == 0.5
    assert m["surface_area"] == 2 * 10 * 12                             # two wall layers, NN = 1 each


def test_nucleation_sites_give_one_site_per_block():
    solid = synth.grf_mask((128, 128, 128), 6, 0.6, 7)
    r = A.nucleation_sites(solid, block=64, seed=1)
    assert r.sum() == 8                                                 # (128/64)^3 blocks
    assert A.reactive_surface_area(r, solid) == 8                       # each site has NN = 1
    nn = A.nearest_solid_count(solid)
    assert (nn[r] == 1).all() and not solid[r].any()


def test_effectiveness_factor_and_fit():
    xi, A_r, phi, V = 1.0, 64, 0.6, 256 ** 3
    m_m = phi * V
    alpha = 0.37
    t = np.arange(0, 50001, 1000, dtype=float)
    m = A.predicted_mass(t, m_m, alpha, xi, A_r, phi, V)
    assert abs(A.fit_effectiveness(t, m, m_m, xi, A_r, phi, V) - alpha) < 1e-12
    rate = -np.gradient(m, t)                                           # consumed per unit time
    al = A.effectiveness_factor(rate, m, xi, A_r, phi, V)
    assert np.abs(al[1:-1] - alpha).max() < 1e-3
    assert abs(A.running_average(np.full(10, 0.5))[-1] - 0.5) < 1e-15
    assert np.allclose(A.running_average([1, 0, 1, 0]), [1, 0.5, 2 / 3, 0.5])
