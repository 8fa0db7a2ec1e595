"""Unit conversions of the input side pinned to the numbers the paper prints
(tests/golden/paper_units.json, Sec. 2.3, Sec. 3.1 and SI Table 1)."""
import json
import math
import os

from paper_1604_01829_gb300 import workloads as W

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_units.json")))


def test_time_unit():
    assert abs(W.t0_seconds() * 1e12 / G["t0_ps"] - 1) < 2e-4


def test_water_density_and_viscosity():
    assert abs(W.density_to_paper_units(G["water_density_kg_m3"]) / G["water_density_M0_per_sigma3"] - 1) < 2e-4
    # printed 5.677 vs 5.6757 from the printed t0: agrees to 3e-4
    assert abs(W.kinematic_viscosity_to_paper_units(G["water_nu_m2_s"]) / G["water_nu_sigma2_per_t0"] - 1) < 5e-4
    assert abs(W.RHO_PAPER - G["water_density_M0_per_sigma3"]) < 1e-12


def test_bead_friction_in_si_and_lattice_units():
    assert abs(W.friction_to_si(G["xi_bead_M0_per_t0"]) / G["xi_bead_kg_s"] - 1) < 2e-3
    # one lattice mass unit is rho a^3, one lattice time unit dt_LB
    assert abs(W.paper_gamma_to_lattice(1000.0) - 1000.0 * G["dt_lb_t0"] / G["water_density_M0_per_sigma3"]) < 1e-12
    # the scaled viscosity in lattice units (grid 1 sigma, step 0.02 t0)
    assert abs(W.NU_PAPER - G["scaled_nu_sigma2_per_t0"] * G["dt_lb_t0"]) < 1e-15


def test_stokes_coefficients():
    eta = G["water_density_kg_m3"] * G["water_nu_m2_s"]
    assert abs(6 * math.pi * eta / G["six_pi_eta_kg_per_m_s"] - 1) < 1e-3
    # the printed 8 pi eta is 0.7 % below 8 pi eta from the same viscosity;
    # recorded as printed, checked only to that precision
    assert abs(8 * math.pi * eta / G["eight_pi_eta_kg_per_m_s_printed"] - 1) < 1e-2
