"""Pins of the oracle's heated-substrate flux (Sec. III.C, Eq. heated) and of its radius law
(Eq. drrr, App. C), each against something other than the oracle's own formula:

  - Eq. drrr against the surface integral it comes from, done independently: Eq. heated
    integrated over the hemisphere in polar angle (dA = 2 pi R^2 sin(theta) dtheta at height
    R cos(theta)), divided by the cap's area rate 2 pi R^2 rho;
  - the Runge-Kutta solution against the separated integral t(R) = int rho R' dR' / (phi_S R0
    ln(1 + R' / (K R0))), done by adaptive quadrature;
  - the limit K -> infinity against the constant-flux law R0 - phi_S t / (rho K);
  - the flux ratio Phi_max / Phi_min of Tab. var_flux (2, 3, 5 for K = 1, 0.5, 0.25);
  - the column height against the height of a sharp step and of a tanh profile (midpoint sums of
    a smooth profile are exact to exponentially small terms), with and without solid cells.
"""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import laws

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "heated_flux.json")))
PHI_S, R0 = GOLDEN["phi_s"], float(GOLDEN["R0"])


@pytest.mark.parametrize("K", [0.25, 0.5, 1.0, 3.0])
@pytest.mark.parametrize("R", [66.0, 40.0, 13.0])
def test_radius_rate_is_the_surface_integral(K, R):
    rho = 1.02
    flux, _ = quad(lambda th: PHI_S / (K + R * np.cos(th) / R0) * 2 * np.pi * R * R * np.sin(th),
                   0.0, np.pi / 2, epsabs=0, epsrel=1e-13)
    want = -flux / (rho * 2 * np.pi * R * R)
    assert laws.heated_radius_rate(R, PHI_S, K, R0, rho) == pytest.approx(want, rel=1e-11)


@pytest.mark.parametrize("K", [0.25, 0.5, 1.0])
def test_runge_kutta_matches_separated_integral(K):
    rho = 1.0
    Rs = np.array([60.0, 45.0, 30.0, 15.0, 8.0])
    ts = [quad(lambda r: rho * r / (PHI_S * R0 * np.log(1.0 + r / (K * R0))), R, R0,
               epsabs=0, epsrel=1e-13)[0] for R in Rs]
    got = laws.heated_radius(np.array(ts), PHI_S, K, R0, rho)
    assert np.max(np.abs(got - Rs)) <= 1e-6 * R0


def test_large_K_is_constant_flux():
    K, rho = 1e5, 1.0
    t = np.linspace(0.0, 0.5 * R0 * rho * K / PHI_S, 6)[1:]
    got = laws.heated_radius(t, PHI_S, K, R0, rho)
    want = laws.constant_flux_length(t, R0, PHI_S / K, rho)
    assert np.max(np.abs(got - want)) <= 1e-4 * R0


@pytest.mark.parametrize("case", GOLDEN["cases"], ids=lambda c: f"K{c['K']}")
def test_flux_ratio_of_table(case):
    # at R = R0 the local height runs from 0 (contact line) to R0 (top)
    ratio = laws.heated_flux(0.0, PHI_S, case["K"], R0) / laws.heated_flux(R0, PHI_S, case["K"], R0)
    assert ratio == pytest.approx(case["phi_max_over_min"], rel=1e-12)


def test_column_height_of_sharp_and_tanh_profiles():
    nz, ny, nx = 64, 3, 4
    z = np.arange(nz)[:, None, None] + 0.5  # cell centres above the wall z = 0
    H = np.array([[20.3, 7.0, 0.0, 33.75], [12.5, 40.0, 18.2, 5.5], [25.0, 9.9, 30.1, 21.0]])
    sharp = (z < H[None]).astype(np.float64)
    rr, rb = sharp, 1.0 - sharp
    assert np.array_equal(laws.column_liquid_height(rr, rb), np.ceil(H - 0.5))
    w = 2.0
    prof = 0.5 * (1.0 + np.tanh((H[None] - z) / w))
    rr, rb = 1.1 * prof, 1.1 * (1.0 - prof)
    h = laws.column_liquid_height(rr, rb)
    far = H > 8 * w
    assert np.max(np.abs(h[far] - H[far])) <= 1e-6
    # a solid plug under the liquid adds nothing
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:5] = 1
    hs = laws.column_liquid_height(np.where(solid, 0.0, rr), np.where(solid, 1.0, rb), solid)
    assert np.max(np.abs((h - hs) - prof[:5].sum(axis=0))) <= 1e-12


def test_flux_field_is_constant_along_columns():
    g = np.random.default_rng(5)
    rr = g.uniform(0.0, 1.0, (6, 3, 4))
    rb = 1.0 - rr + 0.01
    f = laws.heated_flux_field(rr, rb, None, PHI_S, 0.5, R0)
    h = (rr / (rr + rb)).sum(axis=0)
    assert np.allclose(f, PHI_S / (0.5 + h / R0)[None], rtol=1e-15, atol=0)
    assert np.all(f == f[:1])
