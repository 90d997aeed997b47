"""The seeded synthetic input recipe (paper_2412_14859_gb300/inputs.py) on CPU: the geometries and
draws the workloads are stated with, so that every run sees the same inputs.

  - the phase fields: a drop's tanh profile is centred on its centre and crosses zero at R0; the
    cap's centre sits on the wall plane z = -1/2; the pinned cap meets the rim of its cup;
  - the cup (solid ring) lies in the first `depth` planes only, between r_in and r_out;
  - the flux polynomial's basis is (r/R)^k, constant along the wall normal;
  - the random draws repeat bit for bit for a seed and differ between seeds; the 64-member
    ensemble has the stated mix (48 D2Q9 + 16 D3Q19, sides, ranges, 14 056 181 cells)."""
import numpy as np
import pytest

from paper_2412_14859_gb300 import inputs


def test_drop_phase_profile():
    shape = (21, 23, 25)
    c = inputs.centred(shape)
    phi = inputs.sphere_phase(shape, c, 6.0)
    assert phi[10, 11, 12] == pytest.approx(np.tanh(3.0))  # centre: tanh(R0 / 2)
    # along x from the centre: positive inside R0, zero at r = R0 = 6, negative outside
    line = phi[10, 11, 12:]
    assert line[5] > 0 > line[7] and line[6] == pytest.approx(0.0, abs=1e-12)
    assert phi.min() < -0.99 and np.all(np.abs(phi) < 1.0)


def test_cap_centre_on_the_wall_plane():
    case = inputs.sessile_cap_3d((16, 32, 32), R0=8.0)
    phi = case.phase()
    # first plane z = 0 lies 1/2 above the centre: rho^N = tanh((R0 - r) / 2) with r = 1/2 at the axis
    assert phi[0, 15, 15] == pytest.approx(np.tanh((8.0 - np.sqrt(0.5 ** 2 + 2 * 0.5 ** 2)) / 2.0))
    assert np.array_equal(phi[:, :, ::-1], phi) and np.array_equal(phi[:, ::-1, :], phi)
    assert np.all(np.diff(phi[:, 15, 15]) < 0)  # decreasing away from the wall


def test_cup_and_pinned_cap_geometry():
    case = inputs.pinned_cap_3d(128)
    solid = case.solid()
    r_in, r_out, depth = case.extra["r_in"], case.extra["r_out"], case.extra["depth"]
    assert solid.dtype == np.uint8 and not solid[depth:].any()
    n = case.shape[1]
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.hypot(yy - (n - 1) / 2.0, xx - (n - 1) / 2.0)
    ring = (r >= r_in) & (r < r_out)
    assert np.array_equal(solid[0].astype(bool), ring) and all(
        np.array_equal(solid[k], solid[0]) for k in range(depth))
    phi = case.phase()
    # inside the cup liquid, outside it gas; above the rim the cap's edge sits on r = r_out
    assert phi[0][r < r_in - 4].min() > 0.9 and phi[0][r > r_out + 4].max() < -0.9
    th = np.deg2rad(case.extra["angle_deg"])
    R = r_out / np.sin(th)
    zc = depth - 0.5 - r_out / np.tan(th)
    rim = np.hypot(r_out, (depth - 0.5) - zc)
    assert rim == pytest.approx(R)  # the sphere passes through the rim circle


def test_radial_basis_and_flux_polynomial():
    shape = (4, 9, 11)
    B = inputs.radial_basis(shape, (4.0, 5.0), 2.0, 3)
    assert B.shape == (3, 4, 9, 11)
    assert B[0, 0, 4, 7] == pytest.approx(1.0) and B[2, 3, 4, 9] == pytest.approx(8.0)  # r/R = 1, 2
    assert np.array_equal(B[:, 0], B[:, 3])  # constant along the wall normal
    phi = inputs.poly_flux(B, 1e-5, np.array([1.0, 0.0, -0.5]))
    assert phi[0, 4, 9] == pytest.approx(1e-5 * (1.0 + 2.0 - 0.5 * 8.0))


def test_draws_repeat_for_a_seed():
    a = inputs.uniform_noise((2, 19, 3, 4, 5), 1e-6, seed=7)
    assert np.array_equal(a, inputs.uniform_noise((2, 19, 3, 4, 5), 1e-6, seed=7))
    assert not np.array_equal(a, inputs.uniform_noise((2, 19, 3, 4, 5), 1e-6, seed=8))
    assert np.abs(a).max() <= 1e-6
    p1, t1 = inputs.flux_fit_parameters(16)
    p2, t2 = inputs.flux_fit_parameters(16)
    assert np.array_equal(p1, p2) and np.array_equal(t1, t2) and not np.array_equal(p1, t1)


def test_ensemble_member_mix():
    ms = inputs.ensemble_members()
    assert len(ms) == 64
    two, three = ms[:48], ms[48:]
    assert all(m.q == 9 and m.shape[0] == 1 and m.shape[1] == m.shape[2] and m.shape[1] % 32 == 0
               and 16.0 <= m.R0 < 64.0 for m in two)
    assert all(m.q == 19 and len(set(m.shape)) == 1 and m.shape[0] == int(np.ceil(4 * m.R0))
               and 12.0 <= m.R0 < 32.0 for m in three)
    assert all(1e-6 <= m.phi <= 1e-4 and 0.3 <= m.threshold <= 0.7 and m.rho_r_in in (1, 2, 5, 10)
               for m in ms)
    assert sum(m.ncell for m in ms) == 14056181  # the cells the ensemble line reports
    assert [m.seed for m in ms] == [inputs.SEED + 1 + j for j in range(64)]
