"""Pins of the oracle's blue pressure outlet (Sec. III.B.2; the boundary condition of Zou and He),
against things other than its own formula:

  - in 2D it equals the textbook Zou-He pressure condition for D2Q9 at a bottom and a top wall
    (written out here in this file's numbering from the published expressions);
  - in 3D the rebuilt cell holds the prescribed density and no tangential momentum, and an
    equilibrium at that density with any normal velocity comes back unchanged;
  - through whole steps: every outlet cell ends the step at the prescribed blue density with no
    tangential momentum; a uniform plug flow through two outlets is a fixed point; an overdense
    blue box relaxes to the outlet density; red sees a wall, so its mass is conserved.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20241219)


def test_d2q9_matches_textbook_zou_he():
    # numbering: 0 rest, 1 (1,0), 2 (-1,0), 3 (0,1), 4 (0,-1), 5 (1,1), 6 (-1,-1), 7 (1,-1), 8 (-1,1)
    L = oracle.lattice(9)
    assert [tuple(c[:2]) for c in L["c"]] == [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1),
                                             (1, -1), (-1, 1)]
    for _ in range(5):
        g = RNG.uniform(0.01, 0.2, 9)
        rho = RNG.uniform(0.8, 1.3)
        # bottom wall, inward normal +y: 3, 5, 8 unknown
        v = 1.0 - (g[0] + g[1] + g[2] + 2.0 * (g[4] + g[6] + g[7])) / rho
        want = g.copy()
        want[3] = g[4] + 2.0 / 3.0 * rho * v
        want[5] = g[6] - 0.5 * (g[1] - g[2]) + rho * v / 6.0
        want[8] = g[7] + 0.5 * (g[1] - g[2]) + rho * v / 6.0
        assert np.allclose(oracle.outlet_blue(9, +1, rho, g), want, rtol=0, atol=1e-15)
        # top wall, inward normal -y: 4, 6, 7 unknown; v is the inward speed
        v = 1.0 - (g[0] + g[1] + g[2] + 2.0 * (g[3] + g[5] + g[8])) / rho
        want = g.copy()
        want[4] = g[3] + 2.0 / 3.0 * rho * v
        want[6] = g[5] + 0.5 * (g[1] - g[2]) + rho * v / 6.0
        want[7] = g[8] - 0.5 * (g[1] - g[2]) + rho * v / 6.0
        assert np.allclose(oracle.outlet_blue(9, -1, rho, g), want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("inward", [1, -1])
def test_d3q19_moments_and_equilibrium(inward):
    L = oracle.lattice(19)
    c = L["c"].astype(np.float64)
    for _ in range(5):
        g = RNG.uniform(0.01, 0.1, 19)
        rho = RNG.uniform(0.8, 1.3)
        out = oracle.outlet_blue(19, inward, rho, g)
        known = c[:, 2] * inward <= 0
        assert np.array_equal(out[known], g[known])
        assert out.sum() == pytest.approx(rho, rel=1e-14)
        assert abs(out @ c[:, 0]) <= 1e-15 and abs(out @ c[:, 1]) <= 1e-15
    for uz in (-0.07, 0.0, 0.04):
        for abar in (1.0 / 3.0, 0.6):
            fe = oracle.feq(19, 1.1, (0.0, 0.0, uz), abar)
            assert np.allclose(oracle.outlet_blue(19, inward, 1.1, fe), fe, rtol=0, atol=1e-15)


def blue_box(q, shape, outlets, rho_blue=None, noise=0.0, u=None, **kw):
    nz, ny, nx = shape
    periodic = (1, 1, 0) if q == 19 else (1, 0, 1)
    p = oracle.Params(q=q, nx=nx, ny=ny, nz=nz, periodic=periodic, sigma=0.1, beta=0.99,
                      outlet_rho=outlets, phi=0.0, **kw)
    if u is not None:
        lat = oracle.lattice(q)
        fe = oracle.feq(q, 1.0 if rho_blue is None else rho_blue, u, lat["w"][0])
        f = np.zeros((2, q) + p.shape)
        f[1] = fe.reshape((q, 1, 1, 1))
        return p, f
    nzs = np.zeros((2, q) + p.shape)
    nzs[1] = RNG.uniform(-noise, noise, (q,) + p.shape)
    f = oracle.init(p, -np.ones(p.shape), nzs)
    if rho_blue is not None:
        f[1] *= rho_blue
    return p, f


@pytest.mark.parametrize("q", [9, 19])
def test_outlet_planes_hold_density_and_no_tangential_momentum(q):
    shape = (10, 4, 5) if q == 19 else (1, 10, 6)
    p, f = blue_box(q, shape, (1.0, 1.2), noise=1e-3)
    run = oracle.Run(p, f).step(3)
    m = run.macros()
    ax = 0 if q == 19 else 1  # wall-normal axis of the [z][y][x] arrays
    lo = np.take(m["rho_b"], 0, axis=ax)
    hi = np.take(m["rho_b"], -1, axis=ax)
    assert np.max(np.abs(lo - 1.0)) <= 1e-14 and np.max(np.abs(hi - 1.2)) <= 1e-14
    tang = [0, 1] if q == 19 else [0]  # u is (x, y, z)
    for t in tang:
        for plane in (0, -1):
            assert np.max(np.abs(np.take(m["u"][t], plane, axis=ax))) <= 1e-15
    assert np.all(m["rho_r"] == 0.0)


@pytest.mark.parametrize("q", [9, 19])
def test_plug_flow_is_a_fixed_point(q):
    shape = (12, 3, 4) if q == 19 else (1, 12, 5)
    u = (0.0, 0.0, 0.05) if q == 19 else (0.0, 0.05, 0.0)
    p, f = blue_box(q, shape, (1.0, 1.0), rho_blue=1.0, u=u)
    run = oracle.Run(p, f).step(30)
    assert np.max(np.abs(run.f - f)) <= 1e-14


def test_overdense_box_relaxes_to_outlet_density():
    p, f = blue_box(19, (12, 4, 4), (1.0, 1.0), rho_blue=1.05)
    run = oracle.Run(p, f)
    m0 = run.macros()["rho_b"].sum()
    run.step(1500)
    rb = run.macros()["rho_b"]
    assert m0 == pytest.approx(1.05 * rb.size, rel=1e-12)
    assert np.max(np.abs(rb - 1.0)) <= 1e-4
    walled = oracle.Run(blue_box(19, (12, 4, 4), (0.0, 0.0), rho_blue=1.05)[0], f).step(200)
    assert walled.macros()["rho_b"].sum() == pytest.approx(m0, rel=1e-13)  # walls keep the mass


def test_red_sees_a_wall_at_the_outlet():
    shape = (16, 4, 6)
    p = oracle.Params(q=19, nx=6, ny=4, nz=16, periodic=(1, 1, 0), sigma=0.1, beta=0.99,
                      rho_r_in=2.0, rho_b_in=1.0, outlet_rho=(1.0, 1.0), phi=0.0)
    z = np.arange(16)[:, None, None] + 0.5
    rn = np.broadcast_to(np.tanh((6.0 - z) / 2.0), shape).copy()  # red against the lower outlet
    run = oracle.Run(p, oracle.init(p, rn))
    r0 = run.macros()["rho_r"].sum()
    b0 = run.macros()["rho_b"].sum()
    run.step(60)
    m = run.macros()
    assert m["rho_r"].sum() == pytest.approx(r0, rel=1e-13)
    assert abs(m["rho_b"].sum() - b0) > 1e-3  # blue did flow through the outlets
