"""Pins of the oracle's lattice constants and local operators by brute-force identities.

The paper defers A_i, B_i, C_i, W_i and zeta to Leclaire et al. (Sec. II.A); these identities fix
them: isotropy of the weights up to fourth order, normalisation and second moment of the rest
state phi_i(alpha) = A_i + B_i alpha (which with alpha = W_0 must give p = rho c_s^2, Appendix A),
zero mass and momentum of the perturbation of Eq. (perturb) and a purely tangential stress, and the
moments of Eq. (feq).  A dropped term, a wrong sign or a mis-indexed weight fails one of them.
"""
import itertools

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


@pytest.fixture(params=[9, 19])
def L(request, oracle_lib):
    return oracle.lattice(request.param)


def dim(L):
    return 2 if L["c"].shape[0] == 9 else 3


def test_velocity_set(L):
    c = L["c"]
    Q = c.shape[0]
    assert len({tuple(v) for v in c}) == Q
    assert np.all(c[L["opp"]] == -c)
    assert tuple(c[0]) == (0, 0, 0)
    if Q == 9:
        assert np.all(c[:, 2] == 0)
    assert set(np.sum(c * c, axis=1)) == {0, 1, 2}


def test_weight_isotropy(L):
    c, w = L["c"].astype(float), L["w"]
    D = dim(L)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    for a in range(3):
        assert abs(np.sum(w * c[:, a])) < 1e-15
    for a, b in itertools.product(range(D), repeat=2):
        assert np.isclose(np.sum(w * c[:, a] * c[:, b]), CS2 * (a == b), atol=1e-15)
    for a, b, g in itertools.product(range(D), repeat=3):
        assert abs(np.sum(w * c[:, a] * c[:, b] * c[:, g])) < 1e-15
    d = np.eye(3)
    for a, b, g, e in itertools.product(range(D), repeat=4):
        want = CS2 ** 2 * (d[a, b] * d[g, e] + d[a, g] * d[b, e] + d[a, e] * d[b, g])
        assert np.isclose(np.sum(w * c[:, a] * c[:, b] * c[:, g] * c[:, e]), want, atol=1e-15)


@pytest.mark.parametrize("alpha", [0.2, 1.0 / 3.0, 4.0 / 9.0, 0.8, 0.95])
def test_rest_state_moments(L, alpha):
    c = L["c"].astype(float)
    phi = L["a"] + L["b"] * alpha
    D = dim(L)
    assert np.isclose(phi.sum(), 1.0, atol=1e-15)
    assert np.isclose(phi[0], alpha)
    for a, b in itertools.product(range(D), repeat=2):
        assert np.isclose(np.sum(phi * c[:, a] * c[:, b]), L["zeta"] * (1 - alpha) * (a == b),
                          atol=1e-15)


def test_eos_of_least_dense_component(L):
    # Appendix A: p_b = rho_b zeta (1 - W_0) = rho_b c_s^2.
    assert np.isclose(L["zeta"] * (1.0 - L["w"][0]), CS2, atol=1e-15)


@pytest.mark.parametrize("gamma", [1.0, 2.0, 4.0, 10.0])
def test_alphas_and_pressure_ratio(gamma, oracle_lib):
    # Sec. II.A and Appendix A: alpha = W_0 for the least dense component, 1 - (1-W_0)/gamma for
    # the other; then p_r = rho_r c_s^2 / gamma, so equal pressures at rho_r = gamma rho_b.
    for q in (9, 19):
        L = oracle.lattice(q)
        p = oracle.Params(q=q, nx=4, ny=4, nz=1 if q == 9 else 4, rho_r_in=gamma, rho_b_in=1.0)
        ar, ab = oracle.alphas(p)
        assert ab == pytest.approx(L["w"][0], abs=1e-15)
        pr = gamma * L["zeta"] * (1 - ar)
        pb = 1.0 * L["zeta"] * (1 - ab)
        assert pr == pytest.approx(pb, rel=1e-14)
        assert pr == pytest.approx(CS2, rel=1e-14)


def test_perturbation_mass_momentum_stress(L):
    q = L["c"].shape[0]
    c = L["c"].astype(float)
    D = dim(L)
    g = np.random.default_rng(7)
    for _ in range(200):
        F = np.zeros(3)
        F[:D] = g.normal(size=D) * g.uniform(0.01, 2.0)
        s = oracle.perturbation_shape(q, F)
        Fn = np.linalg.norm(F)
        n = F / Fn
        assert abs(s.sum()) < 1e-14 * max(1.0, Fn)
        assert np.all(np.abs(s @ c) < 1e-14 * max(1.0, Fn))
        # second moment: (2/9)|F| (n n - I) restricted to the lattice dimension
        M = np.einsum("i,ia,ib->ab", s, c, c)[:D, :D]
        want = (2.0 / 9.0) * Fn * (np.outer(n[:D], n[:D]) - np.eye(D))
        assert np.allclose(M, want, atol=1e-14 * max(1.0, Fn))
    assert np.all(oracle.perturbation_shape(q, np.zeros(3)) == 0.0)


def test_equilibrium_moments(L):
    q = L["c"].shape[0]
    c = L["c"].astype(float)
    D = dim(L)
    g = np.random.default_rng(11)
    for _ in range(50):
        rho = g.uniform(0.1, 10.0)
        u = np.zeros(3)
        u[:D] = g.normal(scale=0.05, size=D)
        abar = g.uniform(L["w"][0], 0.99)
        f = oracle.feq(q, rho, u, abar)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(f @ c, rho * u, atol=1e-14 * rho)
        P = np.einsum("i,ia,ib->ab", f, c, c)[:D, :D]
        want = rho * L["zeta"] * (1 - abar) * np.eye(D) + rho * np.outer(u[:D], u[:D])
        assert np.allclose(P, want, atol=1e-13 * rho)


def test_recolor_direction_sum_vanishes(L):
    # The recoloring term moves no mass: sum_i cos(theta_i) phi_i(abar) = 0 for any direction.
    c = L["c"].astype(float)
    D = dim(L)
    norms = np.linalg.norm(c, axis=1)
    g = np.random.default_rng(3)
    for abar in (L["w"][0], 0.6, 0.9):
        phi = L["a"] + L["b"] * abar
        for _ in range(20):
            n = np.zeros(3)
            n[:D] = g.normal(size=D)
            n /= np.linalg.norm(n)
            cos = np.where(norms > 0, (c @ n) / np.where(norms > 0, norms, 1), 0.0)
            assert abs(np.sum(cos * phi)) < 1e-15
