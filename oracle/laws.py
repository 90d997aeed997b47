"""Analytic evaporation laws and the heated-substrate flux -- TEST INFRASTRUCTURE ONLY (part of
the oracle; only tests/, __graft_entry__.smoke() and the CPU legs of bench.py use it).

Constant flux (Sec. III.A): a reaction-limited interface recedes at phi / rho along its normal,
so a flat interface, a sphere and a hemisphere all follow  L(t) = L0 - phi t / rho  (Eq.
surface_flux with dM/dt = rho dV/dt).

Heated substrate (Sec. III.C, Eq. heated, App. C): the flux at a surface point of local drop
height h is  Phi = phi_S / (K + h / R0).  On the lattice h is the liquid height of the column
through the cell along the wall normal, i.e. the sum over the column's fluid cells of the liquid
fraction rho_r / (rho_r + rho_b) (reading R25: a diffuse interface of any width integrates to the
height of the equivalent sharp one).  For a hemisphere of radius R the surface integral of
Phi over the cap gives  dR/dt = (phi_S R0 / (rho R)) ln(K R0 / (R + K R0))  (Eq. drrr), which
the paper integrates with an explicit Runge-Kutta 5(4) method from R(0) = R0.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp


def column_liquid_height(rho_r: np.ndarray, rho_b: np.ndarray, solid=None, axis: int = 0) -> np.ndarray:
    """Liquid height of every column along `axis` (the wall normal; axis 0 = z of a [z][y][x]
    field): the sum of rho_r / (rho_r + rho_b) over the column's fluid cells (reading R25)."""
    with np.errstate(invalid="ignore", divide="ignore"):  # solid cells hold no mass
        frac = rho_r / (rho_r + rho_b)
    if solid is not None:
        frac = np.where(np.asarray(solid) != 0, 0.0, frac)
    return frac.sum(axis=axis)


def heated_flux(h: np.ndarray, phi_s: float, K: float, R0: float) -> np.ndarray:
    """Eq. heated in lattice units: Phi = phi_S Phi* = phi_S / (K + h / R0)."""
    return phi_s / (K + np.asarray(h, np.float64) / R0)


def heated_flux_field(rho_r, rho_b, solid, phi_s: float, K: float, R0: float, axis: int = 0):
    """The per-cell flux of a state: every cell takes Eq. heated of its column's height."""
    h = column_liquid_height(rho_r, rho_b, solid, axis)
    return np.broadcast_to(np.expand_dims(heated_flux(h, phi_s, K, R0), axis), rho_r.shape).copy()


def heated_radius_rate(R: float, phi_s: float, K: float, R0: float, rho: float) -> float:
    """Eq. drrr: dR/dt of a hemisphere of radius R under the flux of Eq. heated."""
    return phi_s * R0 / (rho * R) * np.log(K * R0 / (R + K * R0))


def heated_radius(t, phi_s: float, K: float, R0: float, rho: float, rtol: float = 1e-10) -> np.ndarray:
    """R(t) of Eq. drrr from R(0) = R0, by an explicit Runge-Kutta 5(4) integration (App. C);
    0 once the drop has gone (R reaches 1e-6 R0 in finite time)."""
    t = np.atleast_1d(np.asarray(t, np.float64))
    gone = lambda _, y: y[0] - 1e-6 * R0
    gone.terminal = True
    sol = solve_ivp(lambda _, y: [heated_radius_rate(y[0], phi_s, K, R0, rho)], (0.0, float(t.max())),
                    [R0], method="RK45", dense_output=True, events=gone, rtol=rtol, atol=1e-12 * R0)
    if sol.status < 0:
        raise RuntimeError(sol.message)
    out = np.zeros_like(t)
    live = t <= sol.t[-1]
    if live.any():
        out[live] = sol.sol(t[live])[0]
    return out


def constant_flux_length(t, L0: float, phi: float, rho: float):
    """L(t) = L0 - phi t / rho: a flat interface, sphere or hemisphere under constant flux."""
    return L0 - phi * np.asarray(t, np.float64) / rho
