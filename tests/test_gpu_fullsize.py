"""Parity at the workloads' full sizes, in the launch configuration the bench times (the default
kernel of each storage): the GPU advances the lattice, its state is read back, the GPU takes one
more step, and the oracle computes that step one cell at a time (orc_step_cells) for a seeded
sample of cells -- interface cells, cells of the first and last planes and random cells -- from
the same state.

- 192^3 drop (density ratio 10): FP64 (<= 1e-12), FP32 pairs (plain and with exact colour
  masses), F32RC and FP16 recolour on pull (<= 1e-5), BF16 recolour on pull (<= 1e-4), FP16 per-colour deviations (the storage rounding
  of the outputs, <= 2e-4 of the largest population);
- 256 x 256 x 128 sessile cap with walls on z and a flux field: FP32 (<= 1e-5).

Site decisions are compared wherever the GPU did not flag the decision value as lying within
1e-6 of the threshold (bit 2 of the site byte).
"""
import numpy as np
import pytest
import torch

import oracle
from harness import oracle_params
from paper_2412_14859_gb300 import inputs
from paper_2412_14859_gb300.binding import SITES_GRADIENT, Sim

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32x": 1e-5, "f32rc": 1e-5, "f16rc": 1e-5, "bf16rc": 1e-4, "f16dev": 2e-4}


def sample_cells(rhoN, shape, n=2000, seed=inputs.SEED + 31):
    """Half the sample from the interface band |rho^N| < 0.6, a quarter from the first and last
    planes (walls, periodic seams), a quarter anywhere."""
    g = inputs.rng(seed)
    band = np.flatnonzero(np.abs(rhoN.ravel()) < 0.6)
    nz, ny, nx = shape
    plane = ny * nx
    edge = np.concatenate([np.arange(plane), np.arange((nz - 1) * plane, nz * plane)])
    picks = [g.choice(band, n // 2, replace=False), g.choice(edge, n // 4, replace=False),
             g.choice(rhoN.size, n - n // 2 - n // 4, replace=False)]
    return np.unique(np.concatenate(picks)).astype(np.int64)


def run_case(case, storage, phi_field=None, warm=10):
    dev = torch.device("cuda", 0)
    sim = Sim.from_case(case, storage)
    if phi_field is not None:
        sim.set_flux(0.0, torch.from_numpy(phi_field).to(dev))
    else:
        sim.set_flux(case.phi)
    nz = case.noise_array(np.float64)
    sim.init_equilibrium(torch.from_numpy(case.phase()).to(dev),
                         None if nz is None else torch.from_numpy(nz).to(dev))
    sim.step(warm)
    f_in = sim.populations(torch.float64).cpu().numpy()  # the state the next step starts from
    sim.step(1)
    f_out = sim.populations(torch.float64).cpu().numpy()
    mask = sim.mask().cpu().numpy().ravel()
    sim.close()
    p = oracle_params(case, phi_field=phi_field)
    rhoN = oracle.macros(p, f_in)["rhoN"]
    cells = sample_cells(rhoN, case.shape)
    want, _, om = oracle.step_cells(p, f_in, None, cells)
    flat = f_out.reshape(2, case.q, -1)
    got = np.stack([flat[:, :, c] for c in cells])  # [n, 2, Q]
    return got, want, mask[cells], om


def check(got, want, gm, om, tol):
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= tol, err
    far = (gm & 4) == 0
    assert np.array_equal((gm & 1)[far], om[far])
    assert int(om.sum()) > 100  # the sample holds sites


@pytest.mark.parametrize("storage", ["f64", "f32", "f32x", "f32rc", "f16rc", "bf16rc", "f16dev"])
def test_sphere_192_sampled_step(storage):
    case = inputs.sphere_3d(192)
    check(*run_case(case, storage), TOL[storage])


def test_sessile_cap_full_box_sampled_step():
    case = inputs.sessile_cap_3d()
    nz, ny, nx = case.shape
    basis = inputs.radial_basis(case.shape, ((ny - 1) / 2.0, (nx - 1) / 2.0), case.R0, 16)
    a, _ = inputs.flux_fit_parameters(16)
    phi = inputs.poly_flux(basis, case.phi, a)
    check(*run_case(case, "f32", phi_field=phi), TOL["f32"])


def test_density_contrast_outlets_full_box_sampled_step():
    """The density-contrast sphere of Sec. III.B.2 (192^3, gamma = 2, blue outlets at both z ends)
    after ten steps with the outlets on: one more GPU step against the oracle's single-cell step on
    the sampled cells, which include the two outlet planes (FP32)."""
    from harness import oracle_params as op
    n = 192
    case = inputs.Case("density_contrast", 19, (n, n, n), periodic=(1, 1, 0), rho_r_in=2.0,
                       sigma=0.1, beta=0.99, site_rule=SITES_GRADIENT, threshold=0.32, sbar=3.0,
                       phi=0.03, R0=44.0)
    dev = torch.device("cuda", 0)
    sim = Sim.from_case(case, "f32")
    sim.set_flux(case.phi)
    sim.set_outlets(1.0, 1.0)
    sim.init_equilibrium(torch.from_numpy(case.phase()).to(dev))
    sim.step(10)
    f_in = sim.populations(torch.float64).cpu().numpy()
    G_prev = sim.mask().cpu().numpy().ravel()
    sim.step(1)
    f_out = sim.populations(torch.float64).cpu().numpy()
    mask = sim.mask().cpu().numpy().ravel()
    sim.close()
    p = op(case)
    p.outlet_rho = (1.0, 1.0)
    rhoN = oracle.macros(p, f_in)["rhoN"]
    cells = sample_cells(rhoN, case.shape)
    # the gradient rule reads the previous step's decision: hand the oracle |F| > Gamma as bit 1
    G = np.where((G_prev & 2) != 0, case.threshold + 1.0, case.threshold - 1.0).reshape(case.shape)
    want, _, om = oracle.step_cells(p, f_in, G, cells)
    flat = f_out.reshape(2, case.q, -1)
    got = np.stack([flat[:, :, c] for c in cells])
    far = (mask[cells] & 4) == 0
    assert np.array_equal((mask[cells] & 1)[far], om[far])
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= TOL["f32"]
    plane = n * n
    on_outlets = np.isin(cells // plane, [0, n - 1])
    assert on_outlets.sum() > 100


def test_heated_flux_full_box_field_and_step():
    """The heated hemisphere of Sec. III.C at its full size (192^3, R0 = 66): the device-computed
    flux field equals the oracle's field from the same state, and one step with it equals the
    oracle's single-cell step on the sampled cells (FP32)."""
    from oracle import laws
    n = 192
    case = inputs.Case("heated", 19, (n, n, n), periodic=(1, 1, 0), geometry="cap", sigma=0.1,
                       beta=0.99, site_rule=SITES_GRADIENT, threshold=0.305, sbar=3.0, phi=0.0,
                       R0=66.0)
    dev = torch.device("cuda", 0)
    sim = Sim.from_case(case, "f32")
    sim.set_flux(0.0)
    sim.init_equilibrium(torch.from_numpy(case.phase()).to(dev))
    sim.step(20)
    sim.set_flux_heated(1e-3, 0.5, 66.0, every=1)
    f_in = sim.populations(torch.float64).cpu().numpy()
    G_prev = sim.mask().cpu().numpy().ravel()
    field = sim.flux_field().cpu().numpy()
    p = oracle_params(case)
    m = oracle.macros(p, f_in)
    want_field = laws.heated_flux_field(m["rho_r"], m["rho_b"], None, 1e-3, 0.5, 66.0)
    assert np.max(np.abs(field - want_field)) / np.max(want_field) <= 1e-6  # FP32 cell sums
    sim.step(1)
    f_out = sim.populations(torch.float64).cpu().numpy()
    mask = sim.mask().cpu().numpy().ravel()
    sim.close()
    p = oracle_params(case, phi_field=field)
    cells = sample_cells(m["rhoN"], case.shape)
    G = np.where((G_prev & 2) != 0, case.threshold + 1.0, case.threshold - 1.0).reshape(case.shape)
    want, _, om = oracle.step_cells(p, f_in, G, cells)
    flat = f_out.reshape(2, case.q, -1)
    got = np.stack([flat[:, :, c] for c in cells])
    check(got, want, mask[cells], om, TOL["f32"])
