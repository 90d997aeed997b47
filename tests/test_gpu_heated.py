"""The heated-substrate flux (cgevap_set_flux_heated; Sec. III.C, Eq. heated) on the GPU.

- the device-computed flux field equals the oracle's (oracle/laws.py) computed from the same
  state, element by element, for every storage, on a walled cap with a solid block on the wall;
- the field is recomputed exactly when it should be (every `every` steps, before the step);
- one step with the recomputed field equals the oracle's step with the oracle's field (FP64);
- runs repeat bit for bit; a scalar flux switches the mode off; the error paths.
"""
import numpy as np
import pytest
import torch

import oracle
from harness import oracle_params
from oracle import laws
from paper_2412_14859_gb300 import inputs
from paper_2412_14859_gb300.binding import CgevapError, Sim

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 2e-7, "f16dev": 2e-7}  # FP32 fields round the value once
PHI_S, K, L = 2e-3, 0.5, 10.0


def walled_cap():
    case = inputs.sessile_cap_3d((24, 40, 40), R0=10.0, phi0=0.0)
    solid = np.zeros(case.shape, np.uint8)
    solid[0:3, 4:8, 28:33] = 1  # a block on the wall, away from the drop
    return case, solid


def start(case, solid, storage, warm=20):
    sim = Sim.from_case(case, storage)
    sim.set_solid(torch.from_numpy(solid).cuda())
    sim.set_flux(0.0)
    sim.init_equilibrium(torch.from_numpy(case.phase()).cuda())
    sim.step(warm)
    return sim


def oracle_field(sim, solid):
    m = sim.macros()
    return laws.heated_flux_field(m["rho_r"].cpu().numpy(), m["rho_b"].cpu().numpy(), solid, PHI_S, K, L)


def rel(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev"])
def test_field_matches_oracle_and_refresh_cadence(storage):
    case, solid = walled_cap()
    sim = start(case, solid, storage)
    sim.set_flux_heated(PHI_S, K, L, every=3)
    f0 = sim.flux_field().cpu().numpy()
    want0 = oracle_field(sim, solid)
    assert rel(f0, want0) <= TOL[storage]
    assert f0.max() / f0.min() > 1.5  # the drop's columns see a smaller flux than bare wall
    sim.step(3)  # three steps on the field of the starting state
    assert np.array_equal(sim.flux_field().cpu().numpy(), f0)
    want3 = oracle_field(sim, solid)
    sim.step(1)  # recomputed from the state after three steps, then stepped
    f3 = sim.flux_field().cpu().numpy()
    assert rel(f3, want3) <= TOL[storage]
    assert not np.array_equal(f3, f0)


def test_step_with_heated_field_matches_oracle_step():
    case, solid = walled_cap()
    sim = start(case, solid, "f64", warm=30)
    sim.set_flux_heated(PHI_S, K, L, every=1)
    sim.step(5)
    f_in = sim.populations(torch.float64).cpu().numpy()
    want_field = oracle_field(sim, solid)
    sim.step(1)
    f_out = sim.populations(torch.float64).cpu().numpy()
    led = sim.ledger()
    p = oracle_params(case, phi_field=want_field, solid=solid)
    run = oracle.Run(p, f_in).step(1)
    assert int(run.mask.sum()) > 100
    assert rel(f_out, run.f) <= 1e-12
    removed = float(np.sum(want_field[run.mask != 0])) / case.sbar
    assert led["last_removed"] == pytest.approx(removed, rel=1e-12)


def test_repeatable_and_switched_off_by_scalar_flux():
    case, solid = walled_cap()
    out = []
    for _ in range(2):
        sim = start(case, solid, "f32")
        sim.set_flux_heated(PHI_S, K, L, every=2)
        sim.step(7)
        out.append(sim.populations(torch.float32).cpu().numpy())
    assert np.array_equal(out[0], out[1])
    sim.set_flux(1e-3)
    sim.step(2)
    assert torch.all(sim.flux_field() == 1e-3)


def test_heated_error_paths():
    case, solid = walled_cap()
    sim = start(case, solid, "f64", warm=1)
    for args in [(PHI_S, 0.0, L, 1), (PHI_S, K, 0.0, 1), (PHI_S, K, L, 0), (float("nan"), K, L, 1)]:
        with pytest.raises(CgevapError, match="ARG"):
            sim.set_flux_heated(*args)
    sim.set_flux_heated(PHI_S, K, L, 1)
    with pytest.raises(CgevapError, match="UNSUPPORTED"):
        sim.adjoint_forward(4, 2)
    periodic = Sim.from_case(inputs.sphere_3d(16, R0=4.0), "f32")
    with pytest.raises(CgevapError, match="ARG"):
        periodic.set_flux_heated(PHI_S, K, L, 1)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_field_matches_oracle_2d(storage):
    """D2Q9: the substrate normal is y (walls at both ends of y), columns run along y."""
    shape = (1, 40, 64)
    case = inputs.Case("heated2d", 9, shape, periodic=(1, 0, 1), R0=12.0, phi=0.0)
    sim = Sim.from_case(case, storage)
    sim.set_flux(0.0)
    phase = inputs.sphere_phase(shape, (0.0, -0.5, 31.5), 12.0)
    sim.init_equilibrium(torch.from_numpy(phase).cuda())
    sim.step(15)
    sim.set_flux_heated(PHI_S, K, L, every=2)
    m = sim.macros()
    want = laws.heated_flux_field(m["rho_r"].cpu().numpy(), m["rho_b"].cpu().numpy(), None, PHI_S, K,
                                  L, axis=1)
    got = sim.flux_field().cpu().numpy()
    assert rel(got, want) <= TOL[storage]
    assert got.max() / got.min() > 1.5
