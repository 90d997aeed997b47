"""Failure paths of the library, exercised without faulting or hanging the GPU.

- Health check: a non-finite population or a non-positive density written from the host through
  cgevap_set_populations is reported as CGEVAP_ERR_NAN; a healthy state reports OK.
- Checkpoint restart: n steps, save, load into a fresh handle, m steps equals n + m straight steps
  bit for bit in every storage.
- Bounded waits: the ensemble's grid barrier gives up after the limit set from the host.  A test
  hook makes one CTA skip its arrival, so the other CTAs' bounded wait runs out; the launch ends,
  cgevap_ensemble_status reports CGEVAP_ERR_TIMEOUT, and the next launch with the hook off runs
  normally and gives the standalone result.  No wait is unbounded and no memory is touched out
  of turn: the hook only withholds an atomic increment."""
import time

import numpy as np
import pytest
import torch

from harness import gpu_sim
from paper_2412_14859_gb300 import inputs

pytestmark = pytest.mark.gpu

STORAGES = ["f64", "f32", "f16dev", "bf16dev", "f32rc", "f16rc", "bf16rc", "f32x"]


def small_drop(q):
    shape = (10, 17, 35) if q == 19 else (1, 33, 70)
    return inputs.Case(f"fail{q}", q, shape, R0=4.5 if q == 19 else 9.0, noise=1e-6, phi=1e-5)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("q", [9, 19])
def test_health_reports_bad_populations(q, storage):
    from paper_2412_14859_gb300.binding import CgevapError
    case = small_drop(q)
    sim = gpu_sim(case, storage)
    sim.step(2)
    sim.check_health()  # healthy
    f = sim.populations(torch.float64)
    cell = (0, 5, 3 if q == 19 else 0, 4, 7)  # [k][i][z][y][x]
    for bad in (float("nan"), float("inf")):
        g = f.clone()
        g[cell] = bad
        sim.set_populations(g)
        with pytest.raises(CgevapError, match="NAN"):
            sim.check_health()
        sim.step(1)  # the bad value is carried into the storage's own layout
        with pytest.raises(CgevapError, match="NAN"):
            sim.check_health()
    g = f.clone()
    g[:, :, 0, 3, 5] = 0.0  # an empty cell: non-positive density
    sim.set_populations(g)
    with pytest.raises(CgevapError, match="NAN"):
        sim.check_health()
    sim.set_populations(f)
    sim.check_health()
    sim.close()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("q", [9, 19])
def test_checkpoint_restart_is_bit_exact(q, storage, tmp_path):
    case = small_drop(q)
    n, m = 6, 9
    sim = gpu_sim(case, storage)
    sim.step(n)
    path = str(tmp_path / "c.ckpt")
    sim.save(path)
    sim.step(m)
    straight = sim.populations(torch.float64).cpu().numpy()
    mask = sim.mask().cpu().numpy()
    led = sim.ledger()
    other = gpu_sim(case, storage)
    other.step(1)  # the handle holds another state before the load
    other.load(path)
    other.step(m)
    assert np.array_equal(other.populations(torch.float64).cpu().numpy(), straight)
    assert np.array_equal(other.mask().cpu().numpy(), mask)
    assert other.ledger() == led
    sim.close()
    other.close()


def _members():
    return [inputs.Case("t0", 9, (1, 64, 96), R0=14.0, noise=1e-6, phi=1e-4),
            inputs.Case("t1", 9, (1, 40, 128), R0=9.0, noise=1e-6, phi=3e-5),
            inputs.Case("t2", 19, (24, 26, 28), R0=6.0, noise=1e-6, phi=2e-5,
                        sigma=inputs.sigma_from_amplitude(0.005))]


def _init(ens, cases):
    for sim, case in zip(ens.members, cases):
        sim.set_flux(case.phi)
        sim.init_equilibrium(torch.from_numpy(case.phase()).cuda(),
                             torch.from_numpy(case.noise_array()).cuda())


def test_ensemble_barrier_timeout_is_reported_and_recovers():
    from paper_2412_14859_gb300.binding import CgevapError, Ensemble
    cases = _members()
    ens = Ensemble(cases)
    _init(ens, cases)
    ens.step(2)
    ens.status()
    assert ens.grid >= 2
    ens.set_barrier_timeout(50)
    ens.debug_skip_arrival(ens.grid - 1, 1)  # the last CTA withholds its arrival after step 1
    t0 = time.perf_counter()
    ens.step(5)
    with pytest.raises(CgevapError, match="TIMEOUT"):
        ens.status()
    dt = time.perf_counter() - t0
    assert dt < 3.0, dt  # each remaining wait gives up after 50 ms
    ens.status()  # the flag was cleared by the report
    # hook off: a fresh start runs normally and equals standalone runs of the members
    ens.debug_skip_arrival(-1)
    ens.set_barrier_timeout(4000)
    _init(ens, cases)
    ens.step(7)
    ens.status()
    for sim, case in zip(ens.members, cases):
        ref = gpu_sim(case, "f32")
        ref.step(7)
        a, b = sim.populations(torch.float64), ref.populations(torch.float64)
        assert (a - b).abs().max().item() <= 1e-5 * b.abs().max().item(), case.name
        assert sim.ledger()["steps"] == 7
        ref.close()
    ens.close()


def test_ensemble_rejects_bad_hook_and_timeout():
    from paper_2412_14859_gb300.binding import CgevapError, Ensemble
    cases = _members()[:2]
    ens = Ensemble(cases)
    with pytest.raises(CgevapError, match="ARG"):
        ens.set_barrier_timeout(0)
    with pytest.raises(CgevapError, match="ARG"):
        ens.debug_skip_arrival(0, -1)
    ens.close()
