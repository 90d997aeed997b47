"""The blue pressure outlets (cgevap_set_outlets; Sec. III.B.2) on the GPU.

- runs of a density-contrast drop (gamma = 2) with outlets at both ends of the wall-normal axis
  equal the oracle's runs (FP64 <= 1e-12, FP32 <= 1e-5, both kernel families), 2D and 3D;
- one step of every storage from a common state equals the oracle's step from that state within
  the storage's output rounding;
- after each step the outlet planes hold the prescribed blue density; red sees a wall;
- error paths.
"""
import numpy as np
import pytest
import torch

import oracle
from harness import gpu_sim, oracle_params, rel_linf
from paper_2412_14859_gb300 import inputs
from paper_2412_14859_gb300.binding import CgevapError

pytestmark = pytest.mark.gpu

OUT = (1.0, 1.1)


def case(q):
    if q == 19:
        shape, per, R0 = (20, 20, 37), (1, 1, 0), 5.0
    else:
        shape, per, R0 = (1, 40, 70), (1, 0, 1), 9.0
    return inputs.Case(f"outlet{q}", q, shape, periodic=per, R0=R0, rho_r_in=2.0, noise=1e-6,
                       phi=1e-5, sigma=0.1, beta=0.99)


def oracle_run(c, steps):
    p = oracle_params(c)
    p.outlet_rho = OUT
    run = oracle.Run(p, oracle.init(p, c.phase(), c.noise_array()))
    run.step(steps)
    return p, run


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32:reg", 1e-5), ("f32:tma", 1e-5)])
@pytest.mark.parametrize("q", [9, 19])
def test_run_matches_oracle(q, storage, tol):
    c = case(q)
    steps = 20
    _, run = oracle_run(c, steps)
    sim = gpu_sim(c, storage)
    sim.set_outlets(*OUT)
    sim.step(steps)
    g = {k: v.cpu().numpy() for k, v in sim.macros().items()}
    o = run.macros()
    assert rel_linf(g["rho_r"], o["rho_r"]) <= tol
    assert rel_linf(g["rho_b"], o["rho_b"]) <= tol
    assert np.max(np.abs(g["u"] - o["u"])) <= 10 * tol
    if storage == "f64":
        assert rel_linf(sim.populations().cpu().numpy(), run.f) <= tol
    ax = 0 if q == 19 else 1
    for plane, rho in ((0, OUT[0]), (-1, OUT[1])):
        assert np.max(np.abs(np.take(g["rho_b"], plane, axis=ax) - rho)) <= 10 * tol


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-6), ("f16dev", 2e-4), ("bf16dev", 2e-3)])
@pytest.mark.parametrize("q", [9, 19])
def test_one_step_from_common_state(q, storage, tol):
    c = case(q)
    p, run = oracle_run(c, 12)
    sim = gpu_sim(c, storage)
    sim.set_outlets(*OUT)
    sim.set_populations(torch.from_numpy(np.ascontiguousarray(run.f)).cuda())
    f_in = sim.populations().cpu().numpy()  # the state as stored (16-bit storage rounds it)
    sim.step(1)
    got = sim.populations().cpu().numpy()
    want = oracle.Run(p, f_in).step(1).f
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol


def test_red_mass_is_kept_and_blue_flows():
    c = case(19)
    sim = gpu_sim(c, "f64")
    sim.set_flux(0.0)
    sim.set_outlets(1.0, 1.0)
    m0 = sim.macros()
    sim.step(40)
    m1 = sim.macros()
    r0, r1 = float(m0["rho_r"].sum()), float(m1["rho_r"].sum())
    assert r1 == pytest.approx(r0, rel=1e-13)
    assert abs(float(m1["rho_b"].sum()) - float(m0["rho_b"].sum())) > 1e-6


def test_outlet_error_paths():
    sim = gpu_sim(case(19), "f64")
    with pytest.raises(CgevapError, match="ARG"):
        sim.set_outlets(float("nan"), 1.0)
    sim.set_outlets(1.0, 0.0)
    with pytest.raises(CgevapError, match="UNSUPPORTED"):
        sim.adjoint_forward(2, 1)
    sim.set_outlets(0.0, 0.0)
    sim.adjoint_forward(2, 1)  # outlets off again
    periodic = gpu_sim(inputs.sphere_3d(16, R0=4.0), "f32")
    with pytest.raises(CgevapError, match="ARG"):
        periodic.set_outlets(1.0, 1.0)
    periodic.set_outlets(0.0, -1.0)  # walls at both ends: nothing to check
