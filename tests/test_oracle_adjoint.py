"""Pins of the oracle's FP64 autograd statement of the step (oracle/adjoint_ref.py).

The derivative that the library's hand-written adjoint must reproduce is taken by torch.autograd
through a whole-lattice restatement of the step; these tests tie that restatement to things other
than itself:
  - its states equal the C oracle's, step for step (the C oracle is pinned by the physics tests);
  - the C oracle's "given" site rule replays a recorded run bit for bit;
  - its gradient equals central finite differences of the C oracle replaying the same site sets
    (Eq. exchange with x_I held fixed), along random directions of the flux field;
  - for one step it equals the closed form dV(1)/dphi(x) = -m(x) / (rho(x) S-bar): the exchange
    moves phi/S-bar from red to blue at constant rho, and dV/d(rho_r - rho_b) = 1/(2 rho) per cell.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from harness import adjoint_case as case_params
from oracle import adjoint_ref as AR
from paper_2412_14859_gb300 import inputs


STEPS = {9: 8, 19: 6}


@pytest.mark.parametrize("q", [9, 19])
def test_torch_states_equal_c_oracle(q):
    p, f0, phi = case_params(q)
    run = oracle.Run(p, f0)
    ref, sites = [], []
    for _ in range(STEPS[q]):
        run.step(1)
        ref.append(run.f.copy())
        sites.append(run.mask.copy())
    assert sum(int(s.sum()) for s in sites) > 0
    got = AR.states(p, f0, phi, sites)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


@pytest.mark.parametrize("q", [9, 19])
def test_given_rule_replays_run_exactly(q):
    p, f0, phi = case_params(q)
    run = oracle.Run(p, f0)
    sites = []
    for _ in range(STEPS[q]):
        run.step(1)
        sites.append(run.mask.copy())
    rp = dataclasses.replace(p, site_rule=oracle.RULE_GIVEN, mask_given=np.zeros(p.shape, np.uint8))
    rep = oracle.Run(rp, f0)
    for m in sites:
        rep.p.mask_given = m
        rep.step(1)
    assert np.array_equal(rep.f, run.f)
    assert rep.evaporated == run.evaporated


@pytest.mark.parametrize("q", [9, 19])
def test_autograd_gradient_matches_central_differences_of_c_oracle(q):
    p, f0, phi = case_params(q)
    T = STEPS[q]
    sites = AR.record_sites(p, f0, T)
    w = inputs.rng(inputs.SEED + 11).normal(size=T + 1)
    ph = torch.tensor(phi, requires_grad=True)
    V = AR.volume_history(p, f0, ph, sites)
    (V * torch.from_numpy(w)).sum().backward()
    grad = ph.grad.numpy()
    assert np.count_nonzero(grad) > 0
    g = inputs.rng(inputs.SEED + 12)
    for _ in range(3):
        d = g.uniform(-1.0, 1.0, size=phi.shape) * 1e-3
        eps = 1e-3
        Lp = float(w @ AR.replay_volumes(p, f0, phi + eps * d, sites))
        Lm = float(w @ AR.replay_volumes(p, f0, phi - eps * d, sites))
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(grad * d))
        assert ad == pytest.approx(fd, rel=1e-7, abs=1e-15)


@pytest.mark.parametrize("q", [9, 19])
def test_one_step_gradient_closed_form(q):
    p, f0, phi = case_params(q)
    run = oracle.Run(p, f0).step(1)
    site = run.mask.copy()
    ph = torch.tensor(phi, requires_grad=True)
    V = AR.volume_history(p, f0, ph, [site])
    V[1].backward()
    m = run.macros()
    rho = m["rho_r"] + m["rho_b"]
    fluid = np.ones(p.shape, bool) if p.solid is None else p.solid == 0
    want = np.where((site != 0) & fluid, -1.0 / (np.where(fluid, rho, 1.0) * p.sbar), 0.0)
    assert np.count_nonzero(want) > 0
    assert np.max(np.abs(ph.grad.numpy() - want)) <= 1e-14 * np.max(np.abs(want))
