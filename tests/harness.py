"""Shared helpers of the tests: build the oracle's and the CUDA path's inputs from one seeded
`inputs.Case`, run both, and compare.  Nothing here computes the method itself."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2412_14859_gb300 import inputs


def oracle_params(case: inputs.Case, phi_field=None, solid=None) -> oracle.Params:
    nz, ny, nx = case.shape
    return oracle.Params(q=case.q, nx=nx, ny=ny, nz=nz, periodic=tuple(case.periodic),
                         rho_r_in=case.rho_r_in, rho_b_in=case.rho_b_in, tau_r=case.tau_r,
                         tau_b=case.tau_b, sigma=case.sigma, beta=case.beta,
                         site_rule=case.site_rule, threshold=case.threshold, sbar=case.sbar,
                         phi=case.phi, phi_field=phi_field, solid=solid)


def oracle_run(case: inputs.Case, steps: int, phi_field=None, solid=None):
    p = oracle_params(case, phi_field, solid)
    run = oracle.Run(p, oracle.init(p, case.phase(), case.noise_array()))
    run.step(steps)
    return run


def gpu_sim(case: inputs.Case, storage: str, phi_field=None, solid=None, kernel=None):
    """A simulation on the GPU; storage may carry a kernel family as "f32:tma" / "f32:reg"."""
    import torch
    from paper_2412_14859_gb300.binding import Sim
    if ":" in storage:
        storage, kernel = storage.split(":")
    sim = Sim.from_case(case, storage)
    if kernel is not None:
        sim.tune({"reg": 0, "tma": 1}[kernel])
    if solid is not None:
        sim.set_solid(torch.from_numpy(np.ascontiguousarray(solid, np.uint8)).cuda())
    if phi_field is not None:
        sim.set_flux(case.phi, torch.from_numpy(np.ascontiguousarray(phi_field)).cuda())
    else:
        sim.set_flux(case.phi)
    rn = torch.from_numpy(case.phase()).cuda()
    nz = case.noise_array()
    sim.init_equilibrium(rn, None if nz is None else torch.from_numpy(nz).cuda())
    return sim


def adjoint_case(q, bulk=False):
    """Small lattice with sites, walls and (3D) one solid cell, a seeded flux field and a noisy
    initial state: (oracle params, f0, phi field).  bulk: a D2Q9 box large enough that its far
    field holds cells where one colour is a trace (w_r w_b < 1e-6)."""
    if q == 9 and bulk:
        shape = (1, 40, 64)
        per = (1, 0, 1)
        phase = inputs.sphere_phase(shape, (0.0, 19.5, 31.5), 8.0)
    elif q == 9:  # D2Q9 drop touching nothing, walls across y
        shape = (1, 14, 17)
        per = (1, 0, 1)
        phase = inputs.sphere_phase(shape, (0.0, 6.5, 8.0), 4.5)
    else:       # D3Q19 cap on the z = -1/2 wall, walls at both ends of z, one solid cell
        shape = (8, 9, 10)
        per = (1, 1, 0)
        phase = inputs.sphere_phase(shape, (-0.5, 4.0, 4.5), 4.2)
    solid = None
    if q == 19:
        solid = np.zeros(shape, np.uint8)
        solid[5, 1, 1] = 1
    phi = 2e-3 * (1.0 + inputs.uniform_noise(shape, 0.3, seed=inputs.SEED + 7))
    nz, ny, nx = shape
    p = oracle.Params(q, nx, ny, nz, per, rho_r_in=1.0, rho_b_in=1.0, tau_r=1.0, tau_b=0.8,
                      sigma=inputs.sigma_from_amplitude(0.01), beta=0.7,
                      site_rule=oracle.RULE_BAND, threshold=0.5, sbar=3.0, phi_field=phi,
                      solid=solid)
    noise = inputs.uniform_noise((2, q) + shape, 1e-6)
    f0 = oracle.init(p, phase, noise)
    return p, f0, phi


def rel_linf(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def oracle_summary(case: inputs.Case, checkpoints) -> list:
    """What the parity tests compare, after each of the (increasing) step counts in `checkpoints`
    of one oracle run of a case (picklable; runs in a worker process)."""
    p = oracle_params(case)
    run = oracle.Run(p, oracle.init(p, case.phase(), case.noise_array()))
    out = []
    for n in checkpoints:
        run.step(n - run.steps)
        m = run.macros()
        out.append({"steps": n, "rho_r": m["rho_r"], "rho_b": m["rho_b"], "mask": run.mask.copy(),
                    "margin": run.margin.copy(), "evaporated": run.evaporated,
                    "site_steps": run.ledger.site_steps, "min_margin": min(run.min_margin_history)})
    return out


def oracle_summaries(cases, checkpoints, workers: int = 0) -> list:
    """oracle_summary of many cases in a pool of spawned processes (never forked: the parent may
    hold a CUDA context)."""
    import concurrent.futures
    import multiprocessing
    import os
    n = workers or max(1, min(len(cases), os.cpu_count() or 1))
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(n, mp_context=ctx) as ex:
        return list(ex.map(oracle_summary, cases, [tuple(checkpoints)] * len(cases)))
