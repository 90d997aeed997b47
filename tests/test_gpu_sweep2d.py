"""The D2Q9 drop sweep: a drop of R0 = 40 in a 256^2 periodic box, unit density ratio, tau = 1,
A = 0.01, beta = 0.7, seeded U(+-1e-6) noise, constant flux phi log-spaced over 1e-6..1e-4 (5
values) x band thresholds theta = 0.3 / 0.5 / 0.7, FP64 and FP32 populations -- 30 lattices run
as one ensemble (one persistent launch per call, FP64 and FP32 members together).

S-bar: the band rule selects fewer sites per unit length than the paper's gradient rule, so each
theta gets its S-bar the way Sec. II.B calibrates: the time-averaged number of sites per unit
interface length of a flat-interface run (the 64^2 slab) that itself uses that S-bar, a fixed
point reached by iterating.

- Parity: every member equals the oracle on the same seeded input, with identical site masks
  away from the threshold, after 50 and after 500 steps, within bounds stated for those lengths.
  The method amplifies differences of rounding order over hundreds of steps: the oracle itself,
  compiled with multiply-add contraction, departs from the pinned (uncontracted) build by 1e-13
  after 50 steps of the (phi = 1e-6, theta = 0.3) case and by 4e-11 after 300; the GPU's FP64
  arithmetic (contracted multiply-adds, reciprocal and square-root forms of its own) departs by
  3.7e-12 after 50 steps and up to 1e-9 after 500 (measured).  So FP64 is held to 1e-11 at 50
  steps and 1e-8 at 500, FP32 to the short-case 1e-5 at 50 and 1e-4 at 500.
- Radius law (Sec. III.A, R = R0 - phi t / rho_l, the evaporating drop of the paper in 2D): from
  the equilibrated drop, the two largest fluxes run until the law gives R = R0/2 (2e5 and 6.3e5
  steps), each member paused when it gets there; the radius R = sqrt(V / pi) of the liquid area
  V is compared with the law at R/R0 = 3/4 and 1/2."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from harness import gpu_sim, oracle_summaries, rel_linf
from paper_2412_14859_gb300 import inputs

pytestmark = pytest.mark.gpu

THETAS = (0.3, 0.5, 0.7)
# relative L-inf of the densities against the oracle after 50 and 500 steps
BOUND = {"f64": {50: 1e-11, 500: 1e-8}, "f32": {50: 1e-5, 500: 1e-4}}


def band_sbar(theta: float) -> float:
    """S-bar of the band rule at theta: fixed point of S-bar -> time-averaged sites per unit
    length of a flat-interface run with that S-bar (64^2 slab, two interfaces, flux 1e-3)."""
    case = replace(inputs.flat_slab_2d(), phi=1e-3, threshold=theta)
    sbar = 3.0
    for _ in range(4):
        sim = gpu_sim(replace(case, sbar=sbar), "f64")
        sim.step(2000)
        sbar = sim.ledger()["site_steps"] / 2000 / (2 * case.shape[2])
        sim.close()
    return sbar


@pytest.fixture(scope="module")
def sweep():
    sb = {th: band_sbar(th) for th in THETAS}
    print("band-rule S-bar per theta", sb)
    return [replace(c, sbar=sb[c.threshold]) for c in inputs.drop_2d_sweep()]


def init(ens, cases, flux=True):
    for sim, case in zip(ens.members, cases):
        sim.set_flux(case.phi if flux else 0.0)
        sim.init_equilibrium(torch.from_numpy(case.phase()).cuda(),
                             torch.from_numpy(case.noise_array()).cuda())


def test_sweep_first_500_steps_match_oracle(sweep):
    from paper_2412_14859_gb300.binding import Ensemble
    checkpoints = (50, 500)
    want = oracle_summaries(sweep, checkpoints)  # FP64 and FP32 members share their inputs
    cases = sweep + sweep
    storages = ["f64"] * len(sweep) + ["f32"] * len(sweep)
    ens = Ensemble(cases, storages)
    init(ens, cases)
    worst = {}
    done = 0
    for ci, steps in enumerate(checkpoints):
        ens.step(steps - done)
        done = steps
        ens.status()
        for j, (sim, case, st) in enumerate(zip(ens.members, cases, storages)):
            o = want[j % len(sweep)][ci]
            g = {k: v.cpu().numpy() for k, v in sim.macros().items()}
            err = max(rel_linf(g["rho_r"], o["rho_r"]), rel_linf(g["rho_b"], o["rho_b"]))
            worst[(st, steps)] = max(worst.get((st, steps), 0.0), err)
            if st == "f64":  # no decision within reach of FP64 rounding
                assert o["min_margin"] > 1e-9, (case.phi, case.threshold)
            assert err <= BOUND[st][steps], (st, steps, case.phi, case.threshold, err)
            far = o["margin"] > 1e-6
            assert np.array_equal(sim.mask().cpu().numpy()[far] & 1, o["mask"][far])
            led = sim.ledger()
            assert led["steps"] == steps
            assert led["evaporated"] == pytest.approx(o["evaporated"],
                                                      rel=1e-10 if st == "f64" else 1e-3)
    print("worst relative L-inf (storage, steps):", worst)
    ens.close()


def test_sweep_radius_law_to_half_radius(sweep):
    from paper_2412_14859_gb300.binding import Ensemble
    picked = [c for c in sweep if c.phi > 2e-5]  # phi = 1e-4 and 3.16e-5
    cases = picked + picked
    storages = ["f64"] * len(picked) + ["f32"] * len(picked)
    ens = Ensemble(cases, storages)
    init(ens, cases, flux=False)
    ens.step(3000)  # equilibrate with the flux off
    R0, rho_l = [], []
    for sim in ens.members:
        V = float(sim.volume())
        R0.append(float(np.sqrt(V / np.pi)))
        rho_l.append(float(sim.macros()["rho_r"].max()))
    m_red0 = []
    for sim, case in zip(ens.members, cases):
        sim.set_flux(case.phi)
        sim.reset_ledger()
        m_red0.append(float(sim.macros()["rho_r"].sum()))
    # law time of R/R0 = 3/4 and 1/2 for each member
    marks = [[(1.0 - f) * R0[j] * rho_l[j] / c.phi for f in (0.75, 0.5)] for j, c in enumerate(cases)]
    err = [[None, None] for _ in cases]
    t = 0
    active = set(range(len(cases)))
    while active:
        nxt = min(int(round(marks[j][k])) for j in active for k in (0, 1) if err[j][k] is None)
        k = min(nxt - t, 100000)  # launches of at most 1e5 steps
        ens.step(k)
        t += k
        for j in list(active):
            for k in (0, 1):
                if err[j][k] is None and int(round(marks[j][k])) == t:
                    R = float(np.sqrt(float(ens.members[j].volume()) / np.pi))
                    exact = 1.0 - cases[j].phi * t / (R0[j] * rho_l[j])
                    err[j][k] = (R / R0[j] - exact) / exact * 100.0
            if err[j][1] is not None:
                active.discard(j)
                if active:
                    ens.set_active(j, False)
    ens.status()
    for j, c in enumerate(cases):
        # red mass that left against the FP64 ledger of Eq. (exchange)
        sim = ens.members[j]
        lost = m_red0[j] - float(sim.macros()["rho_r"].sum())
        ratio = lost / sim.ledger()["evaporated"]
        print(f"{storages[j]} phi={c.phi:.3g} theta={c.threshold} sbar={c.sbar:.4f} R0={R0[j]:.2f} "
              f"error at R/R0=3/4: {err[j][0]:+.2f} %, at 1/2: {err[j][1]:+.2f} %, "
              f"red mass lost / ledger - 1 = {ratio - 1:+.2e}")
        if storages[j] == "f64":
            assert abs(ratio - 1) <= 1e-9
        bound = {0.3: (2.0, 3.0), 0.5: (3.5, 10.0), 0.7: (2.0, 4.0)}[c.threshold]
        assert abs(err[j][0]) <= bound[0] and abs(err[j][1]) <= bound[1], (c.phi, c.threshold, err[j])
    ens.close()
