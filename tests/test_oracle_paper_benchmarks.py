"""The oracle against numbers the paper prints.

Sec. III.A.1 runs a flat interface on a 4x128x4 lattice and reports the error of the interface
position against h(t) = h0 - (phi/rho0) t at two normalised times, for two thresholds Gamma
(also Tab. fbar).  The oracle, run on the same setup, must reproduce those errors.  This pins
every part of the step at once: lattice constants, Eq. (perturb) amplitude, Eq. (recolor),
the previous-step |F| > Gamma site rule and Eq. (exchange) with S-bar = 3.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2412_14859_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "flat_interface.json")


def interface_height(run):
    """Distance from the wall (y = -1/2) to where rho_r falls to half its maximum."""
    rr = run.macros()["rho_r"].mean(axis=(0, 2))
    half = 0.5 * rr.max()
    j = int(np.argmax(rr < half))
    s = (j - 1) + (rr[j - 1] - half) / (rr[j - 1] - rr[j])
    return s + 0.5


def flat_run(Gamma):
    shape = (4, 128, 4)
    p = oracle.Params(q=19, nx=4, ny=128, nz=4, periodic=(1, 0, 1), sigma=0.1, beta=0.99,
                      site_rule=oracle.RULE_GRADIENT, threshold=Gamma, sbar=3.0, phi=0.0)
    run = oracle.Run(p, oracle.init(p, inputs.half_space_phase(shape, 1, 79.5)))
    # Sec. III: equilibrate with the flux off until the velocity field settles to 1e-7.
    prev = None
    for _ in range(50):
        run.step(100)
        u = run.macros()["u"]
        if prev is not None and np.abs(u - prev).max() < 1e-7:
            break
        prev = u
    return p, run


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"],
                         ids=lambda c: f"Gamma{c['Gamma']}")
def test_flat_interface_errors_match_paper(case):
    p, run = flat_run(case["Gamma"])
    h0 = interface_height(run)
    rho0 = run.macros()["rho_r"].mean(axis=(0, 2))[10]
    assert h0 == pytest.approx(80.0, abs=0.5)
    te = h0 * rho0 / case["phi"]
    p.phi = case["phi"]
    t = 0
    for ts, paper_err in zip(case["t_star"], case["error_percent"]):
        n = int(round(ts * te)) - t
        run.step(n)
        t += n
        exact = 1.0 - t / te
        err = abs(interface_height(run) / h0 - exact) / exact * 100.0
        assert abs(err - paper_err) < 0.3, (ts, err, paper_err)
    # mass bookkeeping of Eq. (exchange) over the whole run
    m = run.macros()
    assert run.evaporated > 0
    assert np.isclose(m["rho_r"].sum() + run.evaporated, 80.0 * 16 * rho0, rtol=2e-3)


def mean_sbar(p, run, Gamma, phi=0.03):
    """Time-averaged sites per step per unit interface area of an evaporation run from the
    equilibrated state to t* = 1/2 (Eq. satisfy: this is S-bar when the mass-loss rate is right)."""
    import copy
    q = copy.copy(p)
    q.threshold, q.phi = Gamma, phi
    r = oracle.Run(q, run.f)
    r.G = run.G.copy()
    steps = int(round(0.5 * 79.5 / phi))
    r.step(steps)
    return r.ledger.site_steps / steps / (p.nx * p.nz)


def test_paper_thresholds_bracket_sbar_3():
    """Sec. III.A.1 finds Gamma = 0.31 accurate on the flat interface and 0.305 slightly too low
    (more mass lost): with S-bar = 3 the mean site count per unit area brackets 3 there."""
    p, run = flat_run(0.31)
    hi, lo = mean_sbar(p, run, 0.305), mean_sbar(p, run, 0.31)
    assert hi > 3.0 > lo
    assert hi - lo < 0.1
