"""What the physics fixes, checked on the GPU path at sizes the oracle would take minutes for.

Laplace's law in 3D: a static drop (flux off) equilibrates to p_in - p_out = 2 sigma / R, with the
pressure of each bulk phase from Eq. (EOS), p = rho zeta (1 - alpha) (unit density ratio), and R
from the liquid volume V = sum (1 + rho^N) / 2 = 4 pi R^3 / 3.  This is the 3D counterpart of the
oracle's 2D pin (test_oracle_physics.py::test_laplace_law_2d) and ties the perturbation amplitude
(9/4) sigma / tau of Eq. (perturb) to sigma in 3D.
"""
import numpy as np
import pytest
import torch

from paper_2412_14859_gb300 import inputs
from paper_2412_14859_gb300.binding import Sim

pytestmark = pytest.mark.gpu


def test_laplace_law_3d():
    n, sigma = 64, 0.05
    zeta, w0 = 0.5, 1.0 / 3.0  # D3Q19: zeta and W_0 = alpha of the least dense component
    vals = []
    for R0 in (12.0, 16.0, 20.0):
        c = inputs.Case("laplace3d", 19, (n, n, n), sigma=sigma, beta=0.99, phi=0.0, R0=R0)
        sim = Sim.from_case(c, "f64")
        sim.set_flux(0.0)
        sim.init_equilibrium(torch.from_numpy(c.phase()).cuda())
        sim.step(4000)
        m = {k: v.cpu().numpy() for k, v in sim.macros().items()}
        rho = m["rho_r"] + m["rho_b"]
        h = n // 2
        p_in = rho[h - 1:h + 1, h - 1:h + 1, h - 1:h + 1].mean() * zeta * (1 - w0)
        p_out = rho[0:2, 0:2, 0:2].mean() * zeta * (1 - w0)
        R = (3.0 * np.sum((1 + m["rhoN"]) / 2) / (4.0 * np.pi)) ** (1.0 / 3.0)
        vals.append((p_in - p_out) * R / (2.0 * sigma))
        sim.close()
    vals = np.array(vals)
    print("laplace 3d: dp R / (2 sigma) =", np.round(vals, 4))
    assert np.all(np.abs(vals - 1.0) < 0.08), vals
    assert vals.max() - vals.min() < 0.05, vals
