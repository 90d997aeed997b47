"""The hand-written adjoint (cgevap_adjoint_forward / _backward, autograd.Function) on the GPU.

- against the oracle's FP64 autograd derivative on small lattices with walls, a solid cell and a
  flux field, several checkpoint segments (FP64: 1e-10 of the largest entry; FP32: 2e-3);
- the flux-fit gradient dL/da_k of the 16 polynomial coefficients against central finite
  differences (h = 1e-3) of runs that replay the base run's site sets (CGEVAP_SITES_GIVEN), on a
  reduced sessile cap (FP64; bound 1e-4 of the largest component);
- FP32 against FP64 on the same problem, and the error paths.
"""
import numpy as np
import pytest
import torch

from harness import adjoint_case
from oracle import adjoint_ref as AR
from paper_2412_14859_gb300 import inputs
from paper_2412_14859_gb300.adjoint import volume_history
from paper_2412_14859_gb300.binding import SITES_BAND, SITES_GIVEN, CgevapError, Sim

pytestmark = pytest.mark.gpu

STEPS = {9: 8, 19: 6}


def sim_for(p, storage, rule=None):
    sim = Sim(p.q, p.nx, p.ny, p.nz, tuple(p.periodic), p.rho_r_in, p.rho_b_in, p.tau_r, p.tau_b,
              p.sigma, p.beta, p.site_rule if rule is None else rule, p.threshold, p.sbar, storage)
    if p.solid is not None:
        sim.set_solid(torch.from_numpy(np.ascontiguousarray(p.solid, np.uint8)).cuda())
    return sim


@pytest.mark.parametrize("q,bulk", [(9, False), (19, False), (9, True)])
@pytest.mark.parametrize("storage,tol,vtol", [("f64", 1e-10, 1e-13), ("f32", 2e-3, 1e-6)])
def test_adjoint_matches_autograd_oracle(q, bulk, storage, tol, vtol):
    p, f0, phi = adjoint_case(q, bulk)
    T = 24 if bulk else STEPS[q]
    if bulk:  # the far field holds trace cells, where the recoloring direction is held fixed
        rr, rb = f0[0].sum(0), f0[1].sum(0)
        assert np.count_nonzero(rr * rb / (rr + rb) ** 2 < AR.BULK_TRACE) > 100
    sites = AR.record_sites(p, f0, T)
    w = inputs.rng(inputs.SEED + 21).normal(size=T + 1)
    ph = torch.tensor(phi, requires_grad=True)
    V = AR.volume_history(p, f0, ph, sites)
    (V * torch.from_numpy(w)).sum().backward()
    want = ph.grad.numpy()

    sim = sim_for(p, storage)
    sim.set_flux(0.0, torch.from_numpy(phi).cuda())
    sim.set_populations_host(np.ascontiguousarray(f0))
    Vg = sim.adjoint_forward(T, 3).cpu().numpy()  # segments of 3, 3 and the rest
    # equal volumes at every step mean equal site sets (one site moves V by ~phi/S-bar)
    assert np.max(np.abs(Vg - V.detach().numpy())) <= vtol * np.max(np.abs(Vg))
    got = sim.adjoint_backward(torch.from_numpy(w).cuda()).cpu().numpy()
    assert np.count_nonzero(want) > 0
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert np.all(got[want == 0] == 0)
    again = sim.adjoint_backward(torch.from_numpy(w).cuda()).cpu().numpy()
    assert np.array_equal(got, again)  # the sweep is deterministic and repeatable


def cap_problem(storage, shape=(32, 64, 64), R0=12.0, K=16):
    case = inputs.sessile_cap_3d(shape, R0=R0, phi0=2e-5)
    nz, ny, nx = shape
    basis = torch.from_numpy(inputs.radial_basis(shape, ((ny - 1) / 2.0, (nx - 1) / 2.0), R0, K)).cuda()
    a, a_t = inputs.flux_fit_parameters(K)
    return case, basis, a, a_t


def flux(case, basis, a):
    return case.phi * (1.0 + torch.tensordot(a, basis, dims=1))


def fresh(case, storage, rule=None):
    sim = Sim.from_case(case, storage)
    if rule is not None:
        sim = Sim(case.q, case.shape[2], case.shape[1], case.shape[0], case.periodic, case.rho_r_in,
                  case.rho_b_in, case.tau_r, case.tau_b, case.sigma, case.beta, rule, case.threshold,
                  case.sbar, storage)
    sim.init_equilibrium(torch.from_numpy(case.phase()).cuda())
    return sim


def loss(V, dVt):
    return ((V[0] - V[1:] - dVt) ** 2).sum()


def fit_gradient(case, basis, a, a_t, storage, T, ckpt):
    st = fresh(case, storage)
    st.set_flux(0.0, flux(case, basis, torch.tensor(a_t).cuda()).contiguous())
    Vt = st.adjoint_forward(T, ckpt)
    dVt = (Vt[0] - Vt[1:]).detach()
    sim = fresh(case, storage)
    at = torch.tensor(a, device="cuda", requires_grad=True)
    V = volume_history(sim, flux(case, basis, at), T, ckpt)
    L = loss(V, dVt)
    L.backward()
    return at.grad.cpu().numpy(), float(L.detach()), dVt, V.detach()


@pytest.mark.parametrize("shape,R0,T,ckpt", [((32, 64, 64), 12.0, 200, 64),
                                             ((128, 256, 256), 48.0, 256, 16)],
                         ids=["reduced_64x64x32", "full_256x256x128"])
def test_flux_fit_gradient_matches_central_differences(shape, R0, T, ckpt):
    """The 16-coefficient flux-fit gradient of the reverse sweep against central differences
    (h = 1e-3) of the forward run with its site sets replayed, FP64: on a reduced cap and on the
    full 256x256x128 box of the sessile-cap workload (R0 = 48, 256 steps)."""
    case, basis, a, a_t = cap_problem("f64", shape, R0)
    grad, L0, dVt, V0 = fit_gradient(case, basis, a, a_t, "f64", T, ckpt)
    # the base run's site sets, step by step
    rec = fresh(case, "f64")
    rec.set_flux(0.0, flux(case, basis, torch.tensor(a).cuda()).contiguous())
    masks = []
    for _ in range(T):
        rec.step(1)
        masks.append(rec.mask().clone())
    assert sum(int((m & 1).sum()) for m in masks) > 1000
    rep = fresh(case, "f64", SITES_GIVEN)

    def replay(av):
        rep.init_equilibrium(torch.from_numpy(case.phase()).cuda())
        rep.set_flux(0.0, flux(case, basis, torch.tensor(av).cuda()).contiguous())
        V = [rep.volume()]
        for m in masks:
            rep.set_mask(m)
            rep.step(1)
            V.append(rep.volume())
        return torch.cat(V)

    Vr = replay(a)
    assert torch.equal(Vr, V0)  # the replay is the base run, bit for bit
    h = 1e-3
    fd = np.empty_like(grad)
    for k in range(len(a)):
        e = np.zeros_like(a)
        e[k] = h
        fd[k] = (float(loss(replay(a + e), dVt)) - float(loss(replay(a - e), dVt))) / (2 * h)
    err = np.max(np.abs(grad - fd)) / np.max(np.abs(fd))
    print(f"{shape}: adjoint vs central differences {err:.2e}")
    assert err <= 1e-4, (err, grad, fd)
    del masks
    torch.cuda.empty_cache()


def test_fp32_adjoint_close_to_fp64():
    case, basis, a, a_t = cap_problem("f32")
    g64, _, _, _ = fit_gradient(case, basis, a, a_t, "f64", 100, 32)
    g32, _, _, _ = fit_gradient(case, basis, a, a_t, "f32", 100, 32)
    assert np.max(np.abs(g32 - g64)) <= 1e-2 * np.max(np.abs(g64))


def test_adjoint_error_paths():
    p, f0, phi = adjoint_case(9)
    sim = sim_for(p, "f16dev")
    sim.set_populations_host(np.ascontiguousarray(f0))
    with pytest.raises(CgevapError, match="UNSUPPORTED"):
        sim.adjoint_forward(4, 2)
    sim = sim_for(p, "f64")
    with pytest.raises(CgevapError, match="ARG"):
        sim.adjoint_backward(None)  # nothing recorded
    with pytest.raises(CgevapError, match="ARG"):
        sim.adjoint_forward(0, 2)
    sim.adjoint_forward(4, 2)
    sim.adjoint_release()
    with pytest.raises(CgevapError, match="ARG"):
        sim.adjoint_backward(None)
    s32 = sim_for(p, "f32")
    s32.tune(1)  # the TMA step
    with pytest.raises(CgevapError, match="UNSUPPORTED"):
        s32.adjoint_forward(4, 2)


def test_volume_matches_macros():
    p, f0, phi = adjoint_case(19)
    sim = sim_for(p, "f64")
    sim.set_populations_host(np.ascontiguousarray(f0))
    sim.step(3)
    m = sim.macros()
    fluid = torch.from_numpy(p.solid == 0).cuda()
    want = float((0.5 * (1.0 + m["rhoN"]))[fluid].sum())
    assert float(sim.volume()) == pytest.approx(want, rel=1e-14)
