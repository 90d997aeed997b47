"""16-bit deviation storage (FP32 rest populations + FP16 / BF16 deviations of the moving ones,
FP32 arithmetic, FP64 ledger) against the FP64 path on the same seeded inputs.

The stated target for the mixed form is a relative error of the red mass <= 1e-5 against FP64.
The default kernel carries each colour's mass exactly through the step (error-free sums, the
rest pair set to the exact mass), so the bounds here are tighter: 1e-7 for FP16 and 2e-6 for
BF16 (measured on this case: 4.7e-9 and 1.3e-7, both kernel families; returning only the 16-bit
encode loss gave about 1.5e-6).  BF16's 8 mantissa bits show in a looser, stated bound on the
density field.  The ledger (FP64 sum of phi / S-bar over sites) must agree
with FP64 up to sites decided differently near the threshold, and the red mass that left must
match it."""
import numpy as np
import pytest

from harness import gpu_sim, oracle_run, rel_linf
from paper_2412_14859_gb300 import inputs

pytestmark = pytest.mark.gpu

BOUNDS = {  # storage: (relative red-mass error, relative L-inf of rho_r)
    "f16dev": (1e-7, 5e-3),
    "bf16dev": (2e-6, 5e-2),
}


def drop3d():
    return inputs.Case("precision", 19, (40, 44, 48), rho_r_in=10.0, rho_b_in=1.0, tau_b=0.8,
                       sigma=inputs.sigma_from_amplitude(0.005), R0=11.0, phi=1e-5, noise=1e-6)


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
def test_mass_and_density_vs_fp64(storage):
    case = drop3d()
    steps = 300
    ref = gpu_sim(case, "f64")
    ref.step(steps)
    sim = gpu_sim(case, storage)
    sim.step(steps)
    a = {k: v.cpu().numpy() for k, v in sim.macros().items()}
    b = {k: v.cpu().numpy() for k, v in ref.macros().items()}
    mass_err = abs(a["rho_r"].sum() - b["rho_r"].sum()) / b["rho_r"].sum()
    linf = rel_linf(a["rho_r"], b["rho_r"])
    mb, lb = BOUNDS[storage]
    assert mass_err <= mb, mass_err
    assert linf <= lb, linf
    ea, eb = sim.ledger()["evaporated"], ref.ledger()["evaporated"]
    assert ea == pytest.approx(eb, rel=5e-3)
    m0 = case.rho_r_in * (1 + case.phase()).sum() / 2
    lost = m0 - a["rho_r"].sum()
    # the red mass that left matches the FP64 ledger of Eq. (exchange); without the compensated
    # encoding BF16 kept only about half of it
    assert lost == pytest.approx(ea, rel=0.05)


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("q,shape", [(9, (1, 36, 70)), (19, (9, 13, 22))])
def test_encode_decode_round_trip(storage, q, shape):
    import torch
    case = inputs.Case("roundtrip", q, shape, R0=4.0, noise=1e-6, rho_r_in=5.0)
    sim = gpu_sim(case, storage)
    f32 = gpu_sim(case, "f64")
    got = sim.populations().cpu().numpy()
    want = f32.populations().cpu().numpy()
    # rest populations are FP32; deviations carry the 16-bit rounding
    eps = 2.0 ** -11 if storage == "f16dev" else 2.0 ** -8
    assert np.max(np.abs(got[:, 0] - want[:, 0])) <= 1e-6 * np.max(np.abs(want[:, 0]))
    assert np.max(np.abs(got - want)) <= 4 * eps * np.max(np.abs(want))
    # set_populations -> get_populations keeps the same values (encode is idempotent on decode)
    sim.set_populations(torch.from_numpy(got).cuda())
    again = sim.populations().cpu().numpy()
    assert np.max(np.abs(again - got)) <= 2 * eps * np.max(np.abs(want))


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("q,shape", [(9, (1, 40, 130)), (19, (12, 21, 37))])
def test_one_step_matches_oracle_within_storage_rounding(storage, q, shape):
    """One step from the same initial state: the 16-bit path differs from the oracle only by the
    storage rounding of the deviations (|deviation| <~ 0.1 at the interface)."""
    case = inputs.Case("onestep", q, shape, R0=5.0, noise=1e-6, phi=1e-5, rho_r_in=2.0)
    run = oracle_run(case, 1)
    sim = gpu_sim(case, storage)
    sim.step(1)
    g = sim.macros()
    tol = 2e-4 if storage == "f16dev" else 2e-3
    assert rel_linf(g["rho_r"].cpu().numpy(), run.macros()["rho_r"]) <= tol
    assert rel_linf(g["rho_b"].cpu().numpy(), run.macros()["rho_b"]) <= tol
    far = run.margin > 1e-4
    assert np.array_equal(sim.mask().cpu().numpy()[far] & 1, run.mask[far])


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("q,shape,nvar", [(9, (1, 40, 130), 2), (19, (12, 21, 37), 5)])
def test_every_variant_within_storage_rounding(storage, q, shape, nvar):
    case = inputs.Case("variants", q, shape, R0=5.0, noise=1e-6, phi=1e-5, rho_r_in=2.0)
    run = oracle_run(case, 3)
    tol = 5e-4 if storage == "f16dev" else 5e-3
    for v in range(nvar):
        sim = gpu_sim(case, storage)
        sim.tune(0, v)
        sim.step(3)
        g = sim.macros()
        assert rel_linf(g["rho_r"].cpu().numpy(), run.macros()["rho_r"]) <= tol, v
        assert rel_linf(g["rho_b"].cpu().numpy(), run.macros()["rho_b"]) <= tol, v
