"""cgevap_step_static_scratch -- the one timestep entry point that allocates nothing.

It exists for callers that cannot allocate device memory (a framework that owns every buffer and
forbids allocation inside its operators, such as a custom call in an XLA/JAX program, or an
application arena with a fixed budget).  Its per-block scratch is a static device array inside
the library.  This test drives it through the C ABI on buffers the test owns, starting from a
state produced by the handle API, and checks two calls in a row against cgevap_step on the same
state, within the parity tolerances of the other GPU tests.  The file is named to be collected
last, so a failure here cannot hide failures of the other tests."""
import ctypes
import os

import numpy as np
import pytest

from harness import gpu_sim
from paper_2412_14859_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
# checkpoint: magic, version, params, phi, flags, ledger, layout flag
HEADER = 8 + 4 + 112 + 8 + 4 + 4 + 40 + 4


def read_checkpoint(sim, path, ncell):
    sim.save(path)
    raw = open(path, "rb").read()
    ledger = raw[HEADER - 44:HEADER - 4]
    state = raw[HEADER:len(raw) - ncell]
    mask = raw[len(raw) - ncell:]
    return state, mask, ledger


def ledger_fields(b):
    ev, last, = np.frombuffer(b[:16], np.float64)
    site_steps, last_sites, steps = np.frombuffer(b[16:40], np.int64)
    return float(ev), float(last), int(site_steps), int(last_sites), int(steps)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_static_scratch_step_matches_handle_step(storage, tmp_path):
    import torch
    from paper_2412_14859_gb300 import binding

    lib = binding.lib()
    case = inputs.Case("noalloc", 19, (12, 21, 37), R0=5.0, noise=1e-6, phi=1e-5)
    sim = gpu_sim(case, storage)
    sim.step(3)
    path = str(tmp_path / "state.ckpt")
    state, mask, ledger = read_checkpoint(sim, path, case.ncell)

    buf = [torch.from_numpy(np.frombuffer(state, np.uint8).copy()).cuda() for _ in range(3)]
    msk = [torch.from_numpy(np.frombuffer(mask, np.uint8).copy()).cuda() for _ in range(3)]
    led = torch.from_numpy(np.frombuffer(ledger, np.uint8).copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    dt = np.float32 if storage == "f32" else np.float64
    for call in (1, 2):
        src, dst = buf[call - 1], buf[call]
        rc = lib.cgevap_step_static_scratch(
            ctypes.byref(sim.params), case.phi, src.data_ptr(), dst.data_ptr(), src.numel(),
            msk[call - 1].data_ptr(), msk[call].data_ptr(), led.data_ptr(), stream)
        assert rc == 0
        sim.step(1)
        ref_state, ref_mask, ref_ledger = read_checkpoint(sim, path, case.ncell)
        torch.cuda.synchronize()
        got = np.frombuffer(dst.cpu().numpy().tobytes(), dt)
        want = np.frombuffer(ref_state, dt)
        assert np.max(np.abs(got - want)) <= TOL[storage] * np.max(np.abs(want))
        assert np.array_equal(msk[call].cpu().numpy(), np.frombuffer(ref_mask, np.uint8))
        g, r = ledger_fields(led.cpu().numpy().tobytes()), ledger_fields(ref_ledger)
        assert g[0] == pytest.approx(r[0], rel=1e-12)
        assert g[1] == pytest.approx(r[1], rel=1e-12)
        assert g[2:] == r[2:]
    sim.close()


def test_static_scratch_rejects_bad_arguments():
    import torch
    from paper_2412_14859_gb300 import binding

    lib = binding.lib()
    case = inputs.Case("noalloc", 19, (12, 21, 37), R0=5.0)
    sim = gpu_sim(case, "f32")
    n = 19 * case.ncell * 8
    a = torch.zeros(n, dtype=torch.uint8, device="cuda")
    b = torch.zeros(n, dtype=torch.uint8, device="cuda")
    m = torch.zeros(case.ncell, dtype=torch.uint8, device="cuda")
    led = torch.zeros(40, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    p = ctypes.byref(sim.params)
    assert lib.cgevap_step_static_scratch(p, 1e-5, a.data_ptr(), b.data_ptr(), n - 8, m.data_ptr(),
                                          m.data_ptr(), led.data_ptr(), s) == -1
    assert lib.cgevap_step_static_scratch(p, 1e-5, a.data_ptr(), a.data_ptr(), n, m.data_ptr(),
                                          m.data_ptr(), led.data_ptr(), s) == -1
    # A lattice whose grid needs more CTAs than the static scratch holds (one plane of 4096 x 2048
    # columns: 65536 tiles of the default 32x4 shape) is refused.  The buffers are full-size, so nothing could run out of bounds
    # even if the size check were missing.
    big = binding.Params.from_buffer_copy(sim.params)
    big.nx, big.ny, big.nz = 4096, 2048, 1
    nb = 19 * 4096 * 2048 * 8
    A = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B = torch.empty(nb, dtype=torch.uint8, device="cuda")
    M0 = torch.zeros(4096 * 2048, dtype=torch.uint8, device="cuda")
    M1 = torch.zeros(4096 * 2048, dtype=torch.uint8, device="cuda")
    assert lib.cgevap_step_static_scratch(ctypes.byref(big), 1e-5, A.data_ptr(), B.data_ptr(), nb,
                                          M0.data_ptr(), M1.data_ptr(), led.data_ptr(), s) == -1
    del A, B, M0, M1
    sim.close()
