"""cgevap_step_static_scratch -- the one timestep entry point that allocates nothing.

It exists for callers that cannot allocate device memory (a framework that owns every buffer and
forbids allocation inside its operators, such as a custom call in an XLA/JAX program, or an
application arena with a fixed budget).  Its per-block scratch is a static device array inside
the library.  These tests drive it through the C ABI on buffers the test owns, starting from a
state produced by the handle API, and check two calls in a row against cgevap_step on the same
state: within the parity tolerances of the other GPU tests for FP64 / FP32, bit for bit for the
16-bit storages (the same kernel on the same input).  The file is named to be collected last, so
a failure here cannot hide failures of the other tests."""
import ctypes

import numpy as np
import pytest

from harness import gpu_sim
from paper_2412_14859_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
# checkpoint: magic, version, params, phi, flags, ledger, layout flag
HEADER = 8 + 4 + 112 + 8 + 4 + 4 + 40 + 4
MAX_CTAS = 16384  # the largest grid the static scratch holds


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


def layout_bytes(q, nx, ny, nz, storage):
    """Size of one state buffer of the padded layout the header states: pitch round_up(nx+18, 16)
    elements per row, ny+4 rows per plane (D3Q19; one row per plane for D2Q9)."""
    pitch = (nx + 18 + 15) // 16 * 16
    rows = ny + 4 if q == 19 else 1
    planes = nz if q == 19 else ny
    E = planes * rows * pitch
    if storage == "f64":
        return 16 * q * E
    if storage == "f32":
        return 8 * q * E
    return (8 * E + 255) // 256 * 256 + 4 * (q - 1) * E


CASES = {
    "d3q19": inputs.Case("noalloc", 19, (12, 21, 37), R0=5.0, noise=1e-6, phi=1e-5),
    "d2q9": inputs.Case("noalloc2d", 9, (1, 40, 70), R0=11.0, noise=1e-6, phi=1e-5),
}


@pytest.mark.parametrize("storage,lattice", [("f32", "d3q19"), ("f64", "d3q19"),
                                             ("f16dev", "d3q19"), ("bf16dev", "d3q19"),
                                             ("f32", "d2q9"), ("f16dev", "d2q9")])
def test_static_scratch_step_matches_handle_step(storage, lattice, tmp_path):
    import torch
    from paper_2412_14859_gb300 import binding

    lib = binding.lib()
    case = CASES[lattice]
    sim = gpu_sim(case, storage)
    sim.step(3)
    path = str(tmp_path / "state.ckpt")
    state, mask, ledger = read_checkpoint(sim, path, case.ncell)
    nz, ny, nx = case.shape
    assert len(state) == layout_bytes(case.q, nx, ny, nz, storage)

    buf = [torch.from_numpy(np.frombuffer(state, np.uint8).copy()).cuda() for _ in range(3)]
    msk = [torch.from_numpy(np.frombuffer(mask, np.uint8).copy()).cuda() for _ in range(3)]
    led = torch.from_numpy(np.frombuffer(ledger, np.uint8).copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in (1, 2):
        src, dst = buf[call - 1], buf[call]
        rc = lib.cgevap_step_static_scratch(
            ctypes.byref(sim.params), case.phi, src.data_ptr(), dst.data_ptr(), src.numel(),
            msk[call - 1].data_ptr(), msk[call].data_ptr(), led.data_ptr(), stream)
        assert rc == 0, lib.cgevap_last_error(None).decode()
        sim.step(1)
        ref_state, ref_mask, ref_ledger = read_checkpoint(sim, path, case.ncell)
        torch.cuda.synchronize()
        raw = dst.cpu().numpy().tobytes()
        if storage in TOL:
            dt = np.float32 if storage == "f32" else np.float64
            got, want = np.frombuffer(raw, dt), np.frombuffer(ref_state, dt)
            assert np.max(np.abs(got - want)) <= TOL[storage] * np.max(np.abs(want))
        else:  # the same kernel on the same bytes: the encoded state agrees bit for bit
            assert raw == ref_state
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
    case = CASES["d3q19"]
    sim = gpu_sim(case, "f32")
    nz, ny, nx = case.shape
    n = layout_bytes(19, nx, ny, nz, "f32")
    a = torch.zeros(n, dtype=torch.uint8, device="cuda")
    b = torch.zeros(n, dtype=torch.uint8, device="cuda")
    m = torch.zeros(case.ncell, dtype=torch.uint8, device="cuda")
    led = torch.zeros(40, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    p = ctypes.byref(sim.params)
    assert lib.cgevap_step_static_scratch(p, 1e-5, a.data_ptr(), b.data_ptr(), n - 8, m.data_ptr(),
                                          m.data_ptr(), led.data_ptr(), s) == -1
    assert b"state_bytes" in lib.cgevap_last_error(None)
    assert lib.cgevap_step_static_scratch(p, 1e-5, a.data_ptr(), a.data_ptr(), n, m.data_ptr(),
                                          m.data_ptr(), led.data_ptr(), s) == -1
    assert b"aliasing" in lib.cgevap_last_error(None)
    sim.close()


def test_static_scratch_grid_limit():
    """A lattice whose grid needs more CTAs than the static scratch holds is refused at the grid
    check; one whose grid just fits gets past it and runs.  One D3Q19 plane of 2048 columns:
    64 tiles of the default 32 x 4 shape across x, ny / 4 across y; ny = 1024 needs exactly
    16384 CTAs, ny = 1028 needs 16448.  The buffers have the layout's exact size, so the state
    check passes and nothing could run out of bounds even if the grid check were missing."""
    import torch
    from paper_2412_14859_gb300 import binding

    lib = binding.lib()
    base = gpu_sim(CASES["d3q19"], "f32")
    s = torch.cuda.current_stream().cuda_stream
    led = torch.zeros(40, dtype=torch.uint8, device="cuda")
    for ny, ok in ((1024, True), (1028, False)):
        p = binding.Params.from_buffer_copy(base.params)
        p.nx, p.ny, p.nz = 2048, ny, 1
        n = layout_bytes(19, 2048, ny, 1, "f32")
        A = torch.full((n // 4,), 0.02, dtype=torch.float32, device="cuda")  # positive densities
        B = torch.zeros(n // 4, dtype=torch.float32, device="cuda")
        M0 = torch.zeros(2048 * ny, dtype=torch.uint8, device="cuda")
        M1 = torch.zeros(2048 * ny, dtype=torch.uint8, device="cuda")
        rc = lib.cgevap_step_static_scratch(ctypes.byref(p), 1e-5, A.data_ptr(), B.data_ptr(), n,
                                            M0.data_ptr(), M1.data_ptr(), led.data_ptr(), s)
        if ok:
            assert rc == 0, lib.cgevap_last_error(None).decode()
            torch.cuda.synchronize()
            assert int(ledger_fields(led.cpu().numpy().tobytes())[4]) == 1  # one step folded
        else:
            assert rc == -1
            msg = lib.cgevap_last_error(None).decode()
            assert f"needs {64 * ny // 4} CTAs" in msg and str(MAX_CTAS) in msg, msg
        del A, B, M0, M1
    base.close()
