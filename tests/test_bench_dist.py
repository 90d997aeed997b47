"""Host logic of bench.py on CPU: the multi-rank aggregation (gloo, world size 2, spawned
processes) and the reference arm's rank handling and JSON line."""
import importlib.util
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = load_bench()
    d = b.Dist("gloo")
    try:
        # rank r updates 1000 + r cells for 10 steps in 5 + r ms
        mlups, ms = b.aggregate(1000 + rank, 10, 5.0 + rank, d)
        d.barrier()
        q.put((rank, mlups, ms))
    finally:
        d.close()


def test_aggregate_is_whole_job_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    want_ms = 6.0
    want = (1000 + 1001) * 10 / (want_ms / 1e3) / 1e6
    for rank, mlups, ms in got:
        assert ms == pytest.approx(want_ms)
        assert mlups == pytest.approx(want)


def test_reference_arm_other_ranks_do_no_work():
    b = load_bench()
    d = SimpleNamespace(rank=1, world=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert b.run_reference(SimpleNamespace(steps=1, warmup=0, size=12), d) is None
    assert buf.getvalue() == ""


def test_reference_arm_line(oracle_lib):
    b = load_bench()
    d = SimpleNamespace(rank=0, world=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        b.run_reference(SimpleNamespace(steps=2, warmup=1, size=12), d)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "MLUPS" and line["value"] > 0
    cores, model = b.host_cpu()
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == cores
    assert line["cpu_baseline"]["cpu_model"] == model
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["steps"] == 2 and line["warmup"] == 1


def test_cpu_baseline_reports_all_cores_and_one(oracle_lib):
    b = load_bench()
    cb = b.cpu_baseline(target_s=0.05)
    cores, model = b.host_cpu()
    assert cb["kind"] == "oracle" and cb["cores"] == cores == cb["nproc"]
    assert cb["cpu_model"] == model and cb["value"] > 0
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0


def test_timing_build_computes_the_oracle_step(oracle_lib):
    """The OpenMP build timed by the CPU baseline runs the same per-cell arithmetic as the pinned
    single-thread oracle: equal populations bit for bit; the ledger's sum may differ only by the
    order of its additions."""
    import numpy as np
    from paper_2412_14859_gb300 import inputs
    b = load_bench()
    case = inputs.shrink(inputs.sphere_3d(), (14, 13, 17), R0=4.5)
    p = b.oracle_params(case)
    f0 = oracle_lib.init(p, case.phase(), case.noise_array())
    plain = oracle_lib.Run(p, f0).step(4)
    omp = oracle_lib.Run(p, f0, omp=True).step(4)
    assert np.array_equal(plain.f, omp.f)
    assert np.array_equal(plain.mask, omp.mask)
    assert omp.evaporated == pytest.approx(plain.evaporated, rel=1e-13)


def test_adjoint_section_times_a_second_iteration(monkeypatch):
    """The adjoint section runs one untimed fit iteration (fresh device memory is slow to write
    the first time) and reports the second; every handle it opens is closed.  The library and
    the CUDA timing are replaced by stand-ins that record the calls."""
    import torch
    import paper_2412_14859_gb300.adjoint as adjoint
    import paper_2412_14859_gb300.binding as binding
    b = load_bench()
    calls = []

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, s=None):
            calls.append("event")

        def elapsed_time(self, other):
            return 10.0

    class FakeSim:
        fluid_cells, bytes_per_update = 1000, 309.0

        def __init__(self, case):
            self.shape, self.closed = case.shape, False
            calls.append("open")

        @classmethod
        def from_case(cls, case, storage):
            return cls(case)

        def init_equilibrium(self, rn):
            pass

        def set_flux(self, phi, field=None):
            pass

        def adjoint_forward(self, T, K):
            return torch.linspace(10.0, 9.0, T + 1, dtype=torch.float64)

        def close(self):
            self.closed = True
            calls.append("close")

    def history(sim, phi, T, K):
        calls.append("iteration")
        return 10.0 - torch.arange(T + 1, dtype=phi.dtype) * phi.mean()

    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(binding, "Sim", FakeSim)
    monkeypatch.setattr(adjoint, "volume_history", history)
    out = b.run_adjoint(SimpleNamespace(adjoint_steps=8, adjoint_shape="8,16,16"),
                        torch.device("cpu"))
    assert calls.count("iteration") == 2
    assert calls.count("open") == calls.count("close") == 3  # target, warm-up, timed
    # the timed events belong to the second iteration: three after its open
    last_open = len(calls) - 1 - calls[::-1].index("open")
    assert calls[last_open + 1:].count("event") == 3
    assert out["forward_ms"] == out["backward_ms"] == 10.0 and "untimed" in out["warmup"]


def test_clock_samples_are_summarised(tmp_path):
    """The clock record of a timed region: median SM clock under load, the maximum clock and the
    throttle reasons seen (nvidia-smi CSV, no header, no units), malformed lines skipped."""
    b = load_bench()
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class Proc:  # stands in for the nvidia-smi sampler process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = b.Clocks(0, enabled=False)
    c.proc, c.path = Proc(), str(path)
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()  # the sample file is removed
    assert b.Clocks(0, enabled=False).stop() is None


def test_traffic_follows_the_kernel_code_not_its_comments(tmp_path, monkeypatch):
    """The committed DRAM-traffic figures stay attached to the step kernel while only comments
    change, and are dropped once its code changes."""
    import shutil
    b = load_bench()
    src = os.path.join(ROOT, "paper_2412_14859_gb300", "csrc")
    fake = tmp_path / "paper_2412_14859_gb300" / "csrc"
    fake.mkdir(parents=True)
    for f in b.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), fake / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    h = b.kernel_hash()
    (tmp_path / "profiles" / "step_traffic.txt").write_text(
        f"# header\nstorage=f32 hash={h} cells=8 dram_read=1 dram_write=1 dram_bytes_per_cell=301.5\n")
    assert b.ncu_traffic("f32", 192) == 301.5
    k = fake / b.KERNEL_SOURCES[-1]
    k.write_text(k.read_text() + "\n// a comment\n/* another\n one */\n")
    assert b.kernel_hash() == h and b.ncu_traffic("f32", 192) == 301.5
    k.write_text(k.read_text() + "\nstatic int changed_code = 1;\n")
    assert b.kernel_hash() != h and b.ncu_traffic("f32", 192) is None
