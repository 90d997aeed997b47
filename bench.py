#!/usr/bin/env python
"""Throughput of the fused colour-gradient LBM + reaction-limited evaporation step on GB300.

Workload (default): D3Q19 spherical drop R0 = 32 in a 192^3 periodic box, density ratio 10,
tau_l = 1, tau_g = 0.8, A = 0.005, beta = 0.7, phi = 1e-5, sites |rho^N| < 0.5, seeded
U(+-1e-6) noise.  One bench step = one timestep of the whole lattice = one launch of the fused
kernel.  The headline line is FP32 storage and arithmetic; FP16 / BF16 deviation storage
(FP32 arithmetic) and FP64 run the same steps from the same initial state and report their
speed and their error against the FP64 path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as N independent replicas (weak scaling, no data-path collective).
`--impl reference` times the FP64 CPU oracle (the only reference this paper has) on the host.

The line also carries the 64-member ensemble (one persistent launch per graph replay) and one
iteration of the adjoint flux fit: a D3Q19 90-degree sessile cap R0 = 48 on a wall of a
256x256x128 box, FP32, 2000 steps with checkpoints every 64, the 16 coefficients of
phi = phi0 (1 + sum_k a_k (r/R)^k) differentiated through the hand-written reverse sweep.
`--adjoint-fd` instead prints the agreement of that gradient with central finite differences.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline, CG-LBM+evaporation step; mixed vs FP64 at stated error"
UNIT = "MLUPS"
KERNEL_SOURCES = ["lattice.cuh", "common.cuh", "step_kernel.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=192)
    ap.add_argument("--storages", default="f32,f32x,f16rc,bf16rc,f32rc,f16dev,bf16dev,f64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="time K eager cgevap_step launches instead of one CUDA-graph replay of them")
    ap.add_argument("--kernel", type=int, default=-1, help="-1 auto, 0 register, 1 TMA pipeline")
    ap.add_argument("--variant", type=int, default=0, help="tile / pipeline variant of the kernel")
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="steps of the adjoint flux-fit iteration (0: skip)")
    ap.add_argument("--adjoint-shape", default="128,256,256",
                    help="nz,ny,nx of the sessile cap (R0 = 48 nx / 256)")
    ap.add_argument("--adjoint-fd", action="store_true",
                    help="only check the flux-fit gradient against finite differences (FP64)")
    ap.add_argument("--ensemble-steps", type=int, default=200,
                    help="steps of the 64-member ensemble workload (0: skip)")
    ap.add_argument("--sweep-2d", default="",
                    help="only run the D2Q9 drop sweep (R0 = 40, 256^2; 5 fluxes x 3 band "
                         "thresholds) to R0/2 as one ensemble in these storages (e.g. f32) and "
                         "print its radius-law errors")
    ap.add_argument("--steady-s", type=float, default=1.0,
                    help="seconds of extra graph replays of the headline storage, timed one by "
                         "one, reported beside the K-step figure (0: skip)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing ------

class Dist:
    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(cells_per_rank: float, steps: int, ms_per_rank: float, d: Dist):
    """Whole-job MLUPS: all ranks' lattice updates over the slowest rank's time."""
    ms = d.max(ms_per_rank)
    total = d.sum(cells_per_rank * steps)
    return total / (ms / 1e3) / 1e6, ms


# ------------------------------------------------------------------ measurement helpers -----

class Clocks:
    """nvidia-smi samples during a timed region (read only; no setting is changed)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool = True):
        self.idx = gpu_index
        try:
            import torch
            gpu_index = "GPU-" + str(torch.cuda.get_device_properties(gpu_index).uuid)
        except Exception:
            pass
        self.proc = None
        self.path = None
        if enabled:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                     "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            except OSError:
                self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def steady_state(graph, stream, ms_first: float, K: int, seconds: float):
    """Replays of the captured K-step graph, each timed with CUDA events on the launching stream,
    until about `seconds` of device time: median and spread of the time per step."""
    import torch
    reps = int(min(200, max(3, seconds * 1e3 / max(ms_first, 1e-3))))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for a, b in evs:
        a.record(stream)
        graph.replay()
        b.record(stream)
    torch.cuda.synchronize()
    per = sorted(a.elapsed_time(b) / K for a, b in evs)
    return {"replays": reps, "steps": reps * K, "ms_per_step": round(statistics.median(per), 5),
            "ms_per_step_min": round(per[0], 5), "ms_per_step_max": round(per[-1], 5),
            "device_s": round(sum(per) * K / 1e3, 3)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def kernel_hash() -> str:
    """sha256 prefix of the step kernel's sources with their comments removed and whitespace
    runs collapsed (a comment edit leaves the kernel, and the traffic measured on it, as they
    were)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, "paper_2412_14859_gb300", "csrc", f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(storage: str, size: int):
    """DRAM bytes per lattice update of the fused kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        kv = dict(p.split("=", 1) for p in line.split() if "=" in p)
        if kv.get("storage") == storage and kv.get("hash") == kernel_hash():
            return float(kv["dram_bytes_per_cell"])
    return None


def workload(size: int):
    from paper_2412_14859_gb300 import inputs
    return inputs.sphere_3d(size, 32.0 * size / 192.0)


def describe(case) -> str:
    n = case.shape[0]
    return (f"sphere_3d: D3Q19 {n}^3 periodic, drop R0={case.R0:g}, rho_l/rho_g="
            f"{case.rho_r_in / case.rho_b_in:g}, tau_l={case.tau_r:g}, tau_g={case.tau_b:g}, "
            f"A=0.005, beta={case.beta:g}, phi={case.phi:g}, sites |rho^N|<{case.threshold:g}, "
            f"noise U(+-1e-6)")


# ------------------------------------------------------------------ CPU oracle timing -------

def oracle_params(case):
    """The oracle's parameter set for a seeded workload case (same fields, oracle's own type)."""
    import oracle
    nz, ny, nx = case.shape
    return oracle.Params(q=case.q, nx=nx, ny=ny, nz=nz, periodic=tuple(case.periodic),
                         rho_r_in=case.rho_r_in, rho_b_in=case.rho_b_in, tau_r=case.tau_r,
                         tau_b=case.tau_b, sigma=case.sigma, beta=case.beta,
                         site_rule=case.site_rule, threshold=case.threshold, sbar=case.sbar,
                         phi=case.phi)


def host_cpu():
    """Host core count (usable by this process) and CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model or "unknown"


def oracle_rate(side: int, steps: int, omp: bool = False):
    """MLUPS of the FP64 C oracle on a side^3 box of the same physics: one thread, or (omp) the
    OpenMP build of the same source on all host cores."""
    import oracle
    case = workload(side)
    p = oracle_params(case)
    run = oracle.Run(p, oracle.init(p, case.phase(), None), omp=omp)
    t0 = time.perf_counter()
    run.step(steps)
    dt = time.perf_counter() - t0
    return case.ncell * steps / dt / 1e6, dt


def cpu_baseline(target_s: float = 10.0):
    """The oracle timed on this host: one thread on a 64^3 box, and the OpenMP build of the same
    source on all host cores on a 128^3 box; each sample sized to about target_s seconds."""
    cores, model = host_cpu()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    out = {}
    for omp, side in ((False, 64), (True, 128)):
        rate, dt = oracle_rate(side, 1, omp)
        steps = max(1, min(200, int(target_s / max(dt, 1e-3))))
        rate, dt = oracle_rate(side, steps, omp)
        out[omp] = (rate, dt, steps, side)
    rate, dt, steps, side = out[True]
    r1, dt1, steps1, side1 = out[False]
    return {"value": round(rate, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": model, "nproc": cores,
            "sample": f"FP64 C oracle built with OpenMP, {cores} threads, {steps} steps of the same "
                      f"physics on a {side}^3 box (drop R0={32 * side / 192:g}), {dt:.1f} s",
            "single_thread": {"value": round(r1, 4), "unit": UNIT, "cores": 1,
                              "sample": f"the plain oracle build, one thread, {steps1} steps on a "
                                        f"{side1}^3 box, {dt1:.1f} s"}}


def run_reference(args, d: Dist):
    if d.rank != 0:
        return
    import oracle
    cores, model = host_cpu()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    # size the sample so warm-up + timed steps take about two minutes
    probe, dt1 = oracle_rate(48, 1, omp=True)
    budget = 120.0 / max(1, args.steps + args.warmup)
    side = int(max(12, min(args.size, round((budget * probe * 1e6) ** (1 / 3)))))
    case = workload(side)
    p = oracle_params(case)
    run = oracle.Run(p, oracle.init(p, case.phase(), None), omp=True)
    run.step(args.warmup)
    t0 = time.perf_counter()
    run.step(args.steps)
    dt = time.perf_counter() - t0
    value = case.ncell * args.steps / dt / 1e6
    full = workload(args.size)
    where = (f"the full {side}^3 box" if side == args.size else
             f"a {side}^3 box (drop R0={case.R0:g}) instead of {args.size}^3")
    sample = (f"FP64 C oracle built with OpenMP, {cores} threads ({model}); each step is one "
              f"timestep of the same physics on {where}")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": d.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(full), "cells": full.ncell, "sample_cells": case.ncell},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": model, "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU path -----------------

def run_ensemble(args, dev):
    """48 D2Q9 + 16 D3Q19 drops of uneven size, flux, density ratio and threshold (FP32), advanced
    by one persistent launch per call from a CUDA graph, tiling chosen by the autotuner."""
    import torch
    from paper_2412_14859_gb300 import inputs
    from paper_2412_14859_gb300.binding import Ensemble
    cases = inputs.ensemble_members()
    ens = Ensemble(cases)
    for sim, case in zip(ens.members, cases):
        sim.set_flux(case.phi)
        sim.init_equilibrium(torch.from_numpy(case.phase()).to(dev))
    best = ens.autotune(probe_steps=4)
    ens.step(3)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    ens.step(args.ensemble_steps)
    e1.record(s)
    torch.cuda.synchronize()
    ens.status()
    ms = e0.elapsed_time(e1)
    cells = ens.cells
    # bytes-weighted roofline: each member's algorithmic bytes per update times its cells
    c2 = sum(m.fluid_cells for m, c in zip(ens.members, cases) if c.q == 9)
    c3 = sum(m.fluid_cells for m, c in zip(ens.members, cases) if c.q == 19)
    nbytes = sum(m.fluid_cells * m.bytes_per_update for m in ens.members)
    gbs = nbytes * args.ensemble_steps / (ms / 1e3) / 1e9
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    out = {"mlups": round(cells * args.ensemble_steps / (ms / 1e3) / 1e6, 1), "cells": cells,
           "cells_d2q9": c2, "cells_d3q19": c3,
           "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(gbs / hbm, 4),
                        "algorithmic_bytes_per_step": nbytes,
                        "note": "sum over members of cells x bytes per update (D2Q9 FP32 145 B, "
                                "D3Q19 FP32 305 B, band rule)"},
           "members": len(cases), "steps": args.ensemble_steps,
           "ms_per_step": round(ms / args.ensemble_steps, 4), "tuning": ens.tuning(),
           "autotune_ms_per_step": round(best, 4),
           "launches": "1 cooperative persistent kernel per call, replayed from a CUDA graph"}
    ens.close()
    return out


def cap_fit(shape, R0, dev, dtype):
    """Sessile-cap flux-fit problem: case, radial basis (r/R0)^k, a, a_target."""
    import torch
    from paper_2412_14859_gb300 import inputs
    case = inputs.sessile_cap_3d(shape, R0=R0, phi0=2e-5)
    nz, ny, nx = shape
    basis = torch.from_numpy(inputs.radial_basis(shape, ((ny - 1) / 2.0, (nx - 1) / 2.0), R0, 16))
    a, a_t = inputs.flux_fit_parameters(16)
    return case, basis.to(device=dev, dtype=dtype), a, a_t


def fit_loss(V, dVt):
    return ((V[0] - V[1:] - dVt) ** 2).sum()


def run_adjoint(args, dev):
    """One iteration of the flux fit (forward run with checkpoints, loss, reverse sweep) in FP32
    on the full sessile cap; throughput as MLUPS-equivalent = cells x steps / (forward + backward)."""
    import torch
    from paper_2412_14859_gb300.adjoint import volume_history
    from paper_2412_14859_gb300.binding import Sim
    T, K = args.adjoint_steps, 64
    shape = tuple(int(v) for v in args.adjoint_shape.split(","))
    case, basis, a, a_t = cap_fit(shape, 48.0 * shape[2] / 256.0, dev, torch.float64)
    rn = torch.from_numpy(case.phase()).to(dev)

    def phi_of(av):
        return case.phi * (1.0 + torch.tensordot(av, basis, dims=1))

    tgt = Sim.from_case(case, "f32")
    tgt.init_equilibrium(rn)
    tgt.set_flux(0.0, phi_of(torch.tensor(a_t, device=dev)).contiguous())
    Vt = tgt.adjoint_forward(T, K)
    dVt = (Vt[0] - Vt[1:]).detach()
    tgt.close()

    def iteration():
        sim = Sim.from_case(case, "f32")
        sim.init_equilibrium(rn)
        at = torch.tensor(a, device=dev, requires_grad=True)
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(s)
        V = volume_history(sim, phi_of(at), T, K)
        ev[1].record(s)
        L = fit_loss(V, dVt)
        L.backward()
        ev[2].record(s)
        torch.cuda.synchronize()
        return sim, at, L, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    # One untimed iteration first: the first writes to freshly allocated device memory cost
    # about 16 GB/s, which the reverse sweep's 93 GB of segment states would otherwise pay inside
    # the timed sweep (a fit loop pays it once); the timed iteration gets the warm memory back.
    iteration()[0].close()
    sim, at, L, fwd, bwd = iteration()
    cells = sim.fluid_cells
    sb = sim.bytes_per_update  # per update of the forward step
    out = {
        "workload": "D3Q19 sessile cap R0=%g, %dx%dx%d, walls on z, FP32, %d steps, "
                    "checkpoint every %d, 16 flux coefficients" % (case.R0, shape[2], shape[1],
                                                                   shape[0], T, K),
        "mlups_equivalent": round(cells * T / ((fwd + bwd) / 1e3) / 1e6, 1),
        "forward_ms": round(fwd, 1), "backward_ms": round(bwd, 1),
        "backward_over_forward": round(bwd / fwd, 2),
        "loss": float(L.detach()), "grad_norm": float(at.grad.norm()),
        "tape_states": -(-T // K) + K + 2, "forward_bytes_per_update": sb,
        "launches": "forward: 1 step + 1 volume kernel per step; backward per step: 1 recomputed "
                    "step + 2 adjoint kernels (A pushes the transposed pull, B1 the stencil)",
        "warmup": "one untimed fit iteration first (first touch of the tape's device memory)",
    }
    sim.close()
    return out


def run_adjoint_fd(args):
    """Gradient of the flux-fit loss vs central differences (h = 1e-3), FP64: the full cap over
    256 steps and a reduced cap (64x64x32, R0 = 12) over 200 steps; site sets replayed from the
    base run (the gate) and, for the reduced cap, also left free (reported)."""
    import numpy as np
    import torch
    from paper_2412_14859_gb300.adjoint import volume_history
    from paper_2412_14859_gb300.binding import SITES_GIVEN, Sim
    dev = torch.device("cuda", 0)
    report = {}
    for name, shape, R0, T, K in (("reduced_64x64x32_R12", (32, 64, 64), 12.0, 200, 64),
                                  ("full_256x256x128_R48", (128, 256, 256), 48.0, 256, 16)):
        case, basis, a, a_t = cap_fit(shape, R0, dev, torch.float64)
        rn = torch.from_numpy(case.phase()).to(dev)

        def phi_of(av):
            return (case.phi * (1.0 + torch.tensordot(torch.as_tensor(av, device=dev), basis, dims=1))).contiguous()

        def run(av, rule=None, masks=None, record=False):
            sim = Sim.from_case(case, "f64") if rule is None else Sim(
                case.q, shape[2], shape[1], shape[0], case.periodic, case.rho_r_in, case.rho_b_in,
                case.tau_r, case.tau_b, case.sigma, case.beta, rule, case.threshold, case.sbar, "f64")
            sim.init_equilibrium(rn)
            sim.set_flux(0.0, phi_of(av))
            V, rec = [sim.volume()], []
            for t in range(T):
                if masks is not None:
                    sim.set_mask(masks[t])
                sim.step(1)
                V.append(sim.volume())
                if record:
                    rec.append(sim.mask())
            sim.close()
            return torch.cat(V), rec

        Vt, _ = run(a_t)
        dVt = Vt[0] - Vt[1:]
        sim = Sim.from_case(case, "f64")
        sim.init_equilibrium(rn)
        at = torch.tensor(a, device=dev, requires_grad=True)
        t0 = time.perf_counter()
        L = fit_loss(volume_history(sim, case.phi * (1.0 + torch.tensordot(at, basis, dims=1)), T, K), dVt)
        L.backward()
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        sim.close()
        grad = at.grad.cpu().numpy()
        _, masks = run(a, record=True)
        h = 1e-3
        fd, fd_free = np.zeros(16), np.zeros(16)
        for k in range(16):
            e = np.zeros(16)
            e[k] = h
            fd[k] = (float(fit_loss(run(a + e, SITES_GIVEN, masks)[0], dVt)) -
                     float(fit_loss(run(a - e, SITES_GIVEN, masks)[0], dVt))) / (2 * h)
            if name.startswith("reduced"):
                fd_free[k] = (float(fit_loss(run(a + e)[0], dVt)) - float(fit_loss(run(a - e)[0], dVt))) / (2 * h)
        del masks
        torch.cuda.empty_cache()
        r = {"steps": T, "ckpt_every": K, "loss": float(L.detach()), "adjoint_s": round(t_adj, 2),
             "grad": [float(v) for v in grad], "fd_replayed_sites": [float(v) for v in fd],
             "max_abs_err_over_max_fd": float(np.max(np.abs(grad - fd)) / np.max(np.abs(fd))),
             "max_rel_err_per_component": float(np.max(np.abs(grad - fd) / np.abs(fd)))}
        if name.startswith("reduced"):
            r["fd_free_sites"] = [float(v) for v in fd_free]
            r["free_sites_err_over_max_fd"] = float(np.max(np.abs(grad - fd_free)) / np.max(np.abs(fd_free)))
        report[name] = r
    print(json.dumps({"adjoint_fd": report}), flush=True)


def band_sbar(theta: float) -> float:
    """S-bar of the band rule at theta: the fixed point of S-bar -> time-averaged sites per unit
    length of a flat-interface run with that S-bar (64^2 slab, two interfaces, flux 1e-3, FP64)."""
    from dataclasses import replace
    from paper_2412_14859_gb300 import inputs
    from paper_2412_14859_gb300.binding import Sim
    import torch
    case = replace(inputs.flat_slab_2d(), phi=1e-3, threshold=theta)
    sbar = 3.0
    for _ in range(4):
        sim = Sim.from_case(replace(case, sbar=sbar), "f64")
        sim.set_flux(case.phi)
        sim.init_equilibrium(torch.from_numpy(case.phase()).cuda())
        sim.step(2000)
        sbar = sim.ledger()["site_steps"] / 2000 / (2 * case.shape[2])
        sim.close()
    return sbar


def run_sweep_2d(args):
    """The D2Q9 drop sweep to R0/2: every (phi, theta) case with its band-rule S-bar, equilibrated
    3000 steps with the flux off, then evaporated; R = sqrt(V / pi) of the liquid area against
    R0 - phi t / rho_l at R/R0 = 3/4 and 1/2; each member is paused once it reaches its second
    mark (the tiling tuned again for the members left), and the launches are cut into calls of
    at most 1e5 steps."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2412_14859_gb300 import inputs
    from paper_2412_14859_gb300.binding import Ensemble
    torch.cuda.set_device(0)
    t_start = time.perf_counter()
    sb = {th: band_sbar(th) for th in (0.3, 0.5, 0.7)}
    storages = [s for s in args.sweep_2d.split(",") if s]
    base = [replace(c, sbar=sb[c.threshold]) for c in inputs.drop_2d_sweep()]
    cases = [c for _ in storages for c in base]
    st_of = [st for st in storages for _ in base]
    ens = Ensemble(cases, st_of)
    for sim, c in zip(ens.members, cases):
        sim.set_flux(0.0)
        sim.init_equilibrium(torch.from_numpy(c.phase()).cuda(), torch.from_numpy(c.noise_array()).cuda())
    ens.autotune(probe_steps=20)
    ens.step(3000)
    R0, rho, m0 = [], [], []
    for sim, c in zip(ens.members, cases):
        R0.append(float(np.sqrt(float(sim.volume()) / np.pi)))
        m = sim.macros()
        rho.append(float(m["rho_r"].max()))
        m0.append(float(m["rho_r"].sum()))
        sim.set_flux(c.phi)
        sim.reset_ledger()
    marks = [[(1.0 - f) * R0[j] * rho[j] / c.phi for f in (0.75, 0.5)] for j, c in enumerate(cases)]
    err = [[None, None] for _ in cases]
    active, t, retune = set(range(len(cases))), 0, False
    while active:
        nxt = min(int(round(marks[j][k])) for j in active for k in (0, 1) if err[j][k] is None)
        ens.step(min(nxt - t, 100000))
        t += min(nxt - t, 100000)
        for j in list(active):
            for k in (0, 1):
                if err[j][k] is None and int(round(marks[j][k])) == t:
                    R = float(np.sqrt(float(ens.members[j].volume()) / np.pi))
                    exact = 1.0 - cases[j].phi * t / (R0[j] * rho[j])
                    err[j][k] = (R / R0[j] - exact) / exact * 100.0
            if err[j][1] is not None:
                active.discard(j)
                if active:
                    ens.set_active(j, False)
                    retune = True
        if retune:  # fewer members: shorter chunks spread the rest over more CTAs
            ens.autotune(probe_steps=20)
            retune = False
    ens.status()
    rows = []
    for j, c in enumerate(cases):
        sim = ens.members[j]
        lost = m0[j] - float(sim.macros()["rho_r"].sum())
        rows.append({"storage": st_of[j], "phi": c.phi, "theta": c.threshold, "sbar": round(c.sbar, 4),
                     "R0": round(R0[j], 3), "steps_to_half": int(round(marks[j][1])),
                     "error_percent_at_3_4": round(err[j][0], 3),
                     "error_percent_at_1_2": round(err[j][1], 3),
                     "red_lost_over_ledger_minus_1": lost / sim.ledger()["evaporated"] - 1.0})
    ens.close()
    print(json.dumps({"sweep_2d": rows, "band_sbar": sb, "wall_s": round(time.perf_counter() - t_start, 1)}),
          flush=True)


def run_ours(args, d: Dist):
    import numpy as np
    import torch
    from paper_2412_14859_gb300.binding import Sim
    from paper_2412_14859_gb300 import inputs

    torch.cuda.set_device(d.local_rank)
    dev = torch.device("cuda", d.local_rank)
    case = workload(args.size)
    rn = torch.from_numpy(case.phase()).to(dev)
    noise = torch.from_numpy(inputs.uniform_noise((2, 19) + case.shape, case.noise, case.seed,
                                                  np.float32)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    storages = [s for s in args.storages.split(",") if s]
    results, rho_r, rho_b = {}, {}, {}

    for st in storages:
        K = args.steps
        with torch.cuda.stream(stream):
            sim = Sim.from_case(case, st)
            sim.tune(args.kernel if st == "f32" else 0, args.variant)
            sim.set_flux(case.phi)
            sim.init_equilibrium(rn, noise)
            sim.step(args.warmup)
            graph = None
            if not args.no_graph:  # the K launches captured once, replayed as one graph
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=stream):
                    sim.step(K)
            torch.cuda.synchronize()
            d.barrier()
            clocks = Clocks(d.local_rank, enabled=(st == storages[0] and not args.no_clocks))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if graph is not None:
                graph.replay()
            else:
                sim.step(K)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            mlups, ms_max = aggregate(sim.fluid_cells, K, ms, d)
            bpu = sim.bytes_per_update
            per_launch_s = ms / K / 1e3
            achieved = bpu * sim.fluid_cells / per_launch_s / 1e9
            # the state after warm-up + K steps, compared across storages below
            m = sim.macros()
            rho_r[st] = m["rho_r"]
            rho_b[st] = m["rho_b"]
            led = sim.ledger()
            mass_r = float(m["rho_r"].sum())
            # headline storage: more replays of the same graph, each timed on its own, so that
            # the fraction also rests on a region of about steady_s seconds (clocks still sampled)
            steady = None
            if st == storages[0] and graph is not None and args.steady_s > 0:
                steady = steady_state(graph, stream, ms, K, args.steady_s)
                steady["mlups"] = round(sim.fluid_cells / (steady["ms_per_step"] / 1e3) / 1e6, 1)
                steady["frac"] = round(bpu * sim.fluid_cells / (steady["ms_per_step"] / 1e3) / 1e9 / hbm, 4)
            del graph
            clk = clocks.stop()
            d.barrier()
            results[st] = {"mlups": mlups, "ms": ms_max, "bytes_per_update": bpu, "tuning": sim.tuning(),
                           "achieved_gbs": achieved, "frac": achieved / hbm, "clocks": clk,
                           "mass_r": mass_r, "ledger": led["evaporated"],
                           "steps_total": led["steps"], "sim": sim, "steady": steady}
        if st != storages[0]:
            sim.close()
            results[st]["sim"] = None

    head = storages[0]
    H = results[head]
    ref = "f64" if "f64" in results else None
    variants = {}
    for st, r in results.items():
        v = {"mlups": round(r["mlups"], 1), "ms_per_step": round(r["ms"] / args.steps, 4),
             "bytes_per_update": r["bytes_per_update"], "hbm_gbs": round(r["achieved_gbs"], 1),
             "hbm_frac": round(r["frac"], 4), "speedup_vs_f32": None}
        if "f32" in results:
            v["speedup_vs_f32"] = round(r["mlups"] / results["f32"]["mlups"], 3)
        if ref and st != ref:
            a, b = rho_r[st], rho_r[ref]
            v["vs_f64"] = {
                "steps": r["steps_total"],
                "rel_mass_error_red": abs(r["mass_r"] - results[ref]["mass_r"]) / results[ref]["mass_r"],
                "rel_linf_rho_r": float((a - b).abs().max() / b.abs().max()),
                "rel_linf_rho_b": float((rho_b[st] - rho_b[ref]).abs().max() / rho_b[ref].abs().max()),
                "rel_error_evaporated_ledger": abs(r["ledger"] - results[ref]["ledger"]) / max(results[ref]["ledger"], 1e-300),
            }
        variants[st] = v

    # ---- end to end through the C ABI with host buffers (headline storage) -------------------
    e2e = None
    sim = H["sim"]
    if not args.no_e2e:
        with torch.cuda.stream(stream):
            f_host = sim.populations(torch.float32).cpu().pin_memory().numpy()
            sim.close()
            sim2 = Sim.from_case(case, head)
            sim2.tune(args.kernel if head == "f32" else 0, args.variant)
            sim2.set_flux(case.phi)
            sim2.set_populations_host(f_host)  # allocates the staging buffer once, untimed
            sim2.step(args.warmup)  # untimed: both state buffers written once (warm memory)
            warm = sim2.macros()    # untimed: the readout's device buffers come from the cache
            out_host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                        for k, v in warm.items()}
            del warm
            # one page-locked 40-byte ledger slot per step: every step's record is read back
            led_host = torch.zeros(40 * args.steps, dtype=torch.uint8, pin_memory=True)
            torch.cuda.synchronize()
            d.barrier()
            # timed: the initial state from pinned host memory, K steps each followed by the
            # copy of its ledger record (40 B) into its host slot, enqueued without waiting, and
            # the final macroscopic fields (rho_r, rho_b, u, rho^N in FP64) copied back into
            # pinned host memory
            t0 = time.perf_counter()
            sim2.set_populations_host(f_host)
            for k in range(args.steps):
                sim2.step(1)
                sim2.ledger_async(led_host[40 * k:40 * (k + 1)])
            fields = sim2.macros()
            for k, v in fields.items():
                out_host[k].copy_(v, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            d.barrier()
            # every slot holds its own step's record
            first = Sim.ledger_from(led_host[:40])["steps"]
            last = Sim.ledger_from(led_host[40 * (args.steps - 1):])["steps"]
            if last - first != args.steps - 1:
                raise RuntimeError(f"ledger slots out of order: {first} .. {last}")
            sim2.ledger()  # the timeout flag of a bounded device-side wait, untimed
            readback = sum(v.numel() * v.element_size() for v in out_host.values())
            e2e_mlups, _ = aggregate(sim2.fluid_cells, args.steps, dt * 1e3, d)
            e2e = {"value": round(e2e_mlups, 1), "unit": UNIT,
                   "h2d_bytes_per_step": int(f_host.nbytes // args.steps),
                   "d2h_bytes_per_step": int((40 * args.steps + readback) // args.steps),
                   "what": "pinned host state in, K steps each followed by an asynchronous "
                           "40-byte ledger read into its own pinned slot, final rho_r, rho_b, u, "
                           "rho^N (FP64) out; wall clock around it"}
            sim2.close()
    elif sim is not None:
        sim.close()

    ensemble = run_ensemble(args, dev) if args.ensemble_steps > 0 else None
    adjoint = run_adjoint(args, dev) if args.adjoint_steps > 0 else None
    if d.rank != 0:
        return
    traffic = ncu_traffic(head, args.size)
    cells = case.ncell
    line = {
        "metric": METRIC, "value": round(H["mlups"], 1), "unit": UNIT, "n_gpus": d.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(H["ms"] / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head if head != "f16dev" else "f32",
        "data": "synthetic",
        "config": {"workload": describe(case), "cells": cells, "storage": head,
                   "timing": ("K eager step launches" if args.no_graph else
                              "the K step launches captured in one CUDA graph, one replay timed"),
                   "parallelism": f"{d.world} independent replicas" if d.world > 1 else "1 GPU",
                   "l2": "no flush: the state (2 x %.2f GB) is larger than L2" % (
                       H["bytes_per_update"] * cells / 2 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": round(H["achieved_gbs"], 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(H["frac"], 4),
                     "traffic": None if traffic is None else round(traffic * cells),
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_update": H["bytes_per_update"],
                     "kernel": ("cg_step_tma_kernel" if H["tuning"]["family"] == 1 else
                                "cg_step_kernel") + " (fused step), tuning %s" % H["tuning"]},
        "variants": variants,
        "gpu_launches": args.steps,
    }
    if ensemble:
        line["ensemble"] = ensemble
    if adjoint:
        line["adjoint"] = adjoint
    if H["clocks"]:
        line["clocks"] = H["clocks"]
    if H["steady"]:
        line["steady_state"] = H["steady"]
    if e2e:
        line["e2e"] = e2e
    if d.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.gpus > 1 and int(os.environ.get("WORLD_SIZE", "1")) != args.gpus:
        sys.exit("--gpus N > 1 must be launched with torchrun --nproc-per-node N")
    if args.adjoint_fd:
        run_adjoint_fd(args)
        return
    if args.sweep_2d:
        run_sweep_2d(args)
        return
    if args.impl == "reference":
        d = Dist("gloo")
        try:
            run_reference(args, d)
        finally:
            d.close()
        return
    d = Dist("nccl")
    try:
        run_ours(args, d)
    finally:
        d.close()


if __name__ == "__main__":
    main()
