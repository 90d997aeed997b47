"""ctypes binding of libcgevap.so (include/cgevap.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch provides device memory (tensors
whose data pointers are passed through) and the current CUDA stream.  ``lib()`` raises if the
library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcgevap.so")

F64, F32, F16DEV, BF16DEV, F32RC, F16RC, BF16RC, F32X = 0, 1, 2, 3, 4, 5, 6, 7
STORAGE = {"f64": F64, "f32": F32, "f16dev": F16DEV, "bf16dev": BF16DEV, "f32rc": F32RC,
           "f16rc": F16RC, "bf16rc": BF16RC, "f32x": F32X}
DTYPE_F64, DTYPE_F32 = 0, 1
SITES_GRADIENT, SITES_BAND, SITES_GIVEN = 0, 1, 2
ERRORS = {-1: "ARG", -2: "CUDA", -3: "OOM", -4: "TIMEOUT", -5: "NAN", -6: "UNSUPPORTED", -7: "IO"}


class CgevapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cgevap error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("rho_r_in", ctypes.c_double), ("rho_b_in", ctypes.c_double),
        ("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
        ("site_rule", ctypes.c_int), ("threshold", ctypes.c_double), ("sbar", ctypes.c_double),
        ("storage", ctypes.c_int),
    ]


class Ledger(ctypes.Structure):
    _fields_ = [
        ("evaporated", ctypes.c_double), ("last_removed", ctypes.c_double),
        ("site_steps", ctypes.c_longlong), ("last_sites", ctypes.c_longlong),
        ("steps", ctypes.c_longlong),
    ]


_lib = None
_vp = ctypes.c_void_p
_SIGS = {
    "cgevap_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    "cgevap_destroy": (ctypes.c_int, [_vp]),
    "cgevap_last_error": (ctypes.c_char_p, [_vp]),
    "cgevap_get_params": (ctypes.c_int, [_vp, ctypes.POINTER(Params)]),
    "cgevap_set_stream": (ctypes.c_int, [_vp, _vp]),
    "cgevap_set_solid": (ctypes.c_int, [_vp, _vp]),
    "cgevap_set_flux": (ctypes.c_int, [_vp, ctypes.c_double, _vp, ctypes.c_int]),
    "cgevap_set_flux_heated": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int]),
    "cgevap_get_flux_field": (ctypes.c_int, [_vp, _vp]),
    "cgevap_set_outlets": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
    "cgevap_init_equilibrium": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "cgevap_set_populations": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "cgevap_set_populations_host": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "cgevap_get_populations": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "cgevap_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "cgevap_get_macros": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "cgevap_get_mask": (ctypes.c_int, [_vp, _vp]),
    "cgevap_calibrate_threshold": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_double,
                                                  ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double)]),
    "cgevap_set_mask": (ctypes.c_int, [_vp, _vp]),
    "cgevap_volume": (ctypes.c_int, [_vp, _vp]),
    "cgevap_adjoint_forward": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "cgevap_adjoint_backward": (ctypes.c_int, [_vp, _vp, _vp]),
    "cgevap_adjoint_run": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "cgevap_adjoint_release": (ctypes.c_int, [_vp]),
    "cgevap_get_ledger": (ctypes.c_int, [_vp, ctypes.POINTER(Ledger)]),
    "cgevap_get_ledger_async": (ctypes.c_int, [_vp, _vp]),
    "cgevap_reset_ledger": (ctypes.c_int, [_vp]),
    "cgevap_check_health": (ctypes.c_int, [_vp]),
    "cgevap_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "cgevap_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "cgevap_bytes_per_update": (ctypes.c_double, [_vp]),
    "cgevap_fluid_cells": (ctypes.c_longlong, [_vp]),
    "cgevap_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cgevap_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cgevap_step_static_scratch": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_double, _vp,
                                                  _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp]),
    "cgevap_ensemble_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(_vp)]),
    "cgevap_ensemble_destroy": (ctypes.c_int, [_vp]),
    "cgevap_ensemble_last_error": (ctypes.c_char_p, [_vp]),
    "cgevap_ensemble_size": (ctypes.c_int, [_vp]),
    "cgevap_ensemble_cells": (ctypes.c_longlong, [_vp]),
    "cgevap_ensemble_member": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "cgevap_ensemble_set_stream": (ctypes.c_int, [_vp, _vp]),
    "cgevap_ensemble_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "cgevap_ensemble_status": (ctypes.c_int, [_vp]),
    "cgevap_ensemble_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cgevap_ensemble_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cgevap_ensemble_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "cgevap_ensemble_set_active": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "cgevap_ensemble_set_barrier_timeout": (ctypes.c_int, [_vp, ctypes.c_int]),
    "cgevap_ensemble_debug_skip_arrival": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "cgevap_ensemble_grid": (ctypes.c_int, [_vp]),
}


def lib() -> ctypes.CDLL:
    """Load libcgevap.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t: Optional[torch.Tensor], dtype=None) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return DTYPE_F64
    if t.dtype == torch.float32:
        return DTYPE_F32
    raise ValueError(f"unsupported dtype {t.dtype}")


class Sim:
    """One lattice on the current CUDA device (a handle of the C ABI)."""

    _borrowed = False

    def __init__(self, q: int, nx: int, ny: int, nz: int = 1, periodic=(1, 1, 1),
                 rho_r_in: float = 1.0, rho_b_in: float = 1.0, tau_r: float = 1.0,
                 tau_b: float = 1.0, sigma: float = 0.0, beta: float = 0.7,
                 site_rule: int = SITES_BAND, threshold: float = 0.5, sbar: float = 3.0,
                 storage="f32"):
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.params = Params(q, nx, ny, nz, (ctypes.c_int * 3)(*periodic), rho_r_in, rho_b_in,
                             tau_r, tau_b, sigma, beta, site_rule, threshold, sbar, st)
        self.q, self.shape = q, (nz, ny, nx)
        self.ncell = nx * ny * nz
        h = _vp()
        rc = lib().cgevap_create(ctypes.byref(self.params), ctypes.byref(h))
        if rc != 0:
            raise CgevapError(rc, lib().cgevap_last_error(None).decode())
        self._h = h
        self._sync_stream()

    @classmethod
    def from_case(cls, case, storage="f32") -> "Sim":
        nz, ny, nx = case.shape
        return cls(case.q, nx, ny, nz, case.periodic, case.rho_r_in, case.rho_b_in, case.tau_r, case.tau_b,
                   case.sigma, case.beta, case.site_rule, case.threshold, case.sbar, storage)

    # -- plumbing -----------------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise CgevapError(rc, lib().cgevap_last_error(self._h).decode())

    def _sync_stream(self):
        s = torch.cuda.current_stream().cuda_stream
        self._check(lib().cgevap_set_stream(self._h, s))

    def close(self):
        if getattr(self, "_h", None) and not self._borrowed:
            lib().cgevap_destroy(self._h)
        self._h = None

    @classmethod
    def _wrap(cls, handle, params: Params, owner) -> "Sim":
        """A member of an ensemble: the ensemble owns (and frees) the handle."""
        obj = cls.__new__(cls)
        obj.params = params
        obj.q = params.q
        obj.shape = (params.nz, params.ny, params.nx)
        obj.ncell = params.nx * params.ny * params.nz
        obj._h = handle
        obj._borrowed = True
        obj._owner = owner
        return obj

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- inputs ---------------------------------------------------------------------------------
    def set_flux(self, phi: float, field: Optional[torch.Tensor] = None):
        self._sync_stream()
        self._check(lib().cgevap_set_flux(self._h, float(phi), _ptr(field),
                                          _dt(field) if field is not None else 0))

    def set_flux_heated(self, phi_s: float, K: float, length: float, every: int = 1):
        """Heated-substrate flux phi_s / (K + h / length), h the liquid height of each cell's
        column along the substrate normal, recomputed on the device every `every` steps."""
        self._sync_stream()
        self._check(lib().cgevap_set_flux_heated(self._h, float(phi_s), float(K), float(length), int(every)))

    def set_outlets(self, rho_lo: float, rho_hi: float):
        """Blue pressure outlets on the first / last plane of the wall-normal axis (<= 0: wall)."""
        self._check(lib().cgevap_set_outlets(self._h, float(rho_lo), float(rho_hi)))

    def flux_field(self) -> torch.Tensor:
        """The flux field the next step reads, FP64, shape of the lattice (device)."""
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_get_flux_field(self._h, out.data_ptr()))
        return out

    def set_solid(self, solid: Optional[torch.Tensor]):
        self._sync_stream()
        self._check(lib().cgevap_set_solid(self._h, _ptr(solid, torch.uint8)))

    def init_equilibrium(self, rhoN0: torch.Tensor, noise: Optional[torch.Tensor] = None):
        self._sync_stream()
        self._check(lib().cgevap_init_equilibrium(self._h, _ptr(rhoN0, torch.float64),
                                                  _ptr(noise), _dt(noise) if noise is not None else 0))

    def set_populations(self, f: torch.Tensor):
        self._sync_stream()
        self._check(lib().cgevap_set_populations(self._h, _ptr(f), _dt(f)))

    def set_populations_host(self, f: np.ndarray):
        if not f.flags.c_contiguous or f.dtype not in (np.float64, np.float32):
            raise ValueError("expected a C-contiguous float64/float32 array")
        self._sync_stream()
        dt = DTYPE_F64 if f.dtype == np.float64 else DTYPE_F32
        self._check(lib().cgevap_set_populations_host(self._h, f.ctypes.data, dt))

    # -- stepping -------------------------------------------------------------------------------
    def step(self, n: int = 1):
        self._sync_stream()
        self._check(lib().cgevap_step(self._h, int(n)))
        return self

    # -- outputs --------------------------------------------------------------------------------
    def populations(self, dtype=torch.float64) -> torch.Tensor:
        out = torch.empty((2, self.q) + self.shape, dtype=dtype, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_get_populations(self._h, out.data_ptr(), _dt(out)))
        return out

    def macros(self) -> dict:
        rr, rb, rn = (torch.empty(self.shape, dtype=torch.float64, device="cuda") for _ in range(3))
        u = torch.empty((3,) + self.shape, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_get_macros(self._h, rr.data_ptr(), rb.data_ptr(), u.data_ptr(),
                                            rn.data_ptr()))
        return {"rho_r": rr, "rho_b": rb, "u": u, "rhoN": rn}

    def mask(self) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.uint8, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_get_mask(self._h, out.data_ptr()))
        return out

    def set_mask(self, mask: torch.Tensor):
        """Site bytes read by the next step (bit 0 = site under SITES_GIVEN)."""
        if mask.dtype != torch.uint8 or not mask.is_contiguous() or mask.numel() != self.ncell:
            raise ValueError("expected a contiguous uint8 tensor of one byte per cell")
        self._sync_stream()
        self._check(lib().cgevap_set_mask(self._h, mask.data_ptr()))

    def volume(self) -> torch.Tensor:
        """Liquid volume sum (1 + rho^N)/2 of the state, FP64, shape [1] (device)."""
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_volume(self._h, out.data_ptr()))
        return out

    # -- adjoint ----------------------------------------------------------------------------------
    def adjoint_forward(self, nsteps: int, ckpt_every: int = 64) -> torch.Tensor:
        """Run nsteps recording checkpoints; returns V(0..nsteps) (FP64, device)."""
        vol = torch.empty(nsteps + 1, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_adjoint_forward(self._h, int(nsteps), int(ckpt_every), vol.data_ptr()))
        return vol

    def adjoint_backward(self, dL_dV: Optional[torch.Tensor]) -> torch.Tensor:
        """dL/dphi per cell (FP64, shape of the lattice) for dL/dV(0..T) of the recorded run."""
        if dL_dV is not None and (dL_dV.dtype != torch.float64 or not dL_dV.is_contiguous()):
            raise ValueError("dL_dV must be a contiguous float64 tensor")
        out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        self._sync_stream()
        self._check(lib().cgevap_adjoint_backward(self._h, _ptr(dL_dV), out.data_ptr()))
        return out

    def adjoint_release(self):
        self._check(lib().cgevap_adjoint_release(self._h))

    def ledger(self) -> dict:
        L = Ledger()
        self._sync_stream()
        self._check(lib().cgevap_get_ledger(self._h, ctypes.byref(L)))
        return {k: getattr(L, k) for k, _ in Ledger._fields_}

    def ledger_async(self, out: torch.Tensor):
        """Enqueue a copy of the ledger into `out`, a page-locked CPU uint8 tensor of at least 40
        bytes (see ledger_from); it holds the record once the current stream has passed here."""
        if out.device.type != "cpu" or out.dtype != torch.uint8 or out.numel() < ctypes.sizeof(Ledger):
            raise ValueError("ledger_async needs a CPU uint8 tensor of at least 40 bytes")
        if not out.is_pinned():
            raise ValueError("ledger_async needs page-locked memory (pin_memory=True)")
        self._sync_stream()
        self._check(lib().cgevap_get_ledger_async(self._h, ctypes.c_void_p(out.data_ptr())))

    @staticmethod
    def ledger_from(buf: torch.Tensor) -> dict:
        """The ledger record held in the first 40 bytes of a CPU uint8 tensor."""
        L = Ledger.from_buffer_copy(bytes(buf[:ctypes.sizeof(Ledger)].numpy()))
        return {k: getattr(L, k) for k, _ in Ledger._fields_}

    def reset_ledger(self):
        self._sync_stream()
        self._check(lib().cgevap_reset_ledger(self._h))

    def check_health(self):
        self._sync_stream()
        self._check(lib().cgevap_check_health(self._h))

    def save(self, path: str):
        self._sync_stream()
        self._check(lib().cgevap_save(self._h, path.encode()))

    def load(self, path: str):
        self._sync_stream()
        self._check(lib().cgevap_load(self._h, path.encode()))

    def tune(self, family: int = -1, variant: int = 0, planes_per_chunk: int = 0):
        """Pick the fused-step kernel (family -1 auto, 0 register, 1 bulk-copy pipeline)."""
        self._check(lib().cgevap_tune(self._h, family, variant, planes_per_chunk))
        return self

    def tuning(self) -> dict:
        f, v, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().cgevap_get_tuning(self._h, ctypes.byref(f), ctypes.byref(v), ctypes.byref(p)))
        return {"family": f.value, "variant": v.value, "planes_per_chunk": p.value}

    @property
    def bytes_per_update(self) -> float:
        return lib().cgevap_bytes_per_update(self._h)

    @property
    def fluid_cells(self) -> int:
        return lib().cgevap_fluid_cells(self._h)


def calibrate_threshold(q: int, nx: int, ny: int, nz: int = 1, periodic=(1, 0, 1), phi: float = 0.03,
                        target_sbar: float = 3.0, rho_r_in: float = 1.0, rho_b_in: float = 1.0,
                        tau_r: float = 1.0, tau_b: float = 1.0, sigma: float = 0.0, beta: float = 0.7,
                        site_rule: int = SITES_GRADIENT, storage="f64"):
    """Threshold for a target S-bar on an evaporating flat interface (cgevap_calibrate_threshold);
    returns (threshold, measured S-bar)."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p = Params(q, nx, ny, nz, (ctypes.c_int * 3)(*periodic), rho_r_in, rho_b_in, tau_r, tau_b, sigma,
               beta, site_rule, 0.0, target_sbar, st)
    thr, sb = ctypes.c_double(), ctypes.c_double()
    rc = lib().cgevap_calibrate_threshold(ctypes.byref(p), float(phi), float(target_sbar),
                                          ctypes.byref(thr), ctypes.byref(sb))
    if rc != 0:
        raise CgevapError(rc, lib().cgevap_last_error(None).decode())
    return thr.value, sb.value


def all_signatures():
    """Names of the C functions this binding declares (kept equal to include/*.h by a test)."""
    return list(_SIGS)


class Ensemble:
    """Independent lattices advanced together by one persistent launch; storage "f32" or "f64",
    one for all members or a list with one per member, or "f32x" for all members."""

    def __init__(self, cases, storage="f32"):
        arr = (Params * len(cases))()
        st = [storage] * len(cases) if isinstance(storage, str) else list(storage)
        for j, c in enumerate(cases):
            nz, ny, nx = c.shape
            arr[j] = Params(c.q, nx, ny, nz, (ctypes.c_int * 3)(*c.periodic), c.rho_r_in,
                            c.rho_b_in, c.tau_r, c.tau_b, c.sigma, c.beta, c.site_rule,
                            c.threshold, c.sbar, STORAGE[st[j]])
        h = _vp()
        rc = lib().cgevap_ensemble_create(arr, len(cases), ctypes.byref(h))
        if rc != 0:
            raise CgevapError(rc, "cgevap_ensemble_create failed")
        self._h = h
        self._params = [arr[j] for j in range(len(cases))]
        self.members = []
        for j in range(len(cases)):
            mh = _vp()
            self._check(lib().cgevap_ensemble_member(self._h, j, ctypes.byref(mh)))
            self.members.append(Sim._wrap(mh, self._params[j], self))
        self._sync_stream()

    def _check(self, rc):
        if rc != 0:
            raise CgevapError(rc, lib().cgevap_ensemble_last_error(self._h).decode())

    def _sync_stream(self):
        s = torch.cuda.current_stream().cuda_stream
        self._check(lib().cgevap_ensemble_set_stream(self._h, s))

    def step(self, n: int = 1):
        self._sync_stream()
        self._check(lib().cgevap_ensemble_step(self._h, int(n)))
        return self

    def status(self):
        self._check(lib().cgevap_ensemble_status(self._h))

    @property
    def cells(self) -> int:
        return lib().cgevap_ensemble_cells(self._h)

    def tuning(self) -> dict:
        g, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().cgevap_ensemble_get_tuning(self._h, ctypes.byref(g), ctypes.byref(a),
                                                     ctypes.byref(b)))
        return {"groups": g.value, "planes_3d": a.value, "planes_2d": b.value}

    def set_tuning(self, groups: int, planes_3d: int, planes_2d: int):
        self._check(lib().cgevap_ensemble_set_tuning(self._h, groups, planes_3d, planes_2d))

    def set_active(self, j: int, active: bool):
        self._check(lib().cgevap_ensemble_set_active(self._h, int(j), 1 if active else 0))

    def set_barrier_timeout(self, ms: int):
        self._check(lib().cgevap_ensemble_set_barrier_timeout(self._h, int(ms)))

    def debug_skip_arrival(self, cta: int, step: int = 0):
        self._check(lib().cgevap_ensemble_debug_skip_arrival(self._h, int(cta), int(step)))

    @property
    def grid(self) -> int:
        return lib().cgevap_ensemble_grid(self._h)

    def autotune(self, probe_steps: int = 4) -> float:
        self._sync_stream()
        ms = ctypes.c_double()
        self._check(lib().cgevap_ensemble_autotune(self._h, probe_steps, ctypes.byref(ms)))
        return ms.value

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            lib().cgevap_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
