"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 CPU statement of the two-component colour-gradient lattice Boltzmann step with
reaction-limited evaporation (arXiv:2412.14859, Sec. II), in C (``cg_oracle.c``) behind ctypes,
plus the analytic evaporation laws of Sec. III and Appendices A-C (``laws.py``) and an FP64
autograd statement of the step used only to check the hand-written adjoint (``adjoint_ref.py``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of ``bench.py`` may import
this package.  The CUDA library neither links nor imports anything here, and nothing here
imports the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcg_oracle.so")
# The same source built with OpenMP: used only to time the oracle on all host cores (the CPU
# baseline of bench.py); every test uses the single-thread library above.
_SO_OMP = os.path.join(_BUILD, "libcg_oracle_omp.so")
# The same source built with multiply-add contraction: only to measure how much the method
# amplifies differences of rounding order (a test of the parity bounds over long runs).
_SO_FMA = os.path.join(_BUILD, "libcg_oracle_fma.so")

RULE_GRADIENT = 0
RULE_BAND = 1
RULE_GIVEN = 2  # replay a recorded site set (bit 0 of ``mask_given``)


def build(force: bool = False, omp: bool = False, contract: bool = False) -> str:
    """Compile the C oracle (plain gcc, IEEE FP64, no contraction into FMA); omp: the OpenMP
    timing build of the same source instead; contract: the build with multiply-adds contracted
    into FMA instructions (x86-64 needs -mfma for them; AArch64 has them in its base ISA)."""
    import platform
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_FMA if contract else (_SO_OMP if omp else _SO)
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cg_oracle.h"))
    ):
        tmp = so + f".{os.getpid()}.tmp"
        fp = ["-ffp-contract=fast"] + (["-mfma"] if platform.machine() in ("x86_64", "AMD64") else []) \
            if contract else ["-ffp-contract=off"]
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11"] + fp + ["-fno-fast-math", "-shared", "-fPIC"]
            + (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, so)
    return so


class _Params(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("rho_r_in", ctypes.c_double), ("rho_b_in", ctypes.c_double),
        ("tau_r", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
        ("site_rule", ctypes.c_int), ("threshold", ctypes.c_double), ("sbar", ctypes.c_double),
        ("phi", ctypes.c_double),
        ("phi_field", ctypes.POINTER(ctypes.c_double)),
        ("solid", ctypes.POINTER(ctypes.c_ubyte)),
        ("mask_given", ctypes.POINTER(ctypes.c_ubyte)),
        ("outlet_rho_lo", ctypes.c_double), ("outlet_rho_hi", ctypes.c_double),
    ]


class _Ledger(ctypes.Structure):
    _fields_ = [
        ("evaporated", ctypes.c_double), ("site_steps", ctypes.c_longlong),
        ("last_sites", ctypes.c_longlong), ("last_removed", ctypes.c_double),
        ("min_margin", ctypes.c_double),
    ]


_lib = None
_lib_omp = None
_lib_fma = None


def _L(omp: bool = False, contract: bool = False):
    global _lib, _lib_omp, _lib_fma
    if contract:
        if _lib_fma is None:
            _lib_fma = _declare(ctypes.CDLL(build(contract=True)))
        return _lib_fma
    if omp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build(omp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument types of the exported oracle functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_ubyte)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(_Params)
    lib.orc_lattice.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp, dp, ip]
    lib.orc_alphas.argtypes = [pp, dp, dp]
    lib.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
    lib.orc_perturbation_shape.argtypes = [ctypes.c_int, dp, dp]
    lib.orc_init.argtypes = [pp, dp, dp, dp]
    lib.orc_gradient_norm.argtypes = [pp, dp, dp]
    lib.orc_step.argtypes = [pp, dp, dp, dp, dp, up, dp, ctypes.POINTER(_Ledger)]
    lib.orc_step_cells.argtypes = [pp, dp, dp, ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.c_longlong, dp, dp, up]
    lib.orc_macros.argtypes = [pp, dp, dp, dp, dp, dp]
    lib.orc_outlet_blue.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
    return lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_ubyte)()
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


@dataclass
class Params:
    """Physical and numerical parameters of one lattice (paper notation, lattice units)."""
    q: int
    nx: int
    ny: int
    nz: int = 1
    periodic: Sequence[int] = (1, 1, 1)
    rho_r_in: float = 1.0
    rho_b_in: float = 1.0
    tau_r: float = 1.0
    tau_b: float = 1.0
    sigma: float = 0.0
    beta: float = 0.7
    site_rule: int = RULE_BAND
    threshold: float = 0.5
    sbar: float = 3.0
    phi: float = 0.0
    phi_field: Optional[np.ndarray] = None
    solid: Optional[np.ndarray] = None
    mask_given: Optional[np.ndarray] = None
    outlet_rho: Sequence[float] = (0.0, 0.0)  # blue outlets on the wall-normal axis (lo, hi); <= 0 wall
    _keep: list = field(default_factory=list, repr=False)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def _c(self) -> _Params:
        pf = None if self.phi_field is None else np.ascontiguousarray(self.phi_field, np.float64)
        sd = None if self.solid is None else np.ascontiguousarray(self.solid, np.uint8)
        mg = None if self.mask_given is None else np.ascontiguousarray(self.mask_given, np.uint8)
        self._keep = [pf, sd, mg]
        return _Params(
            self.q, self.nx, self.ny, self.nz, (ctypes.c_int * 3)(*self.periodic),
            self.rho_r_in, self.rho_b_in, self.tau_r, self.tau_b, self.sigma, self.beta,
            self.site_rule, self.threshold, self.sbar, self.phi, _dp(pf), _up(sd), _up(mg),
            float(self.outlet_rho[0]), float(self.outlet_rho[1]),
        )


def lattice(q: int) -> dict:
    c = np.zeros((q, 3), np.int32)
    w, a, b, cw = (np.zeros(q) for _ in range(4))
    opp = np.zeros(q, np.int32)
    z = ctypes.c_double()
    ip = ctypes.POINTER(ctypes.c_int)
    n = _L().orc_lattice(q, c.ctypes.data_as(ip), _dp(w), _dp(a), _dp(b), _dp(cw),
                         ctypes.byref(z), opp.ctypes.data_as(ip))
    if n != q:
        raise ValueError(f"unsupported lattice q={q}")
    return {"c": c, "w": w, "a": a, "b": b, "cw": cw, "zeta": z.value, "opp": opp}


def alphas(p: Params):
    ar, ab = ctypes.c_double(), ctypes.c_double()
    cp = p._c()
    _L().orc_alphas(ctypes.byref(cp), ctypes.byref(ar), ctypes.byref(ab))
    return ar.value, ab.value


def feq(q: int, rho: float, u, abar: float) -> np.ndarray:
    out = np.zeros(q)
    uu = np.ascontiguousarray(np.asarray(u, np.float64).reshape(3))
    _L().orc_feq(q, rho, _dp(uu), abar, _dp(out))
    return out


def perturbation_shape(q: int, F) -> np.ndarray:
    out = np.zeros(q)
    FF = np.ascontiguousarray(np.asarray(F, np.float64).reshape(3))
    _L().orc_perturbation_shape(q, _dp(FF), _dp(out))
    return out


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle rejected the call (status {rc})")


def init(p: Params, rhoN0: np.ndarray, noise: Optional[np.ndarray] = None) -> np.ndarray:
    f = np.zeros((2, p.q) + p.shape)
    r = np.ascontiguousarray(rhoN0, np.float64).reshape(p.shape)
    nz = None if noise is None else np.ascontiguousarray(noise, np.float64).reshape(f.shape)
    cp = p._c()
    _check(_L().orc_init(ctypes.byref(cp), _dp(r), _dp(nz), _dp(f)))
    return f


def gradient_norm(p: Params, f: np.ndarray) -> np.ndarray:
    G = np.zeros(p.shape)
    cp = p._c()
    _check(_L().orc_gradient_norm(ctypes.byref(cp), _dp(np.ascontiguousarray(f)), _dp(G)))
    return G


def outlet_blue(q: int, inward: int, rho0: float, gb: np.ndarray) -> np.ndarray:
    """The blue outlet (Sec. III.B.2) applied to one cell's pulled blue populations gb [Q] on
    the first (inward = +1) or last (inward = -1) plane of the wall-normal axis."""
    g = np.ascontiguousarray(gb, np.float64).copy()
    _check(_L().orc_outlet_blue(q, inward, rho0, _dp(g)))
    return g


def macros(p: Params, f: np.ndarray):
    rr, rb, rn = (np.zeros(p.shape) for _ in range(3))
    u = np.zeros((3,) + p.shape)
    cp = p._c()
    _check(_L().orc_macros(ctypes.byref(cp), _dp(np.ascontiguousarray(f)), _dp(rr), _dp(rb),
                           _dp(u), _dp(rn)))
    return {"rho_r": rr, "rho_b": rb, "u": u, "rhoN": rn}


class Run:
    """A lattice advanced by the oracle: state f (post-recoloring), |F| of the last step, ledger.
    omp: step with the OpenMP timing build (all host cores; for timing only); contract: step with
    the build whose multiply-adds are contracted (for measuring rounding-order sensitivity)."""

    def __init__(self, p: Params, f: np.ndarray, omp: bool = False, contract: bool = False):
        self.p = p
        self.omp = omp
        self.contract = contract
        self.f = np.ascontiguousarray(f, np.float64).copy()
        self.G = gradient_norm(p, self.f)  # |F| "of the previous step" before step 0
        self.mask = np.zeros(p.shape, np.uint8)
        self.margin = np.full(p.shape, np.inf)
        self.ledger = _Ledger(0.0, 0, 0, 0.0, np.inf)
        self.steps = 0
        self.min_margin_history = []

    def step(self, n: int = 1):
        cp = self.p._c()
        f_out = np.empty_like(self.f)
        G_out = np.empty(self.p.shape)
        for _ in range(n):
            lib = _L(self.omp, self.contract)
            _check(lib.orc_step(ctypes.byref(cp), _dp(self.f), _dp(f_out), _dp(self.G),
                                _dp(G_out), _up(self.mask), _dp(self.margin),
                                ctypes.byref(self.ledger)))
            self.f, f_out = f_out, self.f
            self.G, G_out = G_out, self.G
            self.steps += 1
            self.min_margin_history.append(self.ledger.min_margin)
        return self

    def macros(self):
        return macros(self.p, self.f)

    @property
    def evaporated(self) -> float:
        return self.ledger.evaporated

    @property
    def last_sites(self) -> int:
        return self.ledger.last_sites


def step_cells(p: Params, f: np.ndarray, G_prev: Optional[np.ndarray], cells: np.ndarray):
    """The step evaluated at selected cells only; returns (f_out [n,2,Q], G [n], mask [n])."""
    cells = np.ascontiguousarray(cells, np.int64)
    n = cells.size
    out_f = np.zeros((n, 2, p.q))
    out_G = np.zeros(n)
    out_m = np.zeros(n, np.uint8)
    cp = p._c()
    Gp = None if G_prev is None else np.ascontiguousarray(G_prev, np.float64)
    _check(_L().orc_step_cells(ctypes.byref(cp), _dp(np.ascontiguousarray(f)), _dp(Gp),
                               cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), n,
                               _dp(out_f), _dp(out_G), _up(out_m)))
    return out_f, out_G, out_m
