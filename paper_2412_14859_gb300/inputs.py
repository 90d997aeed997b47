"""Seeded synthetic inputs shared by the CUDA path, the oracle-based tests and the benchmark.

This module holds geometry and random numbers only -- initial phase fields, noise, flux fields
and the parameter sets of the benchmark workloads -- and none of the method's arithmetic
(no equilibria, moments or collision).  Both sides turn these inputs into populations with their
own code.

Workloads (synthetic, lattice units; there is no external dataset in the paper, whose benchmark
geometries in Sec. III are themselves synthetic):
  flat_slab_2d      D2Q9 64x64 periodic, liquid slab of width 32, FP64 reference case
  drop_2d           D2Q9 256x256 periodic, circular drop R0 = 40
  sphere_3d         D3Q19 192^3 periodic, spherical drop R0 = 32, density ratio 10
  ensemble          48 D2Q9 + 16 D3Q19 drops of uneven size, flux, density ratio and threshold
  sessile_cap_3d    D3Q19 256x256x128, walls on the 128 axis, 90-degree cap R0 = 48,
                    flux phi(r) = phi0 (1 + sum_k a_k (r/R)^k)
The surface-tension input of these workloads is given as the perturbation amplitude A at tau = 1,
so sigma = 4 A / 9 (Eq. perturb has amplitude (9/4) sigma / tau).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

SEED = 20241219
RULE_GRADIENT = 0
RULE_BAND = 1


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.default_rng(seed)


def sigma_from_amplitude(A: float) -> float:
    """Surface tension whose perturbation amplitude (9/4) sigma / tau equals A at tau = 1."""
    return 4.0 * A / 9.0


# ------------------------------------------------------------------ geometry ---------------

def slab_phase(shape: Tuple[int, int, int], axis: int, center: float, half_width: float,
               width: float = 2.0) -> np.ndarray:
    """rho^N_0 = tanh(d / width), d = half_width - |s - center| along one axis (z=0,y=1,x=2)."""
    s = np.arange(shape[axis], dtype=np.float64)
    d = half_width - np.abs(s - center)
    prof = np.tanh(d / width)
    sh = [1, 1, 1]
    sh[axis] = shape[axis]
    return np.broadcast_to(prof.reshape(sh), shape).copy()


def half_space_phase(shape: Tuple[int, int, int], axis: int, level: float,
                     width: float = 2.0) -> np.ndarray:
    """rho^N_0 = tanh((level - s) / width): liquid below `level` along one axis."""
    s = np.arange(shape[axis], dtype=np.float64)
    prof = np.tanh((level - s) / width)
    sh = [1, 1, 1]
    sh[axis] = shape[axis]
    return np.broadcast_to(prof.reshape(sh), shape).copy()


def sphere_phase(shape: Tuple[int, int, int], center, R0: float, width: float = 2.0) -> np.ndarray:
    """rho^N_0 = tanh((R0 - r) / width), r the distance from `center` = (cz, cy, cx)."""
    zz, yy, xx = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    r = np.sqrt((zz - center[0]) ** 2 + (yy - center[1]) ** 2 + (xx - center[2]) ** 2)
    return np.tanh((R0 - r) / width)


def cavity_solid(shape, r_in: float, r_out: float, depth: int) -> np.ndarray:
    """A cylindrical cup on the wall z = -1/2: the ring r_in <= r < r_out (r the in-plane distance
    from the box axis) of the first `depth` planes is solid."""
    nz, ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    r = np.sqrt((yy - (ny - 1) / 2.0) ** 2 + (xx - (nx - 1) / 2.0) ** 2)
    out = np.zeros(shape, np.uint8)
    out[:depth] = ((r >= r_in) & (r < r_out)).astype(np.uint8)
    return out


def pinned_cap_phase(shape, r_in: float, r_out: float, depth: int, angle_deg: float,
                     width: float = 2.0) -> np.ndarray:
    """Liquid filling the cup (r < r_in below its rim) and a spherical cap on it whose edge sits
    on the outer rim r_out at the given contact angle: sphere radius r_out / sin(angle), centre
    -r_out / tan(angle) above the rim plane z = depth - 1/2; tanh profiles of the given width."""
    nz, ny, nx = shape
    th = np.deg2rad(angle_deg)
    R = r_out / np.sin(th)
    zc = depth - 0.5 - r_out / np.tan(th)
    zz, yy, xx = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in shape), indexing="ij")
    r = np.sqrt((yy - (ny - 1) / 2.0) ** 2 + (xx - (nx - 1) / 2.0) ** 2)
    cap = np.tanh((R - np.sqrt(r ** 2 + (zz - zc) ** 2)) / width)
    cup = np.tanh((r_in - r) / width)
    return np.where(zz < depth, cup, cap)


def centred(shape) -> Tuple[float, float, float]:
    return tuple((n - 1) / 2.0 for n in shape)


def uniform_noise(shape, amplitude: float, seed: int = SEED, dtype=np.float64) -> np.ndarray:
    return rng(seed).uniform(-amplitude, amplitude, size=shape).astype(dtype)


def radial_basis(shape: Tuple[int, int, int], center_yx, R: float, K: int) -> np.ndarray:
    """(r/R)^k for k = 1..K, r the in-plane (y, x) distance from the cap axis; [K, nz, ny, nx]."""
    nz, ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    r = np.sqrt((yy - center_yx[0]) ** 2 + (xx - center_yx[1]) ** 2) / R
    out = np.empty((K, nz, ny, nx))
    for k in range(1, K + 1):
        out[k - 1] = np.broadcast_to(r ** k, (nz, ny, nx))
    return out


def poly_flux(basis: np.ndarray, phi0: float, a: np.ndarray) -> np.ndarray:
    """phi(x) = phi0 (1 + sum_k a_k (r/R)^k)."""
    return phi0 * (1.0 + np.tensordot(np.asarray(a, np.float64), basis, axes=1))


# ------------------------------------------------------------------ workloads --------------

@dataclass
class Case:
    """One lattice: parameters in the paper's notation plus its initial phase field recipe."""
    name: str
    q: int
    shape: Tuple[int, int, int]          # (nz, ny, nx)
    periodic: Tuple[int, int, int] = (1, 1, 1)   # (x, y, z)
    rho_r_in: float = 1.0
    rho_b_in: float = 1.0
    tau_r: float = 1.0
    tau_b: float = 1.0
    sigma: float = sigma_from_amplitude(0.01)
    beta: float = 0.7
    site_rule: int = RULE_BAND
    threshold: float = 0.5
    sbar: float = 3.0
    phi: float = 1e-5
    steps: int = 1000
    geometry: str = "drop"              # "drop" | "slab" | "cap" | "half"
    R0: float = 0.0
    noise: float = 0.0
    seed: int = SEED
    extra: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.shape))

    def phase(self) -> np.ndarray:
        if self.geometry == "drop":
            return sphere_phase(self.shape, centred(self.shape), self.R0)
        if self.geometry == "slab":
            ax = self.extra.get("axis", 1)
            return slab_phase(self.shape, ax, (self.shape[ax] - 1) / 2.0,
                              self.extra.get("half_width", 16.0))
        if self.geometry == "half":
            return half_space_phase(self.shape, self.extra.get("axis", 1), self.extra["level"])
        if self.geometry == "cap":
            nz, ny, nx = self.shape
            return sphere_phase(self.shape, (-0.5, (ny - 1) / 2.0, (nx - 1) / 2.0), self.R0)
        if self.geometry == "pinned":
            return pinned_cap_phase(self.shape, **self.extra)
        raise ValueError(self.geometry)

    def solid(self) -> Optional[np.ndarray]:
        """Solid cells of the geometry (uint8 [nz, ny, nx]) or None."""
        if self.geometry == "pinned":
            return cavity_solid(self.shape, **{k: self.extra[k] for k in ("r_in", "r_out", "depth")})
        return None

    def noise_array(self, dtype=np.float64) -> Optional[np.ndarray]:
        if self.noise == 0.0:
            return None
        return uniform_noise((2, self.q) + tuple(self.shape), self.noise, self.seed, dtype)


def flat_slab_2d() -> Case:
    """D2Q9, FP64, 64x64 periodic, slab of width 32 across y, phi = 1e-5, band |rho^N| < 0.5."""
    return Case("flat_slab_2d", 9, (1, 64, 64), geometry="slab", phi=1e-5, steps=2000,
                extra={"axis": 1, "half_width": 16.0})


def drop_2d(phi: float = 1e-5, theta: float = 0.5) -> Case:
    """D2Q9 circular drop R0 = 40 centred in a 256x256 periodic box, noise U(-1e-6, 1e-6)."""
    return Case("drop_2d", 9, (1, 256, 256), R0=40.0, phi=phi, threshold=theta, noise=1e-6,
                steps=1000)


def drop_2d_sweep() -> List[Case]:
    out = []
    for phi in np.logspace(-6, -4, 5):
        for theta in (0.3, 0.5, 0.7):
            out.append(drop_2d(float(phi), theta))
    return out


def sphere_3d(n: int = 192, R0: float = 32.0) -> Case:
    """D3Q19 spherical drop R0 = 32 in a 192^3 periodic box, rho_l/rho_g = 10, tau_l = 1,
    tau_g = 0.8, A = 0.005, beta = 0.7, phi = 1e-5, band threshold 0.5, 5000 steps."""
    return Case("sphere_3d", 19, (n, n, n), rho_r_in=10.0, rho_b_in=1.0, tau_r=1.0, tau_b=0.8,
                sigma=sigma_from_amplitude(0.005), beta=0.7, phi=1e-5, R0=R0, steps=5000,
                noise=1e-6)


def sessile_cap_3d(shape=(128, 256, 256), R0: float = 48.0, phi0: float = 2e-5) -> Case:
    """D3Q19 90-degree cap of radius R0 on the bounce-back wall z = -1/2 of a box with walls at
    both ends of z, unit density ratio, A = 0.005, band threshold 0.5, FP32, 2000 steps."""
    return Case("sessile_cap_3d", 19, tuple(shape), periodic=(1, 1, 0), R0=R0, phi=phi0,
                geometry="cap", steps=2000, sigma=sigma_from_amplitude(0.005))


def pinned_cap_3d(n: int = 192, phi: float = 3e-3) -> Case:
    """The pinned spherical cap of Sec. III.A.4: D3Q19 n^3, walls at both ends of z, a cylindrical
    cup (inner radius 50, outer radius 53, depth 8) on the wall z = -1/2, a cap pinned on its outer
    rim at about 120 degrees; unit density ratio, beta = 0.99, sigma = 0.1, Gamma = 0.305 with |F|
    of the previous step, S-bar = 3."""
    return Case("pinned_cap_3d", 19, (n, n, n), periodic=(1, 1, 0), sigma=0.1, beta=0.99,
                site_rule=RULE_GRADIENT, threshold=0.305, sbar=3.0, phi=phi, geometry="pinned",
                extra={"r_in": 50.0, "r_out": 53.0, "depth": 8, "angle_deg": 120.0})


def flux_fit_parameters(K: int = 16, seed: int = SEED):
    """Coefficients of the flux polynomial: a ~ N(0, 0.1) (seed) and the target set a_target ~
    N(0, 0.1) (seed + 1), K each."""
    return (rng(seed).normal(0.0, 0.1, K), rng(seed + 1).normal(0.0, 0.1, K))


def ensemble_members(seed: int = SEED) -> List[Case]:
    """48 D2Q9 drops (R0 ~ U(16, 64), side = 32 ceil(4 R0 / 32)) and 16 D3Q19 drops
    (R0 ~ U(12, 32), side = ceil(4 R0)); phi log-uniform in 1e-6..1e-4, density ratio in
    {1, 2, 5, 10}, threshold ~ U(0.3, 0.7); tau = 1, A = 0.01 (2D) / 0.005 (3D), beta = 0.7."""
    g = rng(seed)
    out = []
    for m in range(64):
        three_d = m >= 48
        if three_d:
            R0 = float(g.uniform(12.0, 32.0))
            side = int(np.ceil(4.0 * R0))
            shape = (side, side, side)
            A = 0.005
        else:
            R0 = float(g.uniform(16.0, 64.0))
            side = int(32 * np.ceil(4.0 * R0 / 32.0))
            shape = (1, side, side)
            A = 0.01
        phi = float(10.0 ** g.uniform(-6.0, -4.0))
        gamma = float(g.choice([1.0, 2.0, 5.0, 10.0]))
        theta = float(g.uniform(0.3, 0.7))
        out.append(Case(f"member{m:02d}", 19 if three_d else 9, shape, rho_r_in=gamma,
                        rho_b_in=1.0, sigma=sigma_from_amplitude(A), phi=phi, threshold=theta,
                        R0=R0, steps=1000, seed=seed + 1 + m))
    return out


def shrink(case: Case, shape, **kw) -> Case:
    """The same physics on another box (used for oracle-sized parity cases)."""
    return replace(case, shape=tuple(shape), **kw)
