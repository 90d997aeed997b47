"""FP64 autograd statement of the step -- TEST INFRASTRUCTURE ONLY (part of the oracle).

The timestep of ``cg_oracle.c`` restated with whole-lattice PyTorch CPU tensor operations in
FP64, so that ``torch.autograd`` supplies the reverse-mode derivative that the library's
hand-written adjoint must reproduce.  The stages follow the paper's Sec. II in the order of its
method summary:

  Eq. (Stream), pull form: f_i^k(x) = f_i^{k*}(x - c_i); halfway bounce-back f_{opp i}^{k*}(x)
      where x - c_i is solid or beyond a wall (Sec. III, first paragraph);
  the site set x_I of the step (given: recorded from a run of the C oracle, so that derivatives
      are taken with x_I held fixed) and Eq. (exchange) with varphi = phi / S-bar (Eq. relation);
  moments rho_k, rho, u; harmonic 1/tau; alpha-bar (Sec. II.A);
  Eq. (cg): F = 3 sum_i W_i rho^N(x + c_i) c_i, rho^N of the cell itself where x + c_i is solid;
  Eq. (feq), Eq. (collision), Eq. (perturb) with amplitude (9/4) sigma / tau, Eq. (recolor) with
      cos(theta_i) = F.c_i / (|F| |c_i|) (0 for i = 0 or |F| = 0), and f^{b*} = f - f^{r*}.

The observable is the liquid volume V = sum over fluid cells of (1 + rho^N)/2 of a stored state.

Where w_r w_b < BULK_TRACE (bulk: one colour is a trace) the recoloring direction F/|F| is held
fixed for differentiation (its value is unchanged): in the bulk that direction is undefined at
F = 0 and the linearised dynamics of trace densities through it is scale-invariant and unstable,
so the exact tangent there says nothing about finite perturbations of the flux.

Pins (tests/test_oracle_adjoint.py): its states equal the C oracle's step for step; its gradient
equals central finite differences of the C oracle replaying the same site sets; and for one
step it equals the closed form dV(1)/dphi(x) = -m(x) / (rho(x) S-bar).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch

from . import RULE_GIVEN, Params, Run, alphas, lattice

torch_dtype = torch.float64
BULK_TRACE = 1e-6


class Geometry:
    """Neighbour masks of a lattice: which pull sources and gradient neighbours are fluid cells."""

    def __init__(self, p: Params):
        self.p = p
        L = lattice(p.q)
        self.Q = p.q
        self.c = [tuple(int(v) for v in L["c"][i]) for i in range(p.q)]  # (cx, cy, cz)
        self.opp = [int(o) for o in L["opp"]]
        self.W = [float(v) for v in L["w"]]
        self.A = [float(v) for v in L["a"]]
        self.B = [float(v) for v in L["b"]]
        self.C = [float(v) for v in L["cw"]]
        shape = p.shape  # (nz, ny, nx)
        solid = np.zeros(shape, bool) if p.solid is None else np.asarray(p.solid).reshape(shape) != 0
        self.fluid = torch.from_numpy(~solid)
        self.coords = [torch.arange(n).view(*[n if d == k else 1 for d in range(3)])
                       for k, n in enumerate(shape)]  # z, y, x index grids
        self.src_ok = [self.inside(tuple(-v for v in self.c[i])) & self.shift(self.fluid, self.c[i])
                       for i in range(self.Q)]
        self.nb_ok = [self.inside(self.c[i]) & self.shift(self.fluid, tuple(-v for v in self.c[i]))
                      for i in range(self.Q)]

    def shift(self, t: torch.Tensor, d) -> torch.Tensor:
        """The value at x - d (periodic wrap; callers mask what lies beyond a wall)."""
        return torch.roll(t, shifts=(d[2], d[1], d[0]), dims=(-3, -2, -1))

    def inside(self, d) -> torch.Tensor:
        """x + d lies inside the box or wraps across a periodic axis."""
        shape = self.p.shape
        ok = torch.ones(shape, dtype=torch.bool)
        per = self.p.periodic  # (x, y, z)
        for axis, dim in ((0, 2), (1, 1), (2, 0)):
            if d[axis] == 0 or per[axis]:
                continue
            s = self.coords[dim] + d[axis]
            ok = ok & ((s >= 0) & (s < shape[dim])).expand(shape)
        return ok


def volume(geo: Geometry, f: torch.Tensor) -> torch.Tensor:
    rr, rb = f[0].sum(0), f[1].sum(0)
    rho = torch.where(geo.fluid, rr + rb, torch.ones_like(rr))
    return torch.where(geo.fluid, 0.5 * (1.0 + (rr - rb) / rho), torch.zeros_like(rr)).sum()


def step(geo: Geometry, f: torch.Tensor, phi: torch.Tensor, site: torch.Tensor) -> torch.Tensor:
    """One timestep of the state f [2, Q, nz, ny, nx] with flux field phi and the site set site."""
    p, Q, c = geo.p, geo.Q, geo.c
    ar, ab = alphas(p)
    # Eq. (Stream), pull form, with halfway bounce-back
    g = torch.stack([
        torch.stack([torch.where(geo.src_ok[i], geo.shift(f[k, i], c[i]), f[k, geo.opp[i]])
                     for i in range(Q)])
        for k in range(2)])
    # Eq. (exchange) at the sites, varphi = phi / S-bar (Eq. relation)
    e = torch.where(site & geo.fluid, phi / p.sbar, torch.zeros_like(phi))
    g = torch.stack([torch.cat([(g[0, 0] - e)[None], g[0, 1:]]),
                     torch.cat([(g[1, 0] + e)[None], g[1, 1:]])])
    # moments (Sec. II.A)
    rr, rb = g[0].sum(0), g[1].sum(0)
    rho = torch.where(geo.fluid, rr + rb, torch.ones_like(rr))
    fc = g[0] + g[1]
    u = [sum(fc[i] * c[i][d] for i in range(Q) if c[i][d] != 0) / rho for d in range(3)]
    u = [ud if torch.is_tensor(ud) else torch.zeros_like(rho) for ud in u]
    itau = (rr / rho) / p.tau_r + (rb / rho) / p.tau_b
    abar = (rr * ar + rb * ab) / rho
    rhoN = torch.where(geo.fluid, (rr - rb) / rho, torch.zeros_like(rho))
    # Eq. (cg)
    F = []
    for d in range(3):
        acc = torch.zeros_like(rho)
        for i in range(1, Q):
            if c[i][d] == 0:
                continue
            nb = torch.where(geo.nb_ok[i], geo.shift(rhoN, tuple(-v for v in c[i])), rhoN)
            acc = acc + 3.0 * geo.W[i] * c[i][d] * nb
        F.append(acc)
    F2 = F[0] ** 2 + F[1] ** 2 + F[2] ** 2
    pos = F2 > 0
    Fn_safe = torch.sqrt(torch.where(pos, F2, torch.ones_like(F2)))
    Fn = torch.where(pos, Fn_safe, torch.zeros_like(F2))
    iFn = torch.where(pos, 1.0 / Fn_safe, torch.zeros_like(F2))
    uu = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    amp = 9.0 * p.sigma / 4.0
    bulk = (rr / rho) * (rb / rho) < BULK_TRACE
    out_r, out_b = [], []
    for i in range(Q):
        cu = sum(c[i][d] * u[d] for d in range(3))
        Fc = sum(c[i][d] * F[d] for d in range(3))
        rest = rho * (geo.A[i] + geo.B[i] * abar)          # f_i^eq(rho, 0) = rho phi_i(alpha-bar)
        feq = rest + rho * geo.W[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)   # Eq. (feq)
        fi = fc[i] - itau * (fc[i] - feq)                                    # Eq. (collision)
        fi = fi + amp * itau * (geo.W[i] * Fc * Fc * iFn - geo.C[i] * Fn)   # Eq. (perturb)
        norm = float(np.sqrt(sum(v * v for v in c[i])))
        cos = Fc * iFn / norm if i else torch.zeros_like(rho)
        cos = torch.where(bulk, cos.detach(), cos)
        fr = (rr / rho) * fi + p.beta * (rr * rb / (rho * rho)) * cos * rest  # Eq. (recolor)
        out_r.append(torch.where(geo.fluid, fr, torch.zeros_like(fr)))
        out_b.append(torch.where(geo.fluid, fi - fr, torch.zeros_like(fr)))
    return torch.stack([torch.stack(out_r), torch.stack(out_b)])


def record_sites(p: Params, f0: np.ndarray, nsteps: int) -> List[np.ndarray]:
    """Site sets x_I of nsteps steps of the C oracle from f0 (the rule of p)."""
    run = Run(p, f0)
    out = []
    for _ in range(nsteps):
        run.step(1)
        out.append(run.mask.copy())
    return out


def volume_history(p: Params, f0: np.ndarray, phi: torch.Tensor,
                   sites: Sequence[np.ndarray]) -> torch.Tensor:
    """V(0..T) of T = len(sites) steps from f0 with flux field phi, differentiable in phi."""
    geo = Geometry(p)
    f = torch.from_numpy(np.ascontiguousarray(f0, np.float64))
    V = [volume(geo, f)]
    for m in sites:
        f = step(geo, f, phi, torch.from_numpy(np.asarray(m).reshape(p.shape) != 0))
        V.append(volume(geo, f))
    return torch.stack(V)


def states(p: Params, f0: np.ndarray, phi: np.ndarray, sites: Sequence[np.ndarray]):
    """The states after each step (numpy), for comparison with the C oracle."""
    geo = Geometry(p)
    f = torch.from_numpy(np.ascontiguousarray(f0, np.float64))
    ph = torch.from_numpy(np.ascontiguousarray(phi, np.float64))
    out = []
    with torch.no_grad():
        for m in sites:
            f = step(geo, f, ph, torch.from_numpy(np.asarray(m).reshape(p.shape) != 0))
            out.append(f.numpy().copy())
    return out


def replay_volumes(p: Params, f0: np.ndarray, phi: np.ndarray,
                   sites: Sequence[np.ndarray]) -> np.ndarray:
    """V(0..T) of the C oracle replaying the site sets (rule "given") with flux field phi."""
    import dataclasses
    q = dataclasses.replace(p, site_rule=RULE_GIVEN, phi_field=np.ascontiguousarray(phi, np.float64),
                            mask_given=np.zeros(p.shape, np.uint8))
    fluid = np.ones(p.shape, bool) if p.solid is None else np.asarray(p.solid).reshape(p.shape) == 0
    run = Run(q, f0)

    def vol():
        m = run.macros()
        return float(np.sum(0.5 * (1.0 + m["rhoN"])[fluid]))

    V = [vol()]
    for m in sites:
        run.p.mask_given = np.ascontiguousarray(np.asarray(m).reshape(p.shape), np.uint8)
        run.step(1)
        V.append(vol())
    return np.array(V)
