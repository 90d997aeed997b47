// step_kernel.cuh -- the fused timestep: one pass over HBM per step.
//
// Work decomposition.  A CTA owns a tile of TX x TY columns of the (a, b) plane (TY = 1 for
// D2Q9) and marches along m through a chunk of PC planes.  For every plane it
//   (1) pulls the populations of plane m+1 (Eq. Stream, pull form, halfway bounce-back),
//       decides the evaporation sites and applies Eq. (exchange), and writes the post-exchange
//       phase field rho^N of the tile plus a one-cell ring into a 4-plane shared-memory ring;
//   (2) after one __syncthreads, collides plane m (moments, Eq. cg stencil from the ring,
//       Eq. collision/feq, Eq. perturb, Eq. recolor) from populations it pulled one iteration
//       earlier and still holds in registers, and stores them.
// The ring cells around the tile (and the planes m0-1, m0+PC at the chunk ends) are pulled by
// this CTA as well -- redundant loads that hit L2 -- so each population is read from HBM once
// and written once per step.  Site counts and the removed mass are reduced with warp shuffles
// into one FP64 partial per CTA; the last CTA to finish folds the partials, in a fixed order,
// into the device ledger (deterministic).
#pragma once

#include "common.cuh"

namespace cgevap {

struct Slot {
  int a, b;                // wrapped coordinates
  int am1, ap1, bm1, bp1;  // neighbours along a and b (-1 beyond a wall)
  bool ok;                 // false beyond a wall
};

template <class L>
__device__ __forceinline__ Slot make_slot(const Geom& g, int ua, int ub) {
  Slot s;
  s.ok = true;
  int a = ua, b = ub;
  if (a < 0 || a >= g.na) {
    if (g.per_a) a = wrap(a, g.na);
    else s.ok = false;
  }
  if (L::D3) {
    if (b < 0 || b >= g.nb) {
      if (g.per_b) b = wrap(b, g.nb);
      else s.ok = false;
    }
  } else {
    b = 0;
  }
  s.a = a;
  s.b = b;
  s.am1 = step_coord(a, -1, g.na, g.per_a);
  s.ap1 = step_coord(a, +1, g.na, g.per_a);
  s.bm1 = L::D3 ? step_coord(b, -1, g.nb, g.per_b) : 0;
  s.bp1 = L::D3 ? step_coord(b, +1, g.nb, g.per_b) : 0;
  return s;
}

struct Plane {
  int m, mm1, mp1;
  bool ok;
};

__device__ __forceinline__ Plane make_plane(const Geom& g, int um) {
  Plane p;
  p.ok = true;
  int m = um;
  if (m < 0 || m >= g.nm) {
    if (g.per_m) {
      m = wrap(m, g.nm);
    } else {
      p.ok = false;
      m = 0;
    }
  }
  p.m = m;
  p.mm1 = step_coord(m, -1, g.nm, g.per_m);
  p.mp1 = step_coord(m, +1, g.nm, g.per_m);
  return p;
}

// Directions whose pull source lies beyond a wall, plus links of solid cells.  Returns false if
// the cell itself is not a fluid cell of the lattice.
template <class L>
__device__ __forceinline__ bool solid_bits(const Geom& g, const Slot& s, const Plane& p, int cell,
                                           uint32_t& bits) {
  constexpr uint32_t APOS = dirs_where<L>(0, +1), ANEG = dirs_where<L>(0, -1);
  constexpr uint32_t BPOS = dirs_where<L>(1, +1), BNEG = dirs_where<L>(1, -1);
  constexpr uint32_t MPOS = dirs_where<L>(2, +1), MNEG = dirs_where<L>(2, -1);
  if (!(s.ok && p.ok)) return false;
  uint32_t w = 0;
  if (s.am1 < 0) w |= APOS;
  if (s.ap1 < 0) w |= ANEG;
  if (L::D3) {
    if (s.bm1 < 0) w |= BPOS;
    if (s.bp1 < 0) w |= BNEG;
  }
  if (p.mm1 < 0) w |= MPOS;
  if (p.mp1 < 0) w |= MNEG;
  if (g.links) {
    uint32_t l = __ldg(g.links + cell);
    if (l >> 31) return false;
    w |= l;
  }
  bits = w;
  return true;
}

template <int S>
__device__ __forceinline__ typename Storage<S>::real flux_at(const Physics& ph, int cell) {
  using R = typename Storage<S>::real;
  if (ph.phi_field == nullptr) return (R)ph.varphi;
  return (R)__ldg(reinterpret_cast<const R*>(ph.phi_field) + cell) * (R)ph.inv_sbar;
}

// Steps 2-4 for one cell whose pulled populations are in g: decide whether it is a site, apply
// Eq. (exchange).  Returns rho^N after the exchange; g, rr, rb become post-exchange.
template <int Q, int S>
__device__ __forceinline__ typename Storage<S>::real site_exchange(
    const StepArgs& A, int cell, V2<typename Storage<S>::real> (&g)[Q],
    typename Storage<S>::real& rr, typename Storage<S>::real& rb, typename Storage<S>::real& e,
    uint32_t& flags) {
  using R = typename Storage<S>::real;
  R sr = R(0), sb = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    sr += g[i].r;
    sb += g[i].b;
  }
  bool site, near;
  if (A.ph.rule == 1) {
    const R rn = (sr - sb) / (sr + sb);
    const R d = fabs(rn) - (R)A.ph.threshold;
    site = d < R(0);
    near = fabs(d) < R(1e-6);
  } else {
    const uint32_t mb = A.mask_in[cell];
    site = (mb >> 1) & 1u;
    near = (mb >> 3) & 1u;
  }
  e = site ? flux_at<S>(A.ph, cell) : R(0);
  g[0].r -= e;
  g[0].b += e;
  rr = sr - e;
  rb = sb + e;
  flags = (site ? 1u : 0u) | (near ? 4u : 0u);
  return (rr - rb) / (rr + rb);
}

// Pull one cell (Eq. Stream, pull form; halfway bounce-back where the source is solid), then
// site_exchange.
template <int Q, int S>
__device__ __forceinline__ typename Storage<S>::real pull_exchange(
    const StepArgs& A, const Slot& s, const Plane& p, int cell, uint32_t sbits,
    V2<typename Storage<S>::real> (&g)[Q], typename Storage<S>::real& rr,
    typename Storage<S>::real& rb, typename Storage<S>::real& e, uint32_t& flags) {
  using L = Lattice<Q>;
  using IO = PopIO<S, Q>;
  const Geom& G = A.g;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ca = L::ca(i), cb = L::cb(i), cm = L::cm(i);
    const int as = ca > 0 ? s.am1 : (ca < 0 ? s.ap1 : s.a);
    const int bs = cb > 0 ? s.bm1 : (cb < 0 ? s.bp1 : s.b);
    const int ms = cm > 0 ? p.mm1 : (cm < 0 ? p.mp1 : p.m);
    const bool bounce = (sbits >> i) & 1u;
    const int src = bounce ? cell : (ms * G.nb + bs) * G.na + as;
    const int dir = bounce ? opp(i) : i;
    g[i] = IO::load(A.pin, G.ncell, i, dir, src, A.ph);
  }
  return site_exchange<Q, S>(A, cell, g, rr, rb, e, flags);
}

template <class R>
__device__ __forceinline__ void norm_pair(R F2, R& Fn, R& iFn);
template <>
__device__ __forceinline__ void norm_pair<double>(double F2, double& Fn, double& iFn) {
  Fn = sqrt(F2);
  iFn = 1.0 / Fn;
}
template <>
__device__ __forceinline__ void norm_pair<float>(float F2, float& Fn, float& iFn) {
  iFn = rsqrtf(F2);
  Fn = F2 * iFn;
}

// Moments, Eq. (collision) with Eq. (feq), Eq. (perturb), Eq. (recolor); stores f^{k*}.
// rnb[i] is rho^N at x + c_i (the cell's own value where that neighbour is solid).
template <int Q, int S>
__device__ __forceinline__ void collide_store(const StepArgs& A, int cell,
                                              const V2<typename Storage<S>::real> (&g)[Q],
                                              typename Storage<S>::real rr,
                                              typename Storage<S>::real rb,
                                              const typename Storage<S>::real (&rnb)[Q],
                                              typename Storage<S>::real& Fn_out) {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  using IO = PopIO<S, Q>;
  const Physics& ph = A.ph;
  const R rho = rr + rb;
  const R irho = R(1) / rho;
  const R wr = rr * irho, wb = rb * irho;
  R f[Q];
  R ja = R(0), jb = R(0), jm = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    f[i] = g[i].r + g[i].b;  // colour-blind population
    if (L::ca(i) > 0) ja += f[i];
    if (L::ca(i) < 0) ja -= f[i];
    if (L::cb(i) > 0) jb += f[i];
    if (L::cb(i) < 0) jb -= f[i];
    if (L::cm(i) > 0) jm += f[i];
    if (L::cm(i) < 0) jm -= f[i];
  }
  const R ua = ja * irho, ub = jb * irho, um = jm * irho;
  const R uu = ua * ua + ub * ub + um * um;
  const R itau = wr * (R)ph.inv_tau_r + wb * (R)ph.inv_tau_b;  // harmonic mean of tau_k
  const R abar = wr * (R)ph.alpha_r + wb * (R)ph.alpha_b;
  // Eq. (cg): F = (1/c_s^2) sum_i W_i rho^N(x + c_i) c_i
  R Fa = R(0), Fb = R(0), Fm = R(0);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const R t = R(3.0 * L::W(i)) * rnb[i];
    if (L::ca(i) > 0) Fa += t;
    if (L::ca(i) < 0) Fa -= t;
    if (L::cb(i) > 0) Fb += t;
    if (L::cb(i) < 0) Fb -= t;
    if (L::cm(i) > 0) Fm += t;
    if (L::cm(i) < 0) Fm -= t;
  }
  const R F2 = Fa * Fa + Fb * Fb + Fm * Fm;
  R Fn = R(0), iFn = R(0);
  if (F2 > R(0)) norm_pair<R>(F2, Fn, iFn);
  const R pamp = (R)ph.amp * itau;       // (9/4) sigma / tau
  const R rcol = (R)ph.beta * wr * wb;   // beta rho_r rho_b / rho^2
  V2<R> f0{R(0), R(0)};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R ca = R(L::ca(i)), cb = R(L::cb(i)), cm = R(L::cm(i));
    const R cu = ca * ua + cb * ub + cm * um;
    const R rest = rho * (R(L::A(i)) + R(L::B(i)) * abar);  // f_i^eq(rho, 0)
    const R feq = rest + rho * R(L::W(i)) * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
    R fi = f[i] - itau * (f[i] - feq);
    const R pc = ca * Fa + cb * Fb + cm * Fm;
    fi += pamp * (R(L::W(i)) * pc * pc * iFn - R(L::C(i)) * Fn);
    const R cosv = (i == 0) ? R(0) : pc * iFn * R(inv_norm<L>(i));
    const R fr = wr * fi + rcol * cosv * rest;
    const R fb = fi - fr;
    if (i == 0) f0 = {fr, fb};
    IO::store(A.pout, A.g.ncell, i, cell, fr, fb, f0, ph);
  }
  Fn_out = Fn;
}

template <int Q, int S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX* TY, MINB) cg_step_kernel(const __grid_constant__ StepArgs A) {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  constexpr int NT = TX * TY;
  constexpr int HX = TX + 2;
  constexpr int HY = L::D3 ? TY + 2 : 1;
  constexpr int OB = L::D3 ? 1 : 0;
  constexpr int NH = HX * HY - TX * TY;
  static_assert(NH <= NT, "one ring cell per thread at most");
  static_assert(L::D3 || TY == 1, "D2Q9 tiles are one row");
  __shared__ R ring[4][HY][HX];
  __shared__ double red_d[NT / 32];
  __shared__ long long red_n[NT / 32];
  __shared__ int is_last;

  const Geom& G = A.g;
  const int tid = threadIdx.x;
  const int a0 = (blockIdx.x % A.ntx) * TX;
  const int b0 = (blockIdx.x / A.ntx) * TY;
  const int m0 = blockIdx.y * A.pc;
  const int m1 = min(m0 + A.pc, G.nm);
  const int lx = tid % TX, ly = tid / TX;
  const bool active = (a0 + lx < G.na) && (b0 + ly < G.nb);
  const Slot me = make_slot<L>(G, a0 + lx, b0 + ly);

  // This thread's ring cell, if any.
  int hx = 0, hy = 0;
  const bool has_halo = tid < NH;
  if (has_halo) {
    if (L::D3) {
      if (tid < HX) {
        hx = tid;
        hy = 0;
      } else if (tid < 2 * HX) {
        hx = tid - HX;
        hy = HY - 1;
      } else {
        const int k = tid - 2 * HX;
        hx = (k & 1) ? HX - 1 : 0;
        hy = 1 + (k >> 1);
      }
    } else {
      hx = tid == 0 ? 0 : HX - 1;
      hy = 0;
    }
  }
  const Slot hs = make_slot<L>(G, a0 + hx - 1, b0 + hy - OB);

  V2<R> cur[Q], nxt[Q];
  R cur_rr = R(0), cur_rb = R(0), cur_e = R(0);
  uint32_t cur_flags = 0, cur_bits = 0;
  bool cur_ok = false;
  long long n_sites = 0;
  double removed = 0.0;

  // rho^N of the own slot and the ring slot in plane um; own populations kept in `keep`.
  auto fill_plane = [&](int um, V2<R>(&keep)[Q], R& k_rr, R& k_rb, R& k_e, uint32_t& k_flags,
                        uint32_t& k_bits, bool& k_ok) {
    const Plane p = make_plane(G, um);
    const int slot = (um - m0 + 1) & 3;
    if (has_halo) {
      const int cell = (p.m * G.nb + hs.b) * G.na + hs.a;
      uint32_t bits = 0;
      R rn = R(0);
      if (solid_bits<L>(G, hs, p, cell, bits)) {
        V2<R> tmp[Q];
        R t_rr, t_rb, t_e;
        uint32_t t_flags;
        rn = pull_exchange<Q, S>(A, hs, p, cell, bits, tmp, t_rr, t_rb, t_e, t_flags);
      }
      ring[slot][hy][hx] = rn;
    }
    {
      const int cell = (p.m * G.nb + me.b) * G.na + me.a;
      uint32_t bits = 0;
      R rn = R(0);
      k_ok = solid_bits<L>(G, me, p, cell, bits);
      if (k_ok) rn = pull_exchange<Q, S>(A, me, p, cell, bits, keep, k_rr, k_rb, k_e, k_flags);
      k_bits = bits;
      ring[slot][ly + OB][lx + 1] = rn;
    }
  };

  {
    V2<R> tmp[Q];
    R t_rr, t_rb, t_e;
    uint32_t t_flags, t_bits;
    bool t_ok;
    fill_plane(m0 - 1, tmp, t_rr, t_rb, t_e, t_flags, t_bits, t_ok);
  }
  fill_plane(m0, cur, cur_rr, cur_rb, cur_e, cur_flags, cur_bits, cur_ok);

  for (int m = m0; m < m1; ++m) {
    R n_rr = R(0), n_rb = R(0), n_e = R(0);
    uint32_t n_flags = 0, n_bits = 0;
    bool n_ok = false;
    fill_plane(m + 1, nxt, n_rr, n_rb, n_e, n_flags, n_bits, n_ok);
    __syncthreads();
    if (active && cur_ok) {
      const int s0 = (m - m0 + 1) & 3;
      const R own = ring[s0][ly + OB][lx + 1];
      R rnb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int s = (m - m0 + 1 + L::cm(i)) & 3;
        const bool solid_nb = (cur_bits >> opp(i)) & 1u;  // x + c_i is the source of opp(i)
        rnb[i] = solid_nb ? own : ring[s][ly + OB + L::cb(i)][lx + 1 + L::ca(i)];
      }
      const Plane p = make_plane(G, m);
      const int cell = (p.m * G.nb + me.b) * G.na + me.a;
      R Fn;
      collide_store<Q, S>(A, cell, cur, cur_rr, cur_rb, rnb, Fn);
      uint32_t mb = cur_flags;
      if (A.ph.rule == 0) {
        const R d = Fn - (R)A.ph.threshold;
        mb |= (d > R(0) ? 2u : 0u) | (fabs(d) < R(1e-6) ? 8u : 0u);
      }
      A.mask_out[cell] = (uint8_t)mb;
      if (cur_flags & 1u) {
        ++n_sites;
        removed += (double)cur_e;
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
    cur_rr = n_rr;
    cur_rb = n_rb;
    cur_e = n_e;
    cur_flags = n_flags;
    cur_bits = n_bits;
    cur_ok = n_ok;
  }

  // ---- ledger: warp shuffle, block, then the last block folds all partials in order ----
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_sites += __shfl_down_sync(0xffffffffu, n_sites, off);
    removed += __shfl_down_sync(0xffffffffu, removed, off);
  }
  if ((tid & 31) == 0) {
    red_d[tid >> 5] = removed;
    red_n[tid >> 5] = n_sites;
  }
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y;
  if (tid == 0) {
    double s = 0.0;
    long long n = 0;
    for (int w = 0; w < NT / 32; ++w) {
      s += red_d[w];
      n += red_n[w];
    }
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    A.red.part_removed[bid] = s;
    A.red.part_sites[bid] = n;
    __threadfence();
    const unsigned prev = atomicAdd(A.red.done, 1u);
    is_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (is_last && tid < 32) {
    __threadfence();
    double s = 0.0;
    long long n = 0;
    for (unsigned j = tid; j < nblk; j += 32) {
      s += __ldcg(A.red.part_removed + j);
      n += __ldcg(A.red.part_sites + j);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, off);
      n += __shfl_down_sync(0xffffffffu, n, off);
    }
    if (tid == 0) {
      DevLedger* led = A.red.ledger;
      led->evaporated += s;
      led->last_removed = s;
      led->site_steps += n;
      led->last_sites = n;
      led->steps += 1;
      *A.red.done = 0u;
    }
  }
}

}  // namespace cgevap
