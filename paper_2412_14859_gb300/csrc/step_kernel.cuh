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

#include <type_traits>

#include "common.cuh"

namespace cgevap {

struct Slot {
  int a, b;                // wrapped coordinates
  int am1, ap1, bm1, bp1;  // neighbours along a and b (-1 beyond a wall)
  int dxm, dxp, dym, dyp;  // storage offsets to the pull sources at a-1, a+1, b-1, b+1
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
  // beyond a wall the offset is never used (the link bounces back); keep it in bounds anyway
  s.dxm = s.am1 >= 0 ? s.am1 - a : 0;
  s.dxp = s.ap1 >= 0 ? s.ap1 - a : 0;
  s.dym = s.bm1 >= 0 ? (s.bm1 - b) * g.pitch : 0;
  s.dyp = s.bp1 >= 0 ? (s.bp1 - b) * g.pitch : 0;
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
  if (ph.phi_field == nullptr) return PHYS(R, ph, varphi);
  return (R)__ldg(reinterpret_cast<const R*>(ph.phi_field) + cell) * PHYS(R, ph, inv_sbar);
}

template <class R>
__device__ __forceinline__ R recip(R x);
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return 1.0 / x;
}
template <>
__device__ __forceinline__ float recip<float>(float x) {
  return __frcp_rn(x);
}

// Steps 2-4 for one cell whose pulled populations are in g: decide whether it is a site, apply
// Eq. (exchange).  Returns rho^N after the exchange; g, rr, rb become post-exchange and irho is
// 1 / rho (rho is not changed by the exchange).
// The decision and Eq. (exchange) from the colour totals sr, sb of the pulled populations:
// returns rho^N after the exchange and sets rr, rb (post-exchange), e (mass moved), flags, irho.
template <int S>
__device__ __forceinline__ typename Storage<S>::real exchange_from_sums(
    const StepArgs& A, int cell, typename Storage<S>::real sr, typename Storage<S>::real sb,
    typename Storage<S>::real& rr, typename Storage<S>::real& rb, typename Storage<S>::real& e,
    uint32_t& flags, typename Storage<S>::real& irho) {
  using R = typename Storage<S>::real;
  irho = recip<R>(sr + sb);
  const R rn_pre = (sr - sb) * irho;
  bool site, near;
  if (A.ph.rule == 1) {
    const R d = fabs(rn_pre) - PHYS(R, A.ph, threshold);
    site = d < R(0);
    near = fabs(d) < R(1e-6);
  } else {
    // gradient rule: the decision of the previous step (bit 1); given rule: bit 0
    const uint32_t mb = A.mask_in[cell];
    const int sh = A.ph.rule == 2 ? 0 : 1;
    site = (mb >> sh) & 1u;
    near = (mb >> (sh + 2)) & 1u;
  }
  e = site ? flux_at<S>(A.ph, cell) : R(0);
  rr = sr - e;
  rb = sb + e;
  flags = (site ? 1u : 0u) | (near ? 4u : 0u);
  return rn_pre - R(2) * e * irho;
}

template <int Q, int S>
__device__ __forceinline__ typename Storage<S>::real site_exchange(
    const StepArgs& A, int cell, V2<typename Storage<S>::real> (&g)[Q],
    typename Storage<S>::real& rr, typename Storage<S>::real& rb, typename Storage<S>::real& e,
    uint32_t& flags, typename Storage<S>::real& irho) {
  using R = typename Storage<S>::real;
  R sr = R(0), sb = R(0);
  if constexpr (std::is_same<R, float>::value) {  // both components in packed FP32
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < Q; ++i) acc = __fadd2_rn(acc, make_float2(g[i].r, g[i].b));
    sr = acc.x;
    sb = acc.y;
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      sr += g[i].r;
      sb += g[i].b;
    }
  }
  const R rn = exchange_from_sums<S>(A, cell, sr, sb, rr, rb, e, flags, irho);
  g[0].r -= e;
  g[0].b += e;
  return rn;
}

// Storage offsets from a cell in plane m to its pull sources in planes m-1 (dm_lo, used by
// directions with c_m = +1) and m+1 (dm_hi); 0 where that plane lies beyond a wall (those links
// bounce back and the offset is never used).
struct PlaneOffsets {
  int dm_lo, dm_hi;
};
__device__ __forceinline__ PlaneOffsets plane_offsets(const Geom& g, int m) {
  const int ps = g.rows * g.pitch;
  PlaneOffsets o;
  o.dm_lo = m > 0 ? -ps : (g.per_m ? (g.nm - 1) * ps : 0);
  o.dm_hi = m < g.nm - 1 ? ps : (g.per_m ? -(g.nm - 1) * ps : 0);
  return o;
}

// Error-free sums (Knuth's TwoSum; Dekker's Fast2Sum where |a| >= |b|): s = fl(a + b) and the
// rounding error a + b - s, exact in round-to-nearest.  Used to carry each colour's mass of a
// cell exactly through the 16-bit storages' step.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {  // fl(a - b), one rounding
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// hi += v with the error added to lo (|hi| >= |v| per component; else lo is approximate)
__device__ __forceinline__ void fast_two_sum_acc(float2& hi, float2& lo, float2 v) {
  const float2 s = __fadd2_rn(hi, v);
  lo = __fadd2_rn(lo, sub2(v, sub2(s, hi)));
  hi = s;
}
// TwoSum error of s = fl(a + b) per component (no ordering needed)
__device__ __forceinline__ float2 two_sum_err2(float2 a, float2 b, float2 s) {
  const float2 bb = sub2(s, a);
  return __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// A running error-free sum per colour starts at the power of two B = Physics::sum_base, which is
// at least any single population, so Fast2Sum's condition |hi| >= |v| holds for every term.
// Started from the first term instead, a larger later term (a red population arriving at a
// gas-side interface cell, whose own red is small) leaves that term's error inexact.  hi - B is
// exact (Sterbenz: B/2 <= hi <= 2B, or hi and B both multiples of ulp(B)).
__device__ __forceinline__ float2 sum_start(const Physics& ph) {
  return make_float2(ph.sum_base, ph.sum_base);
}
// (hi, lo) started at B -> hi = fl(total), lo = total - hi (up to lo's own roundings)
__device__ __forceinline__ void sum_finish(const Physics& ph, float2& hi, float2& lo) {
  const float2 h = sub2(hi, sum_start(ph));
  const float2 t = __fadd2_rn(h, lo);
  lo = two_sum_err2(h, lo, t);
  hi = t;
}

// Pull one cell (Eq. Stream, pull form).  Sources are the slot's wrap-aware in-plane offsets plus
// the plane offsets; where the source is solid or beyond a wall the population leaving the cell
// comes back reversed (halfway bounce-back).
template <int Q, int S>
__device__ __forceinline__ void pull_cell(const StepArgs& A, const Slot& sl, int si,
                                          PlaneOffsets po, uint32_t sbits,
                                          V2<typename Storage<S>::real> (&g)[Q]) {
  using L = Lattice<Q>;
  using IO = PopIO<S, Q>;
  if (sbits == 0) {  // no link of this cell bounces back (the common case)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                      (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                      (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      g[i] = IO::load(A.pin, A.g.nstore, i, i, src, A.ph);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
              (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
              (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
    const bool bounce = (sbits >> i) & 1u;
    src = bounce ? si : src;
    const int dir = bounce ? opp(i) : i;
    g[i] = IO::load(A.pin, A.g.nstore, i, dir, src, A.ph);
  }
}

// Deviation storage: pull one cell whose source rest populations are staged in shared memory.
// restbox(q, y, x) is the (f_0^r, f_0^b) pair of the cell at box row y, column x of plane slot q;
// (ex, ey) is this cell's own box position and ps[k] the slot of plane m + 1 - k, so the source
// plane m - c_m of direction i is ps[1 + c_m].  The step needs of the pulled pairs only the
// colour-blind values and the two colour totals (Eq. exchange changes the totals, not the
// colour-blind rest population), so that is what comes out: g_i = (f_i^r + f_i^b, 0) and
// (sr, sb) = the sums of each colour over i; Q + 2 live values instead of 2Q.  (lr, lb) are the
// rounding errors of those sums: sr + lr is the exact sum of the decoded values (Fast2Sum from
// the base B, see sum_start).
template <int Q, int S, class RestBox>
__device__ __forceinline__ void pull_cell_dev(const StepArgs& A, const Slot& sl, int si,
                                              PlaneOffsets po, uint32_t sbits, int ex, int ey,
                                              const int (&ps)[3], const RestBox& restbox,
                                              V2<float> (&g)[Q], float& sr, float& sb,
                                              float& lr, float& lb) {
  using L = Lattice<Q>;
  using P = typename Storage<S>::packed;
  const Physics& ph = A.ph;
  const P* dev = reinterpret_cast<const P*>(reinterpret_cast<const char*>(A.pin) +
                                            dev_block_offset(A.g.nstore));
  const int ns = A.g.nstore;
  uint32_t raw[Q];
  const float2 r0 = restbox(ps[1], ey, ex);
  g[0] = {r0.x + r0.y, 0.0f};
  float2 acc = sum_start(ph), lo = make_float2(0.0f, 0.0f);
  fast_two_sum_acc(acc, lo, r0);
  if (sbits == 0) {  // no link bounces back: every address is a fixed offset
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                      (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                      (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      const P v = __ldg(dev + (i - 1) * ns + src);
      raw[i] = *reinterpret_cast<const uint32_t*>(&v);
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const float2 rs = restbox(ps[1 + L::cm(i)], ey - L::cb(i), ex - L::ca(i));
      P pv;
      *reinterpret_cast<uint32_t*>(&pv) = raw[i];
      const float2 d = Storage<S>::unpack(pv);
      const float2 v = __ffma2_rn(rs, make_float2(ph.kap_r[i], ph.kap_b[i]),
                                  __fmul2_rn(d, make_float2(ph.inv_scale, ph.inv_scale)));
      fast_two_sum_acc(acc, lo, v);
      g[i] = {v.x + v.y, 0.0f};
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      const bool bounce = (sbits >> i) & 1u;
      src = bounce ? si : src;
      const int dir = bounce ? opp(i) : i;
      const P v = __ldg(dev + (size_t)(dir - 1) * ns + src);
      raw[i] = *reinterpret_cast<const uint32_t*>(&v);
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const bool bounce = (sbits >> i) & 1u;
      // the source's rest pair: box position x - c_i in plane m - c_i,m (own cell if bounced)
      const float2 rs = bounce ? r0 : restbox(ps[1 + L::cm(i)], ey - L::cb(i), ex - L::ca(i));
      P pv;
      *reinterpret_cast<uint32_t*>(&pv) = raw[i];
      const float2 d = Storage<S>::unpack(pv);
      const float2 v = __ffma2_rn(rs, make_float2(ph.kap_r[i], ph.kap_b[i]),
                                  __fmul2_rn(d, make_float2(ph.inv_scale, ph.inv_scale)));
      fast_two_sum_acc(acc, lo, v);
      g[i] = {v.x + v.y, 0.0f};
    }
  }
  sum_finish(ph, acc, lo);
  sr = acc.x;
  sb = acc.y;
  lr = lo.x;
  lb = lo.y;
}

// Recolour-on-pull layout: pull one cell's colour-blind populations and split each into its
// colours with the source cell's record (w_r, V), staged in shared memory; recbox(q, y, x) as
// restbox above.  f_i^r = w_r f_i + s_|c| (c_dir . V) with dir the stored direction (opp(i),
// c_dir = -c_i, for a bounced link, whose source is the cell itself).  Output as for
// pull_cell_dev: g_i = (f_i, 0) and the colour totals; the blue total sums each direction's own
// blue part f_i - f_i^r (small terms, not the difference of two large sums, which would cost the
// density-ratio-10 case its FP32 tolerance).
template <int Q, class RecBox>
__device__ __forceinline__ void pull_cell_rc(const StepArgs& A, const Slot& sl, int si,
                                             PlaneOffsets po, uint32_t sbits, int ex, int ey,
                                             const int (&ps)[3], const RecBox& recbox,
                                             V2<float> (&g)[Q], float& sr, float& sb) {
  using L = Lattice<Q>;
  const float* pop = reinterpret_cast<const float*>(A.pin);
  const int ns = A.g.nstore;
  float fv[Q];
  // all population loads first (fixed offsets unless a link bounces back)
  if (sbits == 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                      (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                      (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      fv[i] = __ldg(pop + i * ns + src);
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      const bool bounce = (sbits >> i) & 1u;
      src = bounce ? si : src;
      const int dir = bounce ? opp(i) : i;
      fv[i] = __ldg(pop + (size_t)dir * ns + src);
    }
  }
  const float4 r0 = recbox(ps[1], ey, ex);
  float2 acc;
  {
    const float fr = r0.x * fv[0];
    acc = make_float2(fr, fv[0] - fr);
    g[0] = {fv[0], 0.0f};
  }
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const bool bounce = sbits && ((sbits >> i) & 1u);
    const float4 r = bounce ? r0 : recbox(ps[1 + L::cm(i)], ey - L::cb(i), ex - L::ca(i));
    float cv = 0.0f;
    if (L::ca(i) > 0) cv += r.y;
    if (L::ca(i) < 0) cv -= r.y;
    if (L::cb(i) > 0) cv += r.z;
    if (L::cb(i) < 0) cv -= r.z;
    if (L::cm(i) > 0) cv += r.w;
    if (L::cm(i) < 0) cv -= r.w;
    if (bounce) cv = -cv;
    const float fr = fmaf(r.x, fv[i], float(rc_factor<L>(i)) * cv);
    acc = __fadd2_rn(acc, make_float2(fr, fv[i] - fr));
    g[i] = {fv[i], 0.0f};
  }
  sr = acc.x;
  sb = acc.y;
}

// 16-bit recolour-on-pull layout: pull one cell.  Each moving population is decoded from its
// 16-bit deviation and the source's rest-state scale Rf, f_i = fl(r_i Rf + dev / s), and split
// with the source's record as pull_cell_rc does.  rec / ref are the staged record and scale boxes
// (flat shared arrays of RS x RY x RX); bx[k] is the flat index of this cell's box position in
// plane m + 1 - k, the plane that the pull sources of the directions with c_m = k - 1 lie in
// (k = 1: this plane), so the source of direction i sits at the compile-time offset
// -(c_i,b RX + c_i,a) from bx[1 + c_i,m].  The rest pair (f_0^r, f_0^b) is the cell's own, read
// from global memory.  Output as pull_cell_dev: g_i = (f_i, 0), the colour totals (sr, sb) summed
// with Fast2Sum from the base B, rest pair first, and their rounding errors (lr, lb): sr + lr is
// the exact sum of the split values.  A cell none of whose links bounces back (sbits == 0, nearly every cell)
// takes a path whose addresses are all fixed offsets; the others take the general one.
// The global loads of pull_cell_rc16: the 16-bit values of the cell's pulled moving populations
// (raw[i], i >= 1) and its own rest pair r0 (they need nothing staged).
template <int Q, int S>
__device__ __forceinline__ void rc16_load(const StepArgs& A, const Slot& sl, int si, PlaneOffsets po,
                                          uint32_t sbits, unsigned short (&raw)[Q], float2& r0) {
  using L = Lattice<Q>;
  const char* base = reinterpret_cast<const char*>(A.pin);
  const Rc16Layout lay = rc16_layout(Q, A.g.nstore);
  const unsigned short* dev = reinterpret_cast<const unsigned short*>(base + lay.dev);
  const int ns = A.g.nstore;
  if (sbits == 0) {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                      (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                      (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      raw[i] = __ldg(dev + (i - 1) * ns + src);
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
                (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
                (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
      const bool bounce = (sbits >> i) & 1u;
      src = bounce ? si : src;
      const int dir = bounce ? opp(i) : i;
      raw[i] = __ldg(dev + (size_t)(dir - 1) * ns + src);
    }
  }
  r0 = __ldg(reinterpret_cast<const float2*>(base) + si);
}

// The arithmetic of pull_cell_rc16 on loaded values (see there).
template <int Q, int S, int RX>
__device__ __forceinline__ void rc16_decode(const StepArgs& A, uint32_t sbits,
                                            const unsigned short (&raw)[Q], float2 r0,
                                            const float4* rec, const float* ref, const int (&bx)[3],
                                            V2<float> (&g)[Q], float& sr, float& sb, float& lr,
                                            float& lb) {
  using L = Lattice<Q>;
  using H = typename Storage<S>::half_t;
  const float inv_scale = A.ph.inv_scale;
  float2 acc = sum_start(A.ph), lo = make_float2(0.0f, 0.0f);
  fast_two_sum_acc(acc, lo, r0);
  g[0] = {r0.x + r0.y, 0.0f};
  if (sbits == 0) {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int e = bx[1 + L::cm(i)] - (L::cb(i) * RX + L::ca(i));
      const float4 rc = rec[e];
      const float rf = ref[e];
      const float f = fmaf(H::unpack_bits(raw[i]), inv_scale, float(rc16_ratio<L>(i)) * rf);
      const float fr = rc_red<L>(i, rc.x, f, rc_cv<L>(i, rc));
      fast_two_sum_acc(acc, lo, make_float2(fr, f - fr));
      g[i] = {f, 0.0f};
    }
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const bool bounce = (sbits >> i) & 1u;
      // the source's record and scale (the cell's own for a bounced link)
      const int e = bounce ? bx[1] : bx[1 + L::cm(i)] - (L::cb(i) * RX + L::ca(i));
      const float4 rc = rec[e];
      const float rf = ref[e];
      const float f = fmaf(H::unpack_bits(raw[i]), inv_scale, float(rc16_ratio<L>(i)) * rf);
      float cv = rc_cv<L>(i, rc);
      if (bounce) cv = -cv;
      const float fr = rc_red<L>(i, rc.x, f, cv);
      fast_two_sum_acc(acc, lo, make_float2(fr, f - fr));
      g[i] = {f, 0.0f};
    }
  }
  sum_finish(A.ph, acc, lo);
  sr = acc.x;
  sb = acc.y;
  lr = lo.x;
  lb = lo.y;
}

// 16-bit recolour-on-pull layout: pull one cell.  Each moving population is decoded from its
// 16-bit deviation and the source's rest-state scale Rf, f_i = fl(r_i Rf + dev / s), and split
// with the source's record as pull_cell_rc does.  rec / ref are the staged record and scale boxes
// (flat shared arrays of RS x RY x RX); bx[k] is the flat index of this cell's box position in
// plane m + 1 - k, the plane that the pull sources of the directions with c_m = k - 1 lie in
// (k = 1: this plane), so the source of direction i sits at the compile-time offset
// -(c_i,b RX + c_i,a) from bx[1 + c_i,m].  The rest pair (f_0^r, f_0^b) is the cell's own, read
// from global memory.  Output as pull_cell_dev: g_i = (f_i, 0), the colour totals (sr, sb) summed
// with Fast2Sum from the base B, rest pair first, and their rounding errors (lr, lb): sr + lr is
// the exact sum of the split values.  A cell none of whose links bounces back (sbits == 0, nearly every cell)
// takes a path whose addresses are all fixed offsets; the others take the general one.
template <int Q, int S, int RX>
__device__ __forceinline__ void pull_cell_rc16(const StepArgs& A, const Slot& sl, int si,
                                               PlaneOffsets po, uint32_t sbits,
                                               const float4* rec, const float* ref,
                                               const int (&bx)[3], V2<float> (&g)[Q],
                                               float& sr, float& sb, float& lr, float& lb) {
  unsigned short raw[Q];
  float2 r0;
  rc16_load<Q, S>(A, sl, si, po, sbits, raw, r0);
  rc16_decode<Q, S, RX>(A, sbits, raw, r0, rec, ref, bx, g, sr, sb, lr, lb);
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

// Moments, Eq. (collision) with Eq. (feq), Eq. (perturb), Eq. (recolor); stores f^{k*} at the
// cell's storage index si and (GHOSTS: the kernel family that keeps periodic images) its ghost
// images si + dimg[j], j < nimg.
// rnb[i] is rho^N at x + c_i (the cell's own value where that neighbour is solid).  The factors
// that depend only on the speed class s = |c_i|^2 are formed once per cell:
//   f_i^eq = rho (A_s + B_s abar) + rho W_s (3 cu + 9/2 cu^2 - 3/2 u^2)            (Eq. feq)
//   (9/4)(sigma/tau)|F|[W_s (F.c_i)^2/|F|^2 - C_s] = kw_s (F.c_i)^2 - kc_s        (Eq. perturb)
//   beta (rho_r rho_b / rho^2) cos(theta_i) f_i^eq(rho, 0) = kr_s (F.c_i)          (Eq. recolor)
// EXACT (16-bit storages): rr + lr and rb + lb are the cell's exact post-exchange colour masses;
// the rest pair, stored last, also takes back the rounding of the collision's FP32 outputs, so
// the stored mass of each colour is that exact mass (to the rest pair's own rounding).
template <int Q, int S, bool GHOSTS = true, bool EXACT = false>
__device__ __forceinline__ void collide_store(const StepArgs& A, int si, int nimg, const int (&dimg)[3],
                                              const typename Storage<S>::real (&fcb)[Q],
                                              typename Storage<S>::real rr,
                                              typename Storage<S>::real rb,
                                              typename Storage<S>::real irho,
                                              const typename Storage<S>::real (&rnb)[Q],
                                              typename Storage<S>::real& Fn_out,
                                              typename Storage<S>::real lr = 0,
                                              typename Storage<S>::real lb = 0) {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  using IO = PopIO<S, Q>;
  const Physics& ph = A.ph;
  const R rho = rr + rb;
  const R wr = rr * irho, wb = rb * irho;
  R f[Q];
  R ja = R(0), jb = R(0), jm = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    f[i] = fcb[i];  // colour-blind population
    if (L::ca(i) > 0) ja += f[i];
    if (L::ca(i) < 0) ja -= f[i];
    if (L::cb(i) > 0) jb += f[i];
    if (L::cb(i) < 0) jb -= f[i];
    if (L::cm(i) > 0) jm += f[i];
    if (L::cm(i) < 0) jm -= f[i];
  }
  const R ua = ja * irho, ub = jb * irho, um = jm * irho;
  const R uu15 = R(1.5) * (ua * ua + ub * ub + um * um);
  const R itau = wr * PHYS(R, ph, inv_tau_r) + wb * PHYS(R, ph, inv_tau_b);  // harmonic mean of tau_k
  const R abar = wr * PHYS(R, ph, alpha_r) + wb * PHYS(R, ph, alpha_b);
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
  const R pamp = PHYS(R, ph, amp) * itau;       // (9/4) sigma / tau
  const R rcol = PHYS(R, ph, beta) * wr * wb;   // beta rho_r rho_b / rho^2
  R restc[3], rwc[3], kw[3], kc[3], kr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int i = c == 0 ? 0 : (c == 1 ? 1 : L::Q - 1);  // a direction of speed class c
    restc[c] = rho * (R(L::A(i)) + R(L::B(i)) * abar);   // f_i^eq(rho, 0)
    rwc[c] = rho * R(L::W(i));
    kw[c] = pamp * R(L::W(i)) * iFn;
    kc[c] = pamp * R(L::C(i)) * Fn;
    kr[c] = rcol * iFn * R(inv_norm<L>(i)) * restc[c];
  }
  // Rest direction: c_0 = 0, so Eq. (feq) is restc - rwc 3/2 u^2, the perturbation -kc and no
  // recoloring term.
  const R f0eq = fma(rwc[0], -uu15, restc[0]);
  const R fi0 = fma(itau, f0eq - f[0], f[0]) - kc[0];
  const V2<R> f0{wr * fi0, fi0 - wr * fi0};
  float* const rc_pop = reinterpret_cast<float*>(A.pout);  // recolour-on-pull layout only
  (void)rc_pop;
  // 16-bit recolour-on-pull: the record, the rest-state scale Rf = f_1^eq(rho, 0) and what the
  // moving populations will deliver per colour, summed without rounding error (rc_out_hi + lo)
  float4 rc16_rec = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float rc16_rf = 0.0f;
  float2 rc_out_hi = sum_start(ph), rc_out_lo = make_float2(0.0f, 0.0f);
  (void)rc16_rec;
  (void)rc16_rf;
  (void)rc_out_hi;
  (void)rc_out_lo;
  if constexpr (Storage<S>::rc16) {
    const R gv = rcol * iFn * rho * (R(1) - abar);
    rc16_rec = make_float4(wr, gv * Fa, gv * Fb, gv * Fm);
    rc16_rf = restc[1];
  } else if constexpr (Storage<S>::rc) {
    // colour-blind populations plus the record (w_r, V) from which the reader recolours:
    // kr_s (F.c_i) = s_|c| (c_i . V) with V = beta (rho_r rho_b / rho) (1 - abar) F / |F|
    const R gv = rcol * iFn * rho * (R(1) - abar);
    const float4 rec = make_float4(wr, gv * Fa, gv * Fb, gv * Fm);
    float4* const rc_rec = reinterpret_cast<float4*>(reinterpret_cast<char*>(A.pout) +
                                                     rc_record_offset(Q, A.g.nstore));
    rc_pop[si] = fi0;
    rc_rec[si] = rec;
    if (GHOSTS && nimg)
      for (int j = 0; j < nimg; ++j) {
        rc_pop[si + dimg[j]] = fi0;
        rc_rec[si + dimg[j]] = rec;
      }
  } else if constexpr (!Storage<S>::dev && !ExactPairs<S>::value) {
    IO::store(A.pout, A.g.nstore, 0, si, f0.r, f0.b, f0, ph);
    if (GHOSTS && nimg)
      for (int j = 0; j < nimg; ++j) IO::store(A.pout, A.g.nstore, 0, si + dimg[j], f0.r, f0.b, f0, ph);
  }
  // deviation storages: the rounding loss of the 16-bit pairs, summed per colour (units of
  // 1 / scale); the rest pair, stored last, takes it back so the cell's stored mass is its mass
  float2 dev_loss = make_float2(0.0f, 0.0f);
  (void)dev_loss;
  // EXACT: the FP32 outputs summed per colour without rounding error (from B), rest pair first
  float2 out_hi = sum_start(ph), out_lo = make_float2(0.0f, 0.0f);
  if constexpr (Storage<S>::dev && EXACT) fast_two_sum_acc(out_hi, out_lo, make_float2(float(f0.r), float(f0.b)));
  (void)out_hi;
  (void)out_lo;
  static_assert(opposites_adjacent<L>(), "directions (i, i+1), i odd, must be opposite");
  // Opposite directions (i, i+1) share |c.u|, |c.F| with opposite signs: the even part of Eq.
  // (feq) and the perturbation are common, the odd part of Eq. (feq) and the recoloring term
  // change sign.
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int j = i + 1;
    const int c = L::speed2(i);
    R cu = R(0), pc = R(0);
    if (L::ca(i) > 0) { cu += ua; pc += Fa; }
    if (L::ca(i) < 0) { cu -= ua; pc -= Fa; }
    if (L::cb(i) > 0) { cu += ub; pc += Fb; }
    if (L::cb(i) < 0) { cu -= ub; pc -= Fb; }
    if (L::cm(i) > 0) { cu += um; pc += Fm; }
    if (L::cm(i) < 0) { cu -= um; pc -= Fm; }
    const R even = fma(rwc[c], fma(R(4.5) * cu, cu, -uu15), restc[c]);
    const R odd = R(3) * rwc[c] * cu;
    const R pert = fma(kw[c], pc * pc, -kc[c]);  // Eq. (perturb), even in c
    const R kp = kr[c] * pc;                     // Eq. (recolor) term, odd in c
    R fi, fj, fri, frj;
    if constexpr (std::is_same<R, float>::value) {
      // both directions of the pair in packed FP32 (same roundings as the scalar form)
      const float2 fv = make_float2(f[i], f[j]);
      const float2 m1 = make_float2(-1.0f, -1.0f);
      const float2 feq = __fadd2_rn(make_float2(even, even), make_float2(odd, -odd));
      float2 post = __ffma2_rn(make_float2(itau, itau), __ffma2_rn(fv, m1, feq), fv);
      post = __fadd2_rn(post, make_float2(pert, pert));
      const float2 fr = __ffma2_rn(make_float2(wr, wr), post, make_float2(kp, -kp));
      fi = post.x;
      fj = post.y;
      fri = fr.x;
      frj = fr.y;
    } else {
      fi = fma(itau, (even + odd) - f[i], f[i]) + pert;  // Eq. (collision) + (perturb)
      fj = fma(itau, (even - odd) - f[j], f[j]) + pert;
      fri = fma(wr, fi, kp);
      frj = fma(wr, fj, -kp);
    }
    if constexpr (Storage<S>::rc16) {
      // encode f - r_i Rf (s scaled) in 16 bits, decode as a reader will, and split the decoded
      // values with this cell's record exactly as the readers will split them
      using H = typename Storage<S>::half_t;
      using P = typename H::packed;
      const Rc16Layout lay = rc16_layout(Q, A.g.nstore);
      P* dev = reinterpret_cast<P*>(reinterpret_cast<char*>(A.pout) + lay.dev);
      const float ri = float(rc16_ratio<L>(i)) * rc16_rf;  // exact (r_i is a power of two)
      const P hi = H::pack((fi - ri) * ph.scale);
      const P hj = H::pack((fj - ri) * ph.scale);
      dev[(size_t)(i - 1) * A.g.nstore + si] = hi;
      dev[(size_t)(j - 1) * A.g.nstore + si] = hj;
      const float di = fmaf(H::unpack(hi), ph.inv_scale, ri);
      const float dj = fmaf(H::unpack(hj), ph.inv_scale, ri);
      const float fr_i = rc_red<L>(i, rc16_rec.x, di, rc_cv<L>(i, rc16_rec));
      const float fr_j = rc_red<L>(j, rc16_rec.x, dj, rc_cv<L>(j, rc16_rec));
      fast_two_sum_acc(rc_out_hi, rc_out_lo, make_float2(fr_i, di - fr_i));
      fast_two_sum_acc(rc_out_hi, rc_out_lo, make_float2(fr_j, dj - fr_j));
    } else if constexpr (Storage<S>::rc) {
      const size_t ns = (size_t)A.g.nstore;
      rc_pop[i * ns + si] = fi;
      rc_pop[j * ns + si] = fj;
      if (GHOSTS && nimg)
        for (int k = 0; k < nimg; ++k) {
          rc_pop[i * ns + si + dimg[k]] = fi;
          rc_pop[j * ns + si + dimg[k]] = fj;
        }
    } else if constexpr (Storage<S>::dev) {
      const float2 vi = make_float2(fri, fi - fri), vj = make_float2(frj, fj - frj);
      const float2 li = IO::store_loss(A.pout, A.g.nstore, i, si, vi.x, vi.y, f0, ph);
      const float2 lj = IO::store_loss(A.pout, A.g.nstore, j, si, vj.x, vj.y, f0, ph);
      if constexpr (EXACT) {  // the stored (decoded) mass: outputs minus the pairs' losses
        const float2 ninv = make_float2(-ph.inv_scale, -ph.inv_scale);
        fast_two_sum_acc(out_hi, out_lo, vi);
        fast_two_sum_acc(out_hi, out_lo, vj);
        out_lo = __ffma2_rn(__fadd2_rn(li, lj), ninv, out_lo);
      } else {
        dev_loss = __fadd2_rn(dev_loss, __fadd2_rn(li, lj));
      }
      if (GHOSTS && nimg) {
        for (int k = 0; k < nimg; ++k) {
          IO::store(A.pout, A.g.nstore, i, si + dimg[k], fri, fi - fri, f0, ph);
          IO::store(A.pout, A.g.nstore, j, si + dimg[k], frj, fj - frj, f0, ph);
        }
      }
    } else {
      IO::store(A.pout, A.g.nstore, i, si, fri, fi - fri, f0, ph);
      IO::store(A.pout, A.g.nstore, j, si, frj, fj - frj, f0, ph);
      if constexpr (ExactPairs<S>::value) {  // what the stored moving pairs carry, exactly
        fast_two_sum_acc(rc_out_hi, rc_out_lo, make_float2(fri, fi - fri));
        fast_two_sum_acc(rc_out_hi, rc_out_lo, make_float2(frj, fj - frj));
      }
      if (GHOSTS && nimg) {  // periodic ghost images: cells within two of a periodic x or y edge
        for (int k = 0; k < nimg; ++k) {
          IO::store(A.pout, A.g.nstore, i, si + dimg[k], fri, fi - fri, f0, ph);
          IO::store(A.pout, A.g.nstore, j, si + dimg[k], frj, fj - frj, f0, ph);
        }
      }
    }
  }
  if constexpr (ExactPairs<S>::value) {
    // the rest pair: the exact colour masses (rr + lr, rb + lb) less the stored moving pairs
    // (rc_out_hi - B + rc_out_lo), as for the 16-bit recolour-on-pull layout
    rc_out_hi = sub2(rc_out_hi, sum_start(ph));  // exact
    const float2 t = make_float2(float(rr), float(rb));
    const float2 s2 = sub2(t, rc_out_hi);
    const float2 e2 = make_float2(two_sum_err(t.x, -rc_out_hi.x, s2.x),
                                  two_sum_err(t.y, -rc_out_hi.y, s2.y));
    const float2 small = __fadd2_rn(e2, sub2(make_float2(float(lr), float(lb)), rc_out_lo));
    const float2 r0 = __fadd2_rn(s2, small);
    IO::store(A.pout, A.g.nstore, 0, si, r0.x, r0.y, f0, ph);
    if (GHOSTS && nimg)
      for (int j = 0; j < nimg; ++j) IO::store(A.pout, A.g.nstore, 0, si + dimg[j], r0.x, r0.y, f0, ph);
  }
  if constexpr (Storage<S>::rc16) {
    // the rest pair carries the exact colour masses (rr + lr, rb + lb) less what the moving
    // populations deliver (rc_out_hi + rc_out_lo): TwoSum of the large terms, then the small ones
    // (the periodic images of the TMA family are not kept for this layout); rc_out_hi - B exact
    rc_out_hi = sub2(rc_out_hi, sum_start(ph));
    const float2 t = make_float2(float(rr), float(rb));
    const float2 s2 = sub2(t, rc_out_hi);
    const float2 e2 = make_float2(two_sum_err(t.x, -rc_out_hi.x, s2.x),
                                  two_sum_err(t.y, -rc_out_hi.y, s2.y));
    const float2 small = __fadd2_rn(e2, sub2(make_float2(float(lr), float(lb)), rc_out_lo));
    char* b = reinterpret_cast<char*>(A.pout);
    const Rc16Layout lay = rc16_layout(Q, A.g.nstore);
    reinterpret_cast<float2*>(b)[si] = __fadd2_rn(s2, small);
    reinterpret_cast<float4*>(b + lay.rec)[si] = rc16_rec;
    reinterpret_cast<float*>(b + lay.ref)[si] = rc16_rf;
  }
  if constexpr (Storage<S>::dev) {
    // decoding gives f_i = f_0 kappa_i + deviation / scale, so raising f_0^k by delta raises the
    // cell's decoded mass by delta / phi_0(alpha_k) = delta / alpha_k; the moving pairs lost
    // dev_loss / scale of mass: delta = alpha_k dev_loss / scale restores it exactly
    V2<R> f0c;
    if constexpr (EXACT) {
      // EXACT: delta = alpha_k times what the stored mass misses of the exact mass, (rr + lr)
      // - (out_hi - B + out_lo); out_hi - B is exact and the high parts agree to a few ulps of
      // B, so their difference is exact too
      out_hi = sub2(out_hi, sum_start(ph));
      const float2 miss = __fadd2_rn(sub2(make_float2(rr, rb), out_hi),
                                     sub2(make_float2(lr, lb), out_lo));
      const float2 c = __ffma2_rn(make_float2(PHYS(R, ph, alpha_r), PHYS(R, ph, alpha_b)), miss,
                                  make_float2(f0.r, f0.b));
      f0c = V2<R>{c.x, c.y};
    } else {
      f0c = V2<R>{fma(PHYS(R, ph, alpha_r) * R(ph.inv_scale), dev_loss.x, f0.r),
                  fma(PHYS(R, ph, alpha_b) * R(ph.inv_scale), dev_loss.y, f0.b)};
    }
    IO::store(A.pout, A.g.nstore, 0, si, f0c.r, f0c.b, f0c, ph);
    if (GHOSTS && nimg)
      for (int j = 0; j < nimg; ++j) IO::store(A.pout, A.g.nstore, 0, si + dimg[j], f0c.r, f0c.b, f0c, ph);
  }
  Fn_out = Fn;
}

// collide_store from the pulled, post-exchange pairs (the colour-blind sums are what it reads).
template <int Q, int S>
__device__ __forceinline__ void collide_store(const StepArgs& A, int si, int nimg, const int (&dimg)[3],
                                              const V2<typename Storage<S>::real> (&g)[Q],
                                              typename Storage<S>::real rr,
                                              typename Storage<S>::real rb,
                                              typename Storage<S>::real irho,
                                              const typename Storage<S>::real (&rnb)[Q],
                                              typename Storage<S>::real& Fn_out) {
  using R = typename Storage<S>::real;
  R f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = g[i].r + g[i].b;
  collide_store<Q, S, true>(A, si, nimg, dimg, f, rr, rb, irho, rnb, Fn_out);
}

// Ghost images of the column (a, b): storage deltas (plane-invariant).
__device__ __forceinline__ int image_deltas(const Geom& g, int a, int b, int (&d)[3]) {
  int da = 0, db = 0;
  if (g.img_a) da = a < 2 ? g.na : (a >= g.na - 2 ? -g.na : 0);
  if (g.img_b) db = b < 2 ? g.nb : (b >= g.nb - 2 ? -g.nb : 0);
  int n = 0;
  if (da) d[n++] = da;
  if (db) d[n++] = db * g.pitch;
  if (da && db) d[n++] = da + db * g.pitch;
  return n;
}

// Per-cell tail of the fused step, called by step_tile for every fluid cell of the tile once the
// colour-blind sums f_i = g_i^r + g_i^b of its pulled, post-exchange populations (the exchange
// keeps each f_i), rho_r, rho_b and the neighbour phase field rnb are at hand: Eq.
// (collision) to Eq. (recolor) and the store, the site byte of this step and the ledger terms.
struct StepEpilogue {
  // Called for each own fluid cell of plane m (storage index si) at the start of the iteration
  // that collides plane m, before the pulls of plane m + 1: an epilogue that reads per-cell data
  // of plane m can start fetching it here (the step itself reads nothing more).
  template <int Q, int S>
  __device__ __forceinline__ void prefetch(const StepArgs&, int /*si*/) const {}
  // Called by every thread of the tile (origin a0, b0), for plane um, before the barrier that
  // precedes the collision of plane um - 1 (and for the chunk's planes m0 - 1 and m0 before the
  // first one): an epilogue that reads per-cell data of the neighbours stages it here.
  template <int Q, int S>
  __device__ __forceinline__ void stage(const StepArgs&, int /*a0*/, int /*b0*/, int /*um*/,
                                        int /*tid*/) const {}
  // sl, sbits, m: the cell's slot, solid-link bits and plane.  (lr, lb): the rounding errors of
  // rr, rb (16-bit storages: rr + lr is the exact mass)
  template <int Q, int S, class R>
  __device__ __forceinline__ void cell(const StepArgs& A, int cell, const Slot& /*sl*/,
                                       uint32_t /*sbits*/, int /*m*/, int si, int nimg,
                                       const int (&dimg)[3], const R (&f)[Q], R rr, R rb,
                                       R irho, R e, uint32_t flags, const R (&rnb)[Q],
                                       int& n_sites, R& removed, R lr = R(0), R lb = R(0)) const {
    R Fn;
    collide_store<Q, S, false, true>(A, si, nimg, dimg, f, rr, rb, irho, rnb, Fn, lr, lb);  // no ghosts
    uint32_t mb = flags;
    if (A.ph.rule == 0) {
      const R d = Fn - PHYS(R, A.ph, threshold);
      mb |= (d > R(0) ? 2u : 0u) | (fabs(d) < R(1e-6) ? 8u : 0u);
    }
    A.mask_out[cell] = (uint8_t)mb;
    if (flags & 1u) {
      ++n_sites;
      removed += e;
    }
  }
};

// Shared-memory footprint of step_tile: the rho^N ring, the deviation storages' rest ring and
// the parking columns (bytes).
template <int Q, int S, int TX, int TY, int CPT>
struct TileSmem {
  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  static constexpr int TH = TY * CPT;
  static constexpr int HX = TX + 2, HY = L::D3 ? TH + 2 : 1;
  static constexpr bool DEV = Storage<S>::dev;
  // source staging: rest pairs (deviation storages), recolouring records (ST_RC), or records
  // plus rest-state scales (16-bit recolour-on-pull)
  static constexpr bool STAGE = DEV || Storage<S>::rc_in;
  static constexpr int BOX = Storage<S>::rc_in ? (Storage<S>::rc16 ? 20 : 16) : 8;
  static constexpr int RX = STAGE ? TX + 4 : 1, RY = STAGE ? (L::D3 ? TH + 4 : 1) : 1, RS = STAGE ? 4 : 1;
  // every part starts on a 16-byte boundary
  static constexpr int RING = ((4 * HY * HX * (int)sizeof(R)) + 15) & ~15;
  static constexpr int REST = ((RS * RY * RX * BOX) + 15) & ~15;
  static constexpr int PARK = ((CPT * Q * TX * TY * (int)sizeof(R)) + 15) & ~15;
  static constexpr int BYTES = RING + REST + PARK;
  static_assert(RING % 16 == 0 && REST % 16 == 0 && BYTES % 16 == 0, "16-byte aligned parts");
};

// One CTA's work of the fused step: tile `tile` of the (a, b) plane, planes of chunk `chunk`
// along m.  CPT cells per thread: thread (lx, ly) owns the columns (lx, ly + c TY), c < CPT, of a
// TX x (TY CPT) tile, so its pulls of all CPT cells are in flight together.  smem points to
// TileSmem<...>::BYTES bytes of shared memory.  Returns this thread's site count and removed mass.
// tid: this thread's index within the TX*TY threads that run the tile; iters >= the number of
// planes of the chunk: the loop runs that many barrier rounds (the extra ones idle), so several
// tiles with different chunk lengths can share one CTA's barriers.  epi: the per-cell tail
// (StepEpilogue for the step itself; the adjoint passes its own).
// PF (storages that pull pairs from global memory without staging): the own cells' pulls of the
// next plane are issued one fill ahead, into registers, so their loads are in flight during the
// rest of that fill, the barrier and the collision of the current plane instead of being waited
// for at once (the same values, loaded earlier; more registers live across the collision).
template <int Q, int S, int TX, int TY, int CPT, class Epi = StepEpilogue, bool PF = false>
__device__ __forceinline__ void step_tile(const StepArgs& A, int tile, int chunk, unsigned char* smem,
                                          long long& n_sites, double& removed,
                                          int tid = threadIdx.x, int iters = -1,
                                          const Epi& epi = Epi()) {
  using SM = TileSmem<Q, S, TX, TY, CPT>;
  unsigned char* ring_mem = smem;
  unsigned char* rest_mem = smem + SM::RING;
  unsigned char* park_mem = smem + SM::RING + SM::REST;

  using L = Lattice<Q>;
  using R = typename Storage<S>::real;
  constexpr int NT = TX * TY;
  constexpr int TH = TY * CPT;  // tile rows
  constexpr int HX = TX + 2;
  constexpr int HY = L::D3 ? TH + 2 : 1;
  constexpr int OB = L::D3 ? 1 : 0;
  constexpr int NH = HX * HY - TX * TH;
  static_assert(NH <= NT, "one ring cell per thread at most");
  static_assert(L::D3 || (TY == 1 && CPT == 1), "D2Q9 tiles are one row");
  R(*ring)[HY][HX] = reinterpret_cast<R(*)[HY][HX]>(ring_mem);
  // deviation storage: rest pairs of the tile plus a two-cell ring, planes m .. m+2
  constexpr bool DEV = Storage<S>::dev;
  constexpr bool EXACTP = ExactPairs<S>::value;      // FP32 pairs with exact colour masses
  constexpr bool RCIN = Storage<S>::rc_in;          // reads a recolour-on-pull layout
  constexpr bool RC16IN = RCIN && Storage<S>::rc16;  // ... the 16-bit one
  constexpr bool STAGE = DEV || RCIN;    // pulls read per-source data staged in shared memory
  constexpr int RX = STAGE ? TX + 4 : 1;
  constexpr int RY = STAGE ? (L::D3 ? TH + 4 : 1) : 1;
  constexpr int RS = STAGE ? 4 : 1;  // planes m-1 .. m+2: one staged ahead, no extra barrier
  constexpr int RN = RX * RY;
  constexpr int RPT = (RN + NT - 1) / NT;  // rest-box elements staged per thread
  float2(*rest_ring)[RY][RX] = reinterpret_cast<float2(*)[RY][RX]>(rest_mem);

  const Geom& G = A.g;
  const int a0 = (tile % A.ntx) * TX;
  const int b0 = (tile / A.ntx) * TH;
  const int m0 = chunk * A.pc;
  const int m1 = min(m0 + A.pc, G.nm);
  const int lx = tid % TX, ly0 = tid / TX;
  bool active[CPT];
  Slot me[CPT];
  int dimg[CPT][3];
  int nimg[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int ly = ly0 + c * TY;
    active[c] = (a0 + lx < G.na) && (b0 + ly < G.nb);
    me[c] = make_slot<L>(G, a0 + lx, b0 + ly);
    dimg[c][0] = dimg[c][1] = dimg[c][2] = 0;
    nimg[c] = active[c] ? image_deltas(G, me[c].a, me[c].b, dimg[c]) : 0;
  }

  // This thread's ring cell, if any (the first NH threads take one each).
  int hx = 0, hy = 0;
  const bool has_halo = tid < NH;
  const int hh = tid;
  if (has_halo) {
    if (L::D3) {
      if (hh < HX) {
        hx = hh;
        hy = 0;
      } else if (hh < 2 * HX) {
        hx = hh - HX;
        hy = HY - 1;
      } else {
        const int k = hh - 2 * HX;
        hx = (k & 1) ? HX - 1 : 0;
        hy = 1 + (k >> 1);
      }
    } else {
      hx = hh == 0 ? 0 : HX - 1;
      hy = 0;
    }
  }
  const Slot hs = make_slot<L>(G, a0 + hx - 1, b0 + hy - OB);

  // deviation storage: in-plane storage offsets of this thread's rest-box elements (-1: beyond a
  // wall or not this thread's)
  int rest_off[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    rest_off[k] = -1;
    const int e = tid + k * NT;
    if (STAGE && e < RN) {
      const int ex = e % RX, ey = e / RX;
      int a = a0 - 2 + ex, b = L::D3 ? b0 - 2 + ey : 0;
      bool ok = true;
      if (a < 0 || a >= G.na) {
        if (G.per_a) a = wrap(a, G.na); else ok = false;
      }
      if (L::D3 && (b < 0 || b >= G.nb)) {
        if (G.per_b) b = wrap(b, G.nb); else ok = false;
      }
      if (ok) rest_off[k] = (b + G.gy) * G.pitch + a + kOx;
    }
  }
  const int plane_stride = G.rows * G.pitch;
  auto rest_slot = [&](int uq) { return (uq - m0 + 4) & 3; };
  // ST_RC: the recolouring records (w_r, V) of the same box, staged the same way; the 16-bit
  // recolour-on-pull layout also stages the rest-state scales, in a second array
  float4(*rec_ring)[RY][RX] = reinterpret_cast<float4(*)[RY][RX]>(rest_mem);
  float(*ref_ring)[RY][RX] = reinterpret_cast<float(*)[RY][RX]>(rest_mem + RS * RY * RX * 16);
  (void)ref_ring;
  auto stage_rest = [&](int uq) {  // rest pairs / records of plane uq (unwrapped) into its slot
    if (!STAGE) return;
    const Plane q = make_plane(G, uq);
    const int sl = rest_slot(uq);
    if constexpr (RC16IN) {
      const Rc16Layout lay = rc16_layout(Q, G.nstore);
      const char* b = reinterpret_cast<const char*>(A.pin);
      const float4* rec = reinterpret_cast<const float4*>(b + lay.rec);
      const float* ref = reinterpret_cast<const float*>(b + lay.ref);
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int e = tid + k * NT;
        if (e < RN && q.ok && rest_off[k] >= 0) {
          rec_ring[sl][e / RX][e % RX] = __ldg(rec + q.m * plane_stride + rest_off[k]);
          ref_ring[sl][e / RX][e % RX] = __ldg(ref + q.m * plane_stride + rest_off[k]);
        }
      }
    } else if constexpr (RCIN) {
      const float4* rec = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(A.pin) +
                                                          rc_record_offset(Q, G.nstore));
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int e = tid + k * NT;
        if (e < RN && q.ok && rest_off[k] >= 0)
          rec_ring[sl][e / RX][e % RX] = __ldg(rec + q.m * plane_stride + rest_off[k]);
      }
    } else {
      const float2* rest = reinterpret_cast<const float2*>(A.pin);
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int e = tid + k * NT;
        if (e < RN && q.ok && rest_off[k] >= 0)
          rest_ring[sl][e / RX][e % RX] = __ldg(rest + q.m * plane_stride + rest_off[k]);
      }
    }
  };
  // the same staging split in two: the loads of plane uq into registers (issued before the
  // pulls of a plane, so their latency overlaps them) and their stores into its slot (after)
  using BoxT = typename std::conditional<RCIN, float4, float2>::type;
  auto stage_load = [&](int uq, BoxT (&v)[RPT]) {
    if constexpr (STAGE) {
      const Plane q = make_plane(G, uq);
      const BoxT* src = reinterpret_cast<const BoxT*>(reinterpret_cast<const char*>(A.pin) +
                                                      (RCIN ? rc_record_offset(Q, G.nstore) : 0));
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int e = tid + k * NT;
        if (e < RN && q.ok && rest_off[k] >= 0) v[k] = __ldg(src + q.m * plane_stride + rest_off[k]);
      }
    }
  };
  auto stage_store = [&](int uq, const BoxT (&v)[RPT]) {
    if constexpr (STAGE) {
      const Plane q = make_plane(G, uq);
      BoxT(*ring_t)[RY][RX] = reinterpret_cast<BoxT(*)[RY][RX]>(rest_mem);
      const int sl = rest_slot(uq);
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int e = tid + k * NT;
        if (e < RN && q.ok && rest_off[k] >= 0) ring_t[sl][e / RX][e % RX] = v[k];
      }
    }
  };
  auto restbox = [&](int slot, int y, int x) -> float2 { return rest_ring[slot][y][x]; };
  auto recbox = [&](int slot, int y, int x) -> float4 { return rec_ring[slot][y][x]; };

  // The colour-blind sums of the next plane's pulled, post-exchange populations wait in
  // thread-private columns of shared memory (only this thread reads or writes its columns, so no
  // barrier guards them).
  R* parked = reinterpret_cast<R*>(park_mem);  // [CPT][Q][NT]

  struct CellScalars {
    R rr, rb, e, irho;
    R lr, lb;  // 16-bit storages: rounding errors of rr, rb
    uint32_t flags, bits;
    bool ok;
  };
  CellScalars cur[CPT], nxt[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
    cur[c] = nxt[c] = CellScalars{R(0), R(0), R(0), R(0), R(0), R(0), 0u, 0u, false};
  // this thread's sites and removed mass (a sum over at most one cell column: the kernel's own
  // real type suffices; the FP64 total is formed below and in the block reduction)
  int nloc = 0;
  R rem = R(0);

  // Pull plane um for the own cells and the ring cell; write rho^N to the ring; the own cells'
  // post-exchange populations are returned in g.
  // PF: the own cells' pulls issued one fill ahead (storages whose pulls need nothing staged; the
  // 16-bit ones are bound by their instruction count, not by load latency, and gain nothing)
  static_assert(!(PF && STAGE), "pulls issued ahead only for storages without staged sources");
  V2<R> pf[CPT][Q];   // PF: the own cells' pulled populations of the next plane to fill
  uint32_t pfbits[CPT];
  bool pfok[CPT];
  (void)pf;
  auto issue = [&](int um) {  // PF: issue the own cells' pulls of plane um
    if constexpr (PF) {
      const Plane p = make_plane(G, um);
      const PlaneOffsets po = plane_offsets(G, p.m);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int cl = (p.m * G.nb + me[c].b) * G.na + me[c].a;
        uint32_t bits = 0;
        pfok[c] = solid_bits<L>(G, me[c], p, cl, bits);
        pfbits[c] = bits;
        if (pfok[c]) pull_cell<Q, S>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits, pf[c]);
      }
    }
  };
  (void)issue;
  auto fill_plane = [&](int um, CellScalars(&out)[CPT], V2<R>(&g)[CPT][Q]) {
    const Plane p = make_plane(G, um);
    const PlaneOffsets po = plane_offsets(G, p.m);
    const int slot = (um - m0 + 1) & 3;
    int ps[3] = {0, 0, 0};
    BoxT staged[RPT];
    if (STAGE) {  // the pulls of plane um read the staged data of planes um-1 .. um+1, staged
                  // before the barrier that ended the previous plane
      ps[0] = rest_slot(um + 1);
      ps[1] = rest_slot(um);
      ps[2] = rest_slot(um - 1);
      if constexpr (DEV) stage_load(um + 2, staged);  // registers to spare: load early
    }
    if (has_halo) {
      const int cell = (p.m * G.nb + hs.b) * G.na + hs.a;
      uint32_t bits = 0;
      R rn = R(0);
      if (solid_bits<L>(G, hs, p, cell, bits)) {
        V2<R> tmp[Q];
        R t_rr, t_rb, t_e, t_irho;
        uint32_t t_flags;
        if constexpr (STAGE) {  // colour-blind values and colour totals
          R sr, sb, lr_unused, lb_unused;
          if constexpr (DEV)
            pull_cell_dev<Q, S>(A, hs, sidx(G, hs.a, hs.b, p.m), po, bits, hx + 1,
                                L::D3 ? hy + 1 : 0, ps, restbox, tmp, sr, sb, lr_unused, lb_unused);
          else if constexpr (RC16IN) {
            const int c0 = (L::D3 ? hy + 1 : 0) * RX + hx + 1;
            const int bx[3] = {ps[0] * RY * RX + c0, ps[1] * RY * RX + c0, ps[2] * RY * RX + c0};
            pull_cell_rc16<Q, S, RX>(A, hs, sidx(G, hs.a, hs.b, p.m), po, bits, &rec_ring[0][0][0],
                                     &ref_ring[0][0][0], bx, tmp, sr, sb, lr_unused, lb_unused);
          }
          else
            pull_cell_rc<Q>(A, hs, sidx(G, hs.a, hs.b, p.m), po, bits, hx + 1,
                            L::D3 ? hy + 1 : 0, ps, recbox, tmp, sr, sb);
          rn = exchange_from_sums<S>(A, cell, sr, sb, t_rr, t_rb, t_e, t_flags, t_irho);
        } else {
          pull_cell<Q, S>(A, hs, sidx(G, hs.a, hs.b, p.m), po, bits, tmp);
          rn = site_exchange<Q, S>(A, cell, tmp, t_rr, t_rb, t_e, t_flags, t_irho);
        }
      }
      ring[slot][hy][hx] = rn;
    }
    int cells[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {  // issue every load of every own cell first
      cells[c] = (p.m * G.nb + me[c].b) * G.na + me[c].a;
      if constexpr (PF) {  // issued one fill ahead
        out[c].ok = pfok[c];
        out[c].bits = pfbits[c];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[c][i] = pf[c][i];
        continue;
      }
      uint32_t bits = 0;
      out[c].ok = solid_bits<L>(G, me[c], p, cells[c], bits);
      out[c].bits = bits;
      if (out[c].ok) {
        // staged storages: g holds the colour-blind values, out.rr / out.rb the colour totals
        if constexpr (DEV)
          pull_cell_dev<Q, S>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits, lx + 2,
                              L::D3 ? ly0 + c * TY + 2 : 0, ps, restbox, g[c], out[c].rr,
                              out[c].rb, out[c].lr, out[c].lb);
        else if constexpr (RC16IN) {
          const int c0 = (L::D3 ? ly0 + c * TY + 2 : 0) * RX + lx + 2;
          const int bx[3] = {ps[0] * RY * RX + c0, ps[1] * RY * RX + c0, ps[2] * RY * RX + c0};
          pull_cell_rc16<Q, S, RX>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits,
                                   &rec_ring[0][0][0], &ref_ring[0][0][0], bx, g[c], out[c].rr,
                                   out[c].rb, out[c].lr, out[c].lb);
        }
        else if constexpr (RCIN)
          pull_cell_rc<Q>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits, lx + 2,
                          L::D3 ? ly0 + c * TY + 2 : 0, ps, recbox, g[c], out[c].rr, out[c].rb);
        else
          pull_cell<Q, S>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits, g[c]);
      }
    }
    issue(um + 1);  // PF: the next fill's own pulls, in flight from here
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      R rn = R(0);
      if (out[c].ok) {
        if constexpr (STAGE) {
          const R sr = out[c].rr, sb = out[c].rb;
          rn = exchange_from_sums<S>(A, cells[c], sr, sb, out[c].rr, out[c].rb, out[c].e,
                                     out[c].flags, out[c].irho);
          if constexpr (DEV || RC16IN) {  // the exchange's own rounding joins the sums' (TwoSum)
            out[c].lr = __fadd_rn(out[c].lr, two_sum_err(sr, -out[c].e, out[c].rr));
            out[c].lb = __fadd_rn(out[c].lb, two_sum_err(sb, out[c].e, out[c].rb));
          }
        } else if constexpr (EXACTP) {
          // the plain sums of the FP32 pairs (those the ring cells form, so rho^N of a cell is
          // the same in every tile that holds it) and the colour totals without rounding error
          // (from B); what the exact totals exceed the plain ones by, and the exchange's own
          // rounding (TwoSum), go to (lr, lb)
          float2 plain = make_float2(0.0f, 0.0f);
          float2 acc = sum_start(A.ph), lo = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const float2 v = make_float2(g[c][i].r, g[c][i].b);
            plain = __fadd2_rn(plain, v);
            fast_two_sum_acc(acc, lo, v);
          }
          // (acc - B) and plain are both within a few ulps of B of the total: exact difference
          lo = __fadd2_rn(sub2(sub2(acc, sum_start(A.ph)), plain), lo);
          rn = exchange_from_sums<S>(A, cells[c], plain.x, plain.y, out[c].rr, out[c].rb,
                                     out[c].e, out[c].flags, out[c].irho);
          out[c].lr = __fadd_rn(lo.x, two_sum_err(plain.x, -out[c].e, out[c].rr));
          out[c].lb = __fadd_rn(lo.y, two_sum_err(plain.y, out[c].e, out[c].rb));
          g[c][0].r -= out[c].e;
          g[c][0].b += out[c].e;
        } else
          rn = site_exchange<Q, S>(A, cells[c], g[c], out[c].rr, out[c].rb, out[c].e,
                                   out[c].flags, out[c].irho);
      }
      ring[slot][ly0 + c * TY + OB][lx + 1] = rn;
    }
    // plane um + 2 into the slot of plane um - 2, which the pulls of plane um - 1 read before
    // the last barrier; the pulls of plane um + 1 read it after the next one
    if constexpr (DEV)
      stage_store(um + 2, staged);
    else
      stage_rest(um + 2);
  };

  epi.template stage<Q, S>(A, a0, b0, m0 - 1, tid);
  epi.template stage<Q, S>(A, a0, b0, m0, tid);
  issue(m0 - 1);  // PF: the first fill's own pulls
  stage_rest(m0 - 2);
  stage_rest(m0 - 1);
  stage_rest(m0);
  if (STAGE) __syncthreads();
  {
    CellScalars t[CPT];
    V2<R> g[CPT][Q];
    fill_plane(m0 - 1, t, g);
  }
  __syncthreads();  // the next fill restages a rest slot the pulls above may still read
  {
    V2<R> g[CPT][Q];
    fill_plane(m0, cur, g);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int i = 0; i < Q; ++i)
        parked[(c * Q + i) * NT + tid] = STAGE ? g[c][i].r : g[c][i].r + g[c][i].b;
  }
  if (STAGE) __syncthreads();  // the first fill below restages a slot the pulls above read

  const int m_end = iters < 0 ? m1 : m0 + iters;
  for (int m = m0; m < m_end; ++m) {
    if (m >= m1) {  // idle barrier rounds of a shorter chunk sharing the CTA
      __syncthreads();
      continue;
    }
    epi.template stage<Q, S>(A, a0, b0, m + 1, tid);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (active[c] && cur[c].ok) epi.template prefetch<Q, S>(A, sidx(G, me[c].a, me[c].b, m));
    V2<R> g[CPT][Q];
    fill_plane(m + 1, nxt, g);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      // plane m of cell c leaves its parking column, plane m+1 takes its place
      R own[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        own[i] = parked[(c * Q + i) * NT + tid];
        // staged storages deliver colour-blind values (g_i.b = 0): park them as they are
        parked[(c * Q + i) * NT + tid] = STAGE ? g[c][i].r : g[c][i].r + g[c][i].b;
      }
      if (!(active[c] && cur[c].ok)) continue;
      const int ly = ly0 + c * TY;
      const int s0 = (m - m0 + 1) & 3;
      const R ownrn = ring[s0][ly + OB][lx + 1];
      R rnb[Q];
      if (cur[c].bits == 0) {  // no neighbour is solid or beyond a wall
#pragma unroll
        for (int i = 0; i < Q; ++i)
          rnb[i] = ring[(m - m0 + 1 + L::cm(i)) & 3][ly + OB + L::cb(i)][lx + 1 + L::ca(i)];
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int s = (m - m0 + 1 + L::cm(i)) & 3;
          const bool solid_nb = (cur[c].bits >> opp(i)) & 1u;  // x + c_i is the source of opp(i)
          rnb[i] = solid_nb ? ownrn : ring[s][ly + OB + L::cb(i)][lx + 1 + L::ca(i)];
        }
      }
      const int cell = (m * G.nb + me[c].b) * G.na + me[c].a;
      if constexpr (DEV || RC16IN || EXACTP)
        epi.template cell<Q, S>(A, cell, me[c], cur[c].bits, m, sidx(G, me[c].a, me[c].b, m),
                                nimg[c], dimg[c], own, cur[c].rr, cur[c].rb, cur[c].irho,
                                cur[c].e, cur[c].flags, rnb, nloc, rem, cur[c].lr, cur[c].lb);
      else
        epi.template cell<Q, S>(A, cell, me[c], cur[c].bits, m, sidx(G, me[c].a, me[c].b, m),
                                nimg[c], dimg[c], own, cur[c].rr, cur[c].rb, cur[c].irho,
                                cur[c].e, cur[c].flags, rnb, nloc, rem);
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) cur[c] = nxt[c];
  }
  n_sites = nloc;
  // a scalar flux moves varphi at every site: n varphi in FP64, exact to one rounding
  removed = A.ph.phi_field ? (double)rem : (double)nloc * A.ph.varphi;
}

// Block-wide sum of (n_sites, removed) into thread 0 (warp shuffles, then shared memory).
template <int NT>
__device__ __forceinline__ void block_sum(long long& n, double& d) {
  __shared__ double red_d[NT / 32];
  __shared__ long long red_n[NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n += __shfl_down_sync(0xffffffffu, n, off);
    d += __shfl_down_sync(0xffffffffu, d, off);
  }
  const int tid = threadIdx.x;
  if ((tid & 31) == 0) {
    red_d[tid >> 5] = d;
    red_n[tid >> 5] = n;
  }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    long long c = 0;
    for (int w = 0; w < NT / 32; ++w) {
      s += red_d[w];
      c += red_n[w];
    }
    d = s;
    n = c;
  }
  __syncthreads();
}

// Ledger fold: per-block partials, then the last block to arrive adds them, in block order, to
// the device ledger (deterministic).
__device__ __forceinline__ void ledger_fold(const Reduce& red, long long n, double d) {
  __shared__ int is_last;
  const int tid = threadIdx.x;
  const unsigned nblk = gridDim.x * gridDim.y;
  if (tid == 0) {
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    red.part_removed[bid] = d;
    red.part_sites[bid] = n;
    __threadfence();
    const unsigned prev = atomicAdd(red.done, 1u);
    is_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (is_last && tid < 32) {
    __threadfence();
    double s = 0.0;
    long long c = 0;
    for (unsigned j = tid; j < nblk; j += 32) {
      s += __ldcg(red.part_removed + j);
      c += __ldcg(red.part_sites + j);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_down_sync(0xffffffffu, s, off);
      c += __shfl_down_sync(0xffffffffu, c, off);
    }
    if (tid == 0) {
      DevLedger* led = red.ledger;
      led->evaporated += s;
      led->last_removed = s;
      led->site_steps += c;
      led->last_sites = c;
      led->steps += 1;
      *red.done = 0u;
    }
  }
}

template <int Q, int S, int TX, int TY, int MINB, int CPT, bool PF = false>
__global__ void __launch_bounds__(TX* TY, MINB) cg_step_kernel(const __grid_constant__ StepArgs A) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  long long n = 0;
  double d = 0.0;
  step_tile<Q, S, TX, TY, CPT, StepEpilogue, PF>(A, blockIdx.x, blockIdx.y, dyn_smem, n, d);
  block_sum<TX * TY>(n, d);
  ledger_fold(A.red, n, d);
}

}  // namespace cgevap
