// adjoint.cuh -- reverse-mode derivative of one fused step with respect to its input state and
// the flux field, with the site set x_I of the step held fixed.
//
// The step maps the stored state f^n to f^{n+1}: for every fluid cell x
//   g(x)    = pulled populations (Eq. Stream, halfway bounce-back), then Eq. (exchange):
//             g_0^r -= m(x) phi(x)/S-bar, g_0^b += m(x) phi(x)/S-bar;
//   F(x)    = 3 sum_i W_i c_i rho^N(n_i(x)),  n_i(x) = x + c_i, or x where x + c_i is solid or
//             beyond a wall (Eq. cg), rho^N = (rho_r - rho_b)/rho of the post-exchange g;
//   f^{n+1}(x) = C(g(x), F(x)): Eq. (feq), (collision), (perturb), (recolor).
// Given lambda^{n+1} = dL/df^{n+1} and w = dL/dV(n+1) for the observable
// V(n+1) = sum_x (1 + rho^N(x))/2 (the stored densities of f^{n+1} are those of g: the
// collision, the perturbation and the recoloring conserve rho_r and rho_b per cell), the sweep is
//   (1) local:   lg(x) = (dC/dg)^T lambda^{n+1}(x),  lF(x) = (dC/dF)^T lambda^{n+1}(x),
//                plus d rho^N/d(rho_r, rho_b) = (2 rho_b, -2 rho_r)/rho^2          [kernel A]
//   (2) stencil: mu(y) = w/2 + sum_{(x,i): n_i(x) = y} 3 W_i c_i . lF(x);
//                lg_total(y) = lg(y) + mu(y) d rho^N/d(rho_r, rho_b) on every direction;
//                dL/dphi(y) += m(y) (lg_total_0^b(y) - lg_total_0^r(y)) / S-bar     [kernel B1]
//   (3) pull^T:  lambda^n_j(y) = lg_total_j(y + c_j), or lg_total_{opp j}(y) where y + c_j is
//                solid or beyond a wall (the transpose of the pull with bounce-back): kernel A
//                pushes the lg part to where the pull read from, the next kernel A adds the ab
//                part of the writer as it reads lambda^{n+1}
// Kernel A recomputes the forward quantities of its tile exactly as the step does (it runs the
// step's own tile code with this file's epilogue in place of the collision/store).
#pragma once

#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

// Minority fraction product w_r w_b below which the adjoint holds the recoloring direction fixed.
constexpr double kBulkTrace = 1e-6;

// Pull source of direction i from the cell with slot sl at storage index si (see pull_cell).
template <class L>
__device__ __forceinline__ int pull_source(const Slot& sl, const PlaneOffsets& po, int si, int i) {
  return si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
         (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
         (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
}

// (1) for one cell: recompute the moments, F and the per-direction terms of collide_store and
// run them backwards.  fcb: colour-blind sums of the post-exchange populations (rho_r, rho_b
// given separately); lam: dL/d(f^{r*}, f^{b*}) of this cell;
// out: lg = dL/dg through this cell's own collision, lF = dL/dF.
// lam_at(i): lambda^{n+1} of direction i (loaded where it is used); lg_out(i, v): stores lg_i.
template <int Q, class R, class LamAt, class LgOut>
__device__ __forceinline__ void collide_adjoint(const Physics& ph, const R (&fcb)[Q], R rr, R rb,
                                                R irho, const R (&rnb)[Q], const LamAt& lam_at,
                                                const LgOut& lg_out, R (&lF)[3]) {
  using L = Lattice<Q>;
  const R rho = rr + rb;
  const R wr = rr * irho, wb = rb * irho;
  R f[Q];
  R ja = R(0), jb = R(0), jm = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    f[i] = fcb[i];
    if (L::ca(i) > 0) ja += f[i];
    if (L::ca(i) < 0) ja -= f[i];
    if (L::cb(i) > 0) jb += f[i];
    if (L::cb(i) < 0) jb -= f[i];
    if (L::cm(i) > 0) jm += f[i];
    if (L::cm(i) < 0) jm -= f[i];
  }
  const R ua = ja * irho, ub = jb * irho, um = jm * irho;
  const R uu15 = R(1.5) * (ua * ua + ub * ub + um * um);
  const R ir = PHYS(R, ph, inv_tau_r), ib = PHYS(R, ph, inv_tau_b);
  const R itau = wr * ir + wb * ib;
  const R abar = wr * PHYS(R, ph, alpha_r) + wb * PHYS(R, ph, alpha_b);
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
  const R amp = PHYS(R, ph, amp), beta = PHYS(R, ph, beta);
  const R pamp = amp * itau;
  const R rcol = beta * wr * wb;
  R restc[3], rwc[3], nrm[3], As[3], Bs[3], Ws[3], Cs[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int i = c == 0 ? 0 : (c == 1 ? 1 : L::Q - 1);
    As[c] = R(L::A(i));
    Bs[c] = R(L::B(i));
    Ws[c] = R(L::W(i));
    Cs[c] = R(L::C(i));
    nrm[c] = R(inv_norm<L>(i));
    restc[c] = rho * (As[c] + Bs[c] * abar);
    rwc[c] = rho * Ws[c];
  }

  // Backwards through recolor -> perturb -> collision -> feq, direction by direction.  The
  // F-dependence is carried by |F| and the unit vector e = F/|F| (nc_i = e.c_i), both bounded:
  //   perturbation  pamp (W_s |F| nc_i^2 - C_s |F|)   -> d/dF = pamp (2 W_s nc_i c_i - (W_s nc_i^2 + C_s) e)
  //   recoloring    rcol nrm_s restc_s nc_i          -> d/dF = rcol nrm_s restc_s (c_i - nc_i e) / |F|
  // so 1/|F| enters once (as in the step itself); far from an interface |F| can be tiny.
  // Where w_r w_b < kBulkTrace (bulk: one colour is a trace) the recoloring direction e is held
  // fixed: that term is homogeneous of degree 1 in the trace, so its derivative with respect to F
  // stays O(beta w_r / |F|) however small the trace, and the linearised trace dynamics grows
  // without bound while the traces themselves stay negligible.
  R A_wr = R(0), A_itau = R(0), A_uu15 = R(0), A_pamp = R(0), A_rcol = R(0);
  R A_rwc[3] = {R(0), R(0), R(0)}, A_restc[3] = {R(0), R(0), R(0)};
  R Aua = R(0), Aub = R(0), Aum = R(0);
  R Pa = R(0), Pb = R(0), Pm = R(0);  // sum_i 2 pamp W_s q_i nc_i c_i
  R Ga = R(0), Gb = R(0), Gm = R(0);  // sum_i g_i c_i, g_i = d_i rcol nrm_s restc_s
  R Sn = R(0), Sg = R(0);             // sum_i q_i (W_s nc_i^2 + C_s), sum_i g_i nc_i
  const bool bulk = wr * wb < R(kBulkTrace);
  R Af[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int c = L::speed2(i);
    R cu = R(0), pc = R(0);
    if (L::ca(i) > 0) { cu += ua; pc += Fa; }
    if (L::ca(i) < 0) { cu -= ua; pc -= Fa; }
    if (L::cb(i) > 0) { cu += ub; pc += Fb; }
    if (L::cb(i) < 0) { cu -= ub; pc -= Fb; }
    if (L::cm(i) > 0) { cu += um; pc += Fm; }
    if (L::cm(i) < 0) { cu -= um; pc -= Fm; }
    const R nc = pc * iFn;  // e.c_i (0 where F = 0)
    const R poly = cu * (R(4.5) * cu + R(3)) - uu15;
    const R feq = rwc[c] * poly + restc[c];
    const R pert = Ws[c] * Fn * nc * nc - Cs[c] * Fn;  // perturbation shape, Eq. (perturb)
    const R fi = f[i] + itau * (feq - f[i]) + pamp * pert;  // post-perturbation
    // Eq. (recolor): f^{r*} = wr fi + rcol nrm restc nc, f^{b*} = fi - f^{r*}
    const V2<R> li = lam_at(i);
    const R d = li.r - li.b;
    const R q = wr * d + li.b;  // dL/dfi
    A_wr += d * fi;
    A_rcol += d * nrm[c] * restc[c] * nc;
    A_restc[c] += d * rcol * nrm[c] * nc;
    const R g = bulk ? R(0) : d * rcol * nrm[c] * restc[c];
    Sg += g * nc;
    // Eq. (perturb)
    A_pamp += q * pert;
    Sn += q * (Ws[c] * nc * nc + Cs[c]);
    const R p2 = R(2) * pamp * Ws[c] * q * nc;
    // Eq. (collision): fi = f + itau (feq - f)
    const R A_feq = q * itau;
    Af[i] = q * (R(1) - itau);
    A_itau += q * (feq - f[i]);
    // Eq. (feq): feq = rwc (cu (9/2 cu + 3) - 3/2 u^2) + restc
    A_rwc[c] += A_feq * poly;
    A_restc[c] += A_feq;
    const R A_cu = A_feq * rwc[c] * (R(9) * cu + R(3));
    A_uu15 -= A_feq * rwc[c];
    if (L::ca(i) > 0) { Aua += A_cu; Pa += p2; Ga += g; }
    if (L::ca(i) < 0) { Aua -= A_cu; Pa -= p2; Ga -= g; }
    if (L::cb(i) > 0) { Aub += A_cu; Pb += p2; Gb += g; }
    if (L::cb(i) < 0) { Aub -= A_cu; Pb -= p2; Gb -= g; }
    if (L::cm(i) > 0) { Aum += A_cu; Pm += p2; Gm += g; }
    if (L::cm(i) < 0) { Aum -= A_cu; Pm -= p2; Gm -= g; }
  }
  // restc_s = rho (A_s + B_s abar), rwc_s = rho W_s
  R A_rho = R(0), A_abar = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    A_rho += A_restc[c] * (As[c] + Bs[c] * abar) + A_rwc[c] * Ws[c];
    A_abar += A_restc[c] * rho * Bs[c];
  }
  A_itau += A_pamp * amp;  // pamp = amp itau
  R A_wb = R(0);
  A_wr += A_rcol * beta * wb + A_itau * ir + A_abar * PHYS(R, ph, alpha_r);  // rcol = beta wr wb
  A_wb += A_rcol * beta * wr + A_itau * ib + A_abar * PHYS(R, ph, alpha_b);
  // u = j / rho, uu15 = 3/2 |u|^2
  Aua += R(3) * A_uu15 * ua;
  Aub += R(3) * A_uu15 * ub;
  Aum += R(3) * A_uu15 * um;
  A_rho -= (Aua * ua + Aub * ub + Aum * um) * irho;
  const R Aja = Aua * irho, Ajb = Aub * irho, Ajm = Aum * irho;
  // dL/dF = P - pamp Sn e + (G - Sg e) / |F|, e = F / |F| (zero where F = 0, as in the step)
  const R ea = Fa * iFn, eb = Fb * iFn, em = Fm * iFn;
  const R se = pamp * Sn + Sg * iFn;
  lF[0] = Pa + Ga * iFn - se * ea;
  lF[1] = Pb + Gb * iFn - se * eb;
  lF[2] = Pm + Gm * iFn - se * em;
  // wr = rr / rho, wb = rb / rho, rho = rr + rb
  const R A_rr = A_rho + (A_wr - A_wb) * wb * irho;
  const R A_rb = A_rho + (A_wb - A_wr) * wr * irho;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R a = Af[i];
    if (L::ca(i) > 0) a += Aja;
    if (L::ca(i) < 0) a -= Aja;
    if (L::cb(i) > 0) a += Ajb;
    if (L::cb(i) < 0) a -= Ajb;
    if (L::cm(i) > 0) a += Ajm;
    if (L::cm(i) < 0) a -= Ajm;
    lg_out(i, V2<R>{a + A_rr, a + A_rb});
  }
}

// Asynchronous copy of `bytes` (8 or 16) from global to shared memory, and its completion for
// the issuing thread (cp.async; the copies land while the thread goes on).
template <int BYTES>
__device__ __forceinline__ void async_copy(void* smem_dst, const void* gsrc) {
  static_assert(BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gsrc), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Kernel A's per-cell tail (replaces StepEpilogue in step_tile).  It reads lambda^{n+1} and
// writes the transpose of the pull of step n directly:
//   lambda^n_j(y) = lg_j(y + c_j) + ab(y + c_j), or lg_{opp j}(y) + ab(y) where y + c_j is solid
// or beyond a wall, with ab = mu d rho^N / d(rho_r, rho_b) from kernel B1 of the same step.  Its
// lg part is pushed here, each cell x writing lg_i(x) where the pull read g_i(x) from -- slot i
// of x - c_i, or slot opp(i) of x itself for a bounced link -- so every slot of a fluid cell has
// exactly one writer.  The ab part is added by the reader: the next adjoint step's kernel A reads
// the pushed values of its own cell (lam_in) and the ab of the writer, x = y + c_j, from a box
// of the tile's neighbourhood staged in shared memory per plane.  lambda^{n+1} of a cell of plane
// m is copied into this thread's shared-memory column `lam` (Q vec slots, stride TX TH) by prefetch(),
// at the start of the iteration that collides plane m, so the copies overlap the pulls of plane
// m + 1; cell() waits for them.  The ab box has four plane slots (m - 1 .. m + 2 in flight): plane
// um is staged at the start of the iteration that collides um - 1, and its slot was last read by
// the collision of um - 4, two barriers earlier.
template <int TX, int TH>
struct AdjointEpilogue {
  AdjointOut o;
  unsigned char* lam;   // this thread's column: Q slots of sizeof(vec), stride TX TH slots
  unsigned char* abox;  // [4][BY][BX] vec: ab of the planes in flight, one-cell halo

  template <int Q>
  static constexpr int box_x() { return TX + 2; }
  template <int Q>
  static constexpr int box_y() { return Lattice<Q>::D3 ? TH + 2 : 1; }
  template <int Q, int S>
  static constexpr int box_bytes() {
    return 4 * box_x<Q>() * box_y<Q>() * (int)sizeof(typename Storage<S>::vec);
  }

  template <int Q, int S>
  __device__ __forceinline__ void prefetch(const StepArgs& A, int si) const {
    using Vec = typename Storage<S>::vec;
    const int ns = A.g.nstore;
    const Vec* lin = reinterpret_cast<const Vec*>(o.lam_in);
    Vec* col = reinterpret_cast<Vec*>(lam);
#pragma unroll
    for (int i = 0; i < Q; ++i) async_copy<sizeof(Vec)>(col + i * (TX * TH), lin + (size_t)i * ns + si);
    async_commit();
  }
  // ab of plane um (unwrapped) over the tile and its one-cell halo into slot um & 3
  template <int Q, int S>
  __device__ __forceinline__ void stage(const StepArgs& A, int a0, int b0, int um, int tid) const {
    using L = Lattice<Q>;
    using Vec = typename Storage<S>::vec;
    constexpr int BX = box_x<Q>(), BY = box_y<Q>(), NB = BX * BY, NT = TX * TH;
    const Geom& G = A.g;
    const Plane p = make_plane(G, um);
    if (!p.ok) return;  // beyond a wall: never read (those links bounce back)
    const Vec* ab = reinterpret_cast<const Vec*>(o.ab);
    Vec* box = reinterpret_cast<Vec*>(abox) + (um & 3) * NB;
    for (int e = tid; e < NB; e += NT) {
      int a = a0 - 1 + e % BX, b = L::D3 ? b0 - 1 + e / BX : 0;
      bool ok = true;
      if (a < 0 || a >= G.na) {
        if (G.per_a) a = wrap(a, G.na); else ok = false;
      }
      if (L::D3 && (b < 0 || b >= G.nb)) {
        if (G.per_b) b = wrap(b, G.nb); else ok = false;
      }
      if (ok) box[e] = __ldg(ab + sidx(G, a, b, p.m));
    }
  }
  template <int Q, int S, class R>
  __device__ __forceinline__ void cell(const StepArgs& A, int /*cell*/, const Slot& sl,
                                       uint32_t sbits, int m, int si, int /*nimg*/,
                                       const int (&)[3], const R (&g)[Q], R rr, R rb, R irho,
                                       R /*e*/, uint32_t /*flags*/, const R (&rnb)[Q],
                                       int&, R&) const {
    using L = Lattice<Q>;
    using Vec = typename Storage<S>::vec;
    constexpr int BX = box_x<Q>(), NB = BX * box_y<Q>();
    const int ns = A.g.nstore;
    Vec* lout = reinterpret_cast<Vec*>(o.lam_g);
    const PlaneOffsets po = plane_offsets(A.g, m);
    // this cell's place in the ab box: the thread's own column of the tile (one cell per thread
    // and plane), one in from the halo
    const int bx = (int)threadIdx.x % TX + 1;
    const int by = L::D3 ? (int)threadIdx.x / TX + 1 : 0;
    const Vec* box = reinterpret_cast<const Vec*>(abox);
    async_wait_all();  // this thread's copies of plane m (only it reads its column)
    const Vec* col = reinterpret_cast<const Vec*>(lam);
    auto lam_at = [&](int i) -> V2<R> {
      const Vec v = col[i * (TX * TH)];
      // ab of the slot's writer: x = y + c_i, or y itself where y + c_i is solid (the source of
      // this cell's direction opp(i))
      const bool self = i == 0 || ((sbits >> opp(i)) & 1u);
      const Vec w = self ? box[(m & 3) * NB + by * BX + bx]
                         : box[((m + L::cm(i)) & 3) * NB + (by + L::cb(i)) * BX + bx + L::ca(i)];
      return {v.x + w.x, v.y + w.y};
    };
    auto lg_out = [&](int i, V2<R> v2) {
      Vec v;
      v.x = v2.r;
      v.y = v2.b;
      // element index in 32 bits (a state holds Q nstore < 2^31 vec2)
      const bool bounce = (sbits >> i) & 1u;
      const int idx = bounce ? opp(i) * ns + si : i * ns + pull_source<L>(sl, po, si, i);
      lout[idx] = v;
    };
    R lF[3];
    collide_adjoint<Q, R>(A.ph, g, rr, rb, irho, rnb, lam_at, lg_out, lF);
    R* ax = reinterpret_cast<R*>(o.aux);
    ax[si] = lF[0];
    ax[(size_t)ns + si] = lF[1];
    ax[2 * (size_t)ns + si] = lF[2];
    ax[3 * (size_t)ns + si] = R(2) * rb * irho * irho;   // d rho^N / d rho_r
    ax[4 * (size_t)ns + si] = -R(2) * rr * irho * irho;  // d rho^N / d rho_b
  }
};

template <int Q, int S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (S == ST_F64 ? 256 : 384) / (TX * TY))
    cg_adjoint_local_kernel(const __grid_constant__ StepArgs A,
                            const __grid_constant__ AdjointOut O) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  long long n = 0;
  double d = 0.0;
  using Vec = typename Storage<S>::vec;
  using Epi = AdjointEpilogue<TX, TY>;
  // lambda columns after the tile's own shared memory (slot i of thread t at i TX TY + t), then
  // the ab box
  constexpr int lam_bytes = Q * TX * TY * (int)sizeof(Vec);
  unsigned char* const lam0 = dyn_smem + TileSmem<Q, S, TX, TY, 1>::BYTES;
  const Epi E{O, lam0 + threadIdx.x * sizeof(Vec), lam0 + lam_bytes};
  step_tile<Q, S, TX, TY, 1, Epi>(A, blockIdx.x, blockIdx.y, dyn_smem, n, d, threadIdx.x, -1, E);
}

__device__ __forceinline__ void cell_coords(const Geom& g, int cell, int& a, int& b, int& m) {
  a = cell % g.na;
  const int t = cell / g.na;
  b = t % g.nb;
  m = t / g.nb;
}

// (2) one thread per cell.  dLdV: pointer to dL/dV(n+1) (nullptr: 0).
template <int Q, class R>
__global__ void __launch_bounds__(256)
    cg_adjoint_stencil_kernel(Geom G, const R* __restrict__ aux, const void* __restrict__ lam_g,
                              void* __restrict__ ab, const uint8_t* __restrict__ mask,
                              double* __restrict__ dphi, double inv_sbar,
                              const double* __restrict__ dLdV) {
  using L = Lattice<Q>;
  using Vec = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= G.ncell) return;
  int a, b, m;
  cell_coords(G, cell, a, b, m);
  const Slot sl = make_slot<L>(G, a, b);
  const Plane p = make_plane(G, m);
  uint32_t bits = 0;
  if (!solid_bits<L>(G, sl, p, cell, bits)) return;
  const PlaneOffsets po = plane_offsets(G, m);
  const int si = sidx(G, a, b, m);
  const size_t ns = G.nstore;
  const R oa = aux[si], ob = aux[ns + si], om = aux[2 * ns + si];
  R mu = dLdV ? R(0.5 * __ldg(dLdV)) : R(0);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    R t = R(0);
    if (!((bits >> i) & 1u)) {  // x = y - c_i is fluid: its F used rho^N(y) with weight 3 W_i c_i
      const int src = pull_source<L>(sl, po, si, i);
      if (L::ca(i)) t += R(L::ca(i)) * __ldg(aux + src);
      if (L::cb(i)) t += R(L::cb(i)) * __ldg(aux + ns + src);
      if (L::cm(i)) t += R(L::cm(i)) * __ldg(aux + 2 * ns + src);
    }
    if ((bits >> opp(i)) & 1u)  // y + c_i is solid: y's own F used rho^N(y) in its place
      t += R(L::ca(i)) * oa + R(L::cb(i)) * ob + R(L::cm(i)) * om;
    mu += R(3.0 * L::W(i)) * t;
  }
  Vec v;
  v.x = mu * aux[3 * ns + si];
  v.y = mu * aux[4 * ns + si];
  reinterpret_cast<Vec*>(ab)[si] = v;
  if (mask[cell] & 1u) {  // Eq. (exchange): d g_0^r / d phi = -1/S-bar, d g_0^b / d phi = +1/S-bar
    const Vec l0 = reinterpret_cast<const Vec*>(lam_g)[si];
    dphi[cell] += ((double)(l0.y + v.y) - (double)(l0.x + v.x)) * inv_sbar;
  }
}

// V = sum over fluid cells of (1 + rho^N)/2 of a stored state, FP64, deterministic: fixed grid,
// per-block partials, the last block to arrive adds them in block order into *out.
template <int Q, int S>
__global__ void __launch_bounds__(256)
    cg_volume_kernel(Geom G, Physics ph, const void* __restrict__ state, double* __restrict__ part,
                     unsigned int* __restrict__ done, double* __restrict__ out) {
  using R = typename Storage<S>::real;
  __shared__ double red[8];
  __shared__ int is_last;
  double v = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < G.ncell; cell += stride) {
    if (G.links && (__ldg(G.links + cell) >> 31)) continue;
    int a, b, m;
    cell_coords(G, cell, a, b, m);
    const int si = sidx(G, a, b, m);
    R rr = R(0), rb = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const V2<R> f = PopIO<S, Q>::load(state, G.nstore, i, i, si, ph);
      rr += f.r;
      rb += f.b;
    }
    // the liquid fraction in the storage's arithmetic (an FP64 division per cell would hold the
    // FP32 kernel to GB300's FP64 rate), summed in FP64
    v += (double)(rr / (rr + rb));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int tid = threadIdx.x;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
    __threadfence();
    is_last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && tid < 32) {
    __threadfence();
    double s = 0.0;
    for (unsigned j = tid; j < gridDim.x; j += 32) s += __ldcg(part + j);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (tid == 0) {
      *out = s;
      *done = 0u;
    }
  }
}

}  // namespace cgevap
