// step_dev_kernel.cuh -- the fused timestep for the 16-bit deviation storages.
//
// Same arithmetic and z-marching tiles as cg_step_kernel (step_kernel.cuh).  What differs is how
// many cells a thread keeps in flight: a pulled direction is one 4-byte word (the FP16 / BF16
// deviation pair), so a thread owns CPT cells and keeps their raw words -- not decoded FP32
// pairs -- in registers and in a thread-private shared-memory parking column between the pull
// of a plane and its collision.  Decoding needs the FP32 rest pair of each source cell; the
// rest pairs of the tile plus a two-cell ring are staged per plane into a five-plane ring of
// shared memory, so every pulled direction costs one global load and one shared-memory read.
#pragma once

#include "step_kernel.cuh"

namespace cgevap {

// Raw deviation words of the pulled directions 1..Q-1 of one cell (bounce-back where the
// source is solid or beyond a wall: the cell's own word of the opposite direction).
template <int Q, int S>
__device__ __forceinline__ void dev_raw_loads(const StepArgs& A, const Slot& sl, int si,
                                              PlaneOffsets po, uint32_t sbits, uint32_t (&raw)[Q]) {
  using L = Lattice<Q>;
  const uint32_t* dev = reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(A.pin) +
                                                          dev_block_offset(A.g.nstore));
  raw[0] = 0u;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int src = si + (L::ca(i) > 0 ? sl.dxm : (L::ca(i) < 0 ? sl.dxp : 0)) +
              (L::cb(i) > 0 ? sl.dym : (L::cb(i) < 0 ? sl.dyp : 0)) +
              (L::cm(i) > 0 ? po.dm_lo : (L::cm(i) < 0 ? po.dm_hi : 0));
    int dir = i;
    if (sbits) {
      const bool bounce = (sbits >> i) & 1u;
      src = bounce ? si : src;
      dir = bounce ? opp(i) : i;
    }
    raw[i] = __ldg(dev + (size_t)(dir - 1) * A.g.nstore + src);
  }
}

// f_i^k = f_0^k(source) kappa_i^k + deviation / s.  (ex, ey): the cell's rest-box position;
// ps[k] = rest slot of plane m + 1 - k, so the source plane m - c_m of direction i is ps[1 + c_m].
template <int Q, int S, int RY, int RX>
__device__ __forceinline__ void dev_decode(const Physics& ph, const uint32_t (&raw)[Q],
                                           uint32_t sbits, int ex, int ey, const int (&ps)[3],
                                           const float2 (*rest)[RY][RX], V2<float> (&g)[Q]) {
  using L = Lattice<Q>;
  using P = typename Storage<S>::packed;
  const float2 r0 = rest[ps[1]][ey][ex];
  g[0] = {r0.x, r0.y};
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const bool bounce = sbits && ((sbits >> i) & 1u);
    const float2 rs = bounce ? r0 : rest[ps[1 + L::cm(i)]][ey - L::cb(i)][ex - L::ca(i)];
    P pv;
    *reinterpret_cast<uint32_t*>(&pv) = raw[i];
    const float2 d = Storage<S>::unpack(pv);
    const float2 v = __ffma2_rn(rs, make_float2(ph.kap_r[i], ph.kap_b[i]),
                                __fmul2_rn(d, make_float2(ph.inv_scale, ph.inv_scale)));
    g[i] = {v.x, v.y};
  }
}

template <int Q, int S, int TX, int TY, int CPT>
struct DevShape {
  using L = Lattice<Q>;
  static constexpr int TH = TY * CPT;
  static constexpr int RX = TX + 4;
  static constexpr int RY = L::D3 ? TH + 4 : 1;
  static constexpr int RS = 5;  // rest planes m-2 .. m+2
  static constexpr int SMEM = RS * RY * RX * 8 + CPT * (Q - 1) * TX * TY * 4;
};

template <int Q, int S, int TX, int TY, int MINB, int CPT>
__global__ void __launch_bounds__(TX* TY, MINB) cg_step_dev_kernel(const __grid_constant__ StepArgs A) {
  using L = Lattice<Q>;
  using R = float;
  using D = DevShape<Q, S, TX, TY, CPT>;
  constexpr int NT = TX * TY;
  constexpr int TH = D::TH;
  constexpr int HX = TX + 2;
  constexpr int HY = L::D3 ? TH + 2 : 1;
  constexpr int OB = L::D3 ? 1 : 0;
  constexpr int NH = HX * HY - TX * TH;
  constexpr int RX = D::RX, RY = D::RY, RS = D::RS;
  constexpr int RN = RX * RY;
  constexpr int RPT = (RN + NT - 1) / NT;
  static_assert(Storage<S>::dev, "deviation storages only");
  static_assert(NH <= NT, "one ring cell per thread at most");
  static_assert(L::D3 || (TY == 1 && CPT == 1), "D2Q9 tiles are one row");
  __shared__ R ring[4][HY][HX];
  __shared__ double red_d[NT / 32];
  __shared__ long long red_n[NT / 32];
  __shared__ int is_last;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float2(*rest_ring)[RY][RX] = reinterpret_cast<float2(*)[RY][RX]>(dyn_smem);
  uint32_t* parked = reinterpret_cast<uint32_t*>(dyn_smem + RS * RY * RX * 8);  // [CPT][Q-1][NT]

  const Geom& G = A.g;
  const int tid = threadIdx.x;
  const int a0 = (blockIdx.x % A.ntx) * TX;
  const int b0 = (blockIdx.x / A.ntx) * TH;
  const int m0 = blockIdx.y * A.pc;
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

  // in-plane storage offsets of this thread's rest-box elements (-1: beyond a wall or unused)
  int rest_off[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    rest_off[k] = -1;
    const int e = tid + k * NT;
    if (e < RN) {
      int a = a0 - 2 + e % RX, b = L::D3 ? b0 - 2 + e / RX : 0;
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
  auto rest_slot = [&](int uq) { return (uq - m0 + 2 + RS) % RS; };
  auto stage_rest = [&](int uq) {
    const Plane q = make_plane(G, uq);
    const float2* rest = reinterpret_cast<const float2*>(A.pin);
    const int sl = rest_slot(uq);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int e = tid + k * NT;
      if (e < RN && q.ok && rest_off[k] >= 0)
        rest_ring[sl][e / RX][e % RX] = __ldg(rest + q.m * plane_stride + rest_off[k]);
    }
  };

  struct CellScalars {
    R rr, rb, e, irho;
    R lr, lb;  // rounding errors of rr, rb: rr + lr is the exact post-exchange red mass
    uint32_t flags, bits;
    bool ok;
  };
  CellScalars cur[CPT], nxt[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
    cur[c] = nxt[c] = CellScalars{R(0), R(0), R(0), R(0), R(0), R(0), 0u, 0u, false};
  long long n_sites = 0;
  double removed = 0.0;

  auto fill_plane = [&](int um, CellScalars(&out)[CPT], uint32_t(&raw)[CPT][Q]) {
    const Plane p = make_plane(G, um);
    const PlaneOffsets po = plane_offsets(G, p.m);
    const int slot = (um - m0 + 1) & 3;
    stage_rest(um + 1);
    __syncthreads();
    const int ps[3] = {rest_slot(um + 1), rest_slot(um), rest_slot(um - 1)};
    if (has_halo) {
      const int cell = (p.m * G.nb + hs.b) * G.na + hs.a;
      uint32_t bits = 0;
      R rn = R(0);
      if (solid_bits<L>(G, hs, p, cell, bits)) {
        uint32_t hraw[Q];
        V2<R> g[Q];
        R t_rr, t_rb, t_e, t_irho;
        uint32_t t_flags;
        dev_raw_loads<Q, S>(A, hs, sidx(G, hs.a, hs.b, p.m), po, bits, hraw);
        dev_decode<Q, S, RY, RX>(A.ph, hraw, bits, hx + 1, L::D3 ? hy + 1 : 0, ps, rest_ring, g);
        rn = site_exchange<Q, S>(A, cell, g, t_rr, t_rb, t_e, t_flags, t_irho);
      }
      ring[slot][hy][hx] = rn;
    }
    int cells[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {  // every load of every own cell first
      cells[c] = (p.m * G.nb + me[c].b) * G.na + me[c].a;
      uint32_t bits = 0;
      out[c].ok = solid_bits<L>(G, me[c], p, cells[c], bits);
      out[c].bits = bits;
      if (out[c].ok) dev_raw_loads<Q, S>(A, me[c], sidx(G, me[c].a, me[c].b, p.m), po, bits, raw[c]);
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      R rn = R(0);
      if (out[c].ok) {
        V2<R> g[Q];
        dev_decode<Q, S, RY, RX>(A.ph, raw[c], out[c].bits, lx + 2, L::D3 ? ly0 + c * TY + 2 : 0,
                                 ps, rest_ring, g);
        // colour totals without rounding error (from the base B, rest pair first), rounded
        // to nearest, then Eq. (exchange) with its own rounding error (the collision re-decodes g)
        float2 hi = sum_start(A.ph), lo = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < Q; ++i) fast_two_sum_acc(hi, lo, make_float2(g[i].r, g[i].b));
        sum_finish(A.ph, hi, lo);
        rn = exchange_from_sums<S>(A, cells[c], hi.x, hi.y, out[c].rr, out[c].rb, out[c].e,
                                   out[c].flags, out[c].irho);
        out[c].lr = __fadd_rn(lo.x, two_sum_err(hi.x, -out[c].e, out[c].rr));
        out[c].lb = __fadd_rn(lo.y, two_sum_err(hi.y, out[c].e, out[c].rb));
      }
      ring[slot][ly0 + c * TY + OB][lx + 1] = rn;
    }
  };

  stage_rest(m0 - 2);
  stage_rest(m0 - 1);
  {
    CellScalars t[CPT];
    uint32_t raw[CPT][Q];
    fill_plane(m0 - 1, t, raw);
  }
  __syncthreads();  // the next fill restages a rest slot the pulls above read
  {
    uint32_t raw[CPT][Q];
    fill_plane(m0, cur, raw);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int i = 1; i < Q; ++i) parked[(c * (Q - 1) + i - 1) * NT + tid] = raw[c][i];
  }

  for (int m = m0; m < m1; ++m) {
    uint32_t own[CPT][Q];
    {
      uint32_t raw[CPT][Q];
      fill_plane(m + 1, nxt, raw);
      // plane m leaves the parking columns, plane m+1 takes its place (thread-private)
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        own[c][0] = 0u;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          own[c][i] = parked[(c * (Q - 1) + i - 1) * NT + tid];
          parked[(c * (Q - 1) + i - 1) * NT + tid] = raw[c][i];
        }
      }
    }
    __syncthreads();
    const int ps[3] = {rest_slot(m + 1), rest_slot(m), rest_slot(m - 1)};
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (!(active[c] && cur[c].ok)) continue;
      const int ly = ly0 + c * TY;
      V2<R> g[Q];
      dev_decode<Q, S, RY, RX>(A.ph, own[c], cur[c].bits, lx + 2, L::D3 ? ly + 2 : 0, ps,
                               rest_ring, g);
      g[0].r -= cur[c].e;  // Eq. (exchange), as applied when the plane was pulled
      g[0].b += cur[c].e;
      const int s0 = (m - m0 + 1) & 3;
      const R ownrn = ring[s0][ly + OB][lx + 1];
      R rnb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int s = (m - m0 + 1 + L::cm(i)) & 3;
        const bool solid_nb = (cur[c].bits >> opp(i)) & 1u;
        rnb[i] = solid_nb ? ownrn : ring[s][ly + OB + L::cb(i)][lx + 1 + L::ca(i)];
      }
      const int cell = (m * G.nb + me[c].b) * G.na + me[c].a;
      R Fn, fcb[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) fcb[i] = g[i].r + g[i].b;
      collide_store<Q, S, true, true>(A, sidx(G, me[c].a, me[c].b, m), nimg[c], dimg[c], fcb,
                                      cur[c].rr, cur[c].rb, cur[c].irho, rnb, Fn, cur[c].lr,
                                      cur[c].lb);
      uint32_t mb = cur[c].flags;
      if (A.ph.rule == 0) {
        const R d = Fn - PHYS(R, A.ph, threshold);
        mb |= (d > R(0) ? 2u : 0u) | (fabs(d) < R(1e-6) ? 8u : 0u);
      }
      A.mask_out[cell] = (uint8_t)mb;
      if (cur[c].flags & 1u) {
        ++n_sites;
        removed += (double)cur[c].e;
      }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) cur[c] = nxt[c];
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
