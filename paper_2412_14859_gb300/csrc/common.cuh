// common.cuh -- kernel argument blocks, the device ledger and population load/store helpers.
#pragma once

#include "lattice.cuh"

namespace cgevap {

// FP64 mass ledger kept on the device (Eq. exchange bookkeeping).
struct DevLedger {
  double evaporated;     // cumulative sum of varphi over (site, step) pairs
  double last_removed;   // sum over the last step's sites
  long long site_steps;
  long long last_sites;
  long long steps;
};

// Geometry shared by all kernels: sizes along (a, b, m), periodicity, optional solid links.
//
// Per-cell fields (site bytes, links, flux) use the compact index cell = (m*nb + b)*na + a.
// Population arrays use the padded storage index sidx(a, b, m): each stored row holds `pitch`
// elements, a = 0 sits at element kOx of its row (x = 0 of FP32 pairs on a 128-byte line) with
// two ghost columns before it and two after a = na-1, and in 3D each plane holds `rows` rows
// with two ghost rows before b = 0 and after b = nb-1.  While img_a / img_b are set (the TMA
// kernel is selected), the ghosts along that periodic axis hold the periodic images of the two
// nearest cells on the other side, written by every kernel that writes populations, so a box of
// the tile plus two cells never has to wrap.
struct Geom {
  int na, nb, nm;          // a = x; b = y (3D) or 1 (2D); m = z (3D) or y (2D)
  int per_a, per_b, per_m;
  int ncell;               // na * nb * nm
  const uint32_t* links;   // per cell: bit i = pull source of direction i is solid or beyond a
                           // wall, bit 31 = the cell itself is solid; nullptr = no solid cells
  int gy;                  // ghost rows on each side of b: 2 in 3D, 0 in 2D (ghost columns: 2)
  int pitch;               // stored elements per row: round_up(na + kOx + 2, 16)
  int rows;                // stored rows per plane: nb + 2 gy
  int nstore;              // stored elements per population array: nm * rows * pitch
  int img_a, img_b;        // 1 where the periodic images along a / b are maintained
};

__host__ __device__ __forceinline__ int sidx(const Geom& g, int a, int b, int m) {
  return (m * g.rows + b + g.gy) * g.pitch + a + kOx;
}

// Storage indices of a cell and of its periodic ghost images (1 to 4 entries).
struct Images {
  int n;
  int s[4];
};

__device__ __forceinline__ Images images_of(const Geom& g, int a, int b, int m) {
  Images im;
  const int base = sidx(g, a, b, m);
  int da = 0, db = 0;
  if (g.img_a) da = a < 2 ? g.na : (a >= g.na - 2 ? -g.na : 0);
  if (g.img_b) db = b < 2 ? g.nb : (b >= g.nb - 2 ? -g.nb : 0);
  im.n = 1;
  im.s[0] = base;
  if (da) im.s[im.n++] = base + da;
  if (db) im.s[im.n++] = base + db * g.pitch;
  if (da && db) im.s[im.n++] = base + da + db * g.pitch;
  return im;
}

struct Physics {
  double inv_tau_r, inv_tau_b;   // 1 / tau_k
  double alpha_r, alpha_b;       // Sec. II.A
  double amp;                    // (9/4) sigma; the perturbation amplitude is amp / tau
  double beta;                   // Eq. (recolor)
  int rule;                      // 0 gradient, 1 band
  double threshold;              // Gamma or theta
  double varphi;                 // scalar phi / S-bar
  double inv_sbar;               // 1 / S-bar for a flux field
  const void* phi_field;         // per-cell phi (double for ST_F64, float otherwise) or nullptr
  float kap_r[19], kap_b[19];    // deviation storage: phi_i(alpha_k) / phi_0(alpha_k)
  float scale, inv_scale;        // deviation storage: power-of-two scale of the deviations
  float sum_base;                // error-free colour sums start here: a power of two at least
                                 // any single population (0: from the first term)
  // FP32 copies of the constants above (rounded to nearest, as a device-side conversion would
  // round them), so FP32 kernels execute no FP64 instruction; filled by mirror_floats().
  float f_inv_tau_r, f_inv_tau_b, f_alpha_r, f_alpha_b, f_amp, f_beta, f_threshold, f_varphi,
      f_inv_sbar;
};

// Start of the error-free colour sums: a power of two at least four times the larger initial
// density (a single population is below the density of its cell).
__host__ inline float sum_base_for(double rho_r_in, double rho_b_in) {
  const double r = 4.0 * (rho_r_in > rho_b_in ? rho_r_in : rho_b_in);
  float b = 1.0f;
  while (b < r && b < 1e30f) b *= 2.0f;
  return b;
}

// Refresh the FP32 copies; every launch that passes a Physics to a kernel calls this first.
__host__ __device__ inline void mirror_floats(Physics& ph) {
  ph.f_inv_tau_r = (float)ph.inv_tau_r;
  ph.f_inv_tau_b = (float)ph.inv_tau_b;
  ph.f_alpha_r = (float)ph.alpha_r;
  ph.f_alpha_b = (float)ph.alpha_b;
  ph.f_amp = (float)ph.amp;
  ph.f_beta = (float)ph.beta;
  ph.f_threshold = (float)ph.threshold;
  ph.f_varphi = (float)ph.varphi;
  ph.f_inv_sbar = (float)ph.inv_sbar;
}

// A physics constant in the kernel's real type R: the double for FP64 kernels, the FP32 copy
// otherwise (the other branch is a compile-time dead one).
#define PHYS(R, ph, name) (sizeof(R) == 8 ? (R)(ph).name : (R)(ph).f_##name)

struct Reduce {
  double* part_removed;          // per-block partial sums (scratch, one slot per block)
  long long* part_sites;
  unsigned int* done;            // arrival counter, returned to 0 by the last block
  DevLedger* ledger;
  int* status;                   // set to 1 by a bounded wait that gave up (may be nullptr)
};

struct StepArgs {
  Geom g;
  Physics ph;
  Reduce red;
  int ntx, nty;                  // tiles along a and b
  int pc;                        // planes per chunk along m
  const void* pin;               // state read (post-recoloring populations of the last step)
  void* pout;                    // state written
  const uint8_t* mask_in;        // site bytes of the last step
  uint8_t* mask_out;             // site bytes of this step
};

template <class T>
struct V2 {
  T r, b;
};

// ---- population access for each storage format ------------------------------------------------

template <int S, int Q, bool DEV = Storage<S>::dev>
struct PopIO;

template <int S, int Q>
struct PopIO<S, Q, false> {
  using R = typename Storage<S>::real;
  using Vec = typename Storage<S>::vec;
  // Population of direction `dir` stored at storage index `si`, delivered as direction i.  The
  // element index is formed in 32 bits: a state holds Q nstore < 2^31 pairs (checked at create).
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int /*i*/, int dir,
                                               int si, const Physics&) {
    const Vec* p = reinterpret_cast<const Vec*>(base) + (dir * nstore + si);
    Vec v = __ldg(p);
    return {v.x, v.y};
  }
  // Stores one population pair at storage index si; f0 is the rest pair (unused here).
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, R r, R b,
                                               V2<R>, const Physics&) {
    Vec* p = reinterpret_cast<Vec*>(base) + (i * nstore + si);
    Vec v;
    v.x = r;
    v.y = b;
    *p = v;
  }
};

// Recolour-on-pull layout: either colour of a direction from the colour-blind population and the
// cell's record (w_r, V); `dir` is the stored direction (opp(i) for a bounced-back link, whose
// c . V is the negative of direction i's).
template <int Q>
struct RcIO {
  using L = Lattice<Q>;
  static __device__ __forceinline__ const float4* rec(const void* base, int nstore) {
    return reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) +
                                           rc_record_offset(Q, nstore));
  }
  static __device__ __forceinline__ V2<float> load(const void* base, int nstore, int i, int dir,
                                                   int si) {
    const float f = __ldg(reinterpret_cast<const float*>(base) + (size_t)dir * nstore + si);
    if (i == 0) {
      const float wr = __ldg(reinterpret_cast<const float*>(rec(base, nstore) + si));
      const float fr = wr * f;
      return {fr, f - fr};
    }
    const float4 r = __ldg(rec(base, nstore) + si);
    float cv = 0.0f;
    if (L::ca(i) > 0) cv += r.y;
    if (L::ca(i) < 0) cv -= r.y;
    if (L::cb(i) > 0) cv += r.z;
    if (L::cb(i) < 0) cv -= r.z;
    if (L::cm(i) > 0) cv += r.w;
    if (L::cm(i) < 0) cv -= r.w;
    if (dir != i) cv = -cv;
    const float fr = fmaf(r.x, f, float(rc_factor<L>(i)) * cv);
    return {fr, f - fr};
  }
  // Writes f = r + b for direction i; with i = 0 also the record (w_r = r / (r + b), V = 0).
  // Exact for the states this layout can hold with V = 0 (used to zero solid cells).
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, float r, float b) {
    const float f = r + b;
    reinterpret_cast<float*>(base)[(size_t)i * nstore + si] = f;
    if (i == 0) {
      float4* rc = reinterpret_cast<float4*>(reinterpret_cast<char*>(base) + rc_record_offset(Q, nstore));
      rc[si] = make_float4(f > 0.0f ? r / f : 0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
};

// c_i . V of a record (w_r, V) for direction i, summed in the order a, b, m: every reader and
// writer of a recolour-on-pull layout forms it with this function, so the colour split of a
// population is the same bits wherever it is computed (c_opp(i) . V is exactly -(c_i . V)).
template <class L>
__device__ __forceinline__ float rc_cv(int i, const float4& r) {
  // the first nonzero term starts the sum (no addition to zero); i is a compile-time constant
  // in every caller, so only the terms of direction i remain
  float cv = 0.0f;
  bool any = false;
  if (L::ca(i) != 0) {
    cv = L::ca(i) > 0 ? r.y : -r.y;
    any = true;
  }
  if (L::cb(i) != 0) {
    const float t = L::cb(i) > 0 ? r.z : -r.z;
    cv = any ? cv + t : t;
    any = true;
  }
  if (L::cm(i) != 0) {
    const float t = L::cm(i) > 0 ? r.w : -r.w;
    cv = any ? cv + t : t;
  }
  return cv;
}

// Red part of a colour-blind population f of direction i whose source record is r; cv is
// rc_cv(i, r), negated for a bounced link (whose stored direction is opp(i)).
template <class L>
__device__ __forceinline__ float rc_red(int i, float w, float f, float cv) {
  return fmaf(w, f, float(rc_factor<L>(i)) * cv);
}

// 16-bit recolour-on-pull layout, one cell at a time (auxiliary kernels).  load() decodes and
// splits as the step's pull does; store() writes exactly only what this layout holds with V = 0
// and deviations measured from Rf = 0 (used to zero solid cells); other states are imported as
// FP32 pairs.
template <int S, int Q>
struct Rc16IO {
  using L = Lattice<Q>;
  using H = typename Storage<S>::half_t;
  using P = typename H::packed;
  static __device__ __forceinline__ V2<float> load(const void* base, int nstore, int i, int dir,
                                                   int si, const Physics& ph) {
    const char* b = reinterpret_cast<const char*>(base);
    if (i == 0) {
      const float2 r0 = __ldg(reinterpret_cast<const float2*>(b) + si);
      return {r0.x, r0.y};
    }
    const Rc16Layout l = rc16_layout(Q, nstore);
    const float4 rec = __ldg(reinterpret_cast<const float4*>(b + l.rec) + si);
    const float rf = __ldg(reinterpret_cast<const float*>(b + l.ref) + si);
    const P d = reinterpret_cast<const P*>(b + l.dev)[(size_t)(dir - 1) * nstore + si];
    const float f = fmaf(H::unpack(d), ph.inv_scale, float(rc16_ratio<L>(i)) * rf);
    float cv = rc_cv<L>(i, rec);
    if (dir != i) cv = -cv;
    const float fr = rc_red<L>(i, rec.x, f, cv);
    return {fr, f - fr};
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, float r, float b) {
    char* p = reinterpret_cast<char*>(base);
    const Rc16Layout l = rc16_layout(Q, nstore);
    if (i == 0) {
      const float f = r + b;
      reinterpret_cast<float2*>(p)[si] = make_float2(r, b);
      reinterpret_cast<float4*>(p + l.rec)[si] = make_float4(f > 0.0f ? r / f : 0.0f, 0.0f, 0.0f, 0.0f);
      reinterpret_cast<float*>(p + l.ref)[si] = 0.0f;
      return;
    }
    reinterpret_cast<P*>(p + l.dev)[(size_t)(i - 1) * nstore + si] = H::pack(r + b);
  }
};

template <int Q>
struct PopIO<ST_H16RC, Q, false> {
  using R = float;
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int i, int dir, int si,
                                               const Physics& ph) {
    return Rc16IO<ST_H16RC, Q>::load(base, nstore, i, dir, si, ph);
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, R r, R b,
                                               V2<R>, const Physics&) {
    Rc16IO<ST_H16RC, Q>::store(base, nstore, i, si, r, b);
  }
};
template <int Q>
struct PopIO<ST_B16RC, Q, false> {
  using R = float;
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int i, int dir, int si,
                                               const Physics& ph) {
    return Rc16IO<ST_B16RC, Q>::load(base, nstore, i, dir, si, ph);
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, R r, R b,
                                               V2<R>, const Physics&) {
    Rc16IO<ST_B16RC, Q>::store(base, nstore, i, si, r, b);
  }
};
// Pairs in (an imported state), 16-bit recolour-on-pull out: the loads of ST_RCI.
template <int Q>
struct PopIO<ST_H16RCI, Q, false> {
  using R = float;
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int, int dir, int si,
                                               const Physics&) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(base) + (size_t)dir * nstore + si);
    return {v.x, v.y};
  }
};
template <int Q>
struct PopIO<ST_B16RCI, Q, false> : PopIO<ST_H16RCI, Q, false> {};

template <int Q>
struct PopIO<ST_RC, Q, false> {
  using R = float;
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int i, int dir, int si,
                                               const Physics&) {
    return RcIO<Q>::load(base, nstore, i, dir, si);
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, R r, R b,
                                               V2<R>, const Physics&) {
    RcIO<Q>::store(base, nstore, i, si, r, b);
  }
};

// Pairs in (an imported state), recolour-on-pull out.
template <int Q>
struct PopIO<ST_RCI, Q, false> {
  using R = float;
  static __device__ __forceinline__ V2<R> load(const void* base, int nstore, int, int dir, int si,
                                               const Physics&) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(base) + (size_t)dir * nstore + si);
    return {v.x, v.y};
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, R r, R b,
                                               V2<R>, const Physics&) {
    RcIO<Q>::store(base, nstore, i, si, r, b);
  }
};

template <int S, int Q>
struct PopIO<S, Q, true> {
  // store() that also returns the rounding loss of the packed pair: (f - f0 kappa) scale minus
  // what the stored 16-bit pair decodes to, in units of 1 / scale (exact in FP32 by Sterbenz's
  // lemma: the stored value is zero or within a factor of two of the unrounded one)
  static __device__ __forceinline__ float2 store_loss(void* base, int nstore, int i, int si,
                                                      float r, float b, V2<float> f0,
                                                      const Physics& ph) {
    P* d = reinterpret_cast<P*>(reinterpret_cast<char*>(base) + dev_block_offset(nstore)) +
           (size_t)(i - 1) * nstore + si;
    const float2 dev = __fmul2_rn(
        __ffma2_rn(make_float2(-f0.r, -f0.b), make_float2(ph.kap_r[i], ph.kap_b[i]), make_float2(r, b)),
        make_float2(ph.scale, ph.scale));
    const P h = Storage<S>::pack(dev.x, dev.y);
    *d = h;
    const float2 back = Storage<S>::unpack(h);
    return make_float2(dev.x - back.x, dev.y - back.y);
  }
  using R = float;
  using P = typename Storage<S>::packed;
  static __device__ __forceinline__ const float2* rest(const void* base) {
    return reinterpret_cast<const float2*>(base);
  }
  // kappa_i = kappa_dir (same speed class), so i selects the constants and dir the address.
  static __device__ __forceinline__ V2<float> load(const void* base, int nstore, int i, int dir,
                                                   int si, const Physics& ph) {
    float2 f0 = __ldg(rest(base) + si);
    if (i == 0) return {f0.x, f0.y};
    const P* d = reinterpret_cast<const P*>(reinterpret_cast<const char*>(base) +
                                            dev_block_offset(nstore)) +
                 (size_t)(dir - 1) * nstore + si;
    const float2 v = Storage<S>::unpack(__ldg(d));
    const float2 r = __ffma2_rn(f0, make_float2(ph.kap_r[i], ph.kap_b[i]),
                                __fmul2_rn(v, make_float2(ph.inv_scale, ph.inv_scale)));
    return {r.x, r.y};
  }
  static __device__ __forceinline__ void store(void* base, int nstore, int i, int si, float r,
                                               float b, V2<float> f0, const Physics& ph) {
    if (i == 0) {
      reinterpret_cast<float2*>(base)[si] = make_float2(r, b);
      return;
    }
    P* d = reinterpret_cast<P*>(reinterpret_cast<char*>(base) + dev_block_offset(nstore)) +
           (size_t)(i - 1) * nstore + si;
    // (f - f0 kappa) scale for both components in packed FP32
    const float2 dev = __fmul2_rn(
        __ffma2_rn(make_float2(-f0.r, -f0.b), make_float2(ph.kap_r[i], ph.kap_b[i]), make_float2(r, b)),
        make_float2(ph.scale, ph.scale));
    *d = Storage<S>::pack(dev.x, dev.y);
  }
};

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Neighbour coordinate along an axis: v+d wrapped if periodic, -1 beyond a wall.
__device__ __forceinline__ int step_coord(int v, int d, int n, int per) {
  int r = v + d;
  if (r < 0 || r >= n) return per ? wrap(r, n) : -1;
  return r;
}

}  // namespace cgevap
