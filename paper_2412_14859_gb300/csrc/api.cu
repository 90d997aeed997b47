// api.cu -- the C ABI of include/cgevap.h: handle lifetime, validation, launch planning and the
// host side of every entry point.  No C++ exception or abort crosses the boundary.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <cuda.h>
#include <string>
#include <vector>

#include "sim.h"

using namespace cgevap;


namespace {
thread_local std::string g_create_error;
}  // namespace

int cgevap::sim_fail(cgevap_sim* s, int code, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_create_error = msg;
  return code;
}

namespace {

int fail(cgevap_sim* s, int code, const std::string& msg) { return sim_fail(s, code, msg); }


double w0_of(int q) { return q == 19 ? Lattice<19>::W(0) : Lattice<9>::W(0); }

std::string validate(const cgevap_params* p) {
  if (!p) return "params is NULL";
  if (p->q != 9 && p->q != 19) return "q must be 9 or 19";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "sizes must be >= 1";
  if (p->q == 9 && p->nz != 1) return "D2Q9 needs nz == 1";
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return "nx*ny*nz must be < 2^31";
  for (int d = 0; d < 3; ++d)
    if (p->periodic[d] != 0 && p->periodic[d] != 1) return "periodic flags must be 0 or 1";
  if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5)) return "tau_r and tau_b must be > 1/2";
  if (!(p->rho_r_in > 0.0) || !(p->rho_b_in > 0.0)) return "initial densities must be > 0";
  if (!(p->beta >= 0.0 && p->beta <= 1.0)) return "beta must lie in [0, 1]";
  if (!(p->sbar > 0.0)) return "sbar must be > 0";
  if (!std::isfinite(p->sigma) || !std::isfinite(p->threshold)) return "sigma/threshold not finite";
  if (p->site_rule != CGEVAP_SITES_GRADIENT && p->site_rule != CGEVAP_SITES_BAND &&
      p->site_rule != CGEVAP_SITES_GIVEN)
    return "unknown site rule";
  if (p->storage < CGEVAP_F64 || p->storage > CGEVAP_F32X) return "unknown storage";
  return "";
}

template <int Q>
void fill_kappa(Physics& ph) {
  using L = Lattice<Q>;
  for (int i = 0; i < 19; ++i) {
    ph.kap_r[i] = ph.kap_b[i] = 0.0f;
    if (i < Q) {
      ph.kap_r[i] = (float)((L::A(i) + L::B(i) * ph.alpha_r) / ph.alpha_r);
      ph.kap_b[i] = (float)((L::A(i) + L::B(i) * ph.alpha_b) / ph.alpha_b);
    }
  }
}

void setup_physics(cgevap_sim* s) {
  const cgevap_params& p = s->p;
  Physics& ph = s->ph;
  const double w0 = w0_of(p.q);
  const double rmin = std::fmin(p.rho_r_in, p.rho_b_in);
  // Sec. II.A: alpha = W_0 for the least dense component, 1 - (1 - W_0)/gamma_k otherwise.
  ph.alpha_r = (p.rho_r_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p.rho_r_in / rmin);
  ph.alpha_b = (p.rho_b_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p.rho_b_in / rmin);
  ph.inv_tau_r = 1.0 / p.tau_r;
  ph.inv_tau_b = 1.0 / p.tau_b;
  ph.amp = 2.25 * p.sigma;
  ph.beta = p.beta;
  ph.rule = p.site_rule;
  ph.threshold = p.threshold;
  ph.inv_sbar = 1.0 / p.sbar;
  ph.varphi = s->phi / p.sbar;
  ph.phi_field = s->phi_field;
  if (p.q == 19)
    fill_kappa<19>(ph);
  else
    fill_kappa<9>(ph);
  if (p.storage == CGEVAP_F16DEV || p.storage == CGEVAP_F16RC) {
    const double rmax = std::fmax(p.rho_r_in, p.rho_b_in);
    int e = (int)std::floor(std::log2(16384.0 / rmax));
    if (e > 10) e = 10;
    if (e < 0) e = 0;
    ph.scale = std::ldexp(1.0f, e);
  } else {
    ph.scale = 1.0f;
  }
  ph.inv_scale = 1.0f / ph.scale;
  ph.sum_base = sum_base_for(p.rho_r_in, p.rho_b_in);
}

}  // namespace

int cgevap::internal_storage(int api_storage) {
  switch (api_storage) {
    case CGEVAP_F64: return ST_F64;
    case CGEVAP_F32: return ST_F32;
    case CGEVAP_F16DEV: return ST_F16;
    case CGEVAP_BF16DEV: return ST_BF16;
    case CGEVAP_F32RC: return ST_RC;
    case CGEVAP_F16RC: return ST_H16RC;
    case CGEVAP_BF16RC: return ST_B16RC;
    case CGEVAP_F32X: return ST_F32X;
    default: return -1;
  }
}

bool cgevap::is_recolour_on_pull(int api_storage) {
  return api_storage == CGEVAP_F32RC || api_storage == CGEVAP_F16RC || api_storage == CGEVAP_BF16RC;
}

AuxArgs cgevap::aux_of(const cgevap_sim* s) {
  AuxArgs a;
  a.g = s->geom;
  a.ph = s->ph;
  mirror_floats(a.ph);
  a.q = s->p.q;
  // the recolour-on-pull layouts hold an imported state as FP32 pairs until the next step; the
  // exact-mass FP32 pairs are FP32 pairs to every kernel but the step
  a.storage = (is_recolour_on_pull(s->p.storage) && s->rc_pairs) || s->p.storage == CGEVAP_F32X
                  ? ST_F32
                  : internal_storage(s->p.storage);
  a.rho_r_in = s->p.rho_r_in;
  a.rho_b_in = s->p.rho_b_in;
  return a;
}

namespace {

// Arguments of the kernels that write a whole imported state: the recolour-on-pull layout takes
// it as FP32 pairs (read by the next step's pairs-in kernel).
AuxArgs import_args(cgevap_sim* s) {
  if (is_recolour_on_pull(s->p.storage)) s->rc_pairs = 1;
  return aux_of(s);
}

// Step kernel of an API storage code; pairs_in: the recolour-on-pull layouts' first step after an
// import, reading FP32 pairs.
KernelRef kernel_for(int q, int storage, int variant, bool pairs_in = false) {
  switch (storage) {
    case CGEVAP_F64: return step_kernel_f64(q, variant);
    case CGEVAP_F32: return step_kernel_f32(q, variant);
    case CGEVAP_F32X: return step_kernel_f32x(q, variant);
    case CGEVAP_F32RC: return step_kernel_rc(q, variant, pairs_in);
    case CGEVAP_F16RC:
    case CGEVAP_BF16RC: return step_kernel_rc16(q, internal_storage(storage), variant, pairs_in);
    default: return step_kernel_dev(q, internal_storage(storage), variant);
  }
}

bool tma_supported(const cgevap_sim* s) {
  const Geom& g = s->geom;
  return s->p.storage == CGEVAP_F32 && (!g.per_a || g.na >= 4) &&
         (s->p.q == 9 || !g.per_b || g.nb >= 4);
}

// Planes per chunk: balance whole waves of resident CTAs against the two extra planes each
// chunk pulls (time ~ waves * (pc + 2)); pc_force > 0 overrides.
int plan_launch(cgevap_sim* s, int family, int variant, int pc_force = 0) {
  KernelRef k = family == 1 ? step_tma_f32(s->p.q, variant)
                            : kernel_for(s->p.q, s->p.storage, variant);
  if (!k.fn) return fail(s, CGEVAP_ERR_UNSUPPORTED, "no step kernel for this configuration");
  KernelRef k_in{nullptr, 0};
  if (is_recolour_on_pull(s->p.storage)) {  // same tiles, FP32 pairs in
    k_in = kernel_for(s->p.q, s->p.storage, variant, true);
    if (!k_in.fn) return fail(s, CGEVAP_ERR_UNSUPPORTED, "no step kernel for this configuration");
  }
  TileCfg t = tile_cfg(s->p.q, variant);
  if (k.tx > 0) t = TileCfg{k.tx, k.ty};
  int occ = 0, sms = 0;
  CG_CUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.threads, k.smem));
  CG_CUDA(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  if (occ < 1) occ = 1;
  const int na = s->geom.na, nb = s->geom.nb, nm = s->geom.nm;
  const int ntx = (na + t.tx - 1) / t.tx;
  const int nty = (nb + t.ty - 1) / t.ty;
  const long long tiles = (long long)ntx * nty;
  const long long slots = (long long)occ * sms;
  int best_pc = nm;
  double best = 1e300;
  for (int pc = 1; pc <= nm; ++pc) {
    const long long nchunk = (nm + pc - 1) / pc;
    if (nchunk > 65535) continue;
    const long long blocks = tiles * nchunk;
    const double waves = std::ceil((double)blocks / (double)slots);
    const double cost = waves * (pc + 2);
    if (cost < best - 1e-9) {
      best = cost;
      best_pc = pc;
    }
  }
  if (pc_force > 0) best_pc = pc_force < nm ? pc_force : nm;
  if (k.needs_map) {
    const int bh = s->p.q == 19 ? t.ty + 2 : 1;
    for (int h = 0; h < 2; ++h) {
      int rc = make_pop_tensor_map(s->tmap[h], s->state[h], s->geom, s->p.q, 8, t.tx + 4, bh);
      if (rc != 0) return fail(s, CGEVAP_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(rc));
    }
  }
  // the TMA kernel reads periodic images from the ghost layers: keep them from now on
  const int want_a = family == 1 && s->geom.per_a && s->geom.na >= 4;
  const int want_b = family == 1 && s->p.q == 19 && s->geom.per_b && s->geom.nb >= 4;
  const bool turn_on = (want_a && !s->geom.img_a) || (want_b && !s->geom.img_b);
  s->geom.img_a = want_a;
  s->geom.img_b = want_b;
  if (turn_on) CG_CUDA(s, launch_fill_ghosts(aux_of(s), s->state[s->cur], s->stream));
  s->family = family;
  s->variant = variant;
  s->kernel = k;
  s->kernel_in = k_in;
  s->ntx = ntx;
  s->nty = nty;
  s->pc = best_pc;
  s->nchunk = (nm + best_pc - 1) / best_pc;
  const long long need = tiles * s->nchunk;
  if (need > s->part_capacity) {
    if (s->part_removed) cudaFree(s->part_removed);
    if (s->part_sites) cudaFree(s->part_sites);
    s->part_removed = nullptr;
    s->part_sites = nullptr;
    if (cudaMalloc(&s->part_removed, need * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->part_sites, need * sizeof(long long)) != cudaSuccess) {
      s->part_capacity = 0;
      return fail(s, CGEVAP_ERR_OOM, "cannot allocate per-block partials");
    }
    s->part_capacity = need;
  }
  return CGEVAP_OK;
}

}  // namespace

StepArgs cgevap::step_args(cgevap_sim* s) {
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = s->geom;
  a.ph = s->ph;
  mirror_floats(a.ph);
  a.red.part_removed = s->part_removed;
  a.red.part_sites = s->part_sites;
  a.red.done = s->done;
  a.red.ledger = s->ledger;
  a.red.status = s->status;
  a.ntx = s->ntx;
  a.nty = s->nty;
  a.pc = s->pc;
  a.pin = s->state[s->cur];
  a.pout = s->state[s->cur ^ 1];
  a.mask_in = s->mask[s->cur];
  a.mask_out = s->mask[s->cur ^ 1];
  return a;
}

namespace {

// Recomputes the heated-substrate flux field from state[cur] (cgevap_set_flux_heated).
int refresh_heated_flux(cgevap_sim* s) {
  CG_CUDA(s, launch_heated_flux(aux_of(s), s->state[s->cur], s->heat.part, s->heat.phi_s, s->heat.K,
                                s->heat.length, s->phi_field, s->p.storage == CGEVAP_F64 ? 1 : 0,
                                s->stream));
  s->heat.since = 0;
  return CGEVAP_OK;
}

int launch_one_step(cgevap_sim* s) {
  if (s->heat.on && s->heat.since >= s->heat.every) {
    const int rc = refresh_heated_flux(s);
    if (rc != CGEVAP_OK) return rc;
  }
  ++s->heat.since;
  if (s->outlet_rho[0] > 0.0 || s->outlet_rho[1] > 0.0)
    CG_CUDA(s, launch_outlets(aux_of(s), s->state[s->cur], s->outlet_rho[0], s->outlet_rho[1], s->stream));
  StepArgs a = step_args(s);
  void* args[] = {&a, s->tmap[s->cur]};
  const KernelRef& k = s->rc_pairs && s->kernel_in.fn ? s->kernel_in : s->kernel;
  CG_CUDA(s, cudaLaunchKernel(k.fn, dim3(s->ntx * s->nty, s->nchunk), dim3(k.threads), args, k.smem,
                              s->stream));
  s->cur ^= 1;
  s->rc_pairs = 0;
  return CGEVAP_OK;
}


}  // namespace

int cgevap::refresh_gradient_sites(cgevap_sim* s) {
  if (s->p.site_rule != CGEVAP_SITES_GRADIENT) {
    CG_CUDA(s, cudaMemsetAsync(s->mask[s->cur], 0, s->N, s->stream));
    return CGEVAP_OK;
  }
  if (!s->tmp_rn && cudaMalloc(&s->tmp_rn, s->N * sizeof(double)) != cudaSuccess)
    return sim_fail(s, CGEVAP_ERR_OOM, "cannot allocate rho^N scratch");
  CG_CUDA(s, launch_gradient_sites(aux_of(s), s->state[s->cur], s->tmp_rn, s->mask[s->cur], s->stream));
  return CGEVAP_OK;
}

namespace {

void release(cgevap_sim* s) {
  if (!s) return;
  adjoint_release(s);
  void* ptrs[] = {s->state[0], s->state[1], s->mask[0],  s->mask[1],  s->links,
                  s->solid,    s->phi_field, s->ledger, s->part_removed, s->part_sites,
                  s->done,     s->tmp_rn,   s->flag,    s->staging, s->status,
                  s->vol_part, s->vol_done, s->heat.part};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete s;
}

}  // namespace

namespace cgevap {
int sim_view(cgevap_sim* s, SimView* v) {
  if (!s || !v) return CGEVAP_ERR_ARG;
  v->g = s->geom;
  v->ph = s->ph;
  mirror_floats(v->ph);
  v->state[0] = s->state[0];
  v->state[1] = s->state[1];
  v->mask[0] = s->mask[0];
  v->mask[1] = s->mask[1];
  v->ledger = s->ledger;
  v->cur = &s->cur;
  v->stream = &s->stream;
  v->state_bytes = s->state_bytes;
  v->ncell = s->N;
  return CGEVAP_OK;
}
}  // namespace cgevap

extern "C" {

int cgevap_create(const cgevap_params* p, cgevap_sim** out) {
  if (!out) return fail(nullptr, CGEVAP_ERR_ARG, "out is NULL");
  *out = nullptr;
  std::string why = validate(p);
  if (!why.empty()) return fail(nullptr, CGEVAP_ERR_ARG, why);
  cgevap_sim* s = new (std::nothrow) cgevap_sim();
  if (!s) return fail(nullptr, CGEVAP_ERR_OOM, "host allocation failed");
  s->p = *p;
  s->Q = p->q;
  s->N = (long long)p->nx * p->ny * p->nz;
  s->nfluid = s->N;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    release(s);
    return fail(nullptr, CGEVAP_ERR_CUDA, "no CUDA device");
  }
  Geom& g = s->geom;
  g.na = p->nx;
  if (p->q == 19) {
    g.nb = p->ny;
    g.nm = p->nz;
    g.per_a = p->periodic[0];
    g.per_b = p->periodic[1];
    g.per_m = p->periodic[2];
  } else {
    g.nb = 1;
    g.nm = p->ny;
    g.per_a = p->periodic[0];
    g.per_b = 1;
    g.per_m = p->periodic[1];
  }
  g.ncell = (int)s->N;
  g.links = nullptr;
  const StoreShape sh = store_shape(p->q, p->nx, p->ny, p->nz);
  if ((long long)p->q * sh.nstore >= (1LL << 31)) {
    release(s);
    return fail(nullptr, CGEVAP_ERR_ARG, "lattice too large for 32-bit storage indices");
  }
  g.gy = p->q == 19 ? 2 : 0;
  g.pitch = sh.pitch;
  g.rows = sh.rows;
  g.nstore = (int)sh.nstore;
  g.img_a = 0;  // ghost images are kept only while the TMA kernel is selected
  g.img_b = 0;
  setup_physics(s);
  s->state_bytes = state_bytes(internal_storage(p->storage), p->q, sh.nstore);
  bool ok = true;
  for (int h = 0; h < 2 && ok; ++h) {
    ok = cudaMalloc(&s->state[h], s->state_bytes) == cudaSuccess &&
         cudaMalloc(&s->mask[h], s->N) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&s->ledger, sizeof(DevLedger)) == cudaSuccess &&
       cudaMalloc(&s->done, sizeof(unsigned int)) == cudaSuccess &&
       cudaMalloc(&s->flag, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&s->status, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release(s);
    return fail(nullptr, CGEVAP_ERR_OOM, "device allocation failed");
  }
  bool z = cudaMemset(s->state[0], 0, s->state_bytes) == cudaSuccess &&
           cudaMemset(s->state[1], 0, s->state_bytes) == cudaSuccess &&
           cudaMemset(s->mask[0], 0, s->N) == cudaSuccess &&
           cudaMemset(s->mask[1], 0, s->N) == cudaSuccess &&
           cudaMemset(s->ledger, 0, sizeof(DevLedger)) == cudaSuccess &&
           cudaMemset(s->done, 0, sizeof(unsigned int)) == cudaSuccess &&
           cudaMemset(s->status, 0, sizeof(int)) == cudaSuccess;
  if (!z) {
    release(s);
    return fail(nullptr, CGEVAP_ERR_CUDA, "initial memset failed");
  }
  int rc = plan_launch(s, 0, 0);
  if (rc != CGEVAP_OK) {
    std::string m = s->err;
    release(s);
    return fail(nullptr, rc, m);
  }
  *out = s;
  return CGEVAP_OK;
}

int cgevap_destroy(cgevap_sim* s) {
  if (!s) return CGEVAP_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  release(s);
  return CGEVAP_OK;
}

const char* cgevap_last_error(const cgevap_sim* s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

int cgevap_get_params(const cgevap_sim* s, cgevap_params* out) {
  if (!s || !out) return CGEVAP_ERR_ARG;
  *out = s->p;
  return CGEVAP_OK;
}

int cgevap_set_stream(cgevap_sim* s, void* stream) {
  if (!s) return CGEVAP_ERR_ARG;
  s->stream = (cudaStream_t)stream;
  return CGEVAP_OK;
}

int cgevap_set_solid(cgevap_sim* s, const uint8_t* dev_solid) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  if (!dev_solid) {
    if (s->links) cudaFree(s->links);
    if (s->solid) cudaFree(s->solid);
    s->links = nullptr;
    s->solid = nullptr;
    s->geom.links = nullptr;
    s->nfluid = s->N;
    return CGEVAP_OK;
  }
  if (!s->solid && cudaMalloc(&s->solid, s->N) != cudaSuccess)
    return fail(s, CGEVAP_ERR_OOM, "cannot allocate solid flags");
  if (!s->links && cudaMalloc(&s->links, s->N * sizeof(uint32_t)) != cudaSuccess)
    return fail(s, CGEVAP_ERR_OOM, "cannot allocate solid links");
  CG_CUDA(s, cudaMemcpyAsync(s->solid, dev_solid, s->N, cudaMemcpyDeviceToDevice, s->stream));
  Geom g = s->geom;
  g.links = nullptr;
  AuxArgs a = aux_of(s);
  a.g = g;
  CG_CUDA(s, launch_links(a, s->solid, s->links, s->stream));
  s->geom.links = s->links;
  CG_CUDA(s, launch_zero_solid(aux_of(s), s->state[s->cur], s->stream));
  std::vector<uint8_t> h(s->N);
  CG_CUDA(s, cudaMemcpyAsync(h.data(), s->solid, s->N, cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  long long nf = 0;
  for (uint8_t v : h) nf += v ? 0 : 1;
  s->nfluid = nf;
  return refresh_gradient_sites(s);
}

int cgevap_set_flux(cgevap_sim* s, double phi, const void* dev_phi_field, int dtype) {
  if (!s) return CGEVAP_ERR_ARG;
  if (!std::isfinite(phi)) return fail(s, CGEVAP_ERR_ARG, "phi is not finite");
  CG_CUDA(s, cudaSetDevice(s->device));
  s->phi = phi;
  s->heat.on = 0;
  if (dev_phi_field) {
    if (dtype != CGEVAP_DTYPE_F64 && dtype != CGEVAP_DTYPE_F32)
      return fail(s, CGEVAP_ERR_ARG, "flux dtype must be F64 or F32");
    const bool dbl = s->p.storage == CGEVAP_F64;
    if (!s->phi_field && cudaMalloc(&s->phi_field, s->N * (dbl ? 8 : 4)) != cudaSuccess)
      return fail(s, CGEVAP_ERR_OOM, "cannot allocate flux field");
    CG_CUDA(s, launch_convert_field(dev_phi_field, dtype, s->phi_field, dbl ? 1 : 0, s->N, s->stream));
  } else if (s->phi_field) {
    cudaFree(s->phi_field);
    s->phi_field = nullptr;
  }
  s->ph.varphi = phi / s->p.sbar;
  s->ph.phi_field = dev_phi_field ? s->phi_field : nullptr;
  return CGEVAP_OK;
}

int cgevap_set_flux_heated(cgevap_sim* s, double phi_s, double K, double length, int every) {
  if (!s) return CGEVAP_ERR_ARG;
  if (!std::isfinite(phi_s) || !(K > 0.0) || !std::isfinite(K) || !(length > 0.0) ||
      !std::isfinite(length) || every < 1)
    return fail(s, CGEVAP_ERR_ARG, "heated flux needs finite phi_s, K > 0, length > 0, every >= 1");
  if (s->geom.per_m)
    return fail(s, CGEVAP_ERR_ARG, "heated flux needs walls on the substrate normal (z in 3D, y in 2D)");
  CG_CUDA(s, cudaSetDevice(s->device));
  const HeatedPlan hp = heated_plan(s->geom);
  if (!s->heat.part &&
      cudaMalloc(&s->heat.part, (size_t)(hp.nchunk + 1) * s->geom.na * s->geom.nb * sizeof(double)) != cudaSuccess)
    return fail(s, CGEVAP_ERR_OOM, "cannot allocate the column partials");
  const bool dbl = s->p.storage == CGEVAP_F64;
  if (!s->phi_field && cudaMalloc(&s->phi_field, s->N * (dbl ? 8 : 4)) != cudaSuccess)
    return fail(s, CGEVAP_ERR_OOM, "cannot allocate flux field");
  s->phi = 0.0;
  s->ph.varphi = 0.0;
  s->ph.phi_field = s->phi_field;
  s->heat.on = 1;
  s->heat.phi_s = phi_s;
  s->heat.K = K;
  s->heat.length = length;
  s->heat.every = every;
  return refresh_heated_flux(s);
}

int cgevap_set_outlets(cgevap_sim* s, double rho_lo, double rho_hi) {
  if (!s) return CGEVAP_ERR_ARG;
  if (is_recolour_on_pull(s->p.storage) && (rho_lo > 0.0 || rho_hi > 0.0))
    return fail(s, CGEVAP_ERR_UNSUPPORTED,
                "outlets need a storage that holds each colour (not a recolour-on-pull layout)");
  if (!std::isfinite(rho_lo) || !std::isfinite(rho_hi))
    return fail(s, CGEVAP_ERR_ARG, "outlet densities must be finite");
  const bool lo = rho_lo > 0.0, hi = rho_hi > 0.0;
  if ((lo || hi) && s->geom.per_m)
    return fail(s, CGEVAP_ERR_ARG, "outlets need walls on the wall-normal axis (z in 3D, y in 2D)");
  if (lo && hi && s->geom.nm < 2)
    return fail(s, CGEVAP_ERR_ARG, "two outlets need at least two planes");
  s->outlet_rho[0] = lo ? rho_lo : 0.0;
  s->outlet_rho[1] = hi ? rho_hi : 0.0;
  return CGEVAP_OK;
}

int cgevap_get_flux_field(cgevap_sim* s, double* dev_out) {
  if (!s || !dev_out) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  if (s->ph.phi_field) {
    CG_CUDA(s, launch_convert_field(s->phi_field, s->p.storage == CGEVAP_F64 ? CGEVAP_DTYPE_F64 : CGEVAP_DTYPE_F32,
                                    dev_out, 1, s->N, s->stream));
  } else {
    CG_CUDA(s, launch_fill(dev_out, s->phi, s->N, s->stream));
  }
  return CGEVAP_OK;
}

int cgevap_init_equilibrium(cgevap_sim* s, const double* dev_rhoN0, const void* dev_noise,
                            int noise_dtype) {
  if (!s || !dev_rhoN0) return CGEVAP_ERR_ARG;
  if (dev_noise && noise_dtype != CGEVAP_DTYPE_F64 && noise_dtype != CGEVAP_DTYPE_F32)
    return fail(s, CGEVAP_ERR_ARG, "noise dtype must be F64 or F32");
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, launch_init_equilibrium(import_args(s), dev_rhoN0, dev_noise, noise_dtype,
                                     s->state[s->cur], s->stream));
  CG_CUDA(s, cudaMemsetAsync(s->ledger, 0, sizeof(DevLedger), s->stream));
  s->heat.since = s->heat.every;  // a heated flux field follows the new state
  return refresh_gradient_sites(s);
}

int cgevap_set_populations(cgevap_sim* s, const void* dev_f, int dtype) {
  if (!s || !dev_f) return CGEVAP_ERR_ARG;
  if (dtype != CGEVAP_DTYPE_F64 && dtype != CGEVAP_DTYPE_F32)
    return fail(s, CGEVAP_ERR_ARG, "dtype must be F64 or F32");
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, launch_set_populations(import_args(s), dev_f, dtype, s->state[s->cur], s->stream));
  s->heat.since = s->heat.every;
  return refresh_gradient_sites(s);
}

int cgevap_set_populations_host(cgevap_sim* s, const void* host_f, int dtype) {
  if (!s || !host_f) return CGEVAP_ERR_ARG;
  if (dtype != CGEVAP_DTYPE_F64 && dtype != CGEVAP_DTYPE_F32)
    return fail(s, CGEVAP_ERR_ARG, "dtype must be F64 or F32");
  CG_CUDA(s, cudaSetDevice(s->device));
  const size_t bytes = (size_t)2 * s->Q * s->N * (dtype == CGEVAP_DTYPE_F64 ? 8 : 4);
  if (s->staging_bytes < bytes) {
    if (s->staging) cudaFree(s->staging);
    s->staging = nullptr;
    s->staging_bytes = 0;
    if (cudaMalloc(&s->staging, bytes) != cudaSuccess)
      return fail(s, CGEVAP_ERR_OOM, "cannot allocate staging buffer");
    s->staging_bytes = bytes;
  }
  CG_CUDA(s, cudaMemcpyAsync(s->staging, host_f, bytes, cudaMemcpyHostToDevice, s->stream));
  int rc = cgevap_set_populations(s, s->staging, dtype);
  if (rc != CGEVAP_OK) return rc;
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  return CGEVAP_OK;
}

int cgevap_get_populations(cgevap_sim* s, void* dev_f, int dtype) {
  if (!s || !dev_f) return CGEVAP_ERR_ARG;
  if (dtype != CGEVAP_DTYPE_F64 && dtype != CGEVAP_DTYPE_F32)
    return fail(s, CGEVAP_ERR_ARG, "dtype must be F64 or F32");
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, launch_get_populations(aux_of(s), s->state[s->cur], dev_f, dtype, s->stream));
  return CGEVAP_OK;
}

int cgevap_step(cgevap_sim* s, int nsteps) {
  if (!s || nsteps < 0) return s ? fail(s, CGEVAP_ERR_ARG, "nsteps < 0") : CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  for (int n = 0; n < nsteps; ++n) {
    int rc = launch_one_step(s);
    if (rc != CGEVAP_OK) return rc;
  }
  return CGEVAP_OK;
}

int cgevap_get_macros(cgevap_sim* s, double* rho_r, double* rho_b, double* u, double* rhoN) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, launch_macros(aux_of(s), s->state[s->cur], rho_r, rho_b, u, rhoN, s->stream));
  return CGEVAP_OK;
}

int cgevap_get_mask(cgevap_sim* s, uint8_t* dev_mask) {
  if (!s || !dev_mask) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaMemcpyAsync(dev_mask, s->mask[s->cur], s->N, cudaMemcpyDeviceToDevice, s->stream));
  return CGEVAP_OK;
}

int cgevap_set_mask(cgevap_sim* s, const uint8_t* dev_mask) {
  if (!s || !dev_mask) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaMemcpyAsync(s->mask[s->cur], dev_mask, s->N, cudaMemcpyDeviceToDevice, s->stream));
  return CGEVAP_OK;
}

int cgevap_get_ledger(cgevap_sim* s, cgevap_ledger* out) {
  if (!s || !out) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  DevLedger d;
  int st = 0;
  CG_CUDA(s, cudaMemcpyAsync(&d, s->ledger, sizeof(d), cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (st) {
    cudaMemsetAsync(s->status, 0, sizeof(int), s->stream);
    return fail(s, CGEVAP_ERR_TIMEOUT, "a device-side wait of the step gave up");
  }
  out->evaporated = d.evaporated;
  out->last_removed = d.last_removed;
  out->site_steps = d.site_steps;
  out->last_sites = d.last_sites;
  out->steps = d.steps;
  return CGEVAP_OK;
}

// The device record is laid out as the public one, so it is copied as it is.
static_assert(sizeof(DevLedger) == sizeof(cgevap_ledger), "ledger layouts");
static_assert(offsetof(DevLedger, evaporated) == offsetof(cgevap_ledger, evaporated) &&
                  offsetof(DevLedger, last_removed) == offsetof(cgevap_ledger, last_removed) &&
                  offsetof(DevLedger, site_steps) == offsetof(cgevap_ledger, site_steps) &&
                  offsetof(DevLedger, last_sites) == offsetof(cgevap_ledger, last_sites) &&
                  offsetof(DevLedger, steps) == offsetof(cgevap_ledger, steps),
              "ledger layouts");

int cgevap_get_ledger_async(cgevap_sim* s, cgevap_ledger* out) {
  if (!s || !out) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaMemcpyAsync(out, s->ledger, sizeof(DevLedger), cudaMemcpyDeviceToHost, s->stream));
  return CGEVAP_OK;
}

int cgevap_reset_ledger(cgevap_sim* s) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaMemsetAsync(s->ledger, 0, sizeof(DevLedger), s->stream));
  return CGEVAP_OK;
}

int cgevap_check_health(cgevap_sim* s) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
  CG_CUDA(s, launch_health(aux_of(s), s->state[s->cur], s->flag, s->stream));
  int h = 0;
  CG_CUDA(s, cudaMemcpyAsync(&h, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (h) return fail(s, CGEVAP_ERR_NAN, "non-finite population or non-positive density");
  return CGEVAP_OK;
}

// Checkpoint file: magic, version, params, then raw device images (bit-exact restart).
static const char kMagic[8] = {'C', 'G', 'E', 'V', 'A', 'P', 'C', 'K'};
static const int kVersion = 2;  // 2 adds the F32RC layout flag after the ledger

int cgevap_save(cgevap_sim* s, const char* path) {
  if (!s || !path) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  std::vector<char> state(s->state_bytes);
  std::vector<uint8_t> mask(s->N), solid;
  std::vector<char> field;
  DevLedger led;
  CG_CUDA(s, cudaMemcpyAsync(state.data(), s->state[s->cur], s->state_bytes, cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaMemcpyAsync(mask.data(), s->mask[s->cur], s->N, cudaMemcpyDeviceToHost, s->stream));
  CG_CUDA(s, cudaMemcpyAsync(&led, s->ledger, sizeof(led), cudaMemcpyDeviceToHost, s->stream));
  const size_t fbytes = s->N * (s->p.storage == CGEVAP_F64 ? 8 : 4);
  if (s->ph.phi_field) {
    field.resize(fbytes);
    CG_CUDA(s, cudaMemcpyAsync(field.data(), s->phi_field, fbytes, cudaMemcpyDeviceToHost, s->stream));
  }
  if (s->solid) {
    solid.resize(s->N);
    CG_CUDA(s, cudaMemcpyAsync(solid.data(), s->solid, s->N, cudaMemcpyDeviceToHost, s->stream));
  }
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(s, CGEVAP_ERR_IO, std::string("cannot open ") + path);
  const int has_field = field.empty() ? 0 : 1, has_solid = solid.empty() ? 0 : 1;
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&kVersion, sizeof(int), 1, f) == 1 &&
            std::fwrite(&s->p, sizeof(s->p), 1, f) == 1 &&
            std::fwrite(&s->phi, sizeof(double), 1, f) == 1 &&
            std::fwrite(&has_field, sizeof(int), 1, f) == 1 &&
            std::fwrite(&has_solid, sizeof(int), 1, f) == 1 &&
            std::fwrite(&led, sizeof(led), 1, f) == 1 &&
            std::fwrite(&s->rc_pairs, sizeof(int), 1, f) == 1 &&
            std::fwrite(state.data(), 1, state.size(), f) == state.size() &&
            std::fwrite(mask.data(), 1, mask.size(), f) == mask.size() &&
            (!has_field || std::fwrite(field.data(), 1, field.size(), f) == field.size()) &&
            (!has_solid || std::fwrite(solid.data(), 1, solid.size(), f) == solid.size());
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(s, CGEVAP_ERR_IO, std::string("write failed: ") + path);
  return CGEVAP_OK;
}

int cgevap_load(cgevap_sim* s, const char* path) {
  if (!s || !path) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(s, CGEVAP_ERR_IO, std::string("cannot open ") + path);
  char magic[8];
  int version = 0, has_field = 0, has_solid = 0, rc_pairs = 1;
  cgevap_params p;
  double phi = 0;
  DevLedger led;
  std::vector<char> state(s->state_bytes), field;
  std::vector<uint8_t> mask(s->N), solid;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(&version, sizeof(int), 1, f) == 1 && (version == 1 || version == kVersion) &&
            std::fread(&p, sizeof(p), 1, f) == 1 && std::fread(&phi, sizeof(double), 1, f) == 1 &&
            std::fread(&has_field, sizeof(int), 1, f) == 1 &&
            std::fread(&has_solid, sizeof(int), 1, f) == 1 &&
            std::fread(&led, sizeof(led), 1, f) == 1 &&
            (version == 1 || std::fread(&rc_pairs, sizeof(int), 1, f) == 1);
  if (ok && std::memcmp(&p, &s->p, sizeof(p)) != 0) {
    std::fclose(f);
    return fail(s, CGEVAP_ERR_ARG, "checkpoint parameters differ from the handle's");
  }
  ok = ok && std::fread(state.data(), 1, state.size(), f) == state.size() &&
       std::fread(mask.data(), 1, mask.size(), f) == mask.size();
  const size_t fbytes = s->N * (s->p.storage == CGEVAP_F64 ? 8 : 4);
  if (ok && has_field) {
    field.resize(fbytes);
    ok = std::fread(field.data(), 1, fbytes, f) == fbytes;
  }
  if (ok && has_solid) {
    solid.resize(s->N);
    ok = std::fread(solid.data(), 1, s->N, f) == (size_t)s->N;
  }
  std::fclose(f);
  if (!ok) return fail(s, CGEVAP_ERR_IO, std::string("malformed checkpoint: ") + path);
  if (has_solid) {
    uint8_t* d = nullptr;
    CG_CUDA(s, cudaMalloc(&d, s->N));
    cudaError_t e = cudaMemcpy(d, solid.data(), s->N, cudaMemcpyHostToDevice);
    int rc = e == cudaSuccess ? cgevap_set_solid(s, d) : CGEVAP_ERR_CUDA;
    cudaStreamSynchronize(s->stream);
    cudaFree(d);
    if (rc != CGEVAP_OK) return rc;
  } else {
    cgevap_set_solid(s, nullptr);
  }
  s->phi = phi;
  s->ph.varphi = phi / s->p.sbar;
  s->heat.on = 0;  // a loaded field is held fixed
  if (has_field) {
    if (!s->phi_field && cudaMalloc(&s->phi_field, fbytes) != cudaSuccess)
      return fail(s, CGEVAP_ERR_OOM, "cannot allocate flux field");
    CG_CUDA(s, cudaMemcpyAsync(s->phi_field, field.data(), fbytes, cudaMemcpyHostToDevice, s->stream));
    s->ph.phi_field = s->phi_field;
  } else {
    s->ph.phi_field = nullptr;
  }
  CG_CUDA(s, cudaMemcpyAsync(s->state[s->cur], state.data(), s->state_bytes, cudaMemcpyHostToDevice, s->stream));
  CG_CUDA(s, cudaMemcpyAsync(s->mask[s->cur], mask.data(), s->N, cudaMemcpyHostToDevice, s->stream));
  CG_CUDA(s, cudaMemcpyAsync(s->ledger, &led, sizeof(led), cudaMemcpyHostToDevice, s->stream));
  s->rc_pairs = rc_pairs;
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  return CGEVAP_OK;
}

int cgevap_tune(cgevap_sim* s, int family, int variant, int planes_per_chunk) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  if (family < 0) family = 0;  // the register-pipelined kernel is the faster one on GB300
  if (family > 1) return fail(s, CGEVAP_ERR_ARG, "kernel family must be -1, 0 or 1");
  if (family == 1 && !tma_supported(s))
    return fail(s, CGEVAP_ERR_UNSUPPORTED,
                "the TMA kernel needs FP32 storage and >= 4 cells along periodic x and y");
  const int nvar = family == 1 ? (s->p.q == 19 ? kNumTmaVariants3D : kNumTmaVariants2D)
                               : num_tile_variants(s->p.q);
  if (variant < 0) variant = 0;
  if (variant >= nvar) return fail(s, CGEVAP_ERR_ARG, "no such kernel variant");
  if (planes_per_chunk < 0) return fail(s, CGEVAP_ERR_ARG, "planes_per_chunk < 0");
  return plan_launch(s, family, variant, planes_per_chunk);
}

int cgevap_get_tuning(const cgevap_sim* s, int* family, int* variant, int* planes_per_chunk) {
  if (!s) return CGEVAP_ERR_ARG;
  if (family) *family = s->family;
  if (variant) *variant = s->variant;
  if (planes_per_chunk) *planes_per_chunk = s->pc;
  return CGEVAP_OK;
}

double cgevap_bytes_per_update(const cgevap_sim* s) {
  if (!s) return 0.0;
  const int Q = s->Q;
  double pops;
  switch (s->p.storage) {
    case CGEVAP_F64: pops = 2.0 * 2 * Q * 8; break;
    case CGEVAP_F32:
    case CGEVAP_F32X: pops = 2.0 * 2 * Q * 4; break;
    case CGEVAP_F32RC: pops = 2.0 * (Q * 4 + 16); break;
    case CGEVAP_F16RC:
    case CGEVAP_BF16RC: pops = 2.0 * (8 + 16 + 4 + (Q - 1) * 2); break;  // rest pair, record, Rf, deviations
    default: pops = 2.0 * (8 + (Q - 1) * 4); break;
  }
  const double mask = s->p.site_rule == CGEVAP_SITES_BAND ? 1.0 : 2.0;  // read + write
  const double field = s->ph.phi_field ? (s->p.storage == CGEVAP_F64 ? 8.0 : 4.0) : 0.0;
  return pops + mask + field;
}

long long cgevap_fluid_cells(const cgevap_sim* s) { return s ? s->nfluid : 0; }

}  // extern "C"
