// calibrate.cu -- cgevap_calibrate_threshold: the site threshold for a target S-bar, found the
// way Sec. II.B fixes it: by requiring the mass-loss rate of an evaporating flat interface to be
// the prescribed one (Eq. satisfy).  Each site removes phi / S-bar per step (Eq. relation,
// Eq. exchange) while the interface of area A should lose phi A per step, so the time-averaged
// number of sites per step must be S-bar A.  The site count of a flat interface at rest only
// takes whole layers, so the average is taken over a run in which the interface recedes.
//
// Host code only; every step runs the library's fused kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sim.h"

namespace {

// The internal handle; its last error, if any, becomes the create error (cgevap_last_error(NULL)).
struct Owned {
  cgevap_sim* s = nullptr;
  ~Owned() {
    if (!s) return;
    if (!s->err.empty()) cgevap::sim_fail(nullptr, 0, s->err);
    cgevap_destroy(s);
  }
};

// max |a - b| over n doubles (host)
double max_abs_diff(const std::vector<double>& a, const std::vector<double>& b) {
  double m = 0.0;
  for (size_t i = 0; i < a.size(); ++i) m = std::fmax(m, std::fabs(a[i] - b[i]));
  return m;
}

}  // namespace

using namespace cgevap;

extern "C" int cgevap_calibrate_threshold(const cgevap_params* p, double phi, double target_sbar,
                                          double* out_threshold, double* out_sbar) {
  if (!p || !out_threshold) return sim_fail(nullptr, CGEVAP_ERR_ARG, "NULL argument");
  if (!(phi > 0.0) || !(target_sbar > 0.0) || !std::isfinite(phi) || !std::isfinite(target_sbar))
    return sim_fail(nullptr, CGEVAP_ERR_ARG, "phi and target_sbar must be finite and > 0");
  if (p->site_rule != CGEVAP_SITES_GRADIENT && p->site_rule != CGEVAP_SITES_BAND)
    return sim_fail(nullptr, CGEVAP_ERR_ARG, "calibration needs the gradient or the band rule");
  if (p->storage != CGEVAP_F64 && p->storage != CGEVAP_F32)
    return sim_fail(nullptr, CGEVAP_ERR_UNSUPPORTED, "calibration runs with F64 or F32 storage");
  if (p->ny < 16) return sim_fail(nullptr, CGEVAP_ERR_ARG, "calibration needs ny >= 16");
  cgevap_params q = *p;
  q.sbar = target_sbar;
  Owned own;
  int rc = cgevap_create(&q, &own.s);
  if (rc != CGEVAP_OK) return rc;
  cgevap_sim* s = own.s;
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  // Flat interface normal to y: liquid (red) below y = 5 ny / 8, tanh profile of width 2.
  const long long N = s->N;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const double level = 5.0 * ny / 8.0 - 0.5;
  std::vector<double> rn(N);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) rn[((size_t)z * ny + y) * nx + x] = std::tanh((level - y) / 2.0);
  const double area = (double)nx * nz * (p->periodic[1] ? 2.0 : 1.0);
  double* d_rn = nullptr;
  double* d_u = nullptr;
  CG_CUDA(s, cudaMalloc(&d_rn, N * sizeof(double)));
  if (cudaMalloc(&d_u, 3 * N * sizeof(double)) != cudaSuccess) {
    cudaFree(d_rn);
    return sim_fail(s, CGEVAP_ERR_OOM, "cannot allocate calibration scratch");
  }
  struct Free {
    void* a;
    void* b;
    ~Free() {
      cudaFree(a);
      cudaFree(b);
    }
  } fr{d_rn, d_u};
  CG_CUDA(s, cudaMemcpy(d_rn, rn.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  rc = cgevap_set_flux(s, 0.0, nullptr, 0);
  if (rc == CGEVAP_OK) rc = cgevap_init_equilibrium(s, d_rn, nullptr, 0);
  if (rc != CGEVAP_OK) return rc;
  // Equilibrate with the flux off until u changes by less than 1e-7 over 100 steps (Sec. III).
  std::vector<double> u(3 * N), u_prev(3 * N);
  bool have_prev = false;
  for (int k = 0; k < 50; ++k) {
    rc = cgevap_step(s, 100);
    if (rc == CGEVAP_OK) rc = cgevap_get_macros(s, nullptr, nullptr, d_u, nullptr);
    if (rc != CGEVAP_OK) return rc;
    CG_CUDA(s, cudaMemcpyAsync(u.data(), d_u, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CG_CUDA(s, cudaStreamSynchronize(s->stream));
    if (have_prev && max_abs_diff(u, u_prev) < 1e-7) break;
    u_prev.swap(u);
    have_prev = true;
  }
  // Keep the equilibrated state; each trial restarts from it.
  void* eq = nullptr;
  CG_CUDA(s, cudaMalloc(&eq, s->state_bytes));
  struct Free1 {
    void* a;
    ~Free1() { cudaFree(a); }
  } fe{eq};
  CG_CUDA(s, cudaMemcpyAsync(eq, s->state[s->cur], s->state_bytes, cudaMemcpyDeviceToDevice, s->stream));
  const int cur0 = s->cur;
  // Evaporation runs to t* = 1/2: the interface recedes by half its height.
  const long long steps = std::max(200LL, (long long)std::llround(0.5 * level * p->rho_r_in / phi));
  if (steps > 2000000) return sim_fail(s, CGEVAP_ERR_ARG, "phi too small for a calibration run");
  auto sbar_at = [&](double thr, double* out) -> int {
    s->p.threshold = thr;
    s->ph.threshold = thr;
    s->cur = cur0;
    CG_CUDA(s, cudaMemcpyAsync(s->state[s->cur], eq, s->state_bytes, cudaMemcpyDeviceToDevice, s->stream));
    int r = cgevap_set_flux(s, 0.0, nullptr, 0);
    if (r != CGEVAP_OK) return r;
    // site bytes of the restart state for this threshold (gradient rule: |F| of that state)
    r = refresh_gradient_sites(s);
    if (r != CGEVAP_OK) return r;
    r = cgevap_set_flux(s, phi, nullptr, 0);
    if (r == CGEVAP_OK) r = cgevap_reset_ledger(s);
    if (r == CGEVAP_OK) r = cgevap_step(s, (int)steps);
    cgevap_ledger led;
    if (r == CGEVAP_OK) r = cgevap_get_ledger(s, &led);
    if (r != CGEVAP_OK) return r;
    *out = (double)led.site_steps / (double)steps / area;
    return CGEVAP_OK;
  };
  // Bisection: the mean site count falls with Gamma (gradient rule), rises with theta (band).
  const bool grad = p->site_rule == CGEVAP_SITES_GRADIENT;
  double lo = 0.0, hi = grad ? 1.5 : 1.0, s_lo = 0.0, s_hi = 0.0;
  rc = sbar_at(lo, &s_lo);
  if (rc == CGEVAP_OK) rc = sbar_at(hi, &s_hi);
  if (rc != CGEVAP_OK) return rc;
  const double s_min = grad ? s_hi : s_lo, s_max = grad ? s_lo : s_hi;
  if (!(target_sbar >= s_min && target_sbar <= s_max))
    return sim_fail(s, CGEVAP_ERR_ARG, "target S-bar outside what a threshold can reach (" +
                                           std::to_string(s_min) + " .. " + std::to_string(s_max) + ")");
  double best = 0.5 * (lo + hi), best_s = 0.0;
  for (int it = 0; it < 30; ++it) {
    const double mid = 0.5 * (lo + hi);
    double sm = 0.0;
    rc = sbar_at(mid, &sm);
    if (rc != CGEVAP_OK) return rc;
    best = mid;
    best_s = sm;
    const bool too_many = sm > target_sbar;
    // gradient rule: too many sites -> raise Gamma; band rule: too many -> lower theta
    if (too_many == grad) lo = mid;
    else hi = mid;
    if (hi - lo < 1e-7) break;
  }
  *out_threshold = best;
  if (out_sbar) *out_sbar = best_s;
  return CGEVAP_OK;
}
