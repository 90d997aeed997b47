// adjoint.cu -- host side of the adjoint entry points and of cgevap_volume: the checkpoint tape,
// segment recomputation and the reverse sweep (kernels in adjoint_kernels.cu).
//
// Memory: the forward run stores the state and the site bytes at every step t = 0, K, 2K, ...
// (ceil(T/K) checkpoints).  The backward sweep walks the segments from the last; for each it
// recomputes the segment's states from its checkpoint into K slots, with the step kernel of the
// forward run (bitwise the same states and site decisions), then runs the adjoint steps of the
// segment from its last step down to its first.  Every step is thus computed twice and the
// device holds ceil(T/K) + K states, plus two adjoint fields of one state each (the pushed lg
// parts of lambda^{n+1} and lambda^n) and one vec2 per cell (their ab part).
#include <cmath>
#include <cstring>
#include <new>

#include "sim.h"

namespace cgevap {

struct AdjointTape {
  int T = 0, K = 0, nseg = 0;
  size_t sb = 0;      // state bytes
  long long N = 0;    // cells
  char* ckpt = nullptr;            // nseg states
  uint8_t* ckpt_mask = nullptr;    // nseg site arrays (the mask read by the segment's first step)
  char* seg = nullptr;             // K states: slot k = state after step k of the segment
  uint8_t* seg_mask = nullptr;     // K site arrays: slot k written by step k of the segment
  char* lam = nullptr;             // 2 states: the lg parts of lambda^{n+1} and lambda^n
  void* aux = nullptr;             // kAdjAuxPlanes planes
  void* ab = nullptr;              // nstore vec2: the ab part of lambda^{n+1} (then of lambda^n)
  DevLedger* led = nullptr;        // ledger of the recomputed steps (discarded)
  // plan of the forward run, checked by the backward sweep
  int family = -1, variant = -1, pc = 0;
  const void* fwd_fn = nullptr;
  // plan of kernel A
  KernelRef adj{nullptr, 0};
  int ntx = 1, nty = 1, apc = 1, anchunk = 1;
  bool recorded = false;
};

namespace {

void free_tape(AdjointTape* t) {
  if (!t) return;
  void* ptrs[] = {t->ckpt, t->ckpt_mask, t->seg, t->seg_mask, t->lam, t->aux, t->ab, t->led};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete t;
}

int volume_into(cgevap_sim* s, const void* state, double* out) {
  if (!s->vol_part) {
    if (cudaMalloc(&s->vol_part, kVolumeBlocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->vol_done, sizeof(unsigned int)) != cudaSuccess)
      return sim_fail(s, CGEVAP_ERR_OOM, "cannot allocate the volume scratch");
    CG_CUDA(s, cudaMemsetAsync(s->vol_done, 0, sizeof(unsigned int), s->stream));
  }
  CG_CUDA(s, launch_volume(aux_of(s), state, s->vol_part, s->vol_done, out, s->stream));
  return CGEVAP_OK;
}

// Launch one fused step of the current plan on explicit buffers (recomputation).
int launch_step_on(cgevap_sim* s, const void* pin, void* pout, const uint8_t* mask_in,
                   uint8_t* mask_out, DevLedger* ledger) {
  StepArgs a = step_args(s);
  a.pin = pin;
  a.pout = pout;
  a.mask_in = mask_in;
  a.mask_out = mask_out;
  a.red.ledger = ledger;
  void* args[] = {&a};
  CG_CUDA(s, cudaLaunchKernel(s->kernel.fn, dim3(s->ntx * s->nty, s->nchunk),
                              dim3(s->kernel.threads), args, s->kernel.smem, s->stream));
  return CGEVAP_OK;
}

// Kernel A's grid: the step's tiles, planes per chunk chosen as the step planner does
// (whole waves of resident CTAs against the two extra planes each chunk pulls).
int plan_adjoint(cgevap_sim* s, AdjointTape* t) {
  t->adj = adjoint_local_kernel(s->p.q, s->p.storage);
  if (!t->adj.fn) return sim_fail(s, CGEVAP_ERR_UNSUPPORTED, "no adjoint kernel for this configuration");
  int occ = 0, sms = 0;
  CG_CUDA(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, t->adj.fn, t->adj.threads, t->adj.smem));
  CG_CUDA(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  if (occ < 1) occ = 1;
  const Geom& g = s->geom;
  t->ntx = (g.na + t->adj.tx - 1) / t->adj.tx;
  t->nty = (g.nb + t->adj.ty - 1) / t->adj.ty;
  const long long tiles = (long long)t->ntx * t->nty;
  const long long slots = (long long)occ * sms;
  int best_pc = g.nm;
  double best = 1e300;
  for (int pc = 1; pc <= g.nm; ++pc) {
    const long long nchunk = (g.nm + pc - 1) / pc;
    if (nchunk > 65535) continue;
    const double waves = std::ceil((double)(tiles * nchunk) / (double)slots);
    const double cost = waves * (pc + 2);
    if (cost < best - 1e-9) {
      best = cost;
      best_pc = pc;
    }
  }
  t->apc = best_pc;
  t->anchunk = (g.nm + best_pc - 1) / best_pc;
  return CGEVAP_OK;
}

template <class T>
bool dev_alloc(T*& p, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) return false;
  p = reinterpret_cast<T*>(q);
  return true;
}

int make_tape(cgevap_sim* s, int T, int K) {
  AdjointTape* t = s->tape;
  const int nseg = (T + K - 1) / K;
  if (t && t->T == T && t->K == K) return CGEVAP_OK;  // same shape: reuse the buffers
  free_tape(t);
  s->tape = nullptr;
  t = new (std::nothrow) AdjointTape();
  if (!t) return sim_fail(s, CGEVAP_ERR_OOM, "host allocation failed");
  t->T = T;
  t->K = K;
  t->nseg = nseg;
  t->sb = s->state_bytes;
  t->N = s->N;
  const size_t real = s->p.storage == CGEVAP_F64 ? 8 : 4;
  const size_t ns = (size_t)s->geom.nstore;
  const bool ok = dev_alloc(t->ckpt, (size_t)nseg * t->sb) &&
                  dev_alloc(t->ckpt_mask, (size_t)nseg * t->N) &&
                  dev_alloc(t->seg, (size_t)K * t->sb) && dev_alloc(t->seg_mask, (size_t)K * t->N) &&
                  dev_alloc(t->lam, 2 * t->sb) &&
                  dev_alloc(t->aux, kAdjAuxPlanes * ns * real) && dev_alloc(t->ab, 2 * ns * real) &&
                  dev_alloc(t->led, sizeof(DevLedger));
  if (!ok) {
    free_tape(t);
    cudaGetLastError();
    return sim_fail(s, CGEVAP_ERR_OOM, "cannot allocate the adjoint tape (" +
                                           std::to_string(nseg + K + 2) + " states of " +
                                           std::to_string(s->state_bytes) + " bytes)");
  }
  s->tape = t;
  return plan_adjoint(s, t);
}

}  // namespace

void adjoint_release(cgevap_sim* s) {
  if (!s) return;
  free_tape(s->tape);
  s->tape = nullptr;
}

}  // namespace cgevap

using namespace cgevap;

extern "C" {

int cgevap_volume(cgevap_sim* s, double* dev_out) {
  if (!s || !dev_out) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  return volume_into(s, s->state[s->cur], dev_out);
}

int cgevap_adjoint_forward(cgevap_sim* s, int nsteps, int ckpt_every, double* dev_volume) {
  if (!s) return CGEVAP_ERR_ARG;
  if (nsteps < 1 || ckpt_every < 1) return sim_fail(s, CGEVAP_ERR_ARG, "nsteps and ckpt_every must be >= 1");
  if (s->p.storage != CGEVAP_F64 && s->p.storage != CGEVAP_F32)
    return sim_fail(s, CGEVAP_ERR_UNSUPPORTED, "the adjoint needs F64 or F32 storage");
  if (s->family != 0)
    return sim_fail(s, CGEVAP_ERR_UNSUPPORTED, "the adjoint needs the register-pipelined step (cgevap_tune family 0)");
  if (s->outlet_rho[0] > 0.0 || s->outlet_rho[1] > 0.0)
    return sim_fail(s, CGEVAP_ERR_UNSUPPORTED, "the adjoint does not differentiate the outlets (cgevap_set_outlets)");
  if (s->heat.on)
    return sim_fail(s, CGEVAP_ERR_UNSUPPORTED, "the adjoint needs a flux that does not depend on the state (heated flux set)");
  CG_CUDA(s, cudaSetDevice(s->device));
  const int K = ckpt_every < nsteps ? ckpt_every : nsteps;
  int rc = make_tape(s, nsteps, K);
  if (rc != CGEVAP_OK) return rc;
  AdjointTape* t = s->tape;
  t->recorded = false;
  if (dev_volume) {
    rc = volume_into(s, s->state[s->cur], dev_volume);
    if (rc != CGEVAP_OK) return rc;
  }
  for (int step = 0; step < nsteps; ++step) {
    if (step % K == 0) {
      const int k = step / K;
      CG_CUDA(s, cudaMemcpyAsync(t->ckpt + (size_t)k * t->sb, s->state[s->cur], t->sb,
                                 cudaMemcpyDeviceToDevice, s->stream));
      CG_CUDA(s, cudaMemcpyAsync(t->ckpt_mask + (size_t)k * t->N, s->mask[s->cur], t->N,
                                 cudaMemcpyDeviceToDevice, s->stream));
    }
    rc = cgevap_step(s, 1);
    if (rc != CGEVAP_OK) return rc;
    if (dev_volume) {
      rc = volume_into(s, s->state[s->cur], dev_volume + step + 1);
      if (rc != CGEVAP_OK) return rc;
    }
  }
  t->family = s->family;
  t->variant = s->variant;
  t->pc = s->pc;
  t->fwd_fn = s->kernel.fn;
  t->recorded = true;
  return CGEVAP_OK;
}

int cgevap_adjoint_backward(cgevap_sim* s, const double* dev_dL_dV, double* dev_dL_dphi) {
  if (!s || !dev_dL_dphi) return CGEVAP_ERR_ARG;
  AdjointTape* t = s->tape;
  if (!t || !t->recorded) return sim_fail(s, CGEVAP_ERR_ARG, "no recorded forward run");
  if (t->family != s->family || t->variant != s->variant || t->pc != s->pc || t->fwd_fn != s->kernel.fn)
    return sim_fail(s, CGEVAP_ERR_ARG, "the step's tuning changed since cgevap_adjoint_forward");
  CG_CUDA(s, cudaSetDevice(s->device));
  cudaStream_t st = s->stream;
  const AuxArgs ax = aux_of(s);
  CG_CUDA(s, cudaMemsetAsync(dev_dL_dphi, 0, (size_t)t->N * sizeof(double), st));
  CG_CUDA(s, cudaMemsetAsync(t->lam, 0, t->sb, st));  // lambda^T = 0: its lg part ...
  CG_CUDA(s, cudaMemsetAsync(t->ab, 0, 2 * (size_t)s->geom.nstore * (s->p.storage == CGEVAP_F64 ? 8 : 4), st));  // ... and its ab part
  int lc = 0;                                             // lambda^{n+1} lives in slot lc
  const double inv_sbar = 1.0 / s->p.sbar;
  for (int sg = t->nseg - 1; sg >= 0; --sg) {
    const int t0 = sg * t->K;
    const int len = (t->T - t0) < t->K ? (t->T - t0) : t->K;
    const char* c0 = t->ckpt + (size_t)sg * t->sb;
    const uint8_t* m0 = t->ckpt_mask + (size_t)sg * t->N;
    // recompute the segment: states after steps t0 .. t0+len-1 and their site bytes
    for (int k = 0; k < len; ++k) {
      const void* pin = k == 0 ? (const void*)c0 : (const void*)(t->seg + (size_t)(k - 1) * t->sb);
      const uint8_t* min = k == 0 ? m0 : t->seg_mask + (size_t)(k - 1) * t->N;
      int rc = launch_step_on(s, pin, t->seg + (size_t)k * t->sb, min,
                              t->seg_mask + (size_t)k * t->N, t->led);
      if (rc != CGEVAP_OK) return rc;
    }
    // adjoint steps t0+len-1 .. t0
    for (int k = len - 1; k >= 0; --k) {
      const int n = t0 + k;
      const void* fn = k == 0 ? (const void*)c0 : (const void*)(t->seg + (size_t)(k - 1) * t->sb);
      const uint8_t* mn = t->seg_mask + (size_t)k * t->N;  // bit 0: the sites of step n
      StepArgs a = step_args(s);
      a.ph.rule = 2;  // the recorded site set, held fixed
      a.pin = fn;
      a.pout = nullptr;
      a.mask_in = mn;
      a.mask_out = nullptr;
      a.red.ledger = nullptr;
      a.ntx = t->ntx;
      a.nty = t->nty;
      a.pc = t->apc;
      AdjointOut o;
      o.lam_in = t->lam + (size_t)lc * t->sb;
      o.ab = t->ab;
      o.lam_g = t->lam + (size_t)(lc ^ 1) * t->sb;
      o.aux = t->aux;
      void* args[] = {&a, &o};
      CG_CUDA(s, cudaLaunchKernel(t->adj.fn, dim3(t->ntx * t->nty, t->anchunk),
                                  dim3(t->adj.threads), args, t->adj.smem, st));
      // B1 reads the ab part of lambda^{n+1} no more (kernel A has): it writes lambda^n's
      CG_CUDA(s, launch_adjoint_stencil(ax, t->aux, o.lam_g, t->ab, mn, dev_dL_dphi, inv_sbar,
                                        dev_dL_dV ? dev_dL_dV + n + 1 : nullptr, st));
      lc ^= 1;
    }
  }
  return CGEVAP_OK;
}

int cgevap_adjoint_run(cgevap_sim* s, int nsteps, int ckpt_every, const double* dev_dL_dV,
                       double* dev_dL_dphi) {
  int rc = cgevap_adjoint_forward(s, nsteps, ckpt_every, nullptr);
  if (rc != CGEVAP_OK) return rc;
  return cgevap_adjoint_backward(s, dev_dL_dV, dev_dL_dphi);
}

int cgevap_adjoint_release(cgevap_sim* s) {
  if (!s) return CGEVAP_ERR_ARG;
  CG_CUDA(s, cudaSetDevice(s->device));
  CG_CUDA(s, cudaStreamSynchronize(s->stream));
  adjoint_release(s);
  return CGEVAP_OK;
}

}  // extern "C"
