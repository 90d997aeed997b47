// noalloc.cu -- cgevap_step_static_scratch: one fused timestep that allocates nothing.
//
// The handle API keeps the per-block ledger partials in memory it allocates with cudaMalloc.
// This entry point is for callers that must not allocate device memory at all -- a framework
// that owns every buffer and forbids allocation inside its operators (custom calls of an XLA /
// JAX program, an application arena with a fixed budget), or code that must not call into the
// allocator at step time.  They pass the state, site bytes and ledger they own; the only scratch
// the kernel needs lives in the file-scope array below, sized for kMaxBlocks CTAs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>

#include "sim.h"

using namespace cgevap;

constexpr int kMaxBlocks = 16384;  // largest grid this entry point accepts
constexpr int kMaxDevices = 64;

// Layout of the scratch: per-block partial sums of the removed mass and the site count, then the
// arrival counter of the last-block fold.
constexpr size_t kRemovedOff = 0;
constexpr size_t kSitesOff = kRemovedOff + sizeof(double) * kMaxBlocks;
constexpr size_t kDoneOff = kSitesOff + sizeof(long long) * kMaxBlocks;
constexpr size_t kScratchBytes = kDoneOff + 256;  // 256 KiB + 256 B

// The scratch, shared by every call on a device and kept until the process exits.  In host code
// `g_scratch` names a host-side stand-in, never the device memory: kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(sizeof(DevLedger) == sizeof(cgevap_ledger), "ledger layouts must match");
static_assert(offsetof(cgevap_ledger, steps) == offsetof(DevLedger, steps), "ledger layouts");

namespace {

// Per device: the scratch's device address and the CUDA context it was resolved in.  A device
// reset (cudaDeviceReset) replaces the primary context and with it the address, so the address is
// resolved again whenever the current context differs from the recorded one.
struct ScratchAddr {
  CUcontext ctx = nullptr;
  unsigned char* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

int fail(int code, const std::string& msg) { return cgevap::sim_fail(nullptr, code, msg); }

// The current context (driver API, through the runtime's entry-point query; nullptr on failure).
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 get = nullptr;
  if (!get) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &qr) !=
            cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  }
  CUcontext c = nullptr;
  return get(&c) == CUDA_SUCCESS ? c : nullptr;
}

// Resolve the device address of g_scratch for the current device, once per device and context.
int scratch_on(int device, unsigned char** out) {
  const CUcontext ctx = current_context();
  if (!ctx) return fail(CGEVAP_ERR_CUDA, "static-scratch step: no current CUDA context");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchAddr& e = g_scratch_addr[device];
  if (!e.addr || e.ctx != ctx) {
    void* addr = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&addr, g_scratch);
    if (rc != cudaSuccess || !addr)
      return fail(CGEVAP_ERR_CUDA, std::string("static-scratch step: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(rc));
    e.addr = static_cast<unsigned char*>(addr);
    e.ctx = ctx;
  }
  *out = e.addr;
  return CGEVAP_OK;
}

bool params_ok(const cgevap_params* p) {
  if (!p) return false;
  if (p->q != 9 && p->q != 19) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  if (p->q == 9 && p->nz != 1) return false;
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return false;
  for (int d = 0; d < 3; ++d)
    if (p->periodic[d] != 0 && p->periodic[d] != 1) return false;
  if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5)) return false;
  if (!(p->rho_r_in > 0.0) || !(p->rho_b_in > 0.0)) return false;
  if (!(p->beta >= 0.0 && p->beta <= 1.0)) return false;
  if (!(p->sbar > 0.0)) return false;
  if (!std::isfinite(p->sigma) || !std::isfinite(p->threshold)) return false;
  if (p->site_rule != CGEVAP_SITES_GRADIENT && p->site_rule != CGEVAP_SITES_BAND) return false;
  if (p->storage < CGEVAP_F64 || p->storage > CGEVAP_BF16DEV) return false;
  return true;
}

template <int Q>
void kappa_of(Physics& ph) {
  using L = Lattice<Q>;
  for (int i = 0; i < 19; ++i) {
    ph.kap_r[i] = ph.kap_b[i] = 0.0f;
    if (i < Q) {
      ph.kap_r[i] = (float)((L::A(i) + L::B(i) * ph.alpha_r) / ph.alpha_r);
      ph.kap_b[i] = (float)((L::A(i) + L::B(i) * ph.alpha_b) / ph.alpha_b);
    }
  }
}

}  // namespace

extern "C" CGEVAP_API int cgevap_step_static_scratch(
    const cgevap_params* p, double phi, const void* dev_state_in, void* dev_state_out,
    size_t state_bytes_in, const uint8_t* dev_mask_in, uint8_t* dev_mask_out,
    cgevap_ledger* dev_ledger, void* cuda_stream) {
  if (!params_ok(p) || !std::isfinite(phi))
    return fail(CGEVAP_ERR_ARG, "static-scratch step: invalid parameters or non-finite phi");
  if (!dev_state_in || !dev_state_out || dev_state_in == dev_state_out || !dev_mask_in ||
      !dev_mask_out || !dev_ledger)
    return fail(CGEVAP_ERR_ARG, "static-scratch step: NULL or aliasing buffers");
  const long long N = (long long)p->nx * p->ny * p->nz;
  const StoreShape sh = store_shape(p->q, p->nx, p->ny, p->nz);
  if ((long long)p->q * sh.nstore >= (1LL << 31))
    return fail(CGEVAP_ERR_ARG, "static-scratch step: lattice too large for 32-bit storage indices");
  const size_t want = state_bytes(internal_storage(p->storage), p->q, sh.nstore);
  if (state_bytes_in != want)
    return fail(CGEVAP_ERR_ARG, "static-scratch step: state_bytes is " + std::to_string(state_bytes_in) +
                                    ", the layout needs " + std::to_string(want));
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return fail(CGEVAP_ERR_CUDA, "static-scratch step: no device");
  if (device < 0 || device >= kMaxDevices)
    return fail(CGEVAP_ERR_UNSUPPORTED, "static-scratch step: device ordinal beyond 63");
  unsigned char* scratch = nullptr;
  const int src = scratch_on(device, &scratch);
  if (src != CGEVAP_OK) return src;

  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  Geom& g = a.g;
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
  g.ncell = (int)N;
  g.links = nullptr;
  g.gy = p->q == 19 ? 2 : 0;
  g.pitch = sh.pitch;
  g.rows = sh.rows;
  g.nstore = (int)sh.nstore;
  g.img_a = 0;  // the register kernel keeps no ghost images
  g.img_b = 0;

  Physics& ph = a.ph;
  const double w0 = p->q == 19 ? Lattice<19>::W(0) : Lattice<9>::W(0);
  const double rmin = std::fmin(p->rho_r_in, p->rho_b_in);
  ph.alpha_r = (p->rho_r_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p->rho_r_in / rmin);
  ph.alpha_b = (p->rho_b_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p->rho_b_in / rmin);
  ph.inv_tau_r = 1.0 / p->tau_r;
  ph.inv_tau_b = 1.0 / p->tau_b;
  ph.amp = 2.25 * p->sigma;
  ph.beta = p->beta;
  ph.rule = p->site_rule;
  ph.threshold = p->threshold;
  ph.inv_sbar = 1.0 / p->sbar;
  ph.varphi = phi / p->sbar;
  ph.phi_field = nullptr;
  mirror_floats(ph);
  if (p->q == 19)
    kappa_of<19>(ph);
  else
    kappa_of<9>(ph);
  if (p->storage == CGEVAP_F16DEV) {
    const double rmax = std::fmax(p->rho_r_in, p->rho_b_in);
    int e = (int)std::floor(std::log2(16384.0 / rmax));
    e = e > 10 ? 10 : (e < 0 ? 0 : e);
    ph.scale = std::ldexp(1.0f, e);
  } else {
    ph.scale = 1.0f;
  }
  ph.inv_scale = 1.0f / ph.scale;
  ph.sum_base = sum_base_for(p->rho_r_in, p->rho_b_in);

  KernelRef k = p->storage == CGEVAP_F64   ? step_kernel_f64(p->q, 0)
                : p->storage == CGEVAP_F32 ? step_kernel_f32(p->q, 0)
                                           : step_kernel_dev(p->q, internal_storage(p->storage), 0);
  if (!k.fn) return fail(CGEVAP_ERR_UNSUPPORTED, "static-scratch step: no kernel for this storage");
  int occ = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.threads, k.smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return fail(CGEVAP_ERR_CUDA, "static-scratch step: occupancy query failed");
  if (occ < 1) occ = 1;
  TileCfg t = tile_cfg(p->q, 0);
  if (k.tx > 0) t = TileCfg{k.tx, k.ty};
  const int ntx = (g.na + t.tx - 1) / t.tx;
  const int nty = (g.nb + t.ty - 1) / t.ty;
  const long long tiles = (long long)ntx * nty;
  const long long slots = (long long)occ * sms;
  int best_pc = g.nm;
  double best = 1e300;
  for (int pc = 1; pc <= g.nm; ++pc) {
    const long long nchunk = (g.nm + pc - 1) / pc;
    if (nchunk > 65535 || tiles * nchunk > kMaxBlocks) continue;
    const double waves = std::ceil((double)(tiles * nchunk) / (double)slots);
    const double cost = waves * (pc + 2);
    if (cost < best - 1e-9) {
      best = cost;
      best_pc = pc;
    }
  }
  const long long nchunk = (g.nm + best_pc - 1) / best_pc;
  if (tiles * nchunk > kMaxBlocks)  // lattice too large for the scratch
    return fail(CGEVAP_ERR_ARG, "static-scratch step: the grid needs " + std::to_string(tiles * nchunk) +
                                    " CTAs, more than the 16384 the static scratch holds");

  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned int* done = reinterpret_cast<unsigned int*>(scratch + kDoneOff);
  if (cudaMemsetAsync(done, 0, sizeof(unsigned int), stream) != cudaSuccess)
    return fail(CGEVAP_ERR_CUDA, "static-scratch step: clearing the arrival counter failed");
  a.red.part_removed = reinterpret_cast<double*>(scratch + kRemovedOff);
  a.red.part_sites = reinterpret_cast<long long*>(scratch + kSitesOff);
  a.red.done = done;
  a.red.ledger = reinterpret_cast<DevLedger*>(dev_ledger);
  a.ntx = ntx;
  a.nty = nty;
  a.pc = best_pc;
  a.pin = dev_state_in;
  a.pout = dev_state_out;
  a.mask_in = dev_mask_in;
  a.mask_out = dev_mask_out;
  void* args[] = {&a};
  const cudaError_t lrc = cudaLaunchKernel(k.fn, dim3((unsigned)tiles, (unsigned)nchunk),
                                           dim3(k.threads), args, k.smem, stream);
  if (lrc != cudaSuccess)
    return fail(CGEVAP_ERR_CUDA, std::string("static-scratch step: launch: ") + cudaGetErrorString(lrc));
  return CGEVAP_OK;
}
