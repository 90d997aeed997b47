// sim.h -- the simulation handle behind include/cgevap.h and the library-internal helpers that
// the entry points in api.cu and adjoint.cu share.  Not installed, not part of the ABI.
#pragma once

#include <string>

#include "../../include/cgevap.h"
#include "launch.h"

namespace cgevap {
struct AdjointTape;
}

struct cgevap_sim {
  cgevap_params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  int Q = 0;
  long long N = 0;
  long long nfluid = 0;
  cgevap::Geom geom{};
  cgevap::Physics ph{};
  size_t state_bytes = 0;
  void* state[2] = {nullptr, nullptr};
  uint8_t* mask[2] = {nullptr, nullptr};
  int cur = 0;
  uint32_t* links = nullptr;
  uint8_t* solid = nullptr;
  void* phi_field = nullptr;  // double (F64 storage) or float, [N]
  double phi = 0.0;
  cgevap::DevLedger* ledger = nullptr;
  double* part_removed = nullptr;
  long long* part_sites = nullptr;
  unsigned int* done = nullptr;
  long long part_capacity = 0;
  double* tmp_rn = nullptr;
  int* flag = nullptr;
  int* status = nullptr;  // set by a bounded device-side wait that gave up
  void* staging = nullptr;  // device staging for host imports
  size_t staging_bytes = 0;
  // launch plan of the fused step
  int family = 0;  // 0 register-pipelined kernel, 1 TMA-pipelined kernel
  int variant = 0;
  cgevap::KernelRef kernel{nullptr, 0};
  cgevap::KernelRef kernel_in{nullptr, 0};  // F32RC: the same step reading FP32 pairs
  int rc_pairs = 1;  // F32RC: state[cur] holds FP32 pairs (created or imported, not yet stepped)
  alignas(64) unsigned char tmap[2][128];  // TMA tensor maps of state[0] and state[1]
  int ntx = 1, nty = 1, pc = 1, nchunk = 1;
  cgevap::AdjointTape* tape = nullptr;  // checkpoints of cgevap_adjoint_forward (adjoint.cu)
  double* vol_part = nullptr;           // cgevap_volume scratch: kVolumeBlocks partials
  unsigned int* vol_done = nullptr;     // and its arrival counter
  // heated-substrate flux (cgevap_set_flux_heated): phi_field is recomputed from the state before
  // a step once `since` reaches `every`; part holds the column partials of launch_heated_flux
  struct Heated {
    int on = 0;
    double phi_s = 0.0, K = 1.0, length = 1.0;
    int every = 1, since = 0;
    double* part = nullptr;
  } heat;
  double outlet_rho[2] = {0.0, 0.0};  // blue pressure outlets (cgevap_set_outlets); <= 0: wall
  std::string err;
};

namespace cgevap {
// Records msg as the handle's last error (or the create error) and returns code.
int sim_fail(cgevap_sim* s, int code, const std::string& msg);
AuxArgs aux_of(const cgevap_sim* s);
// Internal storage code (ST_*) of an API storage code (CGEVAP_*; -1 if unknown).
int internal_storage(int api_storage);
// True for the layouts that hold colour-blind populations and a recolouring record per cell.
bool is_recolour_on_pull(int api_storage);
// Arguments of one fused step of the current plan, reading state[cur] and writing state[cur^1].
StepArgs step_args(cgevap_sim* s);
// Site bytes read by the next step, recomputed from the current state: under the gradient rule
// bit 1 = |F| of the state > threshold (the "previous step" decision before a first step), else 0.
int refresh_gradient_sites(cgevap_sim* s);
// Adjoint tape release (adjoint.cu), called when the handle is destroyed.
void adjoint_release(cgevap_sim* s);
// View of a simulation for the ensemble driver (ensemble.cu): geometry, physics with its FP32
// mirrors, the state and site buffers, the ledger and where the current buffer index lives.
struct SimView {
  Geom g;
  Physics ph;
  void* state[2];
  uint8_t* mask[2];
  DevLedger* ledger;
  int* cur;
  cudaStream_t* stream;
  size_t state_bytes;
  long long ncell;
};
int sim_view(cgevap_sim* s, SimView* v);
}  // namespace cgevap

#define CG_CUDA(s, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return ::cgevap::sim_fail((s), CGEVAP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
