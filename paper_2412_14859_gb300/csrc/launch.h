// launch.h -- host-side launchers of the CUDA kernels (implemented in the .cu files).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace cgevap {

// Tile shapes of the fused step, chosen per lattice by the launch planner / autotuner.
struct TileCfg {
  int tx, ty;
};
constexpr int kNumTiles3D = 5;
constexpr TileCfg kTiles3D[kNumTiles3D] = {{32, 4}, {16, 8}, {16, 16}, {16, 4}, {32, 8}};
constexpr int kNumTiles2D = 2;
constexpr TileCfg kTiles2D[kNumTiles2D] = {{128, 1}, {64, 1}};

inline TileCfg tile_cfg(int q, int variant) {
  return q == 19 ? kTiles3D[variant % kNumTiles3D] : kTiles2D[variant % kNumTiles2D];
}
inline int num_tile_variants(int q) { return q == 19 ? kNumTiles3D : kNumTiles2D; }

// Fused step kernels (step_f64.cu, step_f32.cu, step_dev.cu): the __global__ function of a
// (lattice, storage, tile variant), launched with `threads` threads and one StepArgs argument.
struct KernelRef {
  const void* fn;
  int threads;
  int smem = 0;       // dynamic shared memory bytes
  int tx = 0, ty = 0; // tile shape (0: take it from tile_cfg)
  int needs_map = 0;  // 1: second kernel argument is the TMA tensor map of the input state
};
KernelRef step_kernel_f64(int q, int variant);
KernelRef step_kernel_f32(int q, int variant);
KernelRef step_kernel_f32x(int q, int variant);  // FP32 pairs, exact colour masses (step_f32.cu)
KernelRef step_kernel_dev(int q, int storage, int variant);
// Recolour-on-pull layout (step_rc.cu); pairs_in: the input state holds FP32 pairs (import).
KernelRef step_kernel_rc(int q, int variant, bool pairs_in);
// 16-bit recolour-on-pull layouts (step_rc16.cu); storage is ST_H16RC or ST_B16RC.
KernelRef step_kernel_rc16(int q, int storage, int variant, bool pairs_in);
// TMA-pipelined step (step_tma_f32.cu): FP32 storage; periodic axes need >= 4 cells.
constexpr int kNumTmaVariants3D = 2;
constexpr int kNumTmaVariants2D = 2;
KernelRef step_tma_f32(int q, int variant);
// TMA tensor map (128-byte CUtensorMap written to `map`) of one population buffer: elements of
// elem_bytes, box of box_w x box_h (x, rows) per direction and plane.  Returns 0 on success.
int make_pop_tensor_map(void* map, const void* base, const Geom& g, int q, int elem_bytes,
                        int box_w, int box_h);

// Auxiliary kernels (aux_kernels.cu).
struct AuxArgs {
  Geom g;
  Physics ph;
  int q, storage;
  double rho_r_in, rho_b_in;
};
cudaError_t launch_init_equilibrium(const AuxArgs& a, const double* rhoN0, const void* noise,
                                    int noise_dtype, void* state, cudaStream_t s);
cudaError_t launch_set_populations(const AuxArgs& a, const void* in, int dtype, void* state,
                                   cudaStream_t s);
cudaError_t launch_get_populations(const AuxArgs& a, const void* state, void* out, int dtype,
                                   cudaStream_t s);
cudaError_t launch_macros(const AuxArgs& a, const void* state, double* rho_r, double* rho_b,
                          double* u, double* rhoN, cudaStream_t s);
cudaError_t launch_gradient_sites(const AuxArgs& a, const void* state, double* tmp_rn,
                                  uint8_t* mask, cudaStream_t s);
cudaError_t launch_links(const AuxArgs& a, const uint8_t* solid, uint32_t* links,
                         cudaStream_t s);
cudaError_t launch_zero_solid(const AuxArgs& a, void* state, cudaStream_t s);
cudaError_t launch_health(const AuxArgs& a, const void* state, int* flag, cudaStream_t s);
cudaError_t launch_fill_ghosts(const AuxArgs& a, void* state, cudaStream_t s);
cudaError_t launch_convert_field(const void* in, int in_dtype, void* out, int out_is_double,
                                 long long n, cudaStream_t s);
cudaError_t launch_fill(double* out, double v, long long n, cudaStream_t s);
// Blue pressure outlets (aux_kernels.cu; Sec. III.B.2) on the first / last plane of the march
// axis, prescribed blue density rho_lo / rho_hi (<= 0: wall), written into state before a step.
cudaError_t launch_outlets(const AuxArgs& a, void* state, double rho_lo, double rho_hi, cudaStream_t s);

// Heated-substrate flux field (aux_kernels.cu; Sec. III.C, Eq. heated): every cell of a column
// along the march axis (the wall normal) takes phi_s / (K + h / length), h = the column's summed
// liquid fraction.  `part` holds (heated_plan(g).nchunk + 1) * na * nb doubles; field is double
// (field_double = 1) or float, [N].
struct HeatedPlan {
  int col_blocks = 1, cz = 1, nchunk = 1;
};
HeatedPlan heated_plan(const Geom& g);
cudaError_t launch_heated_flux(const AuxArgs& a, const void* state, double* part, double phi_s,
                               double K, double length, void* field, int field_double, cudaStream_t s);

// Adjoint sweep (adjoint_kernels.cu).  The local kernel (kernel A) takes (StepArgs, AdjointOut)
// and runs on the step's tile grid; F64 / F32 storage only.
// Auxiliary per-cell fields of the sweep, planes of nstore reals in the storage layout:
// dL/dF_a, dL/dF_b, dL/dF_m, d rho^N/d rho_r, d rho^N/d rho_b.
constexpr int kAdjAuxPlanes = 5;
struct AdjointOut {
  const void* lam_in;  // the lg part of lambda^{n+1} = dL/df^{n+1}, pushed by the previous
                       // adjoint step (state layout: vec2 per direction and storage index)
  const void* ab;      // the ab part of lambda^{n+1}: nstore vec2 from kernel B1 of that step
  void* lam_g;         // out: the lg part of lambda^n, pushed to where the pull of step n read
  void* aux;           // out: kAdjAuxPlanes planes
};
KernelRef adjoint_local_kernel(int q, int storage);
// Kernel B1: stencil transpose, exchange derivative into dphi (FP64, compact [N]); aux holds
// kAdjAuxPlanes planes of nstore reals; lam_g is kernel A's pushed output (its rest slot of a
// cell is that cell's own lg_0); ab receives nstore vec2.  dLdV may be nullptr.
cudaError_t launch_adjoint_stencil(const AuxArgs& a, const void* aux, const void* lam_g, void* ab,
                                   const uint8_t* mask, double* dphi, double inv_sbar,
                                   const double* dLdV, cudaStream_t s);
// Liquid volume of a state into *out (FP64); part holds kVolumeBlocks doubles, *done starts at 0.
constexpr int kVolumeBlocks = 152 * 16;  // 16 CTAs of 256 threads per SM: loads in flight
cudaError_t launch_volume(const AuxArgs& a, const void* state, double* part, unsigned int* done,
                          double* out, cudaStream_t s);

}  // namespace cgevap
