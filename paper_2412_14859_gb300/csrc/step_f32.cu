// step_f32.cu -- instantiations of the fused step for ST_F32 storage.
#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

KernelRef step_kernel_f32(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<19, ST_F32, 32, 8, 2>, 256};
      case 1: return {(const void*)cg_step_kernel<19, ST_F32, 32, 4, 4>, 128};
      case 2: return {(const void*)cg_step_kernel<19, ST_F32, 64, 4, 2>, 256};
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<9, ST_F32, 128, 1, 4>, 128};
      case 1: return {(const void*)cg_step_kernel<9, ST_F32, 64, 1, 8>, 64};
    }
  }
  return {nullptr, 0};
}

}  // namespace cgevap
