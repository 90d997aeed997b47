// step_f64.cu -- instantiations of the fused step for ST_F64 storage.
#include "launch.h"
#include "step_kernel.cuh"

namespace cgevap {

KernelRef step_kernel_f64(int q, int variant) {
  if (q == 19) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<19, ST_F64, 32, 8, 1>, 256};
      case 1: return {(const void*)cg_step_kernel<19, ST_F64, 32, 4, 2>, 128};
      case 2: return {(const void*)cg_step_kernel<19, ST_F64, 64, 4, 1>, 256};
    }
  } else if (q == 9) {
    switch (variant) {
      case 0: return {(const void*)cg_step_kernel<9, ST_F64, 128, 1, 1>, 128};
      case 1: return {(const void*)cg_step_kernel<9, ST_F64, 64, 1, 2>, 64};
    }
  }
  return {nullptr, 0};
}

}  // namespace cgevap
