// lin_fp64.cu -- instantiations of the linearization kernel for accumulation mode GLIM_ACC_FP64
// (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernel pick_lin_fp64(int block, int ppt, int lmax) { return pick_lin<GLIM_ACC_FP64>(block, ppt, lmax); }
}  // namespace glim_detail
