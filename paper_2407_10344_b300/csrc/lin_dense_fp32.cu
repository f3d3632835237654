// lin_dense_fp32.cu -- instantiations of the per-lane dense-grid linearization kernel for
// accumulation mode GLIM_ACC_FP32 (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_dense_fp32(int block, int lmax) { return pick_lin_lane<GLIM_ACC_FP32, false>(block, lmax); }
}  // namespace glim_detail
