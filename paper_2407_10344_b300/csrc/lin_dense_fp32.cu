// lin_dense_fp32.cu -- instantiations of the dense-grid linearization kernel for accumulation
// mode GLIM_ACC_FP32 (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_dense_fp32(int block, int lmax) { return pick_lin_dense<GLIM_ACC_FP32>(block, lmax); }
}  // namespace glim_detail
