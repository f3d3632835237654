// lin_dense_kahan.cu -- instantiations of the dense-grid linearization kernel for accumulation
// mode GLIM_ACC_KAHAN (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_dense_kahan(int block, int lmax) { return pick_lin_dense<GLIM_ACC_KAHAN>(block, lmax); }
}  // namespace glim_detail
