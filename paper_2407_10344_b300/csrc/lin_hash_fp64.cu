// lin_hash_fp64.cu -- instantiations of the per-lane hash-table linearization kernel for
// accumulation mode GLIM_ACC_FP64 (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_hash_fp64(int block, int lmax) { return pick_lin_lane<GLIM_ACC_FP64, true>(block, lmax); }
}  // namespace glim_detail
