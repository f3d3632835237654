// lin_hash_kahan.cu -- instantiations of the per-lane hash-table linearization kernel for
// accumulation mode GLIM_ACC_KAHAN (one translation unit per mode so that they compile in parallel).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_hash_kahan(int block, int lmax) { return pick_lin_lane<GLIM_ACC_KAHAN, true>(block, lmax); }
}  // namespace glim_detail
