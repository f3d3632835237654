// lin_ids_hash.cu -- id-recording instantiations of the per-lane hash linearization kernel
// (inspection and parity tests of the correspondences the kernel resolves).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_ids_hash(int block, int lmax) { return pick_lin_ids_lane<2>(block, lmax); }
}  // namespace glim_detail
