// lin_ids_general.cu -- id-recording instantiations of the general linearization kernel
// (inspection and parity tests of the correspondences the kernel resolves).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_ids_general(int block, int lmax) { return pick_lin_ids_lane<0>(block, lmax); }
}  // namespace glim_detail
