// lin_ids_dense.cu -- id-recording instantiations of the per-lane dense-grid linearization kernel
// (inspection and parity tests of the correspondences the kernel resolves).
#include "lin_kernel.cuh"

namespace glim_detail {
LinKernelInfo pick_lin_ids_dense(int block, int lmax) { return pick_lin_ids_lane<1>(block, lmax); }
}  // namespace glim_detail
