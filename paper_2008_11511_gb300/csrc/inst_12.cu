// Kernel instantiations for 12 x 12 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_12() { return make_kernel_set<12>(); }
cudaError_t set_attrs_12() { return set_attrs_t<12>(); }
}  // namespace ptx
