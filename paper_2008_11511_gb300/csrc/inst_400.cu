// Kernel instantiations for 400 x 400 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_400() { return make_kernel_set<400>(); }
cudaError_t set_attrs_400() { return set_attrs_t<400>(); }
}  // namespace ptx
