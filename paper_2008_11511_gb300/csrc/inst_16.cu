// Kernel instantiations for 16 x 16 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_16() { return make_kernel_set<16>(); }
cudaError_t set_attrs_16() { return set_attrs_t<16>(); }
}  // namespace ptx
