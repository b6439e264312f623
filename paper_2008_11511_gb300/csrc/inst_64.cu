// Kernel instantiations for 64 x 64 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_64() { return make_kernel_set<64>(); }
cudaError_t set_attrs_64() { return set_attrs_t<64>(); }
}  // namespace ptx
