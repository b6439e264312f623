// Kernel instantiations for 256 x 256 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_256() { return make_kernel_set<256>(); }
cudaError_t set_attrs_256() { return set_attrs_t<256>(); }
}  // namespace ptx
