// Kernel instantiations for 128 x 128 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_128() { return make_kernel_set<128>(); }
cudaError_t set_attrs_128() { return set_attrs_t<128>(); }
}  // namespace ptx
