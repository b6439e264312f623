// Kernel instantiations for 32 x 32 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_32() { return make_kernel_set<32>(); }
cudaError_t set_attrs_32() { return set_attrs_t<32>(); }
}  // namespace ptx
