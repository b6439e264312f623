// Kernel instantiations for 448 x 448 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_448() { return make_kernel_set<448>(); }
cudaError_t set_attrs_448() { return set_attrs_t<448>(); }
}  // namespace ptx
