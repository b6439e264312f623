// Kernel instantiations for 8 x 8 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_8() { return make_kernel_set<8>(); }
cudaError_t set_attrs_8() { return set_attrs_t<8>(); }
}  // namespace ptx
