// Kernel instantiations for 80 x 80 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_80() { return make_kernel_set<80>(); }
cudaError_t set_attrs_80() { return set_attrs_t<80>(); }
}  // namespace ptx
