// Kernel instantiations for 512 x 512 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_512() { return make_kernel_set<512>(); }
cudaError_t set_attrs_512() { return set_attrs_t<512>(); }
}  // namespace ptx
