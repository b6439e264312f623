// Kernel instantiations for 160 x 160 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_160() { return make_kernel_set<160>(); }
cudaError_t set_attrs_160() { return set_attrs_t<160>(); }
}  // namespace ptx
