// Kernel instantiations for 224 x 224 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_224() { return make_kernel_set<224>(); }
cudaError_t set_attrs_224() { return set_attrs_t<224>(); }
}  // namespace ptx
