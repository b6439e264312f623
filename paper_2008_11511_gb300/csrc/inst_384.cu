// Kernel instantiations for 384 x 384 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_384() { return make_kernel_set<384>(); }
cudaError_t set_attrs_384() { return set_attrs_t<384>(); }
}  // namespace ptx
