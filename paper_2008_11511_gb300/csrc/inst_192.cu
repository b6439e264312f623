// Kernel instantiations for 192 x 192 frames.
#include "kernels.cuh"

namespace ptx {
const KernelSet* kernel_set_192() { return make_kernel_set<192>(); }
cudaError_t set_attrs_192() { return set_attrs_t<192>(); }
}  // namespace ptx
