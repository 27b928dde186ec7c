// Instantiations of the sigma_min kernel for kl = 0 and ku = 0 .. 8.
#include "psa_kernel.cuh"

namespace psa {
KernelOps kernel_ops_kl0(int ku) { return kernel_ops_for_ku<0>(ku); }
}  // namespace psa
