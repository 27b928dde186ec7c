// Instantiations of the gradient kernel for kl = 4 and ku = 0 .. 8.
#include "psa_grad.cuh"

namespace psa {
KernelOps grad_ops_kl4(int ku) { return grad_ops_for_ku<4>(ku); }
}  // namespace psa
