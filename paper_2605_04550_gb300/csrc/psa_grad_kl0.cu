// Instantiations of the gradient kernel for kl = 0 and ku = 0 .. 8.
#include "psa_grad.cuh"

namespace psa {
KernelOps grad_ops_kl0(int ku) { return grad_ops_for_ku<0>(ku); }
}  // namespace psa
