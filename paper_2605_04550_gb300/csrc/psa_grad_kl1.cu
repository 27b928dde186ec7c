// Instantiations of the gradient kernel for kl = 1 and ku = 0 .. 8.
#include "psa_grad.cuh"

namespace psa {
KernelOps grad_ops_kl1(int ku) { return grad_ops_for_ku<1>(ku); }
}  // namespace psa
