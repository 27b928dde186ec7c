// Instantiations of the gradient kernel for kl = 2 and ku = 0 .. 8.
#include "psa_grad.cuh"

namespace psa {
KernelOps grad_ops_kl2(int ku) { return grad_ops_for_ku<2>(ku); }
}  // namespace psa
