// Instantiations of the gradient kernel for kl = 3 and ku = 0 .. 8.
#include "psa_grad.cuh"

namespace psa {
KernelOps grad_ops_kl3(int ku) { return grad_ops_for_ku<3>(ku); }
}  // namespace psa
