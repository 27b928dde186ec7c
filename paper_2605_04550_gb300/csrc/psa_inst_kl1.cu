// Instantiations of the sigma_min kernel for kl = 1 and ku = 0 .. 8.
#include "psa_kernel.cuh"

namespace psa {
launch_fn launcher_kl1(int ku) { return launcher_for_ku<1>(ku); }
}  // namespace psa
