// One variant of the persistent solver kernel: layout BCSR, small tiles of 16 lanes.
#include "solver_impl.cuh"

namespace wbpr {
void *solve_kernel_bcsr_16() { return (void *)solve_kernel<kBCSR, 16>; }
}  // namespace wbpr
